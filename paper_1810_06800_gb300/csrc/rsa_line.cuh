// rsa_line.cuh -- round kernels for long k-mers (any k up to LINE_KMAX, L a
// multiple of 32), sm_103a.
//
// Every pass streams whole contiguous lines.  Horizontal candidates live on
// the rows of the occupancy bit lattice; vertical candidates live on the
// rows of its transpose, which is kept up to date beside it.  One round:
//   k_line_cmin<0>   cA[y][.] = width-k window minima of the live horizontal
//                    priorities along row y            (per-cell minimum, H)
//   k_line_cmin<1>   cB[x][.] = the same along column x (per-cell minimum, V,
//                    stored transposed)
//   k_line_codes     per cell, the smaller of the two minima inverted back to
//                    its candidate (splitmix64 is a bijection): a 2-byte argmin
//                    code in both layouts (32 x 32 tiles through smem)
//   k_line_accept_codes<F>  a live candidate is accepted iff its k cells
//                    carry its codes (start code, then +1 at every step)
// Caller-supplied priorities have no inverse: for them k_line_combine writes
// min(cA, cB) to both layouts and k_line_accept<F> compares values.
// The window minima are van Herk / Gil-Werman over blocks of k cells aligned
// on the staged span, with block-wide segmented prefix / suffix scans, so the
// cost per cell does not depend on k.  Segments and code tiles left without
// live candidates are flagged and skipped in later rounds.
#pragma once
#include "rsa_device.cuh"

namespace rsak {

constexpr u32 LINE_THREADS = 256;
constexpr u32 LINE_KMAX = 4096;

struct LineCfg {
  u32 S;        // segment length along a line (multiple of 32)
  u32 nseg;     // segments per line
  u32 nmax;     // S + k - 1
  u32 T;        // words per line = L / 32
  u32 compact;  // S <= k: the window-minimum pass keeps one value array (below)
};

// Segmented (k-aligned blocks) min-scan of n values held by the whole block.
// FWD: dst[u] = min(src[blockstart(u) .. u]); otherwise dst[u] =
// min(src[u .. blockend(u)]).  src may equal dst.  Thread t owns an odd-sized
// contiguous chunk (bank-conflict free); chunk aggregates are combined with a
// segmented warp scan and a scan over the 8 warp totals.
template <bool FWD>
__device__ void block_seg_scan(const u64* src, u64* dst, u32 n, u32 k, u64* wv, u32* wf) {
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  u32 C = (n + blockDim.x - 1) / blockDim.x;
  C |= 1u;
  const u32 a = min(tid * C, n), b = min(a + C, n);
  u64 run = KEY_NONE;
  bool flag = false;
  // one division per thread: the first block boundary inside the chunk
  if (FWD) {
    u32 nb = (a + k - 1) / k * k;        // next block start >= a
    for (u32 u = a; u < b; ++u) {
      if (u == nb) { run = KEY_NONE; flag = true; nb += k; }
      run = tmin(run, src[u]);
      dst[u] = run;
    }
  } else {
    u32 ne = b / k * k;                  // last block start <= b: p = ne - 1 ends a block
    for (u32 u = b; u > a; --u) {
      const u32 p = u - 1;
      if (p + 1 == ne) { run = KEY_NONE; flag = true; ne -= k; }
      run = tmin(run, src[p]);
      dst[p] = run;
    }
  }
  // inclusive segmented scan of (run, flag) over threads in scan order
  // (ascending tid for FWD, descending for the suffix scan)
  u64 v = run;
  bool f = flag;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u64 o = FWD ? __shfl_up_sync(FULL, v, d) : __shfl_down_sync(FULL, v, d);
    const bool of = FWD ? __shfl_up_sync(FULL, f, d) : __shfl_down_sync(FULL, f, d);
    const bool ok = FWD ? (int)lane >= d : lane + d < 32;
    if (ok) {
      if (!f) v = tmin(v, o);
      f = f || of;
    }
  }
  if (lane == (FWD ? 31u : 0u)) { wv[warp] = v; wf[warp] = f; }
  __syncthreads();
  if (warp == 0) {
    u64 x = lane < nw ? wv[FWD ? lane : nw - 1 - lane] : KEY_NONE;
    bool xf = lane < nw ? wf[FWD ? lane : nw - 1 - lane] != 0 : false;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u64 o = __shfl_up_sync(FULL, x, d);
      const bool of = __shfl_up_sync(FULL, xf, d);
      if ((int)lane >= d) {
        if (!xf) x = tmin(x, o);
        xf = xf || of;
      }
    }
    // exclusive prefix over warps, stored back in scan order
    u64 ex = __shfl_up_sync(FULL, x, 1);
    bool exf = __shfl_up_sync(FULL, xf, 1);
    if (lane == 0) { ex = KEY_NONE; exf = false; }
    __syncwarp();
    if (lane < nw) {
      const u32 at = FWD ? lane : nw - 1 - lane;
      wv[at] = ex;
      wf[at] = exf;
    }
  }
  __syncthreads();
  // carry into this thread = (warps before) combined with (lanes before)
  u64 lv = FWD ? __shfl_up_sync(FULL, v, 1) : __shfl_down_sync(FULL, v, 1);
  bool lf = FWD ? __shfl_up_sync(FULL, f, 1) : __shfl_down_sync(FULL, f, 1);
  if (lane == (FWD ? 0u : 31u)) { lv = KEY_NONE; lf = false; }
  const u64 carry = lf ? lv : tmin(wv[warp], lv);
  if (FWD) {
    if (a < b && (a % k) != 0) {
      const u64 stop = ((u64)a + k - 1) / k * k;
      const u32 e = (u32)(stop < b ? stop : b);
      for (u32 u = a; u < e; ++u) dst[u] = tmin(dst[u], carry);
    }
  } else {
    if (a < b && (b % k) != 0) {
      const u32 s0 = (b / k) * k;
      for (u32 u = (s0 > a ? s0 : a); u < b; ++u) dst[u] = tmin(dst[u], carry);
    }
  }
  __syncthreads();
}

// Number of set bits of the staged span words at bit positions < pos.
__device__ __forceinline__ u32 bits_before(const u32* w, const u32* wpre, u32 pos) {
  const u32 i = pos >> 5, r = pos & 31u;
  return wpre[i] + (r ? __popc(w[i] & ((1u << r) - 1u)) : 0u);
}

// Stage the occupancy words of a span [p0, p0 + nbits) of line `line`
// (p0 a multiple of 32, taken modulo L) and their exclusive popcount prefix.
__device__ __forceinline__ void stage_bits(const u32* occ_line, u32 T, int p0, u32 nwords, u32* w,
                                           u32* wpre, u32* scratch) {
  for (u32 i = threadIdx.x; i < nwords; i += blockDim.x) {
    // p0 / 32 >= -T - 1 and the span is shorter than 3 lines: at most two wraps
    int wi = p0 / 32 + (int)i;
    if (wi < 0) wi += (int)T;
    if (wi < 0) wi += (int)T;
    if (wi >= (int)T) wi -= (int)T;
    if (wi >= (int)T) wi -= (int)T;
    w[i] = occ_line[wi];
  }
  __syncthreads();
  // exclusive prefix sums of popcounts: one thread per 32-word chunk, then a
  // serial pass over the (few) chunk totals
  const u32 nch = (nwords + 31) / 32;
  for (u32 c = threadIdx.x; c < nch; c += blockDim.x) {
    u32 acc = 0;
    for (u32 i = c * 32; i < min(nwords, c * 32 + 32); ++i) {
      wpre[i] = acc;
      acc += __popc(w[i]);
    }
    scratch[c] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 acc = 0;
    for (u32 c = 0; c < nch; ++c) {
      const u32 t = scratch[c];
      scratch[c] = acc;
      acc += t;
    }
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < nwords; i += blockDim.x) wpre[i] += scratch[i >> 5];
  __syncthreads();
}

// Shared-memory carve-up of the line kernels: values / prefix minima V and
// suffix minima Q (nmax u64 each), staged occupancy words and their popcount
// prefix (WN u32 each), scan scratch (64 u32), accepted anchors (ACC u32),
// warp totals (32 u64 + 32 u32).
constexpr u32 LINE_ACC = 128;  // accepted anchors per segment: S / k <= 4096 / 32
struct LineSmem {
  u64* V; u64* Q; u32* w; u32* wpre; u32* scr; u32* acc; u64* wv; u32* wf;
};
__host__ __device__ inline u32 line_wn(u32 S, u32 k) { return (S + 2 * k + 64) / 32 + 3; }
// compact: one value array (Q aliases V), see k_line_cmin.
__host__ __device__ inline size_t line_smem_bytes(u32 nmax, u32 S, u32 k, bool compact = false) {
  return (size_t)nmax * (compact ? 8 : 16) + (size_t)line_wn(S, k) * 8 + 64 * 4 + LINE_ACC * 4 +
         32 * 8 + 32 * 4;
}
__device__ inline LineSmem line_smem(unsigned char* raw, u32 nmax, u32 S, u32 k,
                                     bool compact = false) {
  LineSmem m;
  m.V = reinterpret_cast<u64*>(raw);
  m.Q = compact ? m.V : m.V + nmax;
  m.w = reinterpret_cast<u32*>(m.V + (compact ? nmax : 2 * nmax));
  m.wpre = m.w + line_wn(S, k);
  m.scr = m.wpre + line_wn(S, k);
  m.acc = m.scr + 64;
  // keep the u64 warp totals 8-byte aligned
  size_t off = reinterpret_cast<size_t>(m.acc + LINE_ACC);
  off = (off + 7) & ~size_t(7);
  m.wv = reinterpret_cast<u64*>(off);
  m.wf = reinterpret_cast<u32*>(m.wv + 32);
  return m;
}

// Per-cell minimum of live priorities of one orientation along lines.
// F = 0: lines are rows y of occw, output cA[y][.]; F = 1: lines are columns
// x (rows of the transposed bits occT), output cB[x][.].
// ldead[((s * 2 + F) * L + line) * nseg + seg] is set once a segment's span
// holds no live candidate: its outputs were written as "none" in that round
// and stay so (candidates only die), so later rounds skip it.
template <int F>
__global__ void __launch_bounds__(LINE_THREADS) k_line_cmin(Group g, LineCfg lc, const u32* occw,
                                                            const u32* occT, u64* cA, u64* cB,
                                                            u8* ldead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, T = lc.T;
  const u32 line = blockIdx.x / lc.nseg, seg = blockIdx.x % lc.nseg;
  u8* dflag = ldead + ((size_t)(s * 2 + F) * L + line) * lc.nseg + seg;
  if (*dflag) return;
  const u32 x0 = seg * lc.S;
  const u32 Se = min(lc.S, L - x0);
  if (threadIdx.x == 0) work_add(g, F, Se);
  const u32 n = Se + k - 1;
  const u32 K32 = (k - 1 + 31) / 32 * 32;              // span starts K32 cells before x0
  const u32 nbits = K32 + Se + k - 1 + 32;
  const u32 nwords = (nbits + 31) / 32;
  const LineSmem m = line_smem(smem_raw, lc.nmax, lc.S, k, lc.compact != 0);
  u64 *V = m.V, *Q = m.Q, *wv = m.wv;
  u32 *w = m.w, *wpre = m.wpre, *scr = m.scr, *wf = m.wf;
  const u32* bits = (F == 0 ? occw : occT) + ((size_t)s * L + line) * T;
  stage_bits(bits, T, (int)x0 - (int)K32, nwords, w, wpre, scr);
  const u64 zb = g.base[s] + SM_GAMMA;
  bool any = false;
  // value u is the candidate anchored at position x0 - (k-1) + u, i.e. bit
  // offset K32 - (k-1) + u in the staged span
  for (u32 u = threadIdx.x; u < n; u += blockDim.x) {
    const u32 p = K32 - (k - 1) + u;
    const bool live = bits_before(w, wpre, p + k) == bits_before(w, wpre, p);
    u64 v = KEY_NONE;
    if (live) {
      // position x0 - (k-1) + u lies in [-(k-1), L + k - 1) with k <= L
      int pos = (int)x0 - (int)(k - 1) + (int)u;
      if (pos < 0) pos += (int)L;
      else if (pos >= (int)L) pos -= (int)L;
      const u64 idx = F == 0 ? (u64)line * L + (u32)pos : g.LL + (u64)(u32)pos * L + line;
      v = g.keys ? g.keys[idx] : mix64(zb + SM_GAMMA * idx);
      any = true;
    }
    V[u] = v;
  }
  __syncthreads();
  u64* out = (F == 0 ? cA : cB) + ((size_t)s * L + line) * L;
  if (lc.compact) {
    // Se <= S <= k: the span [0, Se + k - 1) holds two k-blocks.  The windows
    // need suffix minima only inside the first block ([0, k), in place) and
    // prefix minima only inside the second ([k, n), in place); the prefix
    // minimum at k - 1 closing the first block is its suffix minimum at 0.
    block_seg_scan<false>(V, V, k, k, wv, wf);
    if (n > k) block_seg_scan<true>(V + k, V + k, n - k, k, wv, wf);
    for (u32 v = threadIdx.x; v < Se; v += blockDim.x)
      out[x0 + v] = tmin(V[v], v == 0 ? V[0] : V[v + k - 1]);
  } else {
    block_seg_scan<false>(V, Q, n, k, wv, wf);
    block_seg_scan<true>(V, V, n, k, wv, wf);
    for (u32 v = threadIdx.x; v < Se; v += blockDim.x) out[x0 + v] = tmin(Q[v], V[v + k - 1]);
  }
  if (__syncthreads_or(any)) {
    if (threadIdx.x == 0 && !g.st[s].alive) g.st[s].alive = 1;
  } else if (threadIdx.x == 0) {
    *dflag = 1;
  }
}

// cmin = min(cA[y][x], cB[x][y]) into both layouts, one 32 x 32 tile of each.
__global__ void __launch_bounds__(256) k_line_combine(Group g, u64* cA, u64* cB) {
  __shared__ u64 ta[32][33], tb[32][33];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, T = L / 32;
  const u32 ty = blockIdx.x / T, tx = blockIdx.x % T;
  u64* A = cA + (size_t)s * g.LL;
  u64* B = cB + (size_t)s * g.LL;
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;
    ta[r][c] = A[(size_t)(ty * 32 + r) * L + tx * 32 + c];   // (y, x)
    tb[r][c] = B[(size_t)(tx * 32 + r) * L + ty * 32 + c];   // (x, y)
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;
    const u64 m = tmin(ta[r][c], tb[c][r]);  // cell (y = ty*32+r, x = tx*32+c)
    A[(size_t)(ty * 32 + r) * L + tx * 32 + c] = m;
  }
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;
    const u64 m = tmin(ta[c][r], tb[r][c]);  // cell (y = ty*32+c, x = tx*32+r)
    B[(size_t)(tx * 32 + r) * L + ty * 32 + c] = m;
  }
}

// Seeded priorities only: cmin of each cell as a 2-byte argmin code, in both
// layouts.  The winning key is inverted (mix64 is a bijection) back to its
// candidate idx, whose anchor gives the offset d = cell - anchor along the
// line: code d (0 .. k-1) for a horizontal winner, 0x8000 | d for a vertical
// one, CODE_NONE when no live candidate covers the cell.
constexpr u16 CODE_NONE = 0xFFFF;
constexpr u16 CODE_V = 0x8000;

// cdead[s * T^2 + tile] is set once every code of the 32 x 32 tile is
// CODE_NONE; they stay so, and later rounds skip the tile.
__global__ void __launch_bounds__(256) k_line_codes(Group g, const u64* cA, const u64* cB,
                                                    u16* code, u16* codeT, u8* cdead) {
  __shared__ u64 tb[32][33];
  __shared__ u16 tc[32][34];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, T = L / 32;
  u8* dflag = cdead + (size_t)s * T * T + blockIdx.x;
  if (*dflag) return;
  if (threadIdx.x == 0) work_add(g, 3, 1024);
  const u32 ty = blockIdx.x / T, tx = blockIdx.x % T;
  const u64* A = cA + (size_t)s * g.LL;
  const u64* B = cB + (size_t)s * g.LL;
  u16* C = code + (size_t)s * g.LL;
  u16* CT = codeT + (size_t)s * g.LL;
  const u64 zb = g.base[s] + SM_GAMMA;
  // exact division by L = 2^lsh * q (q odd): shift, then multiply by the
  // inverse of q modulo 2^32 (Newton's iteration doubles the correct bits)
  const u32 lsh = __ffs(L) - 1, q = L >> lsh;
  u32 lqinv = q;
#pragma unroll
  for (int i = 0; i < 5; ++i) lqinv *= 2u - q * lqinv;
  bool any = false;
  // the vertical minima of the tile, read along their own rows (columns x)
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;                 // (x, y) = (tx*32 + r, ty*32 + c)
    tb[r][c] = B[(size_t)(tx * 32 + r) * L + ty * 32 + c];
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;                 // cell (y, x) = (ty*32 + r, tx*32 + c)
    const u32 y = ty * 32 + r, x = tx * 32 + c;
    const u64 vh = A[(size_t)y * L + x];
    const u64 vv = tb[c][r];
    u16 out = CODE_NONE;
    if (vh != vv) {
      const u64 m = vh < vv ? vh : vv;
      const u32 idx = (u32)((mix64_inverse(m) - zb) * SM_GAMMA_INV);
      if (vh < vv) {
        // a horizontal candidate covering (y, x) is anchored on row y
        u32 d = x + L - (idx - y * L);
        if (d >= L) d -= L;
        out = (u16)d;
      } else {
        // anchored on column x: idx = L^2 + ya L + x, and (y - ya) mod L is
        // the exact quotient of (y L - ya L) mod L^2 by L
        u32 dl = y * L - (idx - (u32)g.LL - x);
        if ((int)dl < 0) dl += (u32)g.LL;
        const u32 d = (dl >> lsh) * lqinv;
        out = (u16)(CODE_V | d);
      }
    }
    C[(size_t)y * L + x] = out;
    tc[r][c] = out;
    any |= out != CODE_NONE;
  }
  if (!__syncthreads_or(any) && threadIdx.x == 0) *dflag = 1;
  for (u32 i = threadIdx.x; i < 1024; i += blockDim.x) {
    const u32 r = i >> 5, c = i & 31;                 // row x = tx*32 + r of the transpose
    CT[(size_t)(tx * 32 + r) * L + ty * 32 + c] = tc[c][r];
  }
}

// Record an accepted candidate with the whole block: node, occupancy bits in
// both layouts, owner ids of its k cells.
__device__ void accept_block(const Group& g, u32* occw, u32* occT, u32 T, u32 s, u32 idx, u64 key,
                             u32* node_sh) {
  if (threadIdx.x == 0) {
    u32 node = atomicAdd(&g.st[s].n_nodes, 1u);
    if (node >= g.cap_nodes) {
      atomicOr(&g.st[s].status, ST_NODE_OVF);
      node = NONE32;
    }
    *node_sh = node;
  }
  __syncthreads();
  const u32 node = *node_sh;
  __syncthreads();
  if (node == NONE32) return;
  const u32 L = g.L, k = g.k;
  const u32 o = idx / (u32)g.LL, r = idx - o * (u32)g.LL;
  const u32 y0 = r / L, x0 = r - y0 * L;
  if (threadIdx.x == 0) {
    g.node_key[(size_t)s * g.cap_nodes + node] = key;
    g.node_idx[(size_t)s * g.cap_nodes + node] = idx;
    g.node_pos[(size_t)s * g.cap_nodes + node] = (o << 31) | (y0 << 15) | x0;
  }
  u32* ow = occw + (size_t)s * L * T;
  u32* ot = occT + (size_t)s * L * T;
  u32* own = g.owner + (size_t)s * g.LL;
  for (u32 i = threadIdx.x; i < k; i += blockDim.x) {
    u32 y = y0, x = x0;
    if (o == 0) { x += i; if (x >= L) x -= L; }
    else { y += i; if (y >= L) y -= L; }
    atomicOr(ow + (size_t)y * T + (x >> 5), 1u << (x & 31u));
    atomicOr(ot + (size_t)x * T + (y >> 5), 1u << (y & 31u));
    own[(size_t)y * L + x] = node | (o << 31);
  }
}

// Acceptance along lines: F = 0 rows of cA (horizontal candidates), F = 1
// rows of cB (vertical candidates, the columns of the lattice).
template <int F>
__global__ void __launch_bounds__(LINE_THREADS) k_line_accept(Group g, LineCfg lc, u32* occw,
                                                              u32* occT, const u64* cA,
                                                              const u64* cB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, T = lc.T;
  const u32 line = blockIdx.x / lc.nseg, seg = blockIdx.x % lc.nseg;
  const u32 x0 = seg * lc.S;
  const u32 Se = min(lc.S, L - x0);
  const u32 n = Se + k - 1;
  const u32 nbits = Se + k + 32;
  const u32 nwords = (nbits + 31) / 32;
  const LineSmem m = line_smem(smem_raw, lc.nmax, lc.S, k);
  u64 *V = m.V, *Q = m.Q, *wv = m.wv;
  u32 *w = m.w, *wpre = m.wpre, *scr = m.scr, *wf = m.wf;
  const u64* row = (F == 0 ? cA : cB) + ((size_t)s * L + line) * L;
  for (u32 u = threadIdx.x; u < n; u += blockDim.x) {
    u32 p = x0 + u;
    while (p >= L) p -= L;
    V[u] = row[p];
  }
  const u32* bits = (F == 0 ? occw : occT) + ((size_t)s * L + line) * T;
  stage_bits(bits, T, (int)x0, nwords, w, wpre, scr);
  block_seg_scan<false>(V, Q, n, k, wv, wf);
  block_seg_scan<true>(V, V, n, k, wv, wf);
  // window minimum of anchor x0 + v is min(Q[v], P[v + k - 1]); collect the
  // accepted anchors in smem (accepted ones do not overlap: at most S / k)
  u32* acc = m.acc;
  __shared__ u32 nacc, node_sh;
  if (threadIdx.x == 0) nacc = 0;
  __syncthreads();
  const u64 zb = g.base[s] + SM_GAMMA;
  for (u32 v = threadIdx.x; v < Se; v += blockDim.x) {
    const u64 f = tmin(Q[v], V[v + k - 1]);
    if (f == KEY_NONE) continue;
    if (bits_before(w, wpre, v + k) != bits_before(w, wpre, v)) continue;
    const u32 pos = x0 + v;
    const u64 idx = F == 0 ? (u64)line * L + pos : g.LL + (u64)pos * L + line;
    const u64 key = g.keys ? g.keys[idx] : mix64(zb + SM_GAMMA * idx);
    if (f == key) {
      const u32 slot = atomicAdd(&nacc, 1u);
      if (slot < LINE_ACC) acc[slot] = v;
    }
  }
  __syncthreads();
  const u32 na = nacc;
  for (u32 i = 0; i < na && i < LINE_ACC; ++i) {
    const u32 v = acc[i];
    const u32 pos = x0 + v;
    const u64 idx = F == 0 ? (u64)line * L + pos : g.LL + (u64)pos * L + line;
    const u64 key = tmin(Q[v], V[v + k - 1]);
    accept_block(g, occw, occT, T, s, (u32)idx, key, &node_sh);
  }
  if (na > LINE_ACC && threadIdx.x == 0) atomicOr(&g.st[s].status, ST_NODE_OVF);
}

// Acceptance from argmin codes (seeded priorities): along a line (F = 0 a row
// of code, F = 1 a row of codeT), the candidate anchored at position v is
// accepted iff code(v) = base and code(j + 1) = code(j) + 1 for the k-1
// steps j = v .. v+k-2.  "Breaks" of that pattern are packed into words by
// warp ballots; a popcount prefix answers each anchor with two lookups.
template <int F>
__global__ void __launch_bounds__(LINE_THREADS) k_line_accept_codes(Group g, LineCfg lc,
                                                                    u32* occw, u32* occT,
                                                                    const u16* code,
                                                                    const u16* codeT,
                                                                    const u8* ldead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, T = lc.T;
  const u32 line = blockIdx.x / lc.nseg, seg = blockIdx.x % lc.nseg;
  // no live candidate anchored in this segment (its window-minimum span,
  // which contains these anchors, had none this round)
  if (ldead[((size_t)(s * 2 + F) * L + line) * lc.nseg + seg]) return;
  const u32 x0 = seg * lc.S;
  const u32 Se = min(lc.S, L - x0);
  if (threadIdx.x == 0) work_add(g, 2, Se);
  const u32 n = Se + k - 1;                  // codes x0 .. x0+n-1
  const u32 nwords = (n + 31) / 32;
  u16* cv = reinterpret_cast<u16*>(smem_raw);                 // n (+1) codes, 8-code chunks
  u32* brk = reinterpret_cast<u32*>(cv + ((lc.nmax + 9) & ~7u));
  u32* pre = brk + ((lc.nmax + 31) / 32 + 2);
  u32* scr = pre + ((lc.nmax + 31) / 32 + 2);
  __shared__ u32 nacc, node_sh;
  __shared__ u32 acc[LINE_ACC];
  const u16* row = (F == 0 ? code : codeT) + ((size_t)s * L + line) * L;
  // codes x0 .. x0+n (around the torus) in 16-byte chunks: x0 and L are
  // multiples of 32, so a chunk of 8 never crosses the end of the line
  for (u32 u = threadIdx.x * 8; u <= n; u += blockDim.x * 8) {
    u32 p = x0 + u;
    while (p >= L) p -= L;
    *reinterpret_cast<uint4*>(cv + u) = __ldg(reinterpret_cast<const uint4*>(row + p));
  }
  if (threadIdx.x == 0) nacc = 0;
  __syncthreads();
  const u32 base = F == 0 ? 0u : (u32)CODE_V;
  // break bit of step j (code(j) -> code(j+1)); all threads of a warp walk
  // the same 32-position words
  for (u32 w0 = (threadIdx.x >> 5) * 32; w0 < nwords * 32; w0 += blockDim.x) {
    const u32 j = w0 + (threadIdx.x & 31);
    bool b = true;
    if (j < n) {
      const u32 a = cv[j], c = cv[j + 1];
      b = !(a >= base && a + 1 < base + k && c == a + 1);
    }
    const u32 m = __ballot_sync(FULL, b);
    if ((threadIdx.x & 31) == 0) brk[w0 >> 5] = m;
  }
  __syncthreads();
  // exclusive popcount prefix of the break words
  const u32 nch = (nwords + 31) / 32;
  for (u32 c = threadIdx.x; c < nch; c += blockDim.x) {
    u32 a = 0;
    for (u32 i = c * 32; i < min(nwords, c * 32 + 32); ++i) { pre[i] = a; a += __popc(brk[i]); }
    scr[c] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 a = 0;
    for (u32 c = 0; c < nch; ++c) { const u32 t = scr[c]; scr[c] = a; a += t; }
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < nwords; i += blockDim.x) pre[i] += scr[i >> 5];
  __syncthreads();
  const u64 zb = g.base[s] + SM_GAMMA;
  for (u32 v = threadIdx.x; v < Se; v += blockDim.x) {
    if (cv[v] != base) continue;
    if (k > 1 && bits_before(brk, pre, v + k - 1) != bits_before(brk, pre, v)) continue;
    const u32 slot = atomicAdd(&nacc, 1u);
    if (slot < LINE_ACC) acc[slot] = v;
  }
  __syncthreads();
  const u32 na = nacc;
  for (u32 i = 0; i < na && i < LINE_ACC; ++i) {
    const u32 pos = x0 + acc[i];
    const u64 idx = F == 0 ? (u64)line * L + pos : g.LL + (u64)pos * L + line;
    accept_block(g, occw, occT, T, s, (u32)idx, mix64(zb + SM_GAMMA * idx), &node_sh);
  }
  if (na > LINE_ACC && threadIdx.x == 0) atomicOr(&g.st[s].status, ST_NODE_OVF);
}

__host__ __device__ inline size_t line_codes_smem_bytes(u32 nmax) {
  return (size_t)((nmax + 9) & ~7u) * 2 + (size_t)((nmax + 31) / 32 + 2) * 8 + 64 * 4;
}

}  // namespace rsak
