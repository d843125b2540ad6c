// rsa_lwin.cuh -- round kernels of the long-k path for lattices whose lines
// split into whole k-blocks (L a multiple of k and of the CTA span P), sm_103a.
//
// One round, with argmin offsets instead of 8-byte minima:
//   k_lwin<0>   along each row y: for every cell, the live horizontal
//               candidate of smallest priority among those covering it, as
//               its offset d = cell - anchor (0 .. k-1) or CODE_NONE;
//   k_lwin<1>   the same along each column (rows of the transposed
//               occupancy), stored transposed;
//   k_lcomb     per cell, the smaller of the two winners' priorities (both
//               recomputed from their anchors) picks the final winner, kept
//               as bit masks in its orientation's layout (32 x 32 squares,
//               one warp each);
//   k_lacc<F>   acceptance along lines from the masks, 32 anchors per word
//               operation, and the accepted k-mers' nodes, occupancy and
//               owners.
//
// k_lwin is van Herk / Gil-Werman with blocks of k cells aligned on the line
// (L is a multiple of k, so the blocks tile the torus): the window of cell x
// in block b at offset j is the suffix minimum of block b-1 from offset j+1
// and the prefix minimum of block b up to j (the whole of block b if
// j = k-1).  A line is cut into nc = L / P spans of P = NT C cells (NT = 256
// threads, or 128 with C = 32 on 4096-cell spans), one CTA each, launched as
// one thread-block cluster per line.  Thread t holds the C
// consecutive candidates of its chunk in registers: liveness from the staged
// occupancy words (a candidate is live iff the next occupied cell is at
// least k ahead), splitmix64 priorities of the live ones, in-chunk prefix and
// suffix minima, and segmented block scans of the chunk minima within each
// k-block.  Suffix minima go to shared memory; the window of a cell whose
// block b-1 lies in the previous span reads them from that CTA's shared
// memory over the cluster (distributed shared memory), so no priority is
// computed twice.  Every minimum carries the line position of its
// candidate, so the winner's offset is cell - position.
//
// A span with no live anchor has no live anchor in any later round: it is
// flagged and skips hashing and scans; once it and the span before it are
// both flagged, its outputs (written as "none" in the round that made them
// so) are not touched again.
#pragma once
#include <cooperative_groups.h>

#include "rsa_line.cuh"
#include "rsa_tile.cuh"  // cp.async helpers

namespace rsak {

constexpr u32 LW_THREADS = 256;
constexpr u32 LW_INF = 0xFFFFFFFFu;

struct LwinCfg {
  u32 P;   // cells of a line per CTA: 256 * C, a multiple of k and of 32
  u32 nc;  // CTAs per line (cluster size), L = nc * P, nc <= 8
  u32 T;   // occupancy words per line, L / 32
};

constexpr u32 LW_SENT = 0xFFFFu;  // position of "no candidate"

// (key, position) minimum: a = the smaller of a and b with its position.
// Keys are distinct except KEY_NONE, which always carries LW_SENT.
__device__ __forceinline__ void kp_min(u64& a, u32& pa, u64 b, u32 pb) {
  const bool lt = b < a;
  a = lt ? b : a;
  pa = lt ? pb : pa;
}

// Exclusive prefix and suffix (key, position) minima of one value per
// thread, within segments of m consecutive threads (m a power of two, the
// chunks of one k-block): sub-warp shuffles of width min(m, 32), then, for
// segments of several warps, the totals of the other warps of the segment.
__device__ __forceinline__ void lw_block_scans(u64 a, u32 pa, u32 m, u64& ep, u32& epp, u64& es,
                                               u32& esp, u64* wtf, u32* wtfp, u64* wtb,
                                               u32* wtbp) {
  // (m is at most the block's thread count: a k-block never spans CTAs)
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 wd = m < 32 ? m : 32, li = lane & (wd - 1);
  u64 f = a, b = a;
  u32 fp = pa, bp = pa;
#pragma unroll
  for (u32 d = 1; d < 32; d <<= 1) {
    const u64 of = __shfl_up_sync(FULL, f, d, wd);
    const u32 ofp = __shfl_up_sync(FULL, fp, d, wd);
    const u64 ob = __shfl_down_sync(FULL, b, d, wd);
    const u32 obp = __shfl_down_sync(FULL, bp, d, wd);
    if (d < wd) {
      if (li >= d) kp_min(f, fp, of, ofp);
      if (li + d < wd) kp_min(b, bp, ob, obp);
    }
  }
  // exclusive: the inclusive value of the previous (next) thread
  u64 xf = __shfl_up_sync(FULL, f, 1, wd), xb = __shfl_down_sync(FULL, b, 1, wd);
  u32 xfp = __shfl_up_sync(FULL, fp, 1, wd), xbp = __shfl_down_sync(FULL, bp, 1, wd);
  if (li == 0) { xf = KEY_NONE; xfp = LW_SENT; }
  if (li == wd - 1) { xb = KEY_NONE; xbp = LW_SENT; }
  if (m > 32) {
    if (lane == 31) { wtf[warp] = f; wtfp[warp] = fp; }
    if (lane == 0) { wtb[warp] = b; wtbp[warp] = bp; }
    __syncthreads();
    const u32 ws = m / 32, w0 = warp & ~(ws - 1);
    for (u32 w2 = w0; w2 < warp; ++w2) kp_min(xf, xfp, wtf[w2], wtfp[w2]);
    for (u32 w2 = warp + 1; w2 < w0 + ws; ++w2) kp_min(xb, xbp, wtb[w2], wtbp[w2]);
  }
  ep = xf; epp = xfp;
  es = xb; esp = xbp;
}

// F = 0: rows y of occw, offsets to cH[y][.]; F = 1: columns x (rows of the
// transposed occT), offsets to cV[x][.].  lflag[((s * 2 + F) * L + line) *
// nc + r] bit 0: span r of the line has no live anchor (stays so).
// Minima carry the line position of their candidate, so the offset of the
// winner is cell - position; no priority is inverted.
template <int F, int C, int NT>
__global__ void __launch_bounds__(NT) k_lwin(Group g, LwinCfg lc, const u32* occw,
                                             const u32* occT, u16* cout, u8* lflag) {
  namespace cg = cooperative_groups;
  constexpr u32 WPT = (256 + NT - 1) / NT;  // occupancy words staged per thread
  __shared__ u64 Qk[C][NT];      // in-chunk suffix minimum at element e of chunk t: [e][t]
  __shared__ u16 Qp[C][NT];      // its candidate's position on the line
  __shared__ u64 Ek[NT];         // suffix minimum of the chunks after chunk t in its k-block
  __shared__ u16 Ep[NT];
  __shared__ u32 w[256 + 2];     // staged occupancy words
  __shared__ u32 nw[256 + 2];    // first occupied position at / after word i
  __shared__ u32 wmin[NT / 32];
  __shared__ u64 wtf[NT / 32], wtb[NT / 32];
  __shared__ u32 wtfp[NT / 32], wtbp[NT / 32];
  cg::cluster_group cl = cg::this_cluster();
  const u32 nc = lc.nc, r = cl.block_rank();
  const u32 line = blockIdx.x / nc, s = blockIdx.y;
  if (g.st[s].done) return;  // the same for every CTA of the cluster
  const u32 L = g.L, k = g.k, T = lc.T, P = lc.P;
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 rp = r == 0 ? nc - 1 : r - 1;
  u8* fl = lflag + ((size_t)(s * 2 + F) * L + line) * nc;
  // a line whose spans are all flagged has no live anchor and final outputs;
  // every CTA of the cluster reads the same flags (none is written before
  // the cluster's barriers) and leaves before those barriers
  if (__all_sync(FULL, lane >= nc || (fl[lane] & 1u) != 0)) return;
  const bool own_dead = (fl[r] & 1u) != 0, prev_dead = (fl[rp] & 1u) != 0;
  const u32 x0 = r * P;
  const u32 q0 = tid * C;   // first cell of this thread's chunk (relative to x0)
  const u32 xs = x0 + q0;   // its position on the line
  const u32 m = k / C;      // chunks per k-block
  u64 v[C];
#pragma unroll
  for (int e = 0; e < C; ++e) v[e] = KEY_NONE;
  bool any = false;
  u64 ep = KEY_NONE, es = KEY_NONE;
  u32 epp = LW_SENT, esp = LW_SENT;
  if (!own_dead) {
    // occupancy words of [x0, x0 + P + k - 1), around the torus; thread t
    // stages words t WPT .. t WPT + WPT - 1
    const u32 nwords = (P + k + 30) / 32;  // <= 256: P, k <= 4096
    const u32* bits = (F == 0 ? occw : occT) + ((size_t)s * L + line) * T;
    u32 fst[WPT];
#pragma unroll
    for (u32 j = 0; j < WPT; ++j) {
      const u32 i = tid * WPT + j;
      fst[j] = LW_INF;
      if (i < nwords) {
        u32 wi = x0 / 32 + i;
        while (wi >= T) wi -= T;
        const u32 wdd = bits[wi];
        w[i] = wdd;
        if (wdd) fst[j] = i * 32 + __ffs(wdd) - 1;
      }
    }
    // nw[i] = min over words j >= i of their first occupied position
#pragma unroll
    for (int j = (int)WPT - 2; j >= 0; --j) fst[j] = min(fst[j], fst[j + 1]);
    u32 sm = fst[0];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u32 o = __shfl_down_sync(FULL, sm, d);
      if (lane + d < 32) sm = min(sm, o);
    }
    if (lane == 0) wmin[warp] = sm;
    __syncthreads();
    // what follows this thread's words: later lanes of the warp, later warps
    u32 after = __shfl_down_sync(FULL, sm, 1);
    if (lane == 31) after = LW_INF;
    for (u32 w2 = warp + 1; w2 < NT / 32; ++w2) after = min(after, wmin[w2]);
#pragma unroll
    for (u32 j = 0; j < WPT; ++j)
      if (tid * WPT + j < 256) nw[tid * WPT + j] = min(fst[j], after);
    if (tid == 0) nw[256] = LW_INF;
    __syncthreads();
    // the chunk's candidates.  k > 32, so a candidate at q is live iff no
    // cell of its own word from q on is occupied (q is past the word's last
    // occupied bit) and the first occupied cell after that word is at least
    // k ahead: an interval e_lo <= e <= e_hi of the chunk's offsets
    const u32 wi = q0 >> 5, rb = q0 & 31u;  // C divides 32: one word holds the chunk
    const u32 wdd = w[wi], nxtw = nw[wi + 1];
    const int e_lo = wdd ? (int)(31 - __clz(wdd)) - (int)rb + 1 : 0;
    const int e_hi = nxtw == LW_INF ? C : (int)nxtw - (int)k - (int)q0;
    // the chunk's suffix minima, last element first; the one at element 0
    // is the chunk minimum
    u64 rk = KEY_NONE;
    u32 rq = LW_SENT;
    if (e_lo <= e_hi && e_lo < C && e_hi >= 0) {
      any = true;
      const u64 zstep = F == 0 ? SM_GAMMA : SM_GAMMA * (u64)L;
      u64 z = g.base[s] + SM_GAMMA +
              SM_GAMMA * (F == 0 ? (u64)line * L + xs + C - 1 : g.LL + (u64)(xs + C - 1) * L + line);
#pragma unroll
      for (int e = C - 1; e >= 0; --e, z -= zstep) {
        const u64 h = mix64(z);
        v[e] = (e >= e_lo && e <= e_hi) ? h : KEY_NONE;
        kp_min(rk, rq, v[e], xs + e);
        Qk[e][tid] = rk;
        Qp[e][tid] = (u16)rq;
      }
    } else {
#pragma unroll
      for (int e = 0; e < C; ++e) {
        Qk[e][tid] = KEY_NONE;
        Qp[e][tid] = (u16)LW_SENT;
      }
    }
    // chunk minima combined within each k-block (m consecutive chunks)
    lw_block_scans(rk, rq, m, ep, epp, es, esp, wtf, wtfp, wtb, wtbp);
  } else {
    // a span without live anchors publishes "none", so readers need not know
#pragma unroll
    for (int e = 0; e < C; ++e) {
      Qk[e][tid] = KEY_NONE;
      Qp[e][tid] = (u16)LW_SENT;
    }
  }
  Ek[tid] = es;
  Ep[tid] = (u16)esp;
  cl.sync();  // suffix minima of every span of the line are in shared memory
  if (!(own_dead && prev_dead)) {
    // cell q0 + e needs the suffix minimum of its window's first k-block
    // from q0 + e - k + 1 on, in chunk ca = tid - m (the previous span's
    // chunk ca + NT when ca < 0): for e < C - 1 the smaller of ca's in-chunk
    // suffix minimum at element e + 1 and the minimum E of the chunks after
    // ca in that k-block; for e = C - 1 it is E alone (the chunk after ca,
    // or nothing when this chunk ends its k-block, and then E is "none").
    // E is folded into the running prefix minimum once.
    const int ca = (int)tid - (int)m;
    const u64* ka;
    const u16* pa;
    u64 rk;
    u32 rq;
    if (ca >= 0) {
      ka = &Qk[0][ca];
      pa = &Qp[0][ca];
      rk = Ek[ca];
      rq = Ep[ca];
    } else {
      ka = cl.map_shared_rank(&Qk[0][0], rp) + (ca + (int)NT);
      pa = cl.map_shared_rank(&Qp[0][0], rp) + (ca + (int)NT);
      rk = cl.map_shared_rank(&Ek[0], rp)[ca + (int)NT];
      rq = cl.map_shared_rank(&Ep[0], rp)[ca + (int)NT];
    }
    kp_min(rk, rq, ep, epp);
    u32 packed[(C + 1) / 2];
#pragma unroll
    for (int e = 0; e < C; ++e) {
      kp_min(rk, rq, v[e], xs + e);  // prefix minimum within the k-block (and E)
      u64 mk = rk;
      u32 mq = rq;
      if (e < C - 1) kp_min(mk, mq, ka[(e + 1) * NT], pa[(e + 1) * NT]);
      const u32 x = xs + e;
      u32 d = x - mq;
      if (x < mq) d += L;
      const u32 code = mq == LW_SENT ? (u32)CODE_NONE : d;
      if (e & 1) packed[e >> 1] |= code << 16;
      else packed[e >> 1] = code;
    }
    u16* dst = cout + ((size_t)s * L + line) * L + xs;
    if constexpr (C >= 8) {
#pragma unroll
      for (int i = 0; i < C / 8; ++i)
        reinterpret_cast<uint4*>(dst)[i] =
            make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
    } else if constexpr (C == 4) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(packed[0], packed[1]);
    } else if constexpr (C == 2) {
      *reinterpret_cast<u32*>(dst) = packed[0];
    } else {
      *dst = (u16)packed[0];
    }
    if (tid == 0) work_add(g, F, P);
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
  if (!own_dead) {
    if (__syncthreads_or(any)) {
      if (tid == 0 && !g.st[s].alive) g.st[s].alive = 1;
    } else if (tid == 0) {
      fl[r] |= 1u;
    }
  }
}

// Acceptance masks of one orientation: one bit per cell, 32 cells per word
// along that orientation's own lines (rows for horizontal candidates, the
// transposed layout for vertical ones).
struct AccMasks {
  u32* win;    // the cell's final winner has this orientation
  u32* first;  // ... and the cell is its winner's first cell (offset 0)
  u32* last;   // ... and the cell is its winner's last cell (offset k - 1)
};

// Final winner of every cell from the two orientations' argmin offsets: the
// candidate of smaller priority (both recomputed from their anchors), kept
// as the acceptance masks of its orientation.  A candidate anchored at a is
// accepted iff it is the smallest live candidate on each of its k cells, and
// since the winners' anchors are monotone along a line that holds iff cell
// a has it as winner at offset 0, cell a + k - 1 at offset k - 1, and every
// cell in between is won by its orientation (k_lacc).  One warp per square
// of 32 x 32 cells, all its loads (the offsets of both orientations, 4 KB,
// coalesced into shared memory) issued first: lane = column, walking down it (the vertical
// winners' offsets and the high 32 bits of their priorities go to shared
// memory; bits of the cells whose vertical offset is 0 or k - 1), then lane
// = row, walking along it (horizontal winners compared with the vertical
// ones: the row masks, and a bit per cell that the vertical candidate wins);
// a 32 x 32 bit transpose across the warp turns those bits into the column
// masks.  Two priorities with equal high halves (rare) are compared in full,
// the vertical one recomputed from its offset.  A winner's priority is
// recomputed only when its anchor changes along the walk; the hash is an
// out-of-line call so that the fully unrolled walks stay small.
// cdead[s * T^2 + square] is set once no cell of the square is covered by a
// live candidate (it stays so, with its masks zero; later rounds skip it).
constexpr u32 LC_WARPS = 4;
union LcombWarp {
  // the square's offsets as loaded: [orientation][line][16 words], the four
  // 16-byte chunks of line r stored in the order c ^ ((r >> 1) & 3), so that
  // both the coalesced stores and the per-line reads are conflict-free
  u32 stage[2][32][16];
  struct {
    u32 vh[32][33];   // high halves of the vertical winners' priorities [x][y]
    u16 vd[32][34];   // their offsets [x][y], CODE_NONE if none
  } w;
};
struct LcombSmem {
  LcombWarp wp[LC_WARPS];
};

// 32 x 32 bit-matrix transpose across a warp: lane r holds row r (bit c is
// entry (r, c)); on return lane c holds column c (bit r is entry (r, c)).
// Step j swaps the off-diagonal j x j blocks of every 2j x 2j block.
__device__ __forceinline__ u32 warp_transpose32(u32 x, u32 lane) {
  constexpr u32 lo[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const u32 j = 16u >> i, m = lo[i];
    const u32 t = __shfl_xor_sync(FULL, x, j);
    x = (lane & j) ? ((x & ~m) | ((t >> j) & m)) : ((x & m) | ((t << j) & ~m));
  }
  return x;
}

__device__ __noinline__ u64 mix64_call(u64 z) { return mix64(z); }

__global__ void __launch_bounds__(LC_WARPS * 32, 8) k_lcomb(Group g, const u16* cH, const u16* cV,
                                                         AccMasks mh, AccMasks mv, u8* cdead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LcombSmem& sm = *reinterpret_cast<LcombSmem*>(smem_raw);
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, T = L / 32, NQ = T * T;  // squares per sample
  const u32 lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const u32 sq = blockIdx.x * LC_WARPS + wp;
  if (sq >= NQ) return;
  u8* dflag = cdead + (size_t)s * NQ + sq;
  if (*dflag) return;
  const u32 ty = sq / T, tx = sq - ty * T, Y = ty * 32, X = tx * 32;
  const u64 zb = g.base[s] + SM_GAMMA;
  const size_t so = (size_t)s * g.LL;
  LcombWarp& ws = sm.wp[wp];
  u32 (*vh)[33] = ws.w.vh;
  u16 (*vd)[34] = ws.w.vd;
  // the square's 64-byte line pieces, four lanes per line (coalesced), into
  // shared memory: vertical offsets of columns X .. X + 31 (rows Y ..
  // Y + 31), horizontal offsets of rows Y .. Y + 31 (columns X .. X + 31)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const u32 r = 8 * j + (lane >> 2), c = lane & 3, cs = c ^ ((r >> 1) & 3u);
    cp_async16(&ws.stage[0][r][cs * 4], cV + so + (size_t)(X + r) * L + Y + c * 8);
    cp_async16(&ws.stage[1][r][cs * 4], cH + so + (size_t)(Y + r) * L + X + c * 8);
  }
  cp_async_wait_all();
  __syncwarp();
  // lane = line: column X + lane's vertical and row Y + lane's horizontal
  // offsets, 16 words each
  u32 cvw[16], chw[16];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const u32 cs = (u32)j ^ ((lane >> 1) & 3u);
    const uint4 a = *reinterpret_cast<const uint4*>(&ws.stage[0][lane][cs * 4]);
    const uint4 b = *reinterpret_cast<const uint4*>(&ws.stage[1][lane][cs * 4]);
    cvw[4 * j] = a.x, cvw[4 * j + 1] = a.y, cvw[4 * j + 2] = a.z, cvw[4 * j + 3] = a.w;
    chw[4 * j] = b.x, chw[4 * j + 1] = b.y, chw[4 * j + 2] = b.z, chw[4 * j + 3] = b.w;
  }
  __syncwarp();  // the staging area is reused for the vertical winners
  u32 v0 = 0, vl = 0;  // rows of column X + lane with vertical offset 0, k - 1
  {
    const u32 x = X + lane;
    u32 ca = NONE32, ch = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const u32 d = (cvw[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
      const bool has = d != CODE_NONE;
      u32 ya = Y + i + L - d;
      if (ya >= L) ya -= L;
      // the only branch: a new anchor along the column
      if (has && ya != ca) {
        ch = (u32)(mix64_call(zb + SM_GAMMA * (g.LL + (u64)ya * L + x)) >> 32);
        ca = ya;
      }
      vh[lane][i] = ch;
      vd[lane][i] = (u16)d;
      v0 |= (u32)(d == 0) << i;
      vl |= (u32)(d == k - 1) << i;
    }
  }
  __syncwarp();
  u32 bw = 0, b0 = 0, bk = 0, bv = 0;  // row masks; bv: cells the vertical winner takes
  {
    const u32 y = Y + lane;
    u32 ca = NONE32;
    u64 ck = KEY_NONE;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const u32 d = (chw[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
      const bool has = d != CODE_NONE;
      u32 xa = X + i + L - d;
      if (xa >= L) xa -= L;
      if (has && xa != ca) {
        ck = mix64_call(zb + SM_GAMMA * ((u64)y * L + xa));
        ca = xa;
      }
      const u32 dv = vd[i][lane];
      const bool hasv = dv != CODE_NONE;
      const u32 khi = (u32)(ck >> 32), kvhi = vh[i][lane];
      bool hw, vw;
      if (has && hasv && khi == kvhi) {
        // equal high halves: compare the full priorities
        u32 ya = y + L - dv;
        if (ya >= L) ya -= L;
        const u64 kv = mix64_call(zb + SM_GAMMA * (g.LL + (u64)ya * L + X + i));
        hw = ck < kv;
        vw = kv < ck;
      } else {
        hw = has && (!hasv || khi < kvhi);
        vw = hasv && (!has || kvhi < khi);
      }
      bw |= (u32)hw << i;
      bv |= (u32)vw << i;
      b0 |= (u32)(hw && d == 0) << i;
      bk |= (u32)(hw && d == k - 1) << i;
    }
  }
  const size_t wi = ((size_t)s * L + Y + lane) * T + tx;
  mh.win[wi] = bw;
  mh.first[wi] = b0;
  mh.last[wi] = bk;
  const u32 cw = warp_transpose32(bv, lane);  // bit i: cell (Y + i, X + lane)
  const size_t wj = ((size_t)s * L + X + lane) * T + ty;
  mv.win[wj] = cw;
  mv.first[wj] = cw & v0;
  mv.last[wj] = cw & vl;
  if (lane == 0) work_add(g, 3, 1024);
  if (!__any_sync(FULL, (bw | bv) != 0) && lane == 0) *dflag = 1;
}

// Record accepted candidate `idx` (anchor at position `pos` of line `line`,
// orientation F) with one warp: its node (key, idx, packed anchor), its k
// cells in the occupancy bits of both layouts, their owner ids.
template <int F>
__device__ void lacc_record(const Group& g, u32 s, u32 line, u32 pos, u32* occw, u32* occT,
                            u32 T) {
  const u32 lane = threadIdx.x & 31, L = g.L, k = g.k;
  SampleState& st = g.st[s];
  const u32 y0 = F == 0 ? line : pos, x0 = F == 0 ? pos : line;
  const u32 idx = (u32)((u64)F * g.LL + (u64)y0 * L + x0);
  u32 node = 0;
  if (lane == 0) {
    node = atomicAdd(&st.n_nodes, 1u);
    if (node < g.cap_nodes) {
      const size_t nb = (size_t)s * g.cap_nodes + node;
      g.node_key[nb] = mix64(g.base[s] + SM_GAMMA * ((u64)idx + 1));
      g.node_idx[nb] = idx;
      g.node_pos[nb] = ((u32)F << 31) | (y0 << 15) | x0;
    } else {
      atomicOr(&st.status, ST_NODE_OVF);
    }
  }
  node = __shfl_sync(FULL, node, 0);
  if (node >= g.cap_nodes) return;
  u32* own_line = (F == 0 ? occw : occT) + ((size_t)s * L + line) * T;  // along the k-mer
  u32* cross = (F == 0 ? occT : occw) + (size_t)s * L * T;              // across it
  u32* own = g.owner + (size_t)s * g.LL;
  // the k-mer's cells pos .. pos + k - 1 (around the torus): whole and
  // partial words of its own line
  for (u32 j = lane; j * 32 < k + 32; j += 32) {
    const u32 c0 = pos + 32 * j;  // first cell of this piece (unwrapped)
    if (32 * j >= k) break;
    const u32 n = min(32u, k - 32 * j);
    u32 c = c0 >= L ? c0 - L : c0;
    // up to two words: the cells c .. c + n - 1 starting at bit c & 31
    const u32 b = c & 31u, wi = c >> 5;
    const u64 bits = (n == 32 ? 0xFFFFFFFFull : ((1ull << n) - 1ull)) << b;
    atomicOr(own_line + wi, (u32)bits);
    if (bits >> 32) atomicOr(own_line + (wi + 1 == T ? 0 : wi + 1), (u32)(bits >> 32));
  }
  for (u32 i = lane; i < k; i += 32) {
    u32 c = pos + i;
    if (c >= L) c -= L;
    // the cell is (line, c) along the k-mer: bit `line` of word c's column
    atomicOr(cross + (size_t)c * T + (line >> 5), 1u << (line & 31u));
    if (F == 0) own[(size_t)line * L + c] = node;
    else own[(size_t)c * L + line] = node | OWN_V;
  }
}

// Acceptance along lines from the masks of k_lcomb (F = 0: rows, horizontal
// candidates; F = 1: columns, vertical ones).  One CTA per span of P
// anchors (skipped when k_lwin found no live anchor there).  For the 32
// anchors of a word: "won from its first cell" is the first-mask word,
// "won at its last cell" the last-mask shifted by k - 1 cells, and "every
// cell won by this orientation" holds for the anchors a in an interval: past
// the word's last unwon cell and at least k before the next unwon cell
// after the word.  The accepted candidates (disjoint along the line, at
// most P / k + 1) are recorded one per warp.
template <int F>
__global__ void __launch_bounds__(LW_THREADS) k_lacc(Group g, LwinCfg lc, u32* occw, u32* occT,
                                                     AccMasks am, const u8* lflag) {
  __shared__ u32 mw[3][LW_THREADS + 2];  // win, first, last words from x0
  __shared__ u32 nz[LW_THREADS + 2];     // first unwon cell at / after word i
  __shared__ u32 wmin[LW_THREADS / 32];
  __shared__ u32 acc[LINE_ACC];
  __shared__ u32 nacc;
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, T = lc.T, P = lc.P, nc = lc.nc;
  const u32 line = blockIdx.x / nc, r = blockIdx.x - line * nc;
  if (lflag[((size_t)(s * 2 + F) * L + line) * nc + r] & 1u) return;
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 x0 = r * P;
  // words of [x0, x0 + P + k + 32): the last-mask shift reads one word past
  // the last cell of the last anchor
  const u32 nwords = (P + k) / 32 + 1;  // <= 257
  const size_t lb = ((size_t)s * L + line) * T;
  for (u32 i = tid; i < nwords; i += LW_THREADS) {
    u32 wi = x0 / 32 + i;
    while (wi >= T) wi -= T;
    mw[0][i] = am.win[lb + wi];
    mw[1][i] = am.first[lb + wi];
    mw[2][i] = am.last[lb + wi];
  }
  if (tid == 0) nacc = 0;
  __syncthreads();
  // nz[i] = min over words j >= i of their first unwon cell (words past
  // 255 lie beyond every anchor's last cell)
  u32 fz = LW_INF;
  if (tid < nwords && ~mw[0][tid]) fz = tid * 32 + __ffs(~mw[0][tid]) - 1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u32 o = __shfl_down_sync(FULL, fz, d);
    if (lane + d < 32) fz = min(fz, o);
  }
  if (lane == 0) wmin[warp] = fz;
  __syncthreads();
  for (u32 w2 = warp + 1; w2 < LW_THREADS / 32; ++w2) fz = min(fz, wmin[w2]);
  nz[tid] = fz;
  if (tid == 0) nz[LW_THREADS] = LW_INF;
  __syncthreads();
  if (tid == 0) work_add(g, 2, P);
  for (u32 i = tid; i < P / 32; i += LW_THREADS) {
    const u32 unwon = ~mw[0][i], nxt = nz[i + 1];
    // anchors 32 i + b with b > (last unwon bit of word i) and
    // 32 i + b + k <= nxt
    const int lo = unwon ? (int)(31 - __clz(unwon)) + 1 : 0;
    const int hi = nxt == LW_INF ? 31 : min(31, (int)nxt - (int)k - (int)(32 * i));
    u32 run = 0;
    if (lo <= hi) run = (0xFFFFFFFFu >> (31 - hi)) & (0xFFFFFFFFu << lo);
    const u32 base = 32 * i + k - 1, wq = base >> 5, sh = base & 31u;
    const u32 lastw = sh ? (mw[2][wq] >> sh) | (mw[2][wq + 1] << (32 - sh)) : mw[2][wq];
    u32 acc_bits = run & mw[1][i] & lastw;
    while (acc_bits) {
      const u32 b = __ffs(acc_bits) - 1;
      acc_bits &= acc_bits - 1;
      const u32 slot = atomicAdd(&nacc, 1u);
      if (slot < LINE_ACC) acc[slot] = x0 + 32 * i + b;
    }
  }
  __syncthreads();
  const u32 na = nacc;
  if (na > LINE_ACC) {
    if (tid == 0) atomicOr(&g.st[s].status, ST_NODE_OVF);
    return;
  }
  for (u32 j = warp; j < na; j += LW_THREADS / 32)
    lacc_record<F>(g, s, line, acc[j], occw, occT, T);
}

}  // namespace rsak
