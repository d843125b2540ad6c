// rsa_tile.cuh -- tiled round kernels for power-of-two k <= 32 and L a
// multiple of 32 (sm_103a).
//
// The lattice is cut into 32 x 32 tiles; occupancy is one bit per cell
// (row-major, 32 cells per word), so a tile row is exactly one word and a
// window of k <= 32 cells lies in two adjacent words.  One round is two
// passes over the tiles:
//   k_tile_cmin    per cell, which live candidate covering it has the
//                  smallest priority, as a 1-byte argmin code: the
//                  horizontal part along the tile's rows, the vertical part
//                  along its columns, both width-k window minima of the live
//                  priorities anchored in the tile and the tile before it;
//   k_tile_accept  a live candidate anchored in the tile is accepted iff it
//                  is the argmin on every one of its cells (reaching into the
//                  tiles right of and below it), read from the codes alone.
// Window minima are van Herk / Gil-Werman with blocks of k cells (k divides
// 32, so blocks align with tiles): suffix minima Q of the block before, a
// running prefix minimum P of the next, window = min(Q[i+1], P); O(1) 64-bit
// minima per cell and no shuffles.  For k < 32 one thread walks each live
// line in registers; for k = 32 one thread builds Q and another P of each
// live line in shared memory, and the write-out combines them.
// A tile whose codes are all "none" has no live candidate on any of its
// cells; since live candidates only disappear it stays so, is flagged dead
// and is skipped by every later pass.
#pragma once
#include "rsa_device.cuh"

namespace rsak {

struct TileCfg {
  u32 T;        // tiles per side = L / 32
  u32 T2;       // tiles per sample
  u64 items;    // n * T2
};

template <int K>
__device__ __forceinline__ u64 kmask() {
  return K >= 64 ? ~0ull : ((1ull << K) - 1ull);
}

// Line buffers.  A tile line (a row for horizontal candidates, a column for
// vertical ones) holds the live priorities of the candidates anchored at
// positions p = -31 .. 31 along it (negative = the tile before) at slot
// SLOT(p) = 31 + p; position -32 is in no window of k <= 32 cells that
// reaches the tile.  LN = 63 u64 slots: odd, so 32 threads walking 32 lines
// at the same slot hit distinct banks.  The byte buffers of argmin offsets
// use the same slots with a 68-byte pitch (17 words, also conflict-free).
constexpr int LN = 63;
constexpr int LA = 68;
__host__ __device__ constexpr int SLOT(int p) { return 31 + p; }

constexpr u8 ARG_NONE = 0xFF;

// Backward window minima with argmin, one thread per line, K < 32:
//   ln[SLOT(x)] := min(live priorities anchored at x-K+1 .. x),  x in [0, 32),
//   la[SLOT(x)] := x - (anchor of that minimum), or ARG_NONE if none.
// van Herk / Gil-Werman with K-aligned blocks (K divides 32, so blocks align
// with the tile): suffix minima Q of the previous block in registers, running
// prefix minimum P of the current one, window = min(Q[i+1], P).  In place:
// a slot is read before it is overwritten.
template <int K>
__device__ __forceinline__ void line_bwd_arg(u64* ln, u8* la) {
  constexpr int NB = 32 / K;
  u64 q[K];
  int qa[K];  // slot of the suffix minimum, relative to the block start
  q[0] = KEY_NONE;
  qa[0] = 0;
#pragma unroll
  for (int j = 1; j < K; ++j) { q[j] = ln[SLOT(j - K)]; qa[j] = j; }
#pragma unroll
  for (int j = K - 2; j >= 0; --j)
    if (q[j + 1] < q[j]) { q[j] = q[j + 1]; qa[j] = qa[j + 1]; }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    u64 w[K];
    int wa[K];
    u64 P = KEY_NONE;
    int pa = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const u64 v = ln[SLOT(b * K + i)];
      if (b + 1 < NB) { w[i] = v; wa[i] = i; }
      if (v < P) { P = v; pa = i; }
      u64 out = P;
      int d = i - pa;
      if (i + 1 < K && q[(i + 1) % K] < P) {
        out = q[(i + 1) % K];
        d = i + K - qa[(i + 1) % K];
      }
      ln[SLOT(b * K + i)] = out;
      la[SLOT(b * K + i)] = out == KEY_NONE ? ARG_NONE : (u8)d;
    }
    if (b + 1 < NB) {
#pragma unroll
      for (int j = K - 2; j >= 0; --j)
        if (w[j + 1] < w[j]) { w[j] = w[j + 1]; wa[j] = wa[j + 1]; }
#pragma unroll
      for (int j = 0; j < K; ++j) { q[j] = w[j]; qa[j] = wa[j]; }
    }
  }
}

// Position (0-based rank n < popc(m)) of the n-th set bit of m.
__device__ __forceinline__ u32 nth_set_bit(u32 m, u32 n) {
  u32 pos = 0;
#pragma unroll
  for (u32 w = 16; w; w >>= 1) {
    const u32 lo = __popc(m & ((1u << w) - 1u));
    if (n >= lo) {
      n -= lo;
      m >>= w;
      pos += w;
    }
  }
  return pos;
}

// Asynchronous global -> shared copies (cp.async): a tile's staging loads are
// all in flight together instead of one latency per loop iteration.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ u32 wrap_lo(int v, u32 L) {  // v in [-L, 2L) -> [0, L)
  return (u32)(v < 0 ? v + (int)L : (v >= (int)L ? v - (int)L : v));
}

// Persistent loop over (sample, tile) items without 64-bit division.
struct ItemIter {
  u32 s, t;
  __device__ __forceinline__ ItemIter(u32 start, u32 T2) : s(start / T2), t(start % T2) {}
  __device__ __forceinline__ void next(u32 step, u32 T2) {
    t += step;
    while (t >= T2) { t -= T2; ++s; }
  }
};

constexpr u32 TILE_THREADS = 128;

// Pass 1 of a round.  128 threads per tile, persistent over (sample, tile):
// warps 0-1 take the tile's rows (horizontal candidates), warps 2-3 its
// columns (vertical candidates), 16 lines each.
//  (a) lane-parallel: live priorities of the candidates anchored on each line
//      and the K-1 positions before it into the line buffers lh[row],
//      lv[col]; a line with no live candidate is only marked, not written;
//  (b) a tile with no live line is covered by no live candidate: flagged
//      dead, nothing written;
//  (c) one thread per live line: width-K backward window minima with argmin;
//      for K = 32 one thread builds the suffix minima of the previous block
//      and another the prefix minima of the tile's block, the write-out
//      takes min(Q[x+1], P[x]);
//  (d) argmin code of each cell (horizontal offset d, 32 + d vertical,
//      ARG_NONE if uncovered) written out coalesced, 8 cells per store.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, K >= 16 ? 6 : 5)
    k_tile_cmin(Group g, TileCfg tc, u32* occw, u8* dead) {
  __shared__ u32 ow[96][3];     // occupancy words: rows Y-32 .. Y+63, word columns wx-1 .. wx+1
  __shared__ u64 lh[32][LN];
  __shared__ u64 lv[32][LN];
  // occupancy of each tile column (rows Y-32.., rows Y..): short windows only
  __shared__ u32 colmask[K < 16 ? 32 : 1][2];
  __shared__ u32 live_sh[2];      // per direction: bit r = line r has a live candidate
  __shared__ u8 ah[32][LA];       // argmin offsets of the row lines
  __shared__ u8 av[32][LA];       // argmin offsets of the column lines
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 dirw = warp >> 1, half = warp & 1;
  const u32 L = g.L, T = tc.T, T2 = tc.T2;
  u32 cells_sum = 0, keyed_sum = 0;  // work of this block, added once at the end
  for (ItemIter it(blockIdx.x, T2); it.s < g.n; it.next(gridDim.x, T2)) {
    const u32 s = it.s, t = it.t;
    if (g.st[s].done) continue;
    u8* dflag = dead + (size_t)s * T2 + t;
    if (*dflag) continue;
    const u32 ty = t / T, tx = t - ty * T, Y = ty * 32, X = tx * 32;
    const u32* owg = occw + (size_t)s * L * T;
    for (u32 i = threadIdx.x; i < 96 * 3; i += blockDim.x) {
      const u32 r = i / 3, c = i - r * 3;
      const u32 row = wrap_lo((int)(Y + r) - 32, L);
      const u32 wc = wrap_lo((int)(tx + c) - 1, T);
      cp_async4(&ow[r][c], owg + (size_t)row * T + wc);
    }
    if (threadIdx.x < 2) live_sh[threadIdx.x] = 0;
    cp_async_wait_all();
    __syncthreads();
    // splitmix64 input of candidate idx is zb + gamma * idx
    const u64 zb = g.base[s] + SM_GAMMA;
    const bool caller = g.keys != nullptr;
    u32 live = 0;    // lines of this warp with a live candidate (warp-uniform)
    u32 keyed = 0;   // live candidates this lane gave a key
    const u32 l0 = half * 16;
    if constexpr (K >= 16) {
      // long windows: the K-1 positions before the tile are hashed in the
      // same pass as the tile's own, lane = position (lane - 32 before it)
      const bool need_prev = lane >= 33u - K;
      if (dirw == 0) {
        const u64 zstep = SM_GAMMA * (u64)L;
        u64 zc = zb + SM_GAMMA * ((u64)(Y + l0) * L + X + lane);
        u64 zp = zb + SM_GAMMA * ((u64)(Y + l0) * L + wrap_lo((int)(X + lane) - 32, L));
#pragma unroll 2
        for (u32 r = l0; r < l0 + 16; ++r, zc += zstep, zp += zstep) {
          const u64 A = ((u64)ow[32 + r][1] << 32) | ow[32 + r][0];  // positions -32 .. 31
          const u64 B = ((u64)ow[32 + r][2] << 32) | ow[32 + r][1];  // positions 0 .. 63
          const bool ap = need_prev && ((A >> lane) & kmask<K>()) == 0;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          if (__any_sync(FULL, ap || ac)) {
            u64 hp, hc;
            if (caller) {
              hp = g.keys[(u64)(Y + r) * L + wrap_lo((int)(X + lane) - 32, L)];
              hc = g.keys[(u64)(Y + r) * L + X + lane];
            } else {
              hp = mix64(zp);
              hc = mix64(zc);
            }
            if (need_prev) lh[r][SLOT((int)lane - 32)] = ap ? hp : KEY_NONE;
            lh[r][SLOT(lane)] = ac ? hc : KEY_NONE;
            live |= 1u << r;
            keyed += (u32)ap + (u32)ac;
          }
        }
      } else {
        const u32 bp = ow[lane][1], bc = ow[32 + lane][1], bn = ow[64 + lane][1];
        const u64 rowp = g.LL + (u64)wrap_lo((int)(Y + lane) - 32, L) * L + X;
        const u64 rowc = g.LL + (u64)(Y + lane) * L + X;
        u64 zc = zb + SM_GAMMA * (rowc + l0), zp = zb + SM_GAMMA * (rowp + l0);
#pragma unroll 2
        for (u32 c = l0; c < l0 + 16; ++c, zc += SM_GAMMA, zp += SM_GAMMA) {
          const u32 Mp = __ballot_sync(FULL, (bp >> c) & 1u);
          const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
          const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
          const u64 A = ((u64)Mc << 32) | Mp, B = ((u64)Mn << 32) | Mc;
          const bool ap = need_prev && ((A >> lane) & kmask<K>()) == 0;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          if (__any_sync(FULL, ap || ac)) {
            u64 hp, hc;
            if (caller) {
              hp = g.keys[rowp + c];
              hc = g.keys[rowc + c];
            } else {
              hp = mix64(zp);
              hc = mix64(zc);
            }
            if (need_prev) lv[c][SLOT((int)lane - 32)] = ap ? hp : KEY_NONE;
            lv[c][SLOT(lane)] = ac ? hc : KEY_NONE;
            live |= 1u << c;
            keyed += (u32)ap + (u32)ac;
          }
        }
      }
    } else {
      u64 (*ln)[LN] = dirw == 0 ? lh : lv;
      if (dirw == 0) {
        // tile part of each row, lane = position along the row
        u64 z = zb + SM_GAMMA * ((u64)(Y + l0) * L + X + lane);
        const u64 zstep = SM_GAMMA * (u64)L;
#pragma unroll 2
        for (u32 r = l0; r < l0 + 16; ++r, z += zstep) {
          const u64 B = ((u64)ow[32 + r][2] << 32) | ow[32 + r][1];  // positions 0 .. 63
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          const u32 m = __ballot_sync(FULL, ac);
          u64 vc = KEY_NONE;
          if (m) {
            const u64 h = caller ? g.keys[(u64)(Y + r) * L + X + lane] : mix64(z);
            vc = ac ? h : KEY_NONE;
            live |= 1u << r;
            keyed += (u32)ac;
          }
          lh[r][SLOT(lane)] = vc;
        }
      } else {
        // tile part of each column, lane = position along the column
        const u32 bp = ow[lane][1], bc = ow[32 + lane][1], bn = ow[64 + lane][1];
        u64 z = zb + SM_GAMMA * (g.LL + (u64)(Y + lane) * L + X + l0);
#pragma unroll 2
        for (u32 c = l0; c < l0 + 16; ++c, z += SM_GAMMA) {
          const u32 Mp = __ballot_sync(FULL, (bp >> c) & 1u);
          const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
          const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
          if (lane == 0) { colmask[c][0] = Mp; colmask[c][1] = Mc; }
          const u64 B = ((u64)Mn << 32) | Mc;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          const u32 m = __ballot_sync(FULL, ac);
          u64 vc = KEY_NONE;
          if (m) {
            const u64 h = caller ? g.keys[g.LL + (u64)(Y + lane) * L + X + c] : mix64(z);
            vc = ac ? h : KEY_NONE;
            live |= 1u << c;
            keyed += (u32)ac;
          }
          lv[c][SLOT(lane)] = vc;
        }
      }
      __syncthreads();  // colmask complete
      // short windows: the K-1 positions before the tile on every line,
      // packed densely over lanes (item f = i*32 + lane is line f / (K-1),
      // position -(K-1) + f % (K-1)); the two warps of a direction split
      // the K-1 rounds of items
      constexpr u32 KP = K > 1 ? K - 1 : 1;
#pragma unroll 1
      for (u32 i = half; i + 1 < (u32)K; i += 2) {
        const u32 f = i * 32 + lane, line = f / KP, j = f - line * KP;
        const int pos = (int)j - (int)KP;
        const u64 A = dirw == 0 ? (((u64)ow[32 + line][1] << 32) | ow[32 + line][0])
                                : (((u64)colmask[line][1] << 32) | colmask[line][0]);
        const bool ap = ((A >> (pos + 32)) & kmask<K>()) == 0;
        const u64 idx = dirw == 0 ? (u64)(Y + line) * L + wrap_lo((int)X + pos, L)
                                  : g.LL + (u64)wrap_lo((int)Y + pos, L) * L + X + line;
        u64 v = KEY_NONE;
        if (__any_sync(FULL, ap)) {
          const u64 h = caller ? g.keys[idx] : mix64(zb + SM_GAMMA * idx);
          v = ap ? h : KEY_NONE;
          keyed += (u32)ap;
        }
        ln[line][SLOT(pos)] = v;
        live |= __reduce_or_sync(FULL, ap ? 1u << line : 0u);
      }
    }
    if (lane == 0 && live) atomicOr(&live_sh[dirw], live);
    __syncthreads();
    const u32 lhb = live_sh[0], lvb = live_sh[1];
    keyed_sum += __reduce_add_sync(FULL, keyed);
    if ((lhb | lvb) == 0) {
      // no live candidate on or before any line: every cell is uncovered
      if (threadIdx.x == 0) *dflag = 1;
      __syncthreads();
      continue;
    }
    if constexpr (K == 32) {
      // live lines of both directions, numbered densely (rows first);
      // thread t < 64 builds line t's suffix minima Q of the previous block
      // (positions -31 .. -1, Q at SLOT(j - 32) = min over j .. 31, with its
      // argmin j), thread 64 + t its prefix minima P of the tile's block
      const u32 nh = __popc(lhb), nl = nh + __popc(lvb);
      const u32 tt = threadIdx.x & 63;
      if (tt < nl) {
        const bool vert = tt >= nh;
        const u32 line = vert ? nth_set_bit(lvb, tt - nh) : nth_set_bit(lhb, tt);
        u64* ln = vert ? lv[line] : lh[line];
        u8* la = vert ? av[line] : ah[line];
        if (threadIdx.x < 64) {
          u64 q = KEY_NONE;
          int qa = 0;
#pragma unroll 8
          for (int j = 31; j >= 1; --j) {
            const u64 v = ln[SLOT(j - 32)];
            if (v < q) { q = v; qa = j; }
            ln[SLOT(j - 32)] = q;
            la[SLOT(j - 32)] = (u8)qa;
          }
        } else {
          u64 P = KEY_NONE;
          int pa = 0;
#pragma unroll 8
          for (int i = 0; i < 32; ++i) {
            const u64 v = ln[SLOT(i)];
            if (v < P) { P = v; pa = i; }
            ln[SLOT(i)] = P;
            la[SLOT(i)] = (u8)pa;
          }
        }
      }
    } else if (threadIdx.x < 64) {
      const u32 d = threadIdx.x >> 5;
      if ((d == 0 ? lhb : lvb) >> lane & 1u)
        line_bwd_arg<K>((d == 0 ? lh : lv)[lane], (d == 0 ? ah : av)[lane]);
    }
    __syncthreads();
    // argmin code of every cell: offset d of the winning horizontal
    // candidate (0 .. K-1), 32 + d for a vertical one, ARG_NONE if no live
    // candidate covers the cell; 8 cells per thread, one 8-byte store.  Only
    // live lines are read.
    bool any = false;
    u8* cdg = reinterpret_cast<u8*>(g.cmin) + (size_t)s * g.LL;
    {
      const u32 y = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * 8;
      const bool hl = (lhb >> y) & 1u;
      const u32 vm = (lvb >> c0) & 0xFFu;
      u64 pack = ~0ull;
      if (hl || vm) {
        pack = 0;
#pragma unroll
        for (u32 c = c0; c < c0 + 8; ++c) {
          u64 vh = KEY_NONE, vv = KEY_NONE;
          u32 dh = 0, dv = 0;
          if (hl) {
            vh = lh[y][SLOT(c)];
            if constexpr (K == 32) {
              // window of cell c on row y: Q at position c+1-32 vs P[c]
              dh = c - ah[y][SLOT(c)];
              if (c < 31) {
                const u64 q = lh[y][SLOT((int)c - 31)];
                if (q < vh) { vh = q; dh = c + 32 - ah[y][SLOT((int)c - 31)]; }
              }
            } else {
              dh = ah[y][SLOT(c)];
            }
          }
          if ((vm >> (c - c0)) & 1u) {
            vv = lv[c][SLOT(y)];
            if constexpr (K == 32) {
              dv = y - av[c][SLOT(y)];
              if (y < 31) {
                const u64 q = lv[c][SLOT((int)y - 31)];
                if (q < vv) { vv = q; dv = y + 32 - av[c][SLOT((int)y - 31)]; }
              }
            } else {
              dv = av[c][SLOT(y)];
            }
          }
          u32 code = ARG_NONE;
          if (vh < vv) code = dh;
          else if (vv < vh) code = 32u + dv;
          pack |= (u64)code << (8 * (c - c0));
          any |= code != ARG_NONE;
        }
      }
      *reinterpret_cast<u64*>(cdg + (size_t)(Y + y) * L + X + c0) = pack;
    }
    const bool tile_live = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      cells_sum += 1024;
      if (!tile_live) *dflag = 1;
      else if (!g.st[s].alive) g.st[s].alive = 1;
    }
  }
  if (threadIdx.x == 0 && cells_sum) work_add(g, 0, cells_sum);
  if (lane == 0 && keyed_sum) work_add(g, 1, keyed_sum);
}

// Pass 2 of a round: acceptance of candidates anchored in each live tile.
// A live candidate has the smallest key on all of its cells iff each of its
// cells carries its argmin code: a horizontal candidate at x is accepted iff
// code(x + i) = i for i < K, a vertical one iff code(y + i) = 32 + i.  With
// S = "code is the start value" and INC = "the next cell's code is this
// code + 1" as bit masks along a line (ballots), that is S(x) and
// INC(x .. x+K-2).  No priority is needed except for the accepted ones.
//  (a) stage the codes of the tile, the tile to the right (rows) and the
//      tile below (columns); a dead neighbour reads as ARG_NONE;
//  Sixteen 128-thread blocks per SM (32 registers): the pass is latency-bound
//  on its staging and ballots, and full occupancy hides that best (measured
//  3.7% faster for the whole L=1024, k=32 run than twelve blocks at 40).
//  (b) warps 0-1 take 16 rows each, warps 2-3 16 columns each; the accepted
//      candidates of a line (disjoint k-mers) get consecutive nodes from one
//      atomic, each accepting lane records its own node, the union of their
//      cells is OR-ed into the occupancy words once per line, and the owner
//      ids of each accepted k-mer's cells are one warp-wide store.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, 16) k_tile_accept(Group g, TileCfg tc, u32* occw,
                                                              const u8* dead) {
  __shared__ __align__(16) u8 hc[32][80];   // row y: codes of columns X .. X+63 (+ slack)
  __shared__ __align__(16) u8 vc[65][36];   // row j: codes of rows Y .. Y+63, columns X .. X+31
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 dirw = warp >> 1, half = warp & 1;
  const u32 L = g.L, T = tc.T, T2 = tc.T2;
  u32 cells_sum = 0, accepted_sum = 0;  // work of this block, added once at the end
  for (ItemIter it(blockIdx.x, T2); it.s < g.n; it.next(gridDim.x, T2)) {
    const u32 s = it.s, t = it.t;
    if (g.st[s].done) continue;
    const u8* dflag = dead + (size_t)s * T2;
    if (dflag[t]) continue;
    const u32 ty = t / T, tx = t - ty * T, Y = ty * 32, X = tx * 32;
    const u32 txr = tx + 1 == T ? 0 : tx + 1, tyb = ty + 1 == T ? 0 : ty + 1;
    const bool dr = dflag[ty * T + txr] != 0, db = dflag[tyb * T + tx] != 0;
    const u8* cdg = reinterpret_cast<const u8*>(g.cmin) + (size_t)s * g.LL;
    // row lines: 16-byte chunks of the own tile and the tile to the right
    for (u32 i = threadIdx.x; i < 128; i += blockDim.x) {
      const u32 part = i >> 6, r = (i >> 1) & 31, hlf = i & 1;
      u8* dst = &hc[r][part * 32 + hlf * 16];
      if (part == 1 && dr)
        *reinterpret_cast<uint4*>(dst) = make_uint4(~0u, ~0u, ~0u, ~0u);
      else
        cp_async16(dst, cdg + (size_t)(Y + r) * L + (part ? txr * 32 : X) + hlf * 16);
    }
    // column lines (rows of the own tile and the tile below): 4-byte words
    // into a 36-byte row pitch, which keeps the per-column reads conflict-free
    for (u32 i = threadIdx.x; i < 512; i += blockDim.x) {
      const u32 r = i >> 3, wd = i & 7;
      u8* dst = &vc[r][wd * 4];
      if (r >= 32 && db)
        *reinterpret_cast<u32*>(dst) = ~0u;
      else
        cp_async4(dst, cdg + (size_t)(r < 32 ? Y + r : tyb * 32 + r - 32) * L + X + wd * 4);
    }
    if (threadIdx.x < 32) {
      hc[threadIdx.x][64] = ARG_NONE;
      vc[64][threadIdx.x] = ARG_NONE;
    }
    cp_async_wait_all();
    __syncthreads();
    const u64 zb = g.base[s] + SM_GAMMA;
    const bool caller = g.keys != nullptr;
    constexpr u64 KM1 = K > 1 ? ((1ull << (K - 1)) - 1ull) : 0ull;  // INC bits a window needs
    const u32 l0 = half * 16;
    SampleState& st = g.st[s];
    u32* ows = occw + (size_t)s * L * T;
    u32* own = g.owner + (size_t)s * g.LL;
    const size_t nbase = (size_t)s * g.cap_nodes;
    u32 accepted = 0;
    for (u32 line = l0; line < l0 + 16; ++line) {
      u32 c0, c1, c2, c3;
      if (dirw == 0) {
        c0 = hc[line][lane];
        c1 = hc[line][lane + 1];
        c2 = hc[line][32 + lane];
        c3 = hc[line][33 + lane];
      } else {
        c0 = vc[lane][line];
        c1 = vc[lane + 1][line];
        c2 = vc[32 + lane][line];
        c3 = vc[33 + lane][line];
      }
      const u32 base = dirw == 0 ? 0u : 32u;   // code of offset 0
      const u32 top = base + 31u;
      const u32 S = __ballot_sync(FULL, c0 == base);
      if (!S) continue;
      const u64 inc = (u64)__ballot_sync(FULL, c0 >= base && c0 < top && c1 == c0 + 1) |
                      ((u64)__ballot_sync(FULL, c2 >= base && c2 < top && c3 == c2 + 1) << 32);
      const bool acc = ((S >> lane) & 1u) && ((inc >> lane) & KM1) == KM1;
      const u32 m = __ballot_sync(FULL, acc);
      if (!m) continue;
      // nodes for the line's accepted candidates (disjoint k-mers), in lane
      // order from one atomic; each accepting lane records its own
      u32 nb = 0;
      if (lane == 0) nb = atomicAdd(&st.n_nodes, (u32)__popc(m));
      nb = __shfl_sync(FULL, nb, 0);
      if (acc) {
        const u32 node = nb + __popc(m & ((1u << lane) - 1u));
        const u32 y0 = dirw == 0 ? Y + line : Y + lane, x0 = dirw == 0 ? X + lane : X + line;
        const u64 idx = (u64)dirw * g.LL + (u64)y0 * L + x0;
        if (node < g.cap_nodes) {
          g.node_key[nbase + node] = caller ? g.keys[idx] : mix64(zb + SM_GAMMA * idx);
          g.node_idx[nbase + node] = (u32)idx;
          g.node_pos[nbase + node] = (dirw << 31) | (y0 << 15) | x0;
        } else {
          atomicOr(&st.status, ST_NODE_OVF);
        }
      }
      // occupancy: the union of their cells along the line, positions
      // 0 .. 63 from the tile's first row / column, OR-ed in once
      u64 cov = 0;
      for (u32 mm = m; mm; mm &= mm - 1) cov |= kmask<K>() << (__ffs(mm) - 1);
      if (dirw == 0) {
        u32* w = ows + (size_t)(Y + line) * T;
        if (lane == 0) atomicOr(w + tx, (u32)cov);
        if (lane == 1 && (cov >> 32)) atomicOr(w + txr, (u32)(cov >> 32));
      } else {
        const u32 bit = 1u << line;  // column X + line is bit `line` of word tx
        if ((cov >> lane) & 1u) atomicOr(ows + (size_t)(Y + lane) * T + tx, bit);
        if ((cov >> (32 + lane)) & 1u) atomicOr(ows + (size_t)(tyb * 32 + lane) * T + tx, bit);
      }
      // owner ids: one warp-wide store per accepted k-mer (a row run, or a
      // column run whose neighbours the same pass writes soon after)
      for (u32 mm = m; mm; mm &= mm - 1) {
        const u32 src = __ffs(mm) - 1;
        const u32 node = nb + __popc(m & ((1u << src) - 1u));
        if (node < g.cap_nodes && lane < (u32)K) {
          if (dirw == 0)
            own[(size_t)(Y + line) * L + wrap_lo((int)(X + src + lane), L)] = node;
          else
            own[(size_t)wrap_lo((int)(Y + src + lane), L) * L + X + line] = node | OWN_V;
        }
      }
      accepted += __popc(m);
    }
    accepted_sum += accepted;
    cells_sum += 1024;
    __syncthreads();
  }
  if (threadIdx.x == 0 && cells_sum) work_add(g, 2, cells_sum);
  if (lane == 0 && accepted_sum) work_add(g, 3, accepted_sum);
}

}  // namespace rsak
