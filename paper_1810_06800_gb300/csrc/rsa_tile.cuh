// rsa_tile.cuh -- tiled round kernels for power-of-two k <= 32 and L a
// multiple of 32 (sm_103a).
//
// The lattice is cut into 32 x 32 tiles; occupancy is one bit per cell
// (row-major, 32 cells per word), so a tile row is exactly one word and a
// window of k <= 32 cells lies in two adjacent words.  One round is two
// passes over the tiles:
//   k_tile_cmin    cmin(cell) = min over live candidates covering the cell,
//                  horizontal part along the tile's rows, vertical part along
//                  its columns, both as width-k window minima of the live
//                  priorities anchored in the tile and the tile before it;
//   k_tile_accept  a live candidate anchored in the tile is accepted iff the
//                  width-k window minimum of cmin over its cells (reaching
//                  into the tiles right of and below it) equals its key.
// Each thread owns one line of a tile (a row for horizontal candidates, a
// column for vertical ones) and computes its width-k window minima
// sequentially in registers with van Herk / Gil-Werman blocks of k cells
// (k divides 32, so blocks align with tiles): suffix minima Q of one block,
// a running prefix minimum P of the next, window = min(Q[i+1], P).  That is
// O(1) 64-bit minima per cell and no shuffles.
// A tile whose cmin is all "none" has no live candidate on any of its cells;
// since live candidates only disappear it stays so, is flagged dead and is
// skipped by every later pass.
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

// Backward window along one line held in shared memory, one thread:
//   ln[32 + x] := min(ln[32 + x - K + 1 .. 32 + x])   for x in [0, 32),
// the line holding positions -32 .. 31 at ln[0 .. 63] (negative positions =
// the tile before).  van Herk / Gil-Werman with K-aligned blocks: suffix
// minima Q of the previous block in registers, running prefix minimum P of
// the current one, window = min(Q[i+1], P).  In place: position p is read
// before it is overwritten.
template <int K>
__device__ __forceinline__ void line_bwd(u64* ln) {
  constexpr int NB = 32 / K;
  u64 q[K];
  q[0] = KEY_NONE;
#pragma unroll
  for (int j = 1; j < K; ++j) q[j] = ln[32 - K + j];
#pragma unroll
  for (int j = K - 2; j >= 0; --j) q[j] = tmin(q[j], q[j + 1]);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    u64 w[K];
    u64 P = KEY_NONE;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const u64 v = ln[32 + b * K + i];
      if (b + 1 < NB) w[i] = v;
      P = tmin(P, v);
      ln[32 + b * K + i] = (i + 1 < K) ? tmin(q[(i + 1) % K], P) : P;
    }
    if (b + 1 < NB) {
#pragma unroll
      for (int j = K - 2; j >= 0; --j) w[j] = tmin(w[j], w[j + 1]);
#pragma unroll
      for (int j = 0; j < K; ++j) q[j] = w[j];
    }
  }
}

// Forward window along one line in shared memory, one thread:
//   ln[x] := min(ln[x .. x + K - 1])   for x in [0, 32),  ln[0 .. 32+K-2] valid.
// Suffix minima Q of block b, running prefix minimum of block b+1.  In place.
template <int K>
__device__ __forceinline__ void line_fwd(u64* ln) {
  constexpr int NB = 32 / K;
  u64 q[K];
#pragma unroll
  for (int j = 0; j < K; ++j) q[j] = ln[j];
#pragma unroll
  for (int j = K - 2; j >= 0; --j) q[j] = tmin(q[j], q[j + 1]);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    u64 w[K];
    u64 P = KEY_NONE;
    ln[b * K] = q[0];
#pragma unroll
    for (int i = 0; i + 1 < K; ++i) {
      const u64 v = ln[(b + 1) * K + i];
      if (b + 1 < NB) w[i] = v;
      P = tmin(P, v);
      ln[b * K + i + 1] = tmin(q[(i + 1) % K], P);
    }
    if (b + 1 < NB) {
      w[K - 1] = ln[(b + 1) * K + K - 1];
#pragma unroll
      for (int j = K - 2; j >= 0; --j) w[j] = tmin(w[j], w[j + 1]);
#pragma unroll
      for (int j = 0; j < K; ++j) q[j] = w[j];
    }
  }
}

constexpr int LN = 65;  // padded line length (u64) of the tile line buffers

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

// Accept one candidate with the whole warp (k <= 32): lane i writes cell i.
// idx and key are warp-uniform.
__device__ __forceinline__ void accept_warp(const Group& g, u32* occw, u32 T, u32 s, u32 idx,
                                            u64 key) {
  const u32 lane = threadIdx.x & 31;
  SampleState& st = g.st[s];
  u32 node = 0;
  if (lane == 0) node = atomicAdd(&st.n_nodes, 1u);
  node = __shfl_sync(FULL, node, 0);
  if (node >= g.cap_nodes) {
    if (lane == 0) atomicOr(&st.status, ST_NODE_OVF);
    return;
  }
  const u32 L = g.L, k = g.k;
  const u32 o = idx / (u32)g.LL, r = idx - o * (u32)g.LL;
  const u32 y0 = r / L, x0 = r - y0 * L;
  if (lane == 0) {
    g.node_key[(size_t)s * g.cap_nodes + node] = key;
    g.node_idx[(size_t)s * g.cap_nodes + node] = idx;
    g.node_pos[(size_t)s * g.cap_nodes + node] = (o << 31) | (y0 << 15) | x0;
  }
  u32* ow = occw + (size_t)s * L * T;
  u32* own = g.owner + (size_t)s * g.LL;
  if (o == 0) {
    const u32 b = x0 & 31u, w = x0 >> 5;
    const u64 m = (k >= 64 ? ~0ull : ((1ull << k) - 1ull)) << b;
    if (lane == 0) atomicOr(ow + (size_t)y0 * T + w, (u32)m);
    if (lane == 1 && (m >> 32)) atomicOr(ow + (size_t)y0 * T + (w + 1 == T ? 0 : w + 1), (u32)(m >> 32));
    if (lane < k) own[(size_t)y0 * L + wrap_lo((int)(x0 + lane), L)] = node;
  } else if (lane < k) {
    const u32 y = wrap_lo((int)(y0 + lane), L);
    atomicOr(ow + (size_t)y * T + (x0 >> 5), 1u << (x0 & 31u));
    own[(size_t)y * L + x0] = node;
  }
}

// Pass 1 of a round.  64 threads per tile, persistent over (sample, tile).
//  (a) lane-parallel: live priorities of the horizontal candidates anchored
//      in each tile row (and the K-1 before it) and of the vertical ones of
//      each tile column, into line buffers lh[row][.], lv[col][.];
//  (b) one thread per line: width-K backward window minima, in place;
//  (c) cmin(y, x) = min(lh[y][32+x], lv[x][32+y]) written out coalesced.
template <int K>
__global__ void __launch_bounds__(64) k_tile_cmin(Group g, TileCfg tc, u32* occw, u8* dead) {
  __shared__ u32 ow[96][3];     // occupancy words: rows Y-32 .. Y+63, word columns wx-1 .. wx+1
  __shared__ u64 lh[32][LN];    // row lines, positions -32 .. 31
  __shared__ u64 lv[32][LN];    // column lines, positions -32 .. 31
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 L = g.L, T = tc.T, T2 = tc.T2;
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
    cp_async_wait_all();
    __syncthreads();
    // splitmix64 input of candidate idx is zb + gamma * idx
    const u64 zb = g.base[s] + SM_GAMMA;
    const bool caller = g.keys != nullptr;
    u64 (*ln)[LN] = warp == 0 ? lh : lv;
    u32 live = 0;          // bit r: line r has a live candidate (warp-uniform)
    u32 keyed = 0;         // live candidates given a key (warp-uniform)
    if (K >= 16) {
      // long windows: the K-1 positions before the tile are hashed in the
      // same pass as the tile's own, lane = position (slot lane = position
      // lane - 32, slot 32 + lane = position lane)
      const bool need_prev = lane >= 33u - K;
      if (warp == 0) {
        const u64 zstep = SM_GAMMA * (u64)L;
        u64 zc = zb + SM_GAMMA * ((u64)Y * L + X + lane);
        u64 zp = zb + SM_GAMMA * ((u64)Y * L + wrap_lo((int)(X + lane) - 32, L));
#pragma unroll 2
        for (u32 r = 0; r < 32; ++r, zc += zstep, zp += zstep) {
          const u64 A = ((u64)ow[32 + r][1] << 32) | ow[32 + r][0];  // positions -32 .. 31
          const u64 B = ((u64)ow[32 + r][2] << 32) | ow[32 + r][1];  // positions 0 .. 63
          const bool ap = need_prev && ((A >> lane) & kmask<K>()) == 0;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          u64 vp = KEY_NONE, vc = KEY_NONE;
          if (__any_sync(FULL, ap || ac)) {
            u64 hp, hc;
            if (caller) {
              hp = g.keys[(u64)(Y + r) * L + wrap_lo((int)(X + lane) - 32, L)];
              hc = g.keys[(u64)(Y + r) * L + X + lane];
            } else {
              hp = mix64(zp);
              hc = mix64(zc);
            }
            vp = ap ? hp : KEY_NONE;
            vc = ac ? hc : KEY_NONE;
            live |= 1u << r;
            keyed += __popc(__ballot_sync(FULL, ap)) + __popc(__ballot_sync(FULL, ac));
          }
          lh[r][lane] = vp;
          lh[r][32 + lane] = vc;
        }
      } else {
        const u32 bp = ow[lane][1], bc = ow[32 + lane][1], bn = ow[64 + lane][1];
        const u64 rowp = g.LL + (u64)wrap_lo((int)(Y + lane) - 32, L) * L + X;
        const u64 rowc = g.LL + (u64)(Y + lane) * L + X;
        u64 zc = zb + SM_GAMMA * rowc, zp = zb + SM_GAMMA * rowp;
#pragma unroll 2
        for (u32 c = 0; c < 32; ++c, zc += SM_GAMMA, zp += SM_GAMMA) {
          const u32 Mp = __ballot_sync(FULL, (bp >> c) & 1u);
          const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
          const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
          const u64 A = ((u64)Mc << 32) | Mp, B = ((u64)Mn << 32) | Mc;
          const bool ap = need_prev && ((A >> lane) & kmask<K>()) == 0;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          u64 vp = KEY_NONE, vc = KEY_NONE;
          if (__any_sync(FULL, ap || ac)) {
            u64 hp, hc;
            if (caller) {
              hp = g.keys[rowp + c];
              hc = g.keys[rowc + c];
            } else {
              hp = mix64(zp);
              hc = mix64(zc);
            }
            vp = ap ? hp : KEY_NONE;
            vc = ac ? hc : KEY_NONE;
            live |= 1u << c;
            keyed += __popc(__ballot_sync(FULL, ap)) + __popc(__ballot_sync(FULL, ac));
          }
          lv[c][lane] = vp;
          lv[c][32 + lane] = vc;
        }
      }
    } else {
      u32 cp = 0, cc = 0;    // vertical warp: occupancy of column `lane`, rows Y-32.. / Y..
      if (warp == 0) {
        // tile part of each row, lane = position along the row
        u64 z = zb + SM_GAMMA * ((u64)Y * L + X + lane);
        const u64 zstep = SM_GAMMA * (u64)L;
#pragma unroll 2
        for (u32 r = 0; r < 32; ++r, z += zstep) {
          const u64 B = ((u64)ow[32 + r][2] << 32) | ow[32 + r][1];  // positions 0 .. 63
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          const u32 m = __ballot_sync(FULL, ac);
          u64 vc = KEY_NONE;
          if (m) {
            const u64 h = caller ? g.keys[(u64)(Y + r) * L + X + lane] : mix64(z);
            vc = ac ? h : KEY_NONE;
            live |= 1u << r;
            keyed += __popc(m);
          }
          lh[r][32 + lane] = vc;
        }
      } else {
        // tile part of each column, lane = position along the column
        const u32 bp = ow[lane][1], bc = ow[32 + lane][1], bn = ow[64 + lane][1];
        u64 z = zb + SM_GAMMA * (g.LL + (u64)(Y + lane) * L + X);
#pragma unroll 2
        for (u32 c = 0; c < 32; ++c, z += SM_GAMMA) {
          const u32 Mp = __ballot_sync(FULL, (bp >> c) & 1u);
          const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
          const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
          if (lane == c) { cp = Mp; cc = Mc; }
          const u64 B = ((u64)Mn << 32) | Mc;
          const bool ac = ((B >> lane) & kmask<K>()) == 0;
          const u32 m = __ballot_sync(FULL, ac);
          u64 vc = KEY_NONE;
          if (m) {
            const u64 h = caller ? g.keys[g.LL + (u64)(Y + lane) * L + X + c] : mix64(z);
            vc = ac ? h : KEY_NONE;
            live |= 1u << c;
            keyed += __popc(m);
          }
          lv[c][32 + lane] = vc;
        }
      }
      // short windows: the K-1 positions before the tile on every line,
      // packed densely over lanes: item f = i*32 + lane is line f / (K-1),
      // position -(K-1) + f % (K-1)
      constexpr u32 KP = K > 1 ? K - 1 : 1;
#pragma unroll 1
      for (u32 i = 0; i + 1 < (u32)K; ++i) {
        const u32 f = i * 32 + lane, line = f / KP, j = f - line * KP;
        const int pos = (int)j - (int)KP;
        u64 A;
        if (warp == 0) {
          A = ((u64)ow[32 + line][1] << 32) | ow[32 + line][0];  // positions -32 .. 31
        } else {
          const u32 lp = __shfl_sync(FULL, cp, line), lc = __shfl_sync(FULL, cc, line);
          A = ((u64)lc << 32) | lp;
        }
        const bool ap = ((A >> (pos + 32)) & kmask<K>()) == 0;
        const u64 idx = warp == 0 ? (u64)(Y + line) * L + wrap_lo((int)X + pos, L)
                                  : g.LL + (u64)wrap_lo((int)Y + pos, L) * L + X + line;
        u64 v = KEY_NONE;
        if (__any_sync(FULL, ap)) {
          const u64 h = caller ? g.keys[idx] : mix64(zb + SM_GAMMA * idx);
          v = ap ? h : KEY_NONE;
        }
        ln[line][32 + pos] = v;
        live |= __reduce_or_sync(FULL, ap ? 1u << line : 0u);
        keyed += __popc(__ballot_sync(FULL, ap));
      }
    }
    __syncthreads();
    {
      u64* mine_ln = ln[lane];
      if ((live >> lane) & 1u) {
        line_bwd<K>(mine_ln);
      } else {
#pragma unroll 8
        for (int x = 0; x < 32; ++x) mine_ln[32 + x] = KEY_NONE;
      }
    }
    __syncthreads();
    bool any = false;
    u64* cmg = g.cmin + (size_t)s * g.LL;
#pragma unroll 4
    for (u32 i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
      const u32 y = i >> 5, c = i & 31;
      const u64 v = tmin(lh[y][32 + c], lv[c][32 + y]);
      cmg[(size_t)(Y + y) * L + X + c] = v;
      any |= v != KEY_NONE;
    }
    const bool tile_live = __syncthreads_or(any);
    if (lane == 0 && keyed) atomicAdd(g.work + 1, (u64)keyed);
    if (threadIdx.x == 0) {
      atomicAdd(g.work + 0, 1024ull);
      if (!tile_live) *dflag = 1;
      else if (!g.st[s].alive) g.st[s].alive = 1;
    }
  }
}

// Pass 2 of a round: acceptance of candidates anchored in each live tile.
//  (a) stage cmin: row lines (own tile + the tile to the right) and column
//      lines (own tile + the tile below); a dead neighbour reads as "none";
//  (b) one thread per line: width-K forward window minima, in place;
//  (c) lane-parallel: a live candidate whose window minimum equals its key
//      is accepted; accepted candidates are written by the whole warp.
template <int K>
__global__ void __launch_bounds__(64) k_tile_accept(Group g, TileCfg tc, u32* occw,
                                                    const u8* dead) {
  __shared__ u32 ow[64][2];     // occupancy words rows Y .. Y+63, word columns wx, wx+1
  __shared__ u64 lh[32][LN];    // row lines: columns X .. X+63
  __shared__ u64 lv[32][LN];    // column lines: rows Y .. Y+63
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 L = g.L, T = tc.T, T2 = tc.T2;
  for (ItemIter it(blockIdx.x, T2); it.s < g.n; it.next(gridDim.x, T2)) {
    const u32 s = it.s, t = it.t;
    if (g.st[s].done) continue;
    const u8* dflag = dead + (size_t)s * T2;
    if (dflag[t]) continue;
    const u32 ty = t / T, tx = t - ty * T, Y = ty * 32, X = tx * 32;
    const u32 txr = tx + 1 == T ? 0 : tx + 1, tyb = ty + 1 == T ? 0 : ty + 1;
    const bool dr = dflag[ty * T + txr] != 0, db = dflag[tyb * T + tx] != 0;
    const u64* cmg = g.cmin + (size_t)s * g.LL;
    const u32* owg = occw + (size_t)s * L * T;
    for (u32 i = threadIdx.x; i < 64 * 2; i += blockDim.x) {
      const u32 r = i >> 1, c = i & 1;
      cp_async4(&ow[r][c], owg + (size_t)wrap_lo((int)(Y + r), L) * T + (c ? txr : tx));
    }
#pragma unroll 4
    for (u32 i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
      const u32 r = i >> 5, c = i & 31;
      const u64* own = cmg + (size_t)(Y + r) * L + X + c;
      cp_async8(&lh[r][c], own);
      cp_async8(&lv[c][r], own);
      if (dr) lh[r][32 + c] = KEY_NONE;
      else cp_async8(&lh[r][32 + c], cmg + (size_t)(Y + r) * L + txr * 32 + c);
      if (db) lv[c][32 + r] = KEY_NONE;
      else cp_async8(&lv[c][32 + r], cmg + (size_t)(tyb * 32 + r) * L + X + c);
    }
    cp_async_wait_all();
    __syncthreads();
    if (warp == 0) line_fwd<K>(lh[lane]);
    else line_fwd<K>(lv[lane]);
    __syncthreads();
    const u64 zb = g.base[s] + SM_GAMMA;
    const bool caller = g.keys != nullptr;
    u32 keyed = 0;
    if (warp == 0) {
      u64 z = zb + SM_GAMMA * ((u64)Y * L + X + lane);
      const u64 zstep = SM_GAMMA * (u64)L;
#pragma unroll 2
      for (u32 r = 0; r < 32; ++r, z += zstep) {
        const u64 f = lh[r][lane];
        const u64 B = ((u64)ow[r][1] << 32) | ow[r][0];
        const bool cand = f != KEY_NONE && ((B >> lane) & kmask<K>()) == 0;
        if (__any_sync(FULL, cand)) {
          const u64 idx = (u64)(Y + r) * L + X + lane;
          const u64 key = caller ? g.keys[idx] : mix64(z);
          keyed += __popc(__ballot_sync(FULL, cand));
          u32 m = __ballot_sync(FULL, cand && f == key);
          while (m) {
            const u32 src = __ffs(m) - 1;
            m &= m - 1;
            accept_warp(g, occw, T, s, (u32)__shfl_sync(FULL, idx, src), __shfl_sync(FULL, f, src));
          }
        }
      }
    } else {
      const u32 bc = ow[lane][0], bn = ow[32 + lane][0];
      const u64 rowc = g.LL + (u64)(Y + lane) * L + X;
      u64 z = zb + SM_GAMMA * rowc;
#pragma unroll 2
      for (u32 c = 0; c < 32; ++c, z += SM_GAMMA) {
        const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
        const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
        const u64 B = ((u64)Mn << 32) | Mc;
        const u64 f = lv[c][lane];
        const bool cand = f != KEY_NONE && ((B >> lane) & kmask<K>()) == 0;
        if (__any_sync(FULL, cand)) {
          const u64 idx = rowc + c;
          const u64 key = caller ? g.keys[idx] : mix64(z);
          keyed += __popc(__ballot_sync(FULL, cand));
          u32 m = __ballot_sync(FULL, cand && f == key);
          while (m) {
            const u32 src = __ffs(m) - 1;
            m &= m - 1;
            accept_warp(g, occw, T, s, (u32)__shfl_sync(FULL, idx, src), __shfl_sync(FULL, f, src));
          }
        }
      }
    }
    if (lane == 0 && keyed) atomicAdd(g.work + 3, (u64)keyed);
    if (threadIdx.x == 0) atomicAdd(g.work + 2, 1024ull);
    __syncthreads();
  }
}

}  // namespace rsak
