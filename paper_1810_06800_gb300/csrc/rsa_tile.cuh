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

// Occupy the k cells of an accepted candidate in the bit lattice, record
// its node.
__device__ __forceinline__ void accept_bits(const Group& g, u32* occw, u32 T, u32 s, u32 idx,
                                            u64 key) {
  SampleState& st = g.st[s];
  const u32 node = atomicAdd(&st.n_nodes, 1u);
  if (node >= g.cap_nodes) { atomicOr(&st.status, ST_NODE_OVF); return; }
  g.node_key[(size_t)s * g.cap_nodes + node] = key;
  g.node_idx[(size_t)s * g.cap_nodes + node] = idx;
  const u32 L = g.L, k = g.k;
  const u32 o = idx / (u32)g.LL, r = idx % (u32)g.LL;
  const u32 y0 = r / L, x0 = r % L;
  g.node_pos[(size_t)s * g.cap_nodes + node] = (o << 31) | (y0 << 15) | x0;
  u32* ow = occw + (size_t)s * L * T;
  u32* own = g.owner + (size_t)s * g.LL;
  if (o == 0) {
    const u32 b = x0 & 31u, w = x0 >> 5;
    const u64 m = (k >= 64 ? ~0ull : ((1ull << k) - 1ull)) << b;
    atomicOr(ow + (size_t)y0 * T + w, (u32)m);
    if (m >> 32) atomicOr(ow + (size_t)y0 * T + (w + 1 == T ? 0 : w + 1), (u32)(m >> 32));
    u32 x = x0;
    for (u32 i = 0; i < k; ++i) {
      own[(size_t)y0 * L + x] = node;
      if (++x == L) x = 0;
    }
  } else {
    const u32 bit = 1u << (x0 & 31u), w = x0 >> 5;
    u32 y = y0;
    for (u32 i = 0; i < k; ++i) {
      atomicOr(ow + (size_t)y * T + w, bit);
      own[(size_t)y * L + x0] = node;
      if (++y == L) y = 0;
    }
  }
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

__device__ __forceinline__ u64 key_of(const Group& g, u64 base, u64 idx) {
  if (g.keys) return g.keys[idx];
  return mix64(base + SM_GAMMA * (idx + 1));
}

constexpr int LN = 65;  // padded line length (u64) of the tile line buffers

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
  const u32 L = g.L, T = tc.T;
  for (u64 item = blockIdx.x; item < tc.items; item += gridDim.x) {
    const u32 s = (u32)(item / tc.T2), t = (u32)(item % tc.T2);
    if (g.st[s].done) continue;
    u8* dflag = dead + (size_t)s * tc.T2 + t;
    if (*dflag) continue;
    const u32 ty = t / T, tx = t % T, Y = ty * 32, X = tx * 32;
    const u32* owg = occw + (size_t)s * L * T;
    for (u32 i = threadIdx.x; i < 96 * 3; i += blockDim.x) {
      const u32 r = i / 3, c = i % 3;
      ow[r][c] = owg[(size_t)((Y + L + r - 32) % L) * T + (tx + T + c - 1) % T];
    }
    __syncthreads();
    const u64 base = g.base[s];
    const bool need_prev = lane >= 33u - K;  // position lane-32 >= -(K-1)
    if (warp == 0) {
      // horizontal: lane = position along the row
#pragma unroll 2
      for (u32 r = 0; r < 32; ++r) {
        const u64 A = ((u64)ow[32 + r][1] << 32) | ow[32 + r][0];  // positions -32 .. 31
        const u64 B = ((u64)ow[32 + r][2] << 32) | ow[32 + r][1];  // positions 0 .. 63
        const u64 rowbase = (u64)(Y + r) * L;
        u64 vp = KEY_NONE, vc = KEY_NONE;
        if (need_prev && ((A >> lane) & kmask<K>()) == 0)
          vp = key_of(g, base, rowbase + (X + L - 32 + lane) % L);
        if (((B >> lane) & kmask<K>()) == 0) vc = key_of(g, base, rowbase + X + lane);
        lh[r][lane] = vp;
        lh[r][32 + lane] = vc;
      }
    } else {
      // vertical: lane = position along the column
      const u32 bp = ow[lane][1], bc = ow[32 + lane][1], bn = ow[64 + lane][1];
#pragma unroll 2
      for (u32 c = 0; c < 32; ++c) {
        const u32 Mp = __ballot_sync(FULL, (bp >> c) & 1u);
        const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
        const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
        const u64 A = ((u64)Mc << 32) | Mp, B = ((u64)Mn << 32) | Mc;
        const u64 x = X + c;
        u64 vp = KEY_NONE, vc = KEY_NONE;
        if (need_prev && ((A >> lane) & kmask<K>()) == 0)
          vp = key_of(g, base, g.LL + (u64)((Y + L - 32 + lane) % L) * L + x);
        if (((B >> lane) & kmask<K>()) == 0) vc = key_of(g, base, g.LL + (u64)(Y + lane) * L + x);
        lv[c][lane] = vp;
        lv[c][32 + lane] = vc;
      }
    }
    __syncthreads();
    if (warp == 0) line_bwd<K>(lh[lane]);
    else line_bwd<K>(lv[lane]);
    __syncthreads();
    bool any = false;
    u64* cmg = g.cmin + (size_t)s * g.LL;
    for (u32 i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
      const u32 y = i >> 5, c = i & 31;
      const u64 v = tmin(lh[y][32 + c], lv[c][32 + y]);
      cmg[(size_t)(Y + y) * L + X + c] = v;
      any |= v != KEY_NONE;
    }
    const bool live = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      if (!live) *dflag = 1;
      else if (!g.st[s].alive) g.st[s].alive = 1;
    }
  }
}

// Pass 2 of a round: acceptance of candidates anchored in each live tile.
//  (a) stage cmin: row lines (own tile + the tile to the right) and column
//      lines (own tile + the tile below); a dead neighbour reads as "none";
//  (b) one thread per line: width-K forward window minima, in place;
//  (c) lane-parallel: a live candidate whose window minimum equals its key
//      is accepted.
template <int K>
__global__ void __launch_bounds__(64) k_tile_accept(Group g, TileCfg tc, u32* occw,
                                                    const u8* dead) {
  __shared__ u32 ow[64][2];     // occupancy words rows Y .. Y+63, word columns wx, wx+1
  __shared__ u64 lh[32][LN];    // row lines: columns X .. X+63
  __shared__ u64 lv[32][LN];    // column lines: rows Y .. Y+63
  const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 L = g.L, T = tc.T;
  for (u64 item = blockIdx.x; item < tc.items; item += gridDim.x) {
    const u32 s = (u32)(item / tc.T2), t = (u32)(item % tc.T2);
    if (g.st[s].done) continue;
    const u8* dflag = dead + (size_t)s * tc.T2;
    if (dflag[t]) continue;
    const u32 ty = t / T, tx = t % T, Y = ty * 32, X = tx * 32;
    const u32 txr = tx + 1 == T ? 0 : tx + 1, tyb = ty + 1 == T ? 0 : ty + 1;
    const bool dr = dflag[ty * T + txr] != 0, db = dflag[tyb * T + tx] != 0;
    const u64* cmg = g.cmin + (size_t)s * g.LL;
    const u32* owg = occw + (size_t)s * L * T;
    for (u32 i = threadIdx.x; i < 64 * 2; i += blockDim.x) {
      const u32 r = i >> 1, c = i & 1;
      ow[r][c] = owg[(size_t)((Y + r) % L) * T + (c ? txr : tx)];
    }
    for (u32 i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
      const u32 r = i >> 5, c = i & 31;
      const u64 own = cmg[(size_t)(Y + r) * L + X + c];
      lh[r][c] = own;
      lv[c][r] = own;
      lh[r][32 + c] = dr ? KEY_NONE : cmg[(size_t)(Y + r) * L + txr * 32 + c];
      lv[c][32 + r] = db ? KEY_NONE : cmg[(size_t)(tyb * 32 + r) * L + X + c];
    }
    __syncthreads();
    if (warp == 0) line_fwd<K>(lh[lane]);
    else line_fwd<K>(lv[lane]);
    __syncthreads();
    const u64 base = g.base[s];
    if (warp == 0) {
      for (u32 r = 0; r < 32; ++r) {
        const u64 f = lh[r][lane];
        const u64 B = ((u64)ow[r][1] << 32) | ow[r][0];
        if (f != KEY_NONE && ((B >> lane) & kmask<K>()) == 0) {
          const u64 idx = (u64)(Y + r) * L + X + lane;
          if (f == key_of(g, base, idx)) accept_bits(g, occw, T, s, (u32)idx, f);
        }
      }
    } else {
      const u32 bc = ow[lane][0], bn = ow[32 + lane][0];
      for (u32 c = 0; c < 32; ++c) {
        const u32 Mc = __ballot_sync(FULL, (bc >> c) & 1u);
        const u32 Mn = __ballot_sync(FULL, (bn >> c) & 1u);
        const u64 B = ((u64)Mn << 32) | Mc;
        const u64 f = lv[c][lane];
        if (f != KEY_NONE && ((B >> lane) & kmask<K>()) == 0) {
          const u64 idx = g.LL + (u64)(Y + lane) * L + X + c;
          if (f == key_of(g, base, idx)) accept_bits(g, occw, T, s, (u32)idx, f);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace rsak
