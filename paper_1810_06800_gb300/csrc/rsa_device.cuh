// rsa_device.cuh -- device code of the GB300 RSA library (sm_103a).
//
// Exact parallel form of the RSA scan of arXiv:1810.06800 Sec. II.B: the
// viable-list deposition tries each (orientation, y, x) candidate once in
// uniformly random order and accepts it iff its k cells are free.  With the
// order fixed by distinct 64-bit priorities this is the lexicographically
// first maximal independent set of the candidate conflict graph, which is
// reached in rounds: a live candidate whose priority is the smallest over
// every live candidate sharing a cell with it is accepted, and candidates
// touching the newly occupied cells die.  Per round and per cell:
//   cmin(cell) = min over live candidates covering the cell of key,
//   accept c   iff min over c's k cells of cmin == key(c).
// Both minima are sliding-window minima of width k along rows (horizontal
// candidates) and columns (vertical ones), computed with the van Herk /
// Gil-Werman split into k-aligned blocks (segmented prefix and suffix
// minima), so the cost per cell does not depend on k.
//
// Priorities are recomputed from (seed, idx) wherever they are needed
// instead of being stored: splitmix64 costs a few integer instructions,
// while storing 2 L^2 keys would cost 16 bytes per cell of HBM traffic per
// pass and 16 GiB per sample at L = 32768.
#pragma once
#include <cstdint>

namespace rsak {

typedef unsigned long long u64;
typedef uint32_t u32;
typedef uint16_t u16;
typedef uint8_t u8;

constexpr u64 KEY_NONE = 0xFFFFFFFFFFFFFFFFull;  // dead / no candidate
constexpr u64 SM_GAMMA = 0x9E3779B97F4A7C15ull;  // splitmix64 increment
constexpr u32 NONE32 = 0xFFFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr u32 OWN_V = 1u << 31;  // owner word: set for a vertical k-mer's cells
// Work counters are spread over WORK_SLOTS addresses (by block index), so that
// many blocks adding to one counter do not queue on a single L2 address.
constexpr u32 WORK_SLOTS = 32;
constexpr u32 NBKT = 256;  // time buckets (top 8 bits of a priority)

// status bits (per sample), mapped to RSA_E* codes by the host
constexpr u32 ST_NODE_OVF = 1u;     // more accepted k-mers than L^2/k (bug)
constexpr u32 ST_EDGE_OVF = 2u;     // contact-edge buffer too small
constexpr u32 ST_UF_CAP = 4u;       // union-find retry cap hit
constexpr u32 ST_NOWRAP = 8u;       // no wrap at jamming
constexpr u32 ST_SEARCH_CAP = 16u;  // bisection did not converge
constexpr u32 ST_ROUND_CAP = 32u;   // round loop cap hit
constexpr u32 ST_SEARCH_BAD = 64u;  // inconsistent bisection counts

// splitmix64 output finaliser (Stafford "Mix13"), Steele/Lea/Flood 2014.
__device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Inverse of mix64: each xor-shift z ^ (z >> s) is undone by xoring the
// shifts s, 2s, ... below 64, each odd multiplier by its inverse mod 2^64.
__device__ __forceinline__ u64 mix64_inverse(u64 z) {
  z = z ^ (z >> 31) ^ (z >> 62);
  z *= 0x319642B2D24D8EC3ull;  // inverse of 0x94D049BB133111EB
  z = z ^ (z >> 27) ^ (z >> 54);
  z *= 0x96DE1B173F119089ull;  // inverse of 0xBF58476D1CE4E5B9
  z = z ^ (z >> 30) ^ (z >> 60);
  return z;
}
constexpr u64 SM_GAMMA_INV = 0xF1DE83E19937733Dull;  // inverse of the golden gamma

struct Edge {          // one contact between two k-mers (24 bytes)
  u64 time;            // max of the two k-mers' priorities
  u32 m1, m2;          // node ids (acceptance order)
  u32 dxy;             // lifted anchor(m2) - anchor(m1): low 16 dx, high 16 dy
  u32 pad;
};

struct SampleState {   // one per sample, 128 bytes
  u32 n_nodes, n_edges, rounds, probes;
  u32 done, alive, status, wrap;
  u64 lo, hi, mid;
  u32 cnt_lo, cnt_hi, cnt_mid, lo_valid;
  u32 cur, sdone, nc, hi_ok;
  u32 contacts_x, contacts_y, contacts_xy;  // lattice edges between different
                                            // k-mers: both H, both V, mixed
  u32 wdirs;                                // configuration pass: winding bits
  u64 sel;                                  // configuration pass: m-th key
  u32 pad[4];
};
static_assert(sizeof(SampleState) == 128, "SampleState is 128 bytes");

struct Group {         // one batch of samples sharing (L, k)
  u32 L, k, n;
  u32 cap_nodes, cap_edges;
  u32 uf_cap;          // steps of one union-find walk or link retry loop
  u32 edge_limit;      // contact edges stored per sample (<= cap_edges)
  u64 LL;
  u8* occ;             // [n][L][L]   1 = occupied
  u32* owner;          // [n][L][L]   node id (| OWN_V if vertical) or NONE32
  u64* cmin;           // [n][L][L]   per-cell minimum of live priorities
  u64* base;           // [n]         splitmix64 stream base per sample
  const u64* keys;     // caller priorities [2 L^2] (test path), else null
  u64* node_key;       // [n][cap_nodes]
  u32* node_idx;       // [n][cap_nodes]  accepted candidate idx
  u32* node_pos;       // [n][cap_nodes]  o << 31 | y0 << 15 | x0 of the anchor
  u64* uf;             // [n][2][cap_nodes] union-find words
  Edge* edges;         // [n][cap_edges]
  Edge* edges_b;       // [n][cap_edges] edges grouped by time >> 56
  u32* ebkt;           // [n][NBKT + 1] bucket offsets into edges_b
  u64* nkey_b;         // [n][cap_nodes] node keys grouped by key >> 56
  u32* nbkt;           // [n][NBKT + 1] bucket offsets into nkey_b
  SampleState* st;     // [n]
  u64* scratch;        // global scratch for very long windows (or null)
  u64* work;           // [4][WORK_SLOTS] work counters of the round passes (tile path:
                       //     cmin cells, cmin keys, accept cells, accept keys; long-k
                       //     path: horizontal and vertical window-minimum cells,
                       //     acceptance cells, code cells)
};

// Add v to work counter c (slot chosen by the block index).
__device__ __forceinline__ void work_add(const Group& g, u32 c, u64 v) {
  atomicAdd(g.work + c * WORK_SLOTS + (blockIdx.x & (WORK_SLOTS - 1)), v);
}

__device__ __forceinline__ u64 cand_key(const Group& g, u32 s, u64 idx) {
  if (g.keys) return g.keys[idx];
  return mix64(g.base[s] + SM_GAMMA * (idx + 1));
}

template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return b < a ? b : a; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return b > a ? b : a; }

// Shared by the engine and the small-lattice kernel.
// Position of cell (cy, cx) inside the k-mer whose anchor is packed as
// o << 31 | y0 << 15 | x0; *o receives the orientation.
__device__ __forceinline__ u32 pos_in_kmer(u32 pos, u32 cy, u32 cx, u32 L, u32* o) {
  const u32 oo = pos >> 31, y0 = (pos >> 15) & 0x7FFFu, x0 = pos & 0x7FFFu;
  *o = oo;
  const u32 d = oo == 0 ? cx - x0 : cy - y0;
  return (int)d < 0 ? d + L : d;
}

__device__ __forceinline__ u64 uf_pack(u32 p, u32 dx, u32 dy) {
  return (u64)p | ((u64)(dx & 0xFFFFu) << 32) | ((u64)(dy & 0xFFFFu) << 48);
}

constexpr u32 UF_CAP = 1u << 20;  // default walk / retry cap (Group::uf_cap)

// ---------------------------------------------------------------------
// Segmented min-scans used by the window minimum.  A window of width k
// ending at span position v+k-1 (i.e. covering [v, v+k-1]) equals
// min(Q[v], P[v+k-1]) where P / Q are prefix / suffix minima inside blocks
// [m k, (m+1) k) of the span (van Herk / Gil-Werman).  seg == 0 means one
// unbounded segment.
// ---------------------------------------------------------------------

// One warp scans arr[0, n) (contiguous).  Forward = prefix minima.
template <typename T>
__device__ void warp_scan_fwd(const T* src, T* dst, u32 n, u32 seg, T ident) {
  const u32 lane = threadIdx.x & 31;
  u32 C = (n + 31) / 32;
  C |= 1u;  // odd chunk stride keeps the 32 lanes on distinct banks
  const u32 a = min(lane * C, n), b = min(a + C, n);
  T run = ident;
  bool flag = false;
  for (u32 u = a; u < b; ++u) {
    if (seg && (u % seg) == 0) { run = ident; flag = true; }
    run = tmin(run, src[u]);
    dst[u] = run;
  }
  T agg = run;
  bool f = flag;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T oa = __shfl_up_sync(FULL, agg, d);
    bool of = __shfl_up_sync(FULL, f, d);
    if ((int)lane >= d) {
      if (!f) agg = tmin(agg, oa);
      f = f || of;
    }
  }
  T carry = __shfl_up_sync(FULL, agg, 1);
  if (lane == 0) carry = ident;
  if (a < b && !(seg && (a % seg) == 0)) {
    u64 stop = seg ? ((u64)(a + seg - 1) / seg) * seg : (u64)b;
    u32 e = (u32)(stop < b ? stop : b);
    for (u32 u = a; u < e; ++u) dst[u] = tmin(dst[u], carry);
  }
}

// One warp, suffix minima (segments end at multiples of seg minus one).
template <typename T>
__device__ void warp_scan_bwd(const T* src, T* dst, u32 n, u32 seg, T ident) {
  const u32 lane = threadIdx.x & 31;
  u32 C = (n + 31) / 32;
  C |= 1u;
  const u32 a = min(lane * C, n), b = min(a + C, n);
  T run = ident;
  bool flag = false;
  for (u32 u = b; u > a; --u) {
    const u32 p = u - 1;
    if (seg && ((p + 1) % seg) == 0) { run = ident; flag = true; }
    run = tmin(run, src[p]);
    dst[p] = run;
  }
  T agg = run;
  bool f = flag;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T oa = __shfl_down_sync(FULL, agg, d);
    bool of = __shfl_down_sync(FULL, f, d);
    if (lane + d < 32) {
      if (!f) agg = tmin(agg, oa);
      f = f || of;
    }
  }
  T carry = __shfl_down_sync(FULL, agg, 1);
  if (lane == 31) carry = ident;
  if (a < b && !(seg && (b % seg) == 0)) {
    u32 s0 = seg ? (b / seg) * seg : 0u;
    u32 e = s0 > a ? s0 : a;
    for (u32 u = e; u < b; ++u) dst[u] = tmin(dst[u], carry);
  }
}

// Whole block scans W interleaved lines: element (u, line) at [u*W + line].
// Thread t handles line t % W, chunk t / W (G = blockDim / W chunks).
template <typename T>
__device__ void lines_scan_fwd(const T* src, T* dst, u32 n, u32 seg, T ident, u32 W,
                               T* aggv, u8* aggf) {
  const u32 line = threadIdx.x % W, g = threadIdx.x / W, G = blockDim.x / W;
  const u32 C = (n + G - 1) / G;
  const u32 a = min(g * C, n), b = min(a + C, n);
  T run = ident;
  bool flag = false;
  for (u32 u = a; u < b; ++u) {
    if (seg && (u % seg) == 0) { run = ident; flag = true; }
    run = tmin(run, src[(size_t)u * W + line]);
    dst[(size_t)u * W + line] = run;
  }
  aggv[g * W + line] = run;
  aggf[g * W + line] = flag;
  __syncthreads();
  if (a < b && !(seg && (a % seg) == 0)) {
    T carry = ident;
    for (int gg = (int)g - 1; gg >= 0; --gg) {
      carry = tmin(carry, aggv[gg * W + line]);
      if (aggf[gg * W + line]) break;
    }
    u64 stop = seg ? ((u64)(a + seg - 1) / seg) * seg : (u64)b;
    u32 e = (u32)(stop < b ? stop : b);
    for (u32 u = a; u < e; ++u) dst[(size_t)u * W + line] = tmin(dst[(size_t)u * W + line], carry);
  }
  __syncthreads();
}

template <typename T>
__device__ void lines_scan_bwd(const T* src, T* dst, u32 n, u32 seg, T ident, u32 W,
                               T* aggv, u8* aggf) {
  const u32 line = threadIdx.x % W, g = threadIdx.x / W, G = blockDim.x / W;
  const u32 C = (n + G - 1) / G;
  const u32 a = min(g * C, n), b = min(a + C, n);
  T run = ident;
  bool flag = false;
  for (u32 u = b; u > a; --u) {
    const u32 p = u - 1;
    if (seg && ((p + 1) % seg) == 0) { run = ident; flag = true; }
    run = tmin(run, src[(size_t)p * W + line]);
    dst[(size_t)p * W + line] = run;
  }
  aggv[g * W + line] = run;
  aggf[g * W + line] = flag;
  __syncthreads();
  if (a < b && !(seg && (b % seg) == 0)) {
    T carry = ident;
    for (u32 gg = g + 1; gg < G; ++gg) {
      carry = tmin(carry, aggv[gg * W + line]);
      if (aggf[gg * W + line]) break;
    }
    u32 s0 = seg ? (b / seg) * seg : 0u;
    u32 e = s0 > a ? s0 : a;
    for (u32 u = e; u < b; ++u) dst[(size_t)u * W + line] = tmin(dst[(size_t)u * W + line], carry);
  }
  __syncthreads();
}

// Record an accepted candidate: allocate its node, occupy its k cells.
__device__ __forceinline__ void accept_candidate(const Group& g, u32 s, u32 idx, u64 key) {
  SampleState& st = g.st[s];
  const u32 node = atomicAdd(&st.n_nodes, 1u);
  if (node >= g.cap_nodes) { atomicOr(&st.status, ST_NODE_OVF); return; }
  g.node_key[(size_t)s * g.cap_nodes + node] = key;
  g.node_idx[(size_t)s * g.cap_nodes + node] = idx;
  const u32 L = g.L;
  const u32 o = idx / (u32)g.LL, r = idx % (u32)g.LL;
  const u32 y0 = r / L, x0 = r % L;
  g.node_pos[(size_t)s * g.cap_nodes + node] = (o << 31) | (y0 << 15) | x0;
  u8* occ = g.occ + (size_t)s * g.LL;
  u32* own = g.owner + (size_t)s * g.LL;
  if (o == 0) {
    u32 x = x0;
    for (u32 i = 0; i < g.k; ++i) {
      occ[(size_t)y0 * L + x] = 1;
      own[(size_t)y0 * L + x] = node;  // horizontal: bit 31 clear
      if (++x == L) x = 0;
    }
  } else {
    u32 y = y0;
    for (u32 i = 0; i < g.k; ++i) {
      occ[(size_t)y * L + x0] = 1;
      own[(size_t)y * L + x0] = node | OWN_V;
      if (++y == L) y = 0;
    }
  }
}

}  // namespace rsak
