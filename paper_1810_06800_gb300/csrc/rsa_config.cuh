// rsa_config.cuh -- the configuration of the first m accepted k-mers of a
// finished sample (m = n_c: the percolating state, m = n_j: the jamming
// state; Sec. III "Structure of the percolating and jamming states").
//
//   cluster sizes   number of clusters made of exactly s k-mers, s = 1 .. m
//                   (s k sites each; n_s of Eq. CSD is that count over L^2);
//   winding         whether some cluster winds round the torus along x, and
//                   along y (Sec. II.D "in one or both directions").
//
// The k-mers tried first are the ones with the smallest keys, so the first m
// accepted k-mers are the nodes with key <= T_m, the m-th smallest node key,
// and the lattice edges among them are the contact-graph edges with time
// (the larger key of their two ends) <= T_m.  One pass of the bisection
// machinery at that threshold gives both answers:
//   k_select_key   T_m by an 8-bit radix select over the node keys;
//   k_cfg_init     identity union-find, zero sizes and histogram;
//   k_cfg_union    union the edges with time <= T_m; an edge that closes a
//                  cycle of non-zero winding adds its directions;
//   k_cfg_count    k-mers per root;  k_cfg_hist  roots per size.
// A closed cycle's mismatch is its winding (a, b) times L, modulo 2^16.  The
// cycles closed while the union-find grows generate the windings of every
// cycle of the clusters, so "some closed cycle has a != 0" is "the clusters
// wind along x", whatever order the edges are united in.
// Scratch (the sample's search state is no longer needed): union-find words
// in the first half of its uf slot, sizes (u32) in the second half, the
// histogram (u32) in its unsorted edge array.
#pragma once
#include "rsa_kernels.cuh"

namespace rsak {

constexpr u32 CFG_CAPPED = 1u << 31;  // wdirs bit: a union-find walk hit its cap

__device__ __forceinline__ u64* cfg_uf(const Group& g, u32 s) {
  return g.uf + (size_t)s * 2 * g.cap_nodes;
}
__device__ __forceinline__ u32* cfg_size(const Group& g, u32 s) {
  return reinterpret_cast<u32*>(g.uf + ((size_t)s * 2 + 1) * g.cap_nodes);
}
__device__ __forceinline__ u32* cfg_hist(const Group& g, u32 s) {
  return reinterpret_cast<u32*>(g.edges + (size_t)s * g.cap_edges);
}

// T_m (1 <= m <= n_j) into st.sel: eight passes, each fixing the next 8 bits
// of the answer from a histogram of the keys that share the bits fixed so far.
__global__ void __launch_bounds__(1024) k_select_key(Group g, u32 s, u32 m) {
  __shared__ u32 hist[256];
  __shared__ u64 pre_sh;
  __shared__ u32 rank_sh;
  SampleState& st = g.st[s];
  const u32 nn = min(st.n_nodes, g.cap_nodes);
  const u64* K = g.node_key + (size_t)s * g.cap_nodes;
  u64 pre = 0, mask = 0;
  u32 rank = m;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (u32 i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (u32 i = threadIdx.x; i < nn; i += blockDim.x) {
      const u64 kk = K[i];
      if ((kk & mask) == pre) atomicAdd(&hist[(u32)(kk >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 d = 0, below = 0;
      while (d < 255 && below + hist[d] < rank) below += hist[d++];
      rank_sh = rank - below;
      pre_sh = pre | ((u64)d << shift);
    }
    __syncthreads();
    rank = rank_sh;
    pre = pre_sh;
    mask |= 255ull << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st.sel = pre;
    st.wdirs = 0;
  }
}

__global__ void k_cfg_init(Group g, u32 s) {
  const u32 nn = min(g.st[s].n_nodes, g.cap_nodes);
  u64* W = cfg_uf(g, s);
  u32* size = cfg_size(g, s);
  u32* hist = cfg_hist(g, s);
  for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m <= nn; m += gridDim.x * blockDim.x) {
    if (m < nn) {
      W[m] = uf_pack(m, 0, 0);
      size[m] = 0;
    }
    hist[m] = 0;
  }
}

__global__ void k_cfg_union(Group g, u32 s) {
  SampleState& st = g.st[s];
  const u64 T = st.sel;
  const u32* eb = g.ebkt + (size_t)s * (NBKT + 1);
  const u32 e1 = eb[(u32)(T >> 56) + 1];
  const Edge* E = g.edges_b + (size_t)s * g.cap_edges;
  u64* W = cfg_uf(g, s);
  bool capped = false;
  u32 dirs = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < e1; i += gridDim.x * blockDim.x) {
    const Edge e = E[i];
    if (e.time > T) continue;
    u32 mis = 0;
    if (uf_union(W, e.m1, e.m2, e.dxy, &capped, g.uf_cap, &mis))
      dirs |= ((mis & 0xFFFFu) ? 1u : 0u) | ((mis >> 16) ? 2u : 0u);
  }
  if (capped) dirs |= CFG_CAPPED;
  dirs = __reduce_or_sync(FULL, dirs);
  if ((threadIdx.x & 31) == 0 && dirs) atomicOr(&st.wdirs, dirs);
}

__global__ void k_cfg_count(Group g, u32 s) {
  SampleState& st = g.st[s];
  const u64 T = st.sel;
  const u32 nn = min(st.n_nodes, g.cap_nodes);
  const u64* K = g.node_key + (size_t)s * g.cap_nodes;
  u64* W = cfg_uf(g, s);
  u32* size = cfg_size(g, s);
  bool capped = false;
  for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m < nn; m += gridDim.x * blockDim.x) {
    if (K[m] > T) continue;
    u32 ox, oy;
    const u32 r = uf_find(W, m, &ox, &oy, &capped, g.uf_cap);
    atomicAdd(&size[r], 1u);
  }
  if (__any_sync(FULL, capped) && (threadIdx.x & 31) == 0) atomicOr(&st.wdirs, CFG_CAPPED);
}

__global__ void k_cfg_hist(Group g, u32 s) {
  const u32 nn = min(g.st[s].n_nodes, g.cap_nodes);
  const u32* size = cfg_size(g, s);
  u32* hist = cfg_hist(g, s);
  for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m < nn; m += gridDim.x * blockDim.x) {
    const u32 c = size[m];
    if (c) atomicAdd(&hist[c], 1u);
  }
}

}  // namespace rsak
