// rsa_kernels.cuh -- round, contact-graph and bisection kernels (sm_103a).
#pragma once
#include "rsa_device.cuh"

namespace rsak {

// Launch geometry of the row pass: one warp per (row, segment of S cells).
struct RowCfg {
  u32 S, nseg;        // segment length, segments per row
  u32 warps;          // warps per block
  u32 warp_words;     // u64 words of per-warp scratch (A region + B region)
  u32 nmax;           // max span length (S + k - 1)
  int global_scratch; // 1: per-warp scratch in g.scratch instead of smem
};

// Geometry of the column pass: W adjacent columns x (segment of S rows).
struct ColCfg {
  u32 S, nseg;        // segment length (rows), segments per column
  u32 W, nstrip;      // columns per block, column strips
  u32 nmax, nocc;     // value span and occupancy span lengths
  u32 block_words;    // u64 words of scratch per block
  int global_scratch;
};

__device__ __forceinline__ u32 wrap_add(u32 a, u32 b, u32 L) {
  u32 r = a + b;
  return r >= L ? (r % L) : r;
}

// MODE 0: horizontal part of cmin.  For row y and x in the segment,
//   cmin(y,x) = min over live horizontal candidates anchored at
//               (y, x-k+1 .. x) of their key.
// A horizontal candidate is live iff its k cells are free.
// MODE 1: accept horizontal candidates: (y,x) is accepted iff
//   min(cmin(y, x .. x+k-1)) == key(0, y, x).
template <int MODE>
__global__ void __launch_bounds__(256) k_row(Group g, RowCfg rc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 L = g.L, k = g.k;
  u64* A;
  if (rc.global_scratch)
    A = g.scratch +
        (((size_t)blockIdx.y * gridDim.x + blockIdx.x) * rc.warps + warp) * rc.warp_words;
  else
    A = reinterpret_cast<u64*>(smem_raw) + (size_t)warp * rc.warp_words;
  u64* B = A + rc.nmax;          // values -> prefix minima
  u32* N = reinterpret_cast<u32*>(A);  // next-occupied table (aliases A)
  const u8* occ = g.occ + (size_t)s * g.LL;
  u64* cmin = g.cmin + (size_t)s * g.LL;
  bool any_alive = false;
  const u64 total = (u64)L * rc.nseg;
  for (u64 q = (u64)blockIdx.x * rc.warps + warp; q < total; q += (u64)gridDim.x * rc.warps) {
    const u32 y = (u32)(q / rc.nseg), seg = (u32)(q % rc.nseg);
    const u32 x0 = seg * rc.S;
    const u32 Se = min(rc.S, L - x0);
    const u32 n = Se + k - 1;
    const u8* orow = occ + (size_t)y * L;
    u64* crow = cmin + (size_t)y * L;
    if (MODE == 0) {
      const u32 xs = (x0 + L - (k - 1)) % L;
      const u32 nocc = Se + 2 * k - 2;
      for (u32 u = lane; u < nocc; u += 32) N[u] = orow[wrap_add(xs, u % L, L)] ? u : NONE32;
      __syncwarp();
      warp_scan_bwd<u32>(N, N, nocc, 0u, NONE32);
      __syncwarp();
      for (u32 u = lane; u < n; u += 32) {
        const bool alive = N[u] >= u + k;  // NONE32 >= anything
        u64 v = KEY_NONE;
        if (alive) {
          const u32 x = wrap_add(xs, u % L, L);
          v = cand_key(g, s, (u64)y * L + x);
          any_alive = true;
        }
        B[u] = v;
      }
    } else {
      for (u32 u = lane; u < n; u += 32) B[u] = crow[wrap_add(x0, u % L, L)];
    }
    __syncwarp();
    warp_scan_bwd<u64>(B, A, n, k, KEY_NONE);  // suffix minima -> A
    __syncwarp();
    warp_scan_fwd<u64>(B, B, n, k, KEY_NONE);  // prefix minima in place
    __syncwarp();
    for (u32 v = lane; v < Se; v += 32) {
      const u64 w = tmin(A[v], B[v + k - 1]);
      const u32 x = x0 + v;
      if (MODE == 0) {
        crow[x] = w;
      } else if (w != KEY_NONE) {
        const u32 idx = y * L + x;
        if (w == cand_key(g, s, idx)) accept_candidate(g, s, idx, w);
      }
    }
    __syncwarp();
  }
  if (MODE == 0) {
    if (__any_sync(FULL, any_alive) && lane == 0) atomicOr(&g.st[s].alive, 1u);
  }
}

// MODE 0: vertical part of cmin, combined with the horizontal part already
//   in cmin: cmin(y,x) = min(cmin(y,x), min over live vertical candidates
//   anchored at (y-k+1 .. y, x)).
// MODE 1: accept vertical candidates: (y,x) accepted iff
//   min(cmin(y .. y+k-1, x)) == key(1, y, x).
template <int MODE>
__global__ void __launch_bounds__(256) k_col(Group g, ColCfg cc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const u32 s = blockIdx.y;
  if (g.st[s].done) return;
  const u32 L = g.L, k = g.k, W = cc.W, G = blockDim.x / W;
  u64* base;
  if (cc.global_scratch)
    base = g.scratch + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * cc.block_words;
  else
    base = reinterpret_cast<u64*>(smem_raw);
  u64* A = base;                                     // nmax*W (N aliases it)
  const size_t a_words = max((size_t)cc.nmax * W, ((size_t)cc.nocc * W + 1) / 2);
  u64* B = A + a_words;                              // nmax*W
  u64* aggv = B + (size_t)cc.nmax * W;               // G*W
  u8* aggf = reinterpret_cast<u8*>(aggv + (size_t)G * W);  // G*W
  u32* N = reinterpret_cast<u32*>(A);
  const u8* occ = g.occ + (size_t)s * g.LL;
  u64* cmin = g.cmin + (size_t)s * g.LL;
  bool any_alive = false;
  const u32 total = cc.nstrip * cc.nseg;
  for (u32 q = blockIdx.x; q < total; q += gridDim.x) {
    const u32 strip = q / cc.nseg, seg = q % cc.nseg;
    const u32 c0 = strip * W, y0 = seg * cc.S;
    const u32 Se = min(cc.S, L - y0);
    const u32 n = Se + k - 1;
    if (MODE == 0) {
      const u32 ys = (y0 + L - (k - 1)) % L;
      const u32 nocc = Se + 2 * k - 2;
      for (u32 f = threadIdx.x; f < nocc * W; f += blockDim.x) {
        const u32 u = f / W, c = f % W, x = c0 + c;
        u32 v = NONE32;
        if (x < L && occ[(size_t)wrap_add(ys, u % L, L) * L + x]) v = u;
        N[f] = v;
      }
      __syncthreads();
      lines_scan_bwd<u32>(N, N, nocc, 0u, NONE32, W, reinterpret_cast<u32*>(aggv), aggf);
      for (u32 f = threadIdx.x; f < n * W; f += blockDim.x) {
        const u32 u = f / W, c = f % W, x = c0 + c;
        u64 v = KEY_NONE;
        if (x < L && N[f] >= u + k) {
          const u32 y = wrap_add(ys, u % L, L);
          v = cand_key(g, s, (u64)L * L + (u64)y * L + x);
          any_alive = true;
        }
        B[f] = v;
      }
    } else {
      for (u32 f = threadIdx.x; f < n * W; f += blockDim.x) {
        const u32 u = f / W, c = f % W, x = c0 + c;
        B[f] = x < L ? cmin[(size_t)wrap_add(y0, u % L, L) * L + x] : KEY_NONE;
      }
    }
    __syncthreads();
    lines_scan_bwd<u64>(B, A, n, k, KEY_NONE, W, aggv, aggf);
    lines_scan_fwd<u64>(B, B, n, k, KEY_NONE, W, aggv, aggf);
    for (u32 f = threadIdx.x; f < Se * W; f += blockDim.x) {
      const u32 v = f / W, c = f % W, x = c0 + c;
      if (x >= L) continue;
      const u64 w = tmin(A[f], B[f + (size_t)(k - 1) * W]);
      const u32 y = y0 + v;
      if (MODE == 0) {
        u64* p = cmin + (size_t)y * L + x;
        *p = tmin(*p, w);
      } else if (w != KEY_NONE) {
        const u32 idx = (u32)(g.LL + (u64)y * L + x);
        if (w == cand_key(g, s, idx)) accept_candidate(g, s, idx, w);
      }
    }
    __syncthreads();
  }
  if (MODE == 0) {
    if (__syncthreads_or(any_alive) && threadIdx.x == 0) atomicOr(&g.st[s].alive, 1u);
  }
}

// Per-sample set-up: stream base from the seed, state cleared.
__global__ void k_init(Group g, const u64* seeds) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  g.base[s] = mix64(seeds[s] + SM_GAMMA);
  SampleState z = {};
  g.st[s] = z;
}

// End of a round: a sample with no live candidate left is jammed.
__global__ void k_round_end(Group g, u32 round_cap, u32* n_active) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  SampleState& st = g.st[s];
  if (st.done) return;
  if (!st.alive) {
    st.done = 1;
    return;
  }
  st.alive = 0;
  st.rounds += 1;
  if (st.rounds >= round_cap) {
    st.status |= ST_ROUND_CAP;
    st.done = 1;
    return;
  }
  atomicAdd(n_active, 1u);
}

// ---------------------------------------------------------------------
// Contact graph of the jammed lattice.  Nodes are accepted k-mers; a
// lattice edge (a, a+e), e in {+x, +y}, between occupied cells of k-mers
// m1 and m2 says that in the lift anchor(m2) = anchor(m1) + delta with
//   delta = i e(m1) + e - j e(m2)  (i, j = positions of a, a+e inside the
// k-mers).  Runs of identical (m1, m2, delta) along the direction
// perpendicular to e are emitted once; a run start is forced at row 0 (for
// +x) / column 0 (for +y) so that runs that close around the torus are kept.
// Only edges whose m1 == m2 and delta == 0 (inside one k-mer) are dropped.
// ---------------------------------------------------------------------
// Lifted displacement of the contact between cell (y, x) of node m1 and its
// neighbour (by, bx) in direction dir of node m2, packed as 16+16 bits.
__device__ __forceinline__ u32 contact_delta(const Group& g, u32 s, u32 y, u32 x, u32 by, u32 bx,
                                             u32 dir, u32 m1, u32 m2, bool* internal) {
  const u32* npos = g.node_pos + (size_t)s * g.cap_nodes;
  u32 o1, o2;
  const u32 i = pos_in_kmer(npos[m1], y, x, g.L, &o1);
  const u32 j = pos_in_kmer(npos[m2], by, bx, g.L, &o2);
  const int dx = (o1 == 0 ? (int)i : 0) + (dir == 0) - (o2 == 0 ? (int)j : 0);
  const int dy = (o1 == 1 ? (int)i : 0) + (dir == 1) - (o2 == 1 ? (int)j : 0);
  *internal = m1 == m2 && dx == 0 && dy == 0;
  return ((u32)dx & 0xFFFFu) | (((u32)dy & 0xFFFFu) << 16);
}

constexpr u32 EDGES_THREADS = 256;

// The two contacts (+x, +y) of cell (y, x) of owner a, given the owners of
// its neighbours (right, down, up, up-right, left, down-left): counted by
// class into cnt, and emitted as graph edges unless internal to one k-mer or
// a repeat of the previous contact of their run.  Every lane of the warp
// calls it (ballots inside); a lane with nothing to do passes a = NONE32.
__device__ __forceinline__ void edge_cell(const Group& g, u32 s, SampleState& st, const u64* nkey,
                                          Edge* E, bool full_compare, u32 lane, u32 y, u32 x,
                                          u32 yp, u32 yn, u32 xp, u32 xn, u32 a, u32 o_r,
                                          u32 o_d, u32 o_u, u32 o_ur, u32 o_l, u32 o_dl,
                                          u32 cnt[3]) {
#pragma unroll
  for (u32 dir = 0; dir < 2; ++dir) {
    const u32 by = dir ? yn : y, bx = dir ? x : xn;
    bool emit = false;
    u32 b = NONE32, d = 0;
    u32 kind = 3;  // contact class: 0 both horizontal, 1 both vertical, 2 mixed
    if (a != NONE32) {
      b = dir ? o_d : o_r;
      // owner words carry the k-mer's orientation in bit 31
      if (b != NONE32 && b != a) kind = (a ^ b) >> 31 ? 2u : a >> 31;
      if (b != NONE32) {
        bool internal = false;
        // the previous contact of the run: one row up (+x edges) or one
        // column left (+y edges)
        const bool force = dir == 0 ? (y == 0) : (x == 0);
        const u32 py = dir == 0 ? yp : y, px = dir == 0 ? x : xp;
        const u32 qy = dir == 0 ? yp : yn, qx = dir == 0 ? xn : xp;
        const u32 pa = force ? NONE32 : (dir == 0 ? o_u : o_l);
        const u32 pb = force ? NONE32 : (dir == 0 ? o_ur : o_dl);
        const bool same_pair = pa == a && pb == b;
        if (!same_pair || full_compare) {
          d = contact_delta(g, s, y, x, by, bx, dir, a & ~OWN_V, b & ~OWN_V, &internal);
          emit = !internal;
          if (emit && same_pair) {
            bool pint = false;
            const u32 pd = contact_delta(g, s, py, px, qy, qx, dir, pa & ~OWN_V, pb & ~OWN_V,
                                         &pint);
            emit = pd != d;
          }
        }
      }
    }
    // interspecific-contact counts (Sec. II.A): every contact, before the
    // run deduplication of the graph edges
    cnt[0] += kind == 0;
    cnt[1] += kind == 1;
    cnt[2] += kind == 2;
    const u32 mask = __ballot_sync(FULL, emit);
    if (!mask) continue;
    u32 basei = 0;
    const u32 leader = __ffs(mask) - 1;
    if (lane == leader) basei = atomicAdd(&st.n_edges, (u32)__popc(mask));
    basei = __shfl_sync(FULL, basei, leader);
    if (emit) {
      const u32 e = basei + __popc(mask & ((1u << lane) - 1u));
      if (e < g.edge_limit) {
        Edge ed;
        const u32 ma = a & ~OWN_V, mb = b & ~OWN_V;
        ed.time = max(nkey[ma], nkey[mb]);
        ed.m1 = ma;
        ed.m2 = mb;
        ed.dxy = d;
        ed.pad = 0;
        E[e] = ed;
      } else {
        atomicOr(&st.status, ST_EDGE_OVF);
      }
    }
  }
}

__device__ __forceinline__ void edge_counts(SampleState& st, u32 lane, const u32 cnt[3]) {
#pragma unroll
  for (u32 c = 0; c < 3; ++c) {
    const u32 t = __reduce_add_sync(FULL, cnt[c]);
    if (lane == 0 && t)
      atomicAdd(c == 0 ? &st.contacts_x : c == 1 ? &st.contacts_y : &st.contacts_xy, t);
  }
}

// Any L: one cell per thread per step.
__global__ void __launch_bounds__(EDGES_THREADS) k_edges(Group g) {
  const u32 s = blockIdx.y;
  const u32 L = g.L;
  const u32 lane = threadIdx.x & 31;
  SampleState& st = g.st[s];
  const u32* own = g.owner + (size_t)s * g.LL;
  const u64* nkey = g.node_key + (size_t)s * g.cap_nodes;
  Edge* E = g.edges + (size_t)s * g.cap_edges;
  // For k < L (and L > 2) consecutive contacts between the same two k-mers
  // along a run always have the same displacement, so runs are told apart by
  // their owners alone; rings (k = L) and tiny lattices compare displacements.
  const bool full_compare = g.k == L || L <= 2;
  // block b walks rows b, b + gridDim.x, ...; its threads stride along the
  // row (every lane of a warp runs the same number of steps: ballots inside)
  const u32 xsteps = (L + blockDim.x - 1) / blockDim.x;
  u32 cnt[3] = {0, 0, 0};
  for (u32 y = blockIdx.x; y < L; y += gridDim.x)
  for (u32 xs = 0; xs < xsteps; ++xs) {
    const u32 xx = xs * blockDim.x + threadIdx.x;
    const bool inb = xx < L;
    const u32 x = inb ? xx : 0;
    const u32 yp = y == 0 ? L - 1 : y - 1, yn = y + 1 == L ? 0 : y + 1;
    const u32 xp = x == 0 ? L - 1 : x - 1, xn = x + 1 == L ? 0 : x + 1;
    // the cell, its +x / +y neighbours, and the cells whose contact precedes
    // each of the two in its run (up, up-right for +x; left, down-left for
    // +y): all loaded at once, so their latencies overlap
    const u32 a = inb ? __ldg(own + (size_t)y * L + x) : NONE32;
    const u32 o_r = __ldg(own + (size_t)y * L + xn), o_d = __ldg(own + (size_t)yn * L + x);
    const u32 o_u = __ldg(own + (size_t)yp * L + x), o_ur = __ldg(own + (size_t)yp * L + xn);
    const u32 o_l = __ldg(own + (size_t)y * L + xp), o_dl = __ldg(own + (size_t)yn * L + xp);
    edge_cell(g, s, st, nkey, E, full_compare, lane, y, x, yp, yn, xp, xn, a, o_r, o_d, o_u,
              o_ur, o_l, o_dl, cnt);
  }
  edge_counts(st, lane, cnt);
}

// L a multiple of 4 (and at least 8): four consecutive cells per thread per
// step, from one 16-byte load of each of the three rows involved plus the
// four neighbour cells outside the quad.
__global__ void __launch_bounds__(EDGES_THREADS) k_edges4(Group g) {
  const u32 s = blockIdx.y;
  const u32 L = g.L, L4 = L / 4;
  const u32 lane = threadIdx.x & 31;
  SampleState& st = g.st[s];
  const u32* own = g.owner + (size_t)s * g.LL;
  const u64* nkey = g.node_key + (size_t)s * g.cap_nodes;
  Edge* E = g.edges + (size_t)s * g.cap_edges;
  const bool full_compare = g.k == L;
  const u32 xsteps = (L4 + blockDim.x - 1) / blockDim.x;
  u32 cnt[3] = {0, 0, 0};
  for (u32 y = blockIdx.x; y < L; y += gridDim.x)
  for (u32 xs = 0; xs < xsteps; ++xs) {
    const u32 qq = xs * blockDim.x + threadIdx.x;
    const bool inb = qq < L4;
    const u32 x0 = inb ? 4 * qq : 0;
    const u32 yp = y == 0 ? L - 1 : y - 1, yn = y + 1 == L ? 0 : y + 1;
    const u32 xl = x0 == 0 ? L - 1 : x0 - 1, xr = x0 + 4 == L ? 0 : x0 + 4;
    const u32* ry = own + (size_t)y * L;
    const u32* rn = own + (size_t)yn * L;
    const u32* rp = own + (size_t)yp * L;
    const uint4 A = __ldg(reinterpret_cast<const uint4*>(ry + x0));
    const uint4 D = __ldg(reinterpret_cast<const uint4*>(rn + x0));
    const uint4 U = __ldg(reinterpret_cast<const uint4*>(rp + x0));
    const u32 a_r = __ldg(ry + xr), a_l = __ldg(ry + xl);
    const u32 d_l = __ldg(rn + xl), u_r = __ldg(rp + xr);
    const u32 av[4] = {A.x, A.y, A.z, A.w}, dv[4] = {D.x, D.y, D.z, D.w};
    const u32 uv[4] = {U.x, U.y, U.z, U.w};
#pragma unroll
    for (u32 i = 0; i < 4; ++i) {
      const u32 x = x0 + i;
      const u32 xp = i == 0 ? xl : x - 1, xn = i == 3 ? xr : x + 1;
      edge_cell(g, s, st, nkey, E, full_compare, lane, y, x, yp, yn, xp, xn,
                inb ? av[i] : NONE32, i < 3 ? av[i + 1] : a_r, dv[i], uv[i],
                i < 3 ? uv[i + 1] : u_r, i > 0 ? av[i - 1] : a_l, i > 0 ? dv[i - 1] : d_l, cnt);
    }
  }
  edge_counts(st, lane, cnt);
}

// Group one sample's edges by time >> 56 and its node keys by key >> 56
// (counting sort into NBKT buckets), so that a bisection probe touches only
// the edges whose time can lie in its window.  One block per sample.
__global__ void __launch_bounds__(1024) k_bucket(Group g) {
  __shared__ u32 he[NBKT], hn[NBKT], ce[NBKT], cn[NBKT];
  const u32 s = blockIdx.x;
  SampleState& st = g.st[s];
  const u32 ne = min(st.n_edges, g.edge_limit), nn = min(st.n_nodes, g.cap_nodes);
  const Edge* E = g.edges + (size_t)s * g.cap_edges;
  Edge* E2 = g.edges_b + (size_t)s * g.cap_edges;
  const u64* K = g.node_key + (size_t)s * g.cap_nodes;
  u64* K2 = g.nkey_b + (size_t)s * g.cap_nodes;
  u32* eb = g.ebkt + (size_t)s * (NBKT + 1);
  u32* nb = g.nbkt + (size_t)s * (NBKT + 1);
  for (u32 i = threadIdx.x; i < NBKT; i += blockDim.x) he[i] = hn[i] = 0;
  __syncthreads();
  for (u32 i = threadIdx.x; i < ne; i += blockDim.x) atomicAdd(&he[(u32)(E[i].time >> 56)], 1u);
  for (u32 i = threadIdx.x; i < nn; i += blockDim.x) atomicAdd(&hn[(u32)(K[i] >> 56)], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 a = 0, b = 0;
    for (u32 i = 0; i < NBKT; ++i) {
      eb[i] = a; ce[i] = a; a += he[i];
      nb[i] = b; cn[i] = b; b += hn[i];
    }
    eb[NBKT] = a;
    nb[NBKT] = b;
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < ne; i += blockDim.x) {
    const Edge e = E[i];
    E2[atomicAdd(&ce[(u32)(e.time >> 56)], 1u)] = e;
  }
  for (u32 i = threadIdx.x; i < nn; i += blockDim.x) {
    const u64 kk = K[i];
    K2[atomicAdd(&cn[(u32)(kk >> 56)], 1u)] = kk;
  }
}

// ---------------------------------------------------------------------
// First wrap by bisection over the number of placed k-mers (Sec. II.D).
// wrap(m): does the graph of the first m accepted k-mers (the m smallest
// keys) contain a cycle of non-zero winding?  It is monotone in m, and n_c
// is the smallest m with wrap(m).  The first probe takes every k-mer (the
// jammed lattice must wrap); later probes bisect the rank interval
// (cnt_lo, cnt_hi] and take mid = T_r, the key of rank r, so that the edges
// of a probe are those with time (the larger key of their two ends) <= T_r.
// Each probe starts from the union-find state of the last non-wrapping rank
// cnt_lo (threshold `lo`) and adds only edges with lo < time <= mid, so the
// probes after the first non-wrapping one touch a halving share of edges.  Union-find words: parent (bits 0-31) and the lifted
// offset of the node from its parent, dx (32-47), dy (48-63), modulo 2^16.
// A wrap is a cycle of primitive winding (a, b) times L; for L < 65536 its
// offset is never 0 modulo 2^16, so 16-bit offsets decide exactly.
// ---------------------------------------------------------------------

// Root of x and x's offset from it.  Path halving by CAS; a failed CAS is
// harmless because every stored (parent, offset) pair stays a true ancestor
// relation.  Loads bypass L1 (other SMs write these words).
__device__ __forceinline__ u32 uf_find(u64* W, u32 x, u32* ox, u32* oy, bool* capped, u32 cap) {
  u32 sx = 0, sy = 0;
  for (u32 it = 0; it < cap; ++it) {
    const u64 wx = __ldcg(W + x);
    const u32 p = (u32)wx;
    if (p == x) {
      *ox = sx;
      *oy = sy;
      return x;
    }
    const u64 wp = __ldcg(W + p);
    const u32 gp = (u32)wp;
    if (gp != p) {
      const u64 nw = uf_pack(gp, (u32)(wx >> 32) + (u32)(wp >> 32),
                             (u32)(wx >> 48) + (u32)(wp >> 48));
      atomicCAS(W + x, wx, nw);
    }
    sx += (u32)(wx >> 32);
    sy += (u32)(wx >> 48);
    x = p;
  }
  *capped = true;
  *ox = sx;
  *oy = sy;
  return x;
}

// Add edge "anchor(m2) = anchor(m1) + d"; returns true if it closes a cycle
// of non-zero winding, and then, if mis is given, stores the cycle's lifted
// mismatch (x in bits 0-15, y in 16-31, modulo 2^16).  Roots are linked
// larger-id under smaller-id, so the forest stays acyclic under concurrent
// unions.
__device__ bool uf_union(u64* W, u32 m1, u32 m2, u32 dxy, bool* capped, u32 cap,
                         u32* mis = nullptr) {
  const u32 dx = dxy & 0xFFFFu, dy = dxy >> 16;
  for (u32 it = 0; it < cap; ++it) {
    u32 o1x, o1y, o2x, o2y;
    const u32 r1 = uf_find(W, m1, &o1x, &o1y, capped, cap);
    const u32 r2 = uf_find(W, m2, &o2x, &o2y, capped, cap);
    if (*capped) return false;
    // lifted position of r2 minus r1
    const u32 Dx = o1x + dx - o2x, Dy = o1y + dy - o2y;
    if (r1 == r2) {
      if (mis) *mis = (Dx & 0xFFFFu) | ((Dy & 0xFFFFu) << 16);
      return ((Dx | Dy) & 0xFFFFu) != 0;
    }
    if (r1 < r2) {
      if (atomicCAS(W + r2, uf_pack(r2, 0, 0), uf_pack(r1, Dx, Dy)) == uf_pack(r2, 0, 0))
        return false;
    } else {
      if (atomicCAS(W + r1, uf_pack(r1, 0, 0), uf_pack(r2, 0u - Dx, 0u - Dy)) ==
          uf_pack(r1, 0, 0))
        return false;
    }
  }
  *capped = true;
  return false;
}

__global__ void k_search_init(Group g) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  SampleState& st = g.st[s];
  st.lo = 0;
  st.lo_valid = 0;
  st.cnt_lo = 0;
  st.hi = KEY_NONE;
  st.cnt_hi = min(st.n_nodes, g.cap_nodes);
  st.mid = KEY_NONE;  // first probe: the whole jammed lattice must wrap
  st.cnt_mid = st.cnt_hi;
  st.hi_ok = 0;
  st.cur = 0;
  st.sdone = (st.status & (ST_NODE_OVF | ST_EDGE_OVF | ST_ROUND_CAP)) ? 1u : 0u;
  st.nc = NONE32;
  st.probes = 0;
}

__global__ void k_uf_identity(Group g) {
  const u32 s = blockIdx.y;
  const u32 nn = min(g.st[s].n_nodes, g.cap_nodes);
  u64* U = g.uf + (size_t)s * 2 * g.cap_nodes;
  for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m < nn; m += gridDim.x * blockDim.x)
    U[m] = uf_pack(m, 0, 0);
}

// Working copy of the union-find state at `lo`.
__global__ void k_probe_copy(Group g) {
  const u32 s = blockIdx.y;
  SampleState& st = g.st[s];
  if (st.sdone) return;
  if (threadIdx.x == 0 && blockIdx.x == 0) st.wrap = 0;
  const u32 nn = min(st.n_nodes, g.cap_nodes);
  const u64* S = g.uf + ((size_t)s * 2 + st.cur) * g.cap_nodes;
  u64* Wd = g.uf + ((size_t)s * 2 + (st.cur ^ 1u)) * g.cap_nodes;
  for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m < nn; m += gridDim.x * blockDim.x)
    Wd[m] = S[m];
}

// Eight 256-thread blocks per SM (32 registers): probes are latency-bound
// union-find walks, and full occupancy hides more of that latency.
__global__ void __launch_bounds__(256, 8) k_probe(Group g) {
  const u32 s = blockIdx.y;
  SampleState& st = g.st[s];
  if (st.sdone) return;
  const u64 lo = st.lo, mid = st.mid;
  const bool lo_valid = st.lo_valid != 0;
  const u32* eb = g.ebkt + (size_t)s * (NBKT + 1);
  const u32 blo = lo_valid ? (u32)(lo >> 56) : 0u, bmid = (u32)(mid >> 56);
  const u32 e0 = eb[blo], e1 = eb[bmid + 1];
  u64* Wd = g.uf + ((size_t)s * 2 + (st.cur ^ 1u)) * g.cap_nodes;
  const Edge* E = g.edges_b + (size_t)s * g.cap_edges;
  bool wrap = false, capped = false;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 i = e0 + blockIdx.x * blockDim.x + threadIdx.x; i < e1; i += stride) {
    const Edge e = E[i];
    if (e.time > mid || (lo_valid && e.time <= lo)) continue;
    if (uf_union(Wd, e.m1, e.m2, e.dxy, &capped, g.uf_cap)) wrap = true;
  }
  const bool bw = __syncthreads_or(wrap);
  const bool bc = __syncthreads_or(capped);
  if (threadIdx.x == 0) {
    if (bw) atomicOr(&st.wrap, 1u);
    if (bc) atomicOr(&st.status, ST_UF_CAP);
  }
}

// One bisection step of sample s (one thread): read the probe's wrap flag,
// move lo or hi, finish or pick the next rank.  True if another probe follows.
__device__ bool search_step(Group& g, SampleState& st, u32 probe_cap, u32* n_open) {
  st.probes += 1;
  if (st.status & ST_UF_CAP) {
    st.sdone = 1;
    return false;
  }
  const bool w = st.wrap != 0;
  if (!st.hi_ok) {
    if (!w) {
      st.status |= ST_NOWRAP;
      st.nc = NONE32;
      st.sdone = 1;
      return false;
    }
    st.hi_ok = 1;
    st.cnt_hi = st.cnt_mid;
  } else if (w) {
    st.hi = st.mid;
    st.cnt_hi = st.cnt_mid;
  } else {
    st.lo = st.mid;
    st.lo_valid = 1;
    st.cnt_lo = st.cnt_mid;
    st.cur ^= 1u;
  }
  if (st.cnt_hi <= st.cnt_lo) {
    st.status |= ST_SEARCH_BAD;
    st.sdone = 1;
    return false;
  }
  if (st.cnt_hi - st.cnt_lo == 1) {
    st.nc = st.cnt_hi;
    st.sdone = 1;
    return false;
  }
  if (st.probes >= probe_cap) {
    st.status |= ST_SEARCH_CAP;
    st.sdone = 1;
    return false;
  }
  // next rank, strictly inside (cnt_lo, cnt_hi)
  st.cnt_mid = st.cnt_lo + (st.cnt_hi - st.cnt_lo) / 2;
  atomicAdd(n_open, 1u);
  return true;
}

// mid := the key of rank r (1-based) among the sample's node keys, by the
// whole block.  The keys are grouped by their top byte (k_bucket); the rank's
// bucket is found from the bucket offsets and the key inside it by an 8-bit
// radix select over the remaining 56 bits.
__device__ u64 select_rank(const Group& g, u32 s, u32 r) {
  __shared__ u32 hist[256];
  __shared__ u32 bk_sh, rank_sh;
  __shared__ u64 pre_sh;
  const u32* nb = g.nbkt + (size_t)s * (NBKT + 1);
  const u64* K = g.nkey_b + (size_t)s * g.cap_nodes;
  if (threadIdx.x == 0) bk_sh = 0;
  __syncthreads();
  for (u32 b = threadIdx.x; b < NBKT; b += blockDim.x)
    if (nb[b] < r && r <= nb[b + 1]) bk_sh = b;
  __syncthreads();
  const u32 nn = min(g.st[s].n_nodes, g.cap_nodes);
  const u32 bk = bk_sh, k0 = min(nb[bk], nn), k1 = min(nb[bk + 1], nn);
  u64 pre = (u64)bk << 56, mask = 0xFFull << 56;
  u32 rank = r - k0;
  for (int shift = 48; shift >= 0; shift -= 8) {
    for (u32 i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (u32 i = k0 + threadIdx.x; i < k1; i += blockDim.x) {
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
  return pre;
}

// After a probe: one block per sample takes the bisection step and, if the
// search goes on, selects the key of the next rank as the next threshold.
__global__ void __launch_bounds__(256) k_search_decide(Group g, u32 probe_cap, u32* n_open) {
  __shared__ u32 go;
  const u32 s = blockIdx.x;
  SampleState& st = g.st[s];
  if (st.sdone) return;
  if (threadIdx.x == 0) go = search_step(g, st, probe_cap, n_open) ? 1u : 0u;
  __syncthreads();
  if (!go) return;
  const u64 mid = select_rank(g, s, st.cnt_mid);
  if (threadIdx.x == 0) st.mid = mid;
}

}  // namespace rsak
