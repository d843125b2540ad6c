// rsa_small.cuh -- one CTA runs one whole sample in shared memory (small
// lattices: L <= SMALL_LMAX and at most SMALL_NMAX k-mers), sm_103a.
//
// The same exact method as the tiled and long-k paths (Sec. II.B to II.D of
// arXiv:1810.06800 recast as a round-parallel greedy over splitmix64
// priorities), but with every structure of the sample in the CTA's shared
// memory, so all greedy rounds and the whole first-wrap search run inside
// one launch with no host round trip:
//   round:  live bits of every candidate (its k cells free) per row and per
//           column; per cell the smallest live priority covering it (direct
//           window minima, priorities recomputed, never stored); every live
//           candidate that is that minimum on all of its k cells is accepted
//           (accepted candidates of one round never overlap) and occupies
//           its cells;
//   n_c:    contacts between k-mers read off the owner grid; bisection over
//           the number m of placed k-mers, each probe a union-find over the
//           contacts among the first m k-mers with 16-bit periodic offsets
//           (a non-zero mismatch inside one cluster is a wrap).
// The kernel is persistent over a job table: each CTA takes the next sample
// from a global counter, so samples of different (L, k) share one launch.
#pragma once
#include "rsa_device.cuh"

namespace rsak {

constexpr u32 SMALL_LMAX = 128;
constexpr u32 SMALL_NMAX = 4096;  // k-mers of a sample: L^2 / k
constexpr u16 SMALL_NONE = 0xFFFFu;

struct SmallJob {  // one sample
  u32 L, k;
  u64 seed;
};
struct SmallOut {  // its results
  u32 n_j, n_c, rounds, status;
};

// Shared-memory carve-up for lattices up to Lm (words per bit row: Lm / 32
// rounded up).  The per-cell minima (8 B per cell) are no longer needed once
// the sample is jammed; the union-find words and the sorted node priorities
// of the first-wrap search reuse that space.
struct SmallSmem {
  u64* cmin;    // [Lm^2] per-cell minimum; after jamming: uf [NMAX] + sorted keys [NMAX]
  u64* nkey;    // [NMAX] node priorities (acceptance order)
  u32* npos;    // [NMAX] o << 31 | y0 << 15 | x0 of the node's anchor
  u32* rowb;    // [Lm][W] occupancy, row-major bits
  u32* colb;    // [Lm][W] occupancy, column-major bits
  u32* liveH;   // [Lm][W] live horizontal anchors per row
  u32* liveV;   // [Lm][W] live vertical anchors per column
  u16* owner;   // [Lm^2] node of the cell or SMALL_NONE
};
__host__ __device__ inline u32 small_words(u32 Lm) { return (Lm + 31) / 32; }
__host__ __device__ inline size_t small_smem_bytes(u32 Lm) {
  const size_t LL = (size_t)Lm * Lm, W = small_words(Lm);
  const size_t cmin = LL * 8 > 2 * SMALL_NMAX * 8 ? LL * 8 : 2 * SMALL_NMAX * 8;
  return cmin + SMALL_NMAX * 12 + 4 * Lm * W * 4 + LL * 2 + 64;
}
__device__ inline SmallSmem small_smem(unsigned char* raw, u32 Lm) {
  const size_t LL = (size_t)Lm * Lm, W = small_words(Lm);
  const size_t cmin = LL * 8 > 2 * SMALL_NMAX * 8 ? LL * 8 : 2 * SMALL_NMAX * 8;
  SmallSmem m;
  m.cmin = reinterpret_cast<u64*>(raw);
  m.nkey = reinterpret_cast<u64*>(raw + cmin);
  m.npos = reinterpret_cast<u32*>(m.nkey + SMALL_NMAX);
  m.rowb = m.npos + SMALL_NMAX;
  m.colb = m.rowb + Lm * W;
  m.liveH = m.colb + Lm * W;
  m.liveV = m.liveH + Lm * W;
  m.owner = reinterpret_cast<u16*>(m.liveV + Lm * W);
  return m;
}

// Bits x .. x + n - 1 (around a circular line of L bits) of a bit row.
__device__ __forceinline__ bool small_run_free(const u32* row, u32 L, u32 x, u32 n) {
  u32 p = x;
  while (n) {
    const u32 b = p & 31u, take = min(min(32u - b, n), L - p);
    const u32 m = take == 32 ? 0xFFFFFFFFu : ((1u << take) - 1u);
    if ((row[p >> 5] >> b) & m) return false;
    n -= take;
    p += take;
    if (p == L) p = 0;
  }
  return true;
}

__device__ __forceinline__ bool small_bit(const u32* row, u32 i) { return (row[i >> 5] >> (i & 31u)) & 1u; }

// Union-find on shared-memory words {parent, dx:16, dy:16} (the global
// path's layout), walks and link retries capped at `cap` steps.
__device__ __forceinline__ u32 small_find(u64* W, u32 x, u32* ox, u32* oy, bool* capped, u32 cap) {
  u32 sx = 0, sy = 0;
  for (u32 it = 0; it < cap; ++it) {
    const u64 wx = *(volatile u64*)(W + x);
    const u32 p = (u32)wx;
    if (p == x) {
      *ox = sx;
      *oy = sy;
      return x;
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

__device__ bool small_union(u64* W, u32 m1, u32 m2, u32 dxy, bool* capped, u32 cap) {
  const u32 dx = dxy & 0xFFFFu, dy = dxy >> 16;
  for (u32 it = 0; it < cap; ++it) {
    u32 o1x, o1y, o2x, o2y;
    const u32 r1 = small_find(W, m1, &o1x, &o1y, capped, cap);
    const u32 r2 = small_find(W, m2, &o2x, &o2y, capped, cap);
    if (*capped) return false;
    const u32 Dx = o1x + dx - o2x, Dy = o1y + dy - o2y;  // r2 relative to r1
    if (r1 == r2) return ((Dx | Dy) & 0xFFFFu) != 0;
    // the larger root goes under the smaller one, with its offset from it
    const u32 hi = r1 < r2 ? r2 : r1;
    const u64 want = uf_pack(hi, 0, 0);
    const u64 link = r1 < r2 ? uf_pack(r1, Dx, Dy) : uf_pack(r2, 0u - Dx, 0u - Dy);
    if (atomicCAS((unsigned long long*)(W + hi), want, link) == want) return false;
  }
  *capped = true;
  return false;
}

// Cell i of the k-mer of node n (anchor packed as o << 31 | y0 << 15 | x0).
__device__ __forceinline__ u32 small_cell(u32 pos, u32 L, u32 i) {
  const u32 o = pos >> 31, y0 = (pos >> 15) & 0x7FFFu, x0 = pos & 0x7FFFu;
  u32 y = y0, x = x0;
  if (o == 0) { x += i; if (x >= L) x -= L; }
  else { y += i; if (y >= L) y -= L; }
  return y * L + x;
}

// One sample per CTA, persistent over the job table.  out[j] receives n_j,
// n_c, the number of greedy rounds and the status bits of job j.  Every
// loop is bounded: rounds by n_j + 2, union-find walks by uf_cap.
__global__ void __launch_bounds__(1024) k_small(const SmallJob* jobs, u32 n_jobs, SmallOut* out,
                                                u32* next, u32 Lm, u32 uf_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmallSmem m = small_smem(smem_raw, Lm);
  __shared__ u32 item_sh, nn_sh, status_sh;
  const u32 tid = threadIdx.x, nt = blockDim.x, W = small_words(Lm);
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(next, 1u);
    __syncthreads();
    const u32 it = item_sh;
    if (it >= n_jobs) return;
    const SmallJob J = jobs[it];
    const u32 L = J.L, k = J.k, LL = L * L;
    const u64 zb = mix64(J.seed + SM_GAMMA) + SM_GAMMA;  // key(idx) = mix64(zb + gamma idx)
    for (u32 i = tid; i < Lm * W; i += nt) m.rowb[i] = m.colb[i] = 0;
    for (u32 i = tid; i < LL; i += nt) m.owner[i] = SMALL_NONE;
    if (tid == 0) { nn_sh = 0; status_sh = 0; }
    __syncthreads();
    const u32 round_cap = LL / k + 2;
    u32 rounds = 0;
    for (;;) {
      // (a) live anchors: a candidate is live iff its k cells are free
      for (u32 i = tid; i < Lm * W; i += nt) m.liveH[i] = m.liveV[i] = 0;
      __syncthreads();
      bool any = false;
      for (u32 c = tid; c < 2 * LL; c += nt) {
        const u32 o = c >= LL, r = c - o * LL, y = r / L, x = r - y * L;
        const bool live = o == 0 ? small_run_free(m.rowb + y * W, L, x, k)
                                 : small_run_free(m.colb + x * W, L, y, k);
        if (live) {
          any = true;
          if (o == 0) atomicOr(m.liveH + y * W + (x >> 5), 1u << (x & 31u));
          else atomicOr(m.liveV + x * W + (y >> 5), 1u << (y & 31u));
        }
      }
      if (!__syncthreads_or(any)) break;  // jammed
      if (rounds >= round_cap) {
        if (tid == 0) status_sh |= ST_ROUND_CAP;
        break;
      }
      // (b) per cell, the smallest live priority covering it
      for (u32 cell = tid; cell < LL; cell += nt) {
        const u32 y = cell / L, x = cell - y * L;
        u64 mn = KEY_NONE;
        for (u32 i = 0; i < k; ++i) {
          const u32 a = x >= i ? x - i : x + L - i;
          if (small_bit(m.liveH + y * W, a)) mn = tmin(mn, mix64(zb + SM_GAMMA * (u64)(y * L + a)));
          const u32 b = y >= i ? y - i : y + L - i;
          if (small_bit(m.liveV + x * W, b))
            mn = tmin(mn, mix64(zb + SM_GAMMA * ((u64)LL + b * L + x)));
        }
        m.cmin[cell] = mn;
      }
      __syncthreads();
      // (c) a live candidate that is the minimum on all of its cells is
      // accepted; accepted ones never overlap, so each occupies its cells
      for (u32 c = tid; c < 2 * LL; c += nt) {
        const u32 o = c >= LL, r = c - o * LL, y = r / L, x = r - y * L;
        if (!small_bit(o == 0 ? m.liveH + y * W : m.liveV + x * W, o == 0 ? x : y)) continue;
        const u64 key = mix64(zb + SM_GAMMA * (u64)c);
        const u32 pos = (o << 31) | (y << 15) | x;
        bool ok = true;
        for (u32 i = 0; i < k && ok; ++i) ok = m.cmin[small_cell(pos, L, i)] == key;
        if (!ok) continue;
        const u32 node = atomicAdd(&nn_sh, 1u);
        if (node >= SMALL_NMAX) {
          atomicOr(&status_sh, ST_NODE_OVF);
          continue;
        }
        m.nkey[node] = key;
        m.npos[node] = pos;
        for (u32 i = 0; i < k; ++i) {
          const u32 cl = small_cell(pos, L, i), cy = cl / L, cx = cl - cy * L;
          atomicOr(m.rowb + cy * W + (cx >> 5), 1u << (cx & 31u));
          atomicOr(m.colb + cx * W + (cy >> 5), 1u << (cy & 31u));
          m.owner[cl] = (u16)node;
        }
      }
      __syncthreads();
      ++rounds;
    }
    const u32 nj = min(nn_sh, SMALL_NMAX);
    // ---- first wrap: bisection over m, the number of k-mers placed ----
    u64* uf = m.cmin;                 // the per-cell minima are no longer needed
    u64* srt = m.cmin + SMALL_NMAX;   // node priorities, ascending
    u32 P2 = 1;
    while (P2 < nj) P2 <<= 1;
    for (u32 i = tid; i < P2; i += nt) srt[i] = i < nj ? m.nkey[i] : KEY_NONE;
    __syncthreads();
    for (u32 kk = 2; kk <= P2; kk <<= 1)
      for (u32 j = kk >> 1; j > 0; j >>= 1) {
        for (u32 i = tid; i < P2; i += nt) {
          const u32 ixj = i ^ j;
          if (ixj > i) {
            const u64 a = srt[i], b = srt[ixj];
            if ((a > b) == ((i & kk) == 0)) { srt[i] = b; srt[ixj] = a; }
          }
        }
        __syncthreads();
      }
    // wrap(mm): do the contacts among the first mm k-mers close a cycle of
    // non-zero winding?  A contact is a lattice edge (cell, cell + x / + y)
    // between two occupied cells; its time is the larger of the two nodes'
    // priorities.
    auto probe = [&](u32 mm) -> bool {
      const u64 T = srt[mm - 1];
      for (u32 j = tid; j < nj; j += nt) uf[j] = uf_pack(j, 0, 0);
      __syncthreads();
      bool wrap = false, capped = false;
      for (u32 cell = tid; cell < LL; cell += nt) {
        const u32 na = m.owner[cell];
        if (na == SMALL_NONE) continue;
        const u32 y = cell / L, x = cell - y * L;
        for (u32 dir = 0; dir < 2; ++dir) {
          const u32 by = dir ? (y + 1 == L ? 0 : y + 1) : y, bx = dir ? x : (x + 1 == L ? 0 : x + 1);
          const u32 nb = m.owner[by * L + bx];
          if (nb == SMALL_NONE) continue;
          if (tmax(m.nkey[na], m.nkey[nb]) > T) continue;
          // lifted anchor(nb) - anchor(na) across this contact
          u32 oa, ob;
          const u32 i = pos_in_kmer(m.npos[na], y, x, L, &oa);
          const u32 j = pos_in_kmer(m.npos[nb], by, bx, L, &ob);
          const int dx = (oa == 0 ? (int)i : 0) + (dir == 0) - (ob == 0 ? (int)j : 0);
          const int dy = (oa == 1 ? (int)i : 0) + (dir == 1) - (ob == 1 ? (int)j : 0);
          if (na == nb && dx == 0 && dy == 0) continue;  // inside one k-mer
          const u32 dxy = ((u32)dx & 0xFFFFu) | (((u32)dy & 0xFFFFu) << 16);
          if (small_union(uf, na, nb, dxy, &capped, uf_cap)) wrap = true;
        }
      }
      if (__syncthreads_or(capped) && tid == 0) status_sh |= ST_UF_CAP;
      return __syncthreads_or(wrap);
    };
    u32 nc = NONE32, probes = 0;
    if (nj > 0 && !(status_sh & (ST_ROUND_CAP | ST_NODE_OVF))) {
      ++probes;
      if (!probe(nj)) {
        if (tid == 0) status_sh |= ST_NOWRAP;
      } else {
        u32 lo = 0, hi = nj;  // wrap(lo) is false, wrap(hi) true
        while (hi - lo > 1 && !(status_sh & ST_UF_CAP)) {
          const u32 mid = lo + (hi - lo) / 2;
          ++probes;
          if (probe(mid)) hi = mid;
          else lo = mid;
        }
        nc = hi;
      }
    }
    __syncthreads();
    if (tid == 0) {
      SmallOut r;
      r.n_j = nj;
      r.n_c = (status_sh & (ST_UF_CAP | ST_NOWRAP)) ? NONE32 : nc;
      r.rounds = rounds;
      r.status = status_sh;
      out[it] = r;
    }
    __syncthreads();
  }
}

}  // namespace rsak
