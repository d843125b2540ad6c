// rsa.cu -- host engine and C ABI (include/rsa.h) of the GB300 RSA library.
//
// One handle = one lattice shape (L, k).  A run processes a batch of samples
// in lock-step: every kernel takes the whole batch (grid.y = sample), so one
// launch covers all samples and per-sample "done" flags let finished samples
// drop out.  The data-dependent loops (greedy rounds, bisection probes) are
// driven from the host with one small device->host read per few iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rsa.h"
#include "rsa_kernels.cuh"

using namespace rsak;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(RSA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

constexpr size_t ALIGN = 256;
constexpr u32 ROUND_CHECK = 4;   // greedy rounds between host checks
constexpr u32 PROBE_CHECK = 4;   // bisection probes between host checks
constexpr u32 PROBE_CAP = 72;    // 64-bit bisection plus the initial probe
constexpr size_t SMEM_BUDGET = 160 * 1024;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t occ, owner, cmin, base, node_key, node_idx, uf, edges, st, seeds, counters, keys,
      scratch, total;
};

struct Geometry {
  RowCfg row;
  ColCfg col;
  u32 row_threads, col_threads;
  size_t row_smem, col_smem;
  dim3 row_grid_x, col_grid_x;  // .x only
  size_t scratch_words;         // per sample
};

u32 cap_nodes_of(u32 L, u32 k) { return (u32)(((u64)L * L) / k); }
u32 cap_edges_of(u32 L, u32 k) {
  u64 LL = (u64)L * L;
  u64 c = std::min<u64>(2 * LL, 6ull * cap_nodes_of(L, k) + 4ull * L) + 64;
  return (u32)c;
}

Geometry plan(u32 L, u32 k) {
  Geometry G{};
  // ---- row pass: one warp per (row, segment) ----
  RowCfg& r = G.row;
  r.S = L <= 4096 ? L : 4096;
  r.nseg = (L + r.S - 1) / r.S;
  r.nmax = r.S + k - 1;
  r.warp_words = 2 * r.nmax;
  size_t warp_bytes = (size_t)r.warp_words * 8;
  if (warp_bytes <= 200 * 1024) {
    r.global_scratch = 0;
    r.warps = (u32)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / warp_bytes));
    G.row_smem = warp_bytes * r.warps;
    G.row_grid_x = dim3((unsigned)(((u64)L * r.nseg + r.warps - 1) / r.warps));
  } else {
    r.global_scratch = 1;
    r.warps = 8;
    G.row_smem = 0;
    G.row_grid_x = dim3(16);
  }
  G.row_threads = 32 * r.warps;
  // ---- column pass: W columns x S rows per block ----
  ColCfg& c = G.col;
  const u32 T = 256;
  u32 W = k <= 64 ? 32 : k <= 256 ? 16 : k <= 1024 ? 8 : k <= 2048 ? 4 : 2;
  c.W = W;
  auto bytes_for = [&](u32 S) {
    size_t nmax = (size_t)S + k - 1, nocc = (size_t)S + 2 * k - 2;
    size_t a_words = std::max(nmax * W, (nocc * W + 1) / 2);
    size_t Gc = T / W;
    size_t words = a_words + nmax * W + Gc * W + (Gc * W + 7) / 8;
    return words * 8;
  };
  u32 S = std::min<u32>(L, 1024);
  while (S > 32 && bytes_for(S) > SMEM_BUDGET) S /= 2;
  c.S = S;
  c.nseg = (L + S - 1) / S;
  c.nstrip = (L + W - 1) / W;
  c.nmax = S + k - 1;
  c.nocc = S + 2 * k - 2;
  size_t bb = bytes_for(S);
  c.block_words = (u32)(bb / 8);
  G.col_threads = T;
  if (bb <= 200 * 1024) {
    c.global_scratch = 0;
    G.col_smem = bb;
    G.col_grid_x = dim3(c.nstrip * c.nseg);
  } else {
    c.global_scratch = 1;
    G.col_smem = 0;
    G.col_grid_x = dim3(16);
  }
  size_t row_scr = r.global_scratch ? (size_t)G.row_grid_x.x * r.warps * r.warp_words : 0;
  size_t col_scr = c.global_scratch ? (size_t)G.col_grid_x.x * c.block_words : 0;
  G.scratch_words = std::max(row_scr, col_scr);
  return G;
}

Layout layout_of(u32 L, u32 k, u32 n, bool with_keys, const Geometry& G) {
  Layout l{};
  const u64 LL = (u64)L * L;
  const size_t cn = cap_nodes_of(L, k), ce = cap_edges_of(L, k);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  l.occ = take(n * LL);
  l.owner = take(n * LL * 4);
  l.cmin = take(n * LL * 8);
  l.base = take((size_t)n * 8);
  l.node_key = take(n * cn * 8);
  l.node_idx = take(n * cn * 4);
  l.uf = take(n * cn * 16);
  l.edges = take(n * ce * sizeof(Edge));
  l.st = take((size_t)n * sizeof(SampleState));
  l.seeds = take((size_t)n * 8);
  l.counters = take(64);
  l.keys = take(with_keys ? 2 * LL * 8 : 0);
  // scratch blocks are indexed by (sample, block) in the kernels
  l.scratch = take(G.scratch_words * 8 * n);
  l.total = off;
  return l;
}

template <typename F>
int set_smem(F* fn, size_t bytes) {
  if (bytes > 48 * 1024)
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return 0;
}

}  // namespace

struct rsa {
  u32 L, k;
  u64 seed;
  Geometry geo;
  // device memory owned by the library
  void* own_ptr = nullptr;
  size_t own_bytes = 0;
  // caller-bound workspace
  void* bound_ptr = nullptr;
  size_t bound_bytes = 0;
  // last run
  void* ws = nullptr;
  Layout lay{};
  u32 last_n = 0;
  bool with_keys = false;
  cudaStream_t stream = nullptr;
  u32* h_counter = nullptr;  // pinned
  int device = -1;
};

namespace {

int ensure_workspace(rsa_t* h, u32 n, bool with_keys) {
  Layout l = layout_of(h->L, h->k, n, with_keys, h->geo);
  if (h->bound_ptr) {
    if (l.total > h->bound_bytes)
      return fail(RSA_ENOMEM, "bound workspace too small: need " + std::to_string(l.total) +
                                  " bytes, have " + std::to_string(h->bound_bytes));
    h->ws = h->bound_ptr;
  } else {
    if (l.total > h->own_bytes) {
      if (h->own_ptr) cudaFree(h->own_ptr);
      h->own_ptr = nullptr;
      h->own_bytes = 0;
      cudaError_t e = cudaMalloc(&h->own_ptr, l.total);
      if (e != cudaSuccess) {
        cudaGetLastError();
        h->own_ptr = nullptr;
        return fail(RSA_ENOMEM, "cudaMalloc(" + std::to_string(l.total) +
                                    ") failed: " + cudaGetErrorString(e));
      }
      h->own_bytes = l.total;
    }
    h->ws = h->own_ptr;
  }
  h->lay = l;
  return 0;
}

Group group_of(rsa_t* h, u32 n) {
  char* b = static_cast<char*>(h->ws);
  const Layout& l = h->lay;
  Group g{};
  g.L = h->L;
  g.k = h->k;
  g.n = n;
  g.cap_nodes = cap_nodes_of(h->L, h->k);
  g.cap_edges = cap_edges_of(h->L, h->k);
  g.LL = (u64)h->L * h->L;
  g.occ = reinterpret_cast<u8*>(b + l.occ);
  g.owner = reinterpret_cast<u32*>(b + l.owner);
  g.cmin = reinterpret_cast<u64*>(b + l.cmin);
  g.base = reinterpret_cast<u64*>(b + l.base);
  g.keys = h->with_keys ? reinterpret_cast<const u64*>(b + l.keys) : nullptr;
  g.node_key = reinterpret_cast<u64*>(b + l.node_key);
  g.node_idx = reinterpret_cast<u32*>(b + l.node_idx);
  g.uf = reinterpret_cast<u64*>(b + l.uf);
  g.edges = reinterpret_cast<Edge*>(b + l.edges);
  g.st = reinterpret_cast<SampleState*>(b + l.st);
  g.scratch = reinterpret_cast<u64*>(b + l.scratch);
  return g;
}

int launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(RSA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return 0;
}

int read_counter(rsa_t* h, u32* dev_counter, u32* out) {
  CUDA_TRY(cudaMemcpyAsync(h->h_counter, dev_counter, 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  *out = *h->h_counter;
  return 0;
}

int run_impl(rsa_t* h, const uint64_t* seeds, u32 n, const uint64_t* keys, cudaStream_t stream) {
  if (n == 0) return fail(RSA_EINVAL, "n_samples must be >= 1");
  int rc;
  CUDA_TRY(cudaGetDevice(&h->device));
  if (!h->h_counter) CUDA_TRY(cudaMallocHost(&h->h_counter, 16));
  h->with_keys = keys != nullptr;
  if ((rc = ensure_workspace(h, n, h->with_keys))) return rc;
  h->stream = stream;
  h->last_n = n;
  Group g = group_of(h, n);
  const Geometry& G = h->geo;
  const Layout& l = h->lay;
  char* b = static_cast<char*>(h->ws);
  u64* d_seeds = reinterpret_cast<u64*>(b + l.seeds);
  u32* d_counter = reinterpret_cast<u32*>(b + l.counters);
  const u64 LL = g.LL;

  CUDA_TRY(cudaMemcpyAsync(d_seeds, seeds, (size_t)n * 8, cudaMemcpyHostToDevice, stream));
  if (keys)
    CUDA_TRY(cudaMemcpyAsync(b + l.keys, keys, 2 * LL * 8, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemsetAsync(g.occ, 0, (size_t)n * LL, stream));
  CUDA_TRY(cudaMemsetAsync(g.owner, 0xFF, (size_t)n * LL * 4, stream));
  k_init<<<(n + 127) / 128, 128, 0, stream>>>(g, d_seeds);
  if ((rc = launch_check("k_init"))) return rc;

  if ((rc = set_smem(k_row<0>, G.row_smem))) return rc;
  if ((rc = set_smem(k_row<1>, G.row_smem))) return rc;
  if ((rc = set_smem(k_col<0>, G.col_smem))) return rc;
  if ((rc = set_smem(k_col<1>, G.col_smem))) return rc;
  const dim3 rg(G.row_grid_x.x, n), cg(G.col_grid_x.x, n);
  // every round accepts at least the smallest live key, so n_j + 1 rounds
  // always suffice
  const u32 round_cap = cap_nodes_of(h->L, h->k) + 2;
  for (u32 r = 0;; ++r) {
    CUDA_TRY(cudaMemsetAsync(d_counter, 0, 4, stream));
    k_row<0><<<rg, G.row_threads, G.row_smem, stream>>>(g, G.row);
    k_col<0><<<cg, G.col_threads, G.col_smem, stream>>>(g, G.col);
    k_row<1><<<rg, G.row_threads, G.row_smem, stream>>>(g, G.row);
    k_col<1><<<cg, G.col_threads, G.col_smem, stream>>>(g, G.col);
    k_round_end<<<(n + 127) / 128, 128, 0, stream>>>(g, round_cap, d_counter);
    if ((rc = launch_check("round kernels"))) return rc;
    if ((r + 1) % ROUND_CHECK == 0) {
      u32 active;
      if ((rc = read_counter(h, d_counter, &active))) return rc;
      if (active == 0) break;
    }
  }
  // contact graph of the jammed lattice
  {
    u32 bx = (u32)std::min<u64>((LL + 255) / 256, 4096);
    k_edges<<<dim3(bx, n), 256, 0, stream>>>(g);
    if ((rc = launch_check("k_edges"))) return rc;
  }
  // bisection for the first wrap
  k_search_init<<<(n + 127) / 128, 128, 0, stream>>>(g);
  {
    u32 bx = (u32)std::min<u64>(((u64)g.cap_nodes + 255) / 256, 1024);
    k_uf_identity<<<dim3(bx, n), 256, 0, stream>>>(g);
  }
  if ((rc = launch_check("search init"))) return rc;
  const u32 copy_bx = (u32)std::min<u64>(((u64)g.cap_nodes + 255) / 256, 1024);
  const u32 probe_bx = (u32)std::min<u64>(((u64)g.cap_edges + 255) / 256, 512);
  for (u32 p = 0; p < PROBE_CAP + 1; ++p) {
    CUDA_TRY(cudaMemsetAsync(d_counter + 1, 0, 4, stream));
    k_probe_copy<<<dim3(copy_bx, n), 256, 0, stream>>>(g);
    k_probe<<<dim3(probe_bx, n), 256, 0, stream>>>(g);
    k_search_decide<<<(n + 127) / 128, 128, 0, stream>>>(g, PROBE_CAP, d_counter + 1);
    if ((rc = launch_check("probe kernels"))) return rc;
    if ((p + 1) % PROBE_CHECK == 0) {
      u32 open;
      if ((rc = read_counter(h, d_counter + 1, &open))) return rc;
      if (open == 0) break;
    }
  }
  return 0;
}

int status_code(u32 bits) {
  if (bits & ST_NOWRAP) return RSA_ENOWRAP;
  if (bits & (ST_UF_CAP | ST_SEARCH_CAP | ST_ROUND_CAP)) return RSA_ETIMEOUT;
  if (bits & (ST_NODE_OVF | ST_EDGE_OVF)) return RSA_ENOMEM;
  if (bits & ST_SEARCH_BAD) return RSA_ETIMEOUT;
  return 0;
}

int fetch_states(rsa_t* h, std::vector<SampleState>& out) {
  if (!h->ws || h->last_n == 0) return fail(RSA_ESTATE, "no run to read");
  out.resize(h->last_n);
  const char* b = static_cast<const char*>(h->ws);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(out.data(), b + h->lay.st, sizeof(SampleState) * h->last_n,
                      cudaMemcpyDeviceToHost));
  return 0;
}

}  // namespace

extern "C" {

int rsa_create(uint32_t L, uint32_t k, uint64_t seed, rsa_t** out) {
  if (!out) return fail(RSA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!(k >= 1 && k <= L && L <= 32768))
    return fail(RSA_EINVAL, "need 1 <= k <= L <= 32768");
  rsa_t* h = new (std::nothrow) rsa_t();
  if (!h) return fail(RSA_ENOMEM, "host allocation failed");
  h->L = L;
  h->k = k;
  h->seed = seed;
  h->geo = plan(L, k);
  *out = h;
  g_err.clear();
  return 0;
}

int rsa_run_seeds(rsa_t* h, const uint64_t* seeds, uint32_t n, void* stream) {
  if (!h || !seeds) return fail(RSA_EINVAL, "null handle or seeds");
  return run_impl(h, seeds, n, nullptr, static_cast<cudaStream_t>(stream));
}

int rsa_run_batch(rsa_t* h, uint32_t n_samples, void* stream) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  std::vector<uint64_t> seeds(n_samples);
  for (uint32_t i = 0; i < n_samples; ++i) seeds[i] = h->seed + i;
  return run_impl(h, seeds.data(), n_samples, nullptr, static_cast<cudaStream_t>(stream));
}

int rsa_run_keys(rsa_t* h, const uint64_t* keys, void* stream) {
  if (!h || !keys) return fail(RSA_EINVAL, "null handle or keys");
  const u64 n = 2ull * h->L * h->L;
  std::vector<uint64_t> sorted(keys, keys + n);
  std::sort(sorted.begin(), sorted.end());
  for (u64 i = 0; i < n; ++i) {
    if (sorted[i] == KEY_NONE) return fail(RSA_EINVAL, "key 2^64-1 is reserved");
    if (i && sorted[i] == sorted[i - 1]) return fail(RSA_EINVAL, "keys are not distinct");
  }
  uint64_t seed = h->seed;
  return run_impl(h, &seed, 1, keys, static_cast<cudaStream_t>(stream));
}

int rsa_results(rsa_t* h, uint32_t* n_j, uint32_t* n_c, uint32_t n) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (n > h->last_n) return fail(RSA_EINVAL, "n exceeds samples of the last run");
  std::vector<SampleState> st;
  int rc = fetch_states(h, st);
  if (rc) return rc;
  int first = 0;
  for (u32 i = 0; i < n; ++i) {
    if (n_j) n_j[i] = st[i].n_nodes;
    if (n_c) n_c[i] = st[i].nc;
    int c = status_code(st[i].status);
    if (c && !first) {
      first = c;
      g_err = "sample " + std::to_string(i) + " status bits " + std::to_string(st[i].status);
    }
  }
  return first;
}

int rsa_sample_stats(rsa_t* h, uint32_t* rounds, uint32_t* probes, uint32_t* edges,
                     int32_t* status, uint32_t n) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (n > h->last_n) return fail(RSA_EINVAL, "n exceeds samples of the last run");
  std::vector<SampleState> st;
  int rc = fetch_states(h, st);
  if (rc) return rc;
  for (u32 i = 0; i < n; ++i) {
    if (rounds) rounds[i] = st[i].rounds;
    if (probes) probes[i] = st[i].probes;
    if (edges) edges[i] = st[i].n_edges;
    if (status) status[i] = status_code(st[i].status);
  }
  return 0;
}

int rsa_accepted(rsa_t* h, uint32_t sample, uint32_t* idx, uint32_t cap, uint32_t* count) {
  if (!h || !count) return fail(RSA_EINVAL, "null argument");
  if (sample >= h->last_n) return fail(RSA_EINVAL, "sample out of range");
  std::vector<SampleState> st;
  int rc = fetch_states(h, st);
  if (rc) return rc;
  const u32 cn = cap_nodes_of(h->L, h->k);
  const u32 nj = std::min(st[sample].n_nodes, cn);
  std::vector<uint32_t> v(nj);
  const char* b = static_cast<const char*>(h->ws);
  if (nj)
    CUDA_TRY(cudaMemcpy(v.data(), b + h->lay.node_idx + (size_t)sample * cn * 4, (size_t)nj * 4,
                        cudaMemcpyDeviceToHost));
  std::sort(v.begin(), v.end());
  *count = nj;
  if (idx) std::memcpy(idx, v.data(), (size_t)std::min(cap, nj) * 4);
  return 0;
}

int rsa_workspace_bytes(uint32_t L, uint32_t k, uint32_t n_samples, uint64_t* bytes) {
  if (!bytes || !(k >= 1 && k <= L && L <= 32768) || n_samples == 0)
    return fail(RSA_EINVAL, "bad arguments");
  Geometry G = plan(L, k);
  *bytes = layout_of(L, k, n_samples, false, G).total;
  return 0;
}

int rsa_bind_workspace(rsa_t* h, void* dev_ptr, uint64_t bytes) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) % ALIGN))
    return fail(RSA_EINVAL, "workspace must be 256-byte aligned");
  h->bound_ptr = dev_ptr;
  h->bound_bytes = dev_ptr ? bytes : 0;
  return 0;
}

void rsa_destroy(rsa_t* h) {
  if (!h) return;
  if (h->own_ptr) cudaFree(h->own_ptr);
  if (h->h_counter) cudaFreeHost(h->h_counter);
  delete h;
}

const char* rsa_last_error(void) { return g_err.c_str(); }

}  // extern "C"
