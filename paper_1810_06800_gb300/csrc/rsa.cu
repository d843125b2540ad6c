// rsa.cu -- host engine and C ABI (include/rsa.h) of the GB300 RSA library.
//
// One handle = one lattice shape (L, k).  A run processes a batch of samples
// in lock-step: every kernel takes the whole batch (grid.y = sample), so one
// launch covers all samples and per-sample "done" flags let finished samples
// drop out.  The data-dependent loops (greedy rounds, bisection probes) are
// driven from the host with one small device->host read per few iterations.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstddef>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rsa.h"
#include "rsa_kernels.cuh"
#include "rsa_tile.cuh"
#include "rsa_line.cuh"
#include "rsa_lwin.cuh"
#include "rsa_config.cuh"

using namespace rsak;

namespace {

// An NVTX range for the lifetime of a scope (a no-op unless a profiler that
// collects NVTX ranges is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

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
constexpr u32 ROUND_CHECK = 4;   // greedy rounds between host checks (default)
constexpr u32 PROBE_CHECK = 4;   // bisection probes between host checks
constexpr u32 PROBE_CAP = 40;    // rank bisection (<= 31 halvings) plus the initial probe
constexpr size_t SMEM_BUDGET = 160 * 1024;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t occ, occw, occT, cB, code16, code16T, cH, cV, masks, dead, owner, cmin, base, node_key, node_idx, node_pos, uf, edges, edges_b,
      ebkt, nkey_b, nbkt, st, seeds, counters, work, keys,
      scratch, total;
};

struct Geometry {
  bool tile;                    // power-of-two k <= 32 and L % 32 == 0
  bool line;                    // 32 <= k <= LINE_KMAX, L % 32 == 0, not tile
  LineCfg lc;
  // long-k lines made of whole k-blocks and whole CTA spans (rsa_lwin.cuh),
  // used for seeded priorities; caller priorities keep the lc kernels
  bool lw;
  LwinCfg lw_cfg;
  u32 lw_C;                     // cells per thread of k_lwin
  size_t line_smem, line_acc_smem, line_codes_smem;
  TileCfg tc;                   // (items filled per run)
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

bool tile_shape(u32 L, u32 k) { return k <= 32 && (k & (k - 1)) == 0 && L % 32 == 0; }

Geometry plan(u32 L, u32 k) {
  Geometry G{};
  G.tile = tile_shape(L, k);
  G.tc.T = L / 32;
  G.tc.T2 = G.tc.T * G.tc.T;
  G.line = !G.tile && L % 32 == 0 && k >= 32 && k <= LINE_KMAX;
  if (G.line) {
    // longest segment (multiple of 32, <= 4096) whose buffers stay near 100 KB,
    // so at least two blocks fit on an SM
    u32 S = std::min<u32>(L, 4096);
    while (S > 256 && line_smem_bytes(S + k - 1, S, k) > 100 * 1024) S -= 256;
    // very long windows: if that cap leaves segments shorter than k, take
    // S = k (rounded down to 32, at most L) with the one-array layout, which
    // halves the bytes per value: fewer halo values per output cell
    G.lc.compact = 0;
    if (S < k) {
      S = std::min<u32>(L, k & ~31u);
      G.lc.compact = 1;
    }
    G.lc.S = S;
    G.lc.nseg = (L + S - 1) / S;
    G.lc.nmax = S + k - 1;
    G.lc.T = L / 32;
    G.line_smem = line_smem_bytes(G.lc.nmax, S, k, G.lc.compact != 0);
    G.line_acc_smem = line_smem_bytes(G.lc.nmax, S, k);
    G.line_codes_smem = line_codes_smem_bytes(G.lc.nmax);
    const u32 P = std::min<u32>(L, 4096), C = P / LW_THREADS;
    G.lw = P % LW_THREADS == 0 && C >= 1 && C <= 16 && (C & (C - 1)) == 0 && L % P == 0 &&
           P % k == 0 && k % C == 0 && L / P <= 8;
    if (G.lw) {
      G.lw_cfg.P = P;
      G.lw_cfg.nc = L / P;
      G.lw_cfg.T = L / 32;
      G.lw_C = C;
    }
  }
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
  const bool bits = G.tile || G.line;
  const bool lw = G.lw && !with_keys;        // argmin-offset round (rsa_lwin.cuh)
  const bool lold = G.line && !lw;           // 8-byte minima round (rsa_line.cuh)
  l.occ = take(bits ? 0 : n * LL);
  l.occw = take(bits ? n * LL / 8 : 0);
  l.occT = take(G.line ? n * LL / 8 : 0);
  l.cB = take(lold ? n * LL * 8 : 0);
  l.code16 = take(lold ? n * LL * 2 : 0);
  l.code16T = take(lold ? n * LL * 2 : 0);
  l.cH = take(lw ? n * LL * 2 : 0);
  l.cV = take(lw ? n * LL * 2 : 0);
  // acceptance masks: win / first / last, rows then the transposed layout
  l.masks = take(lw ? 6 * (n * LL / 8) : 0);
  // dead flags: per 32 x 32 tile (tile path); per line segment (or span) of
  // each orientation, then per 32 x 32 code tile (long-k path; 32 x 32
  // combine squares on the argmin-offset path)
  const u32 nseg = lw ? G.lw_cfg.nc : G.lc.nseg;
  const size_t ncode = G.tc.T2;
  l.dead = take(G.tile ? (size_t)n * G.tc.T2
                       : G.line ? (size_t)n * (2ull * L * nseg + ncode) : 0);
  l.owner = take(n * LL * 4);
  // tile path: one argmin code byte per cell; none on the argmin-offset path
  l.cmin = take(n * LL * (G.tile ? 1 : lw ? 0 : 8));
  l.base = take((size_t)n * 8);
  l.node_key = take(n * cn * 8);
  l.node_idx = take(n * cn * 4);
  l.node_pos = take(n * cn * 4);
  l.uf = take(n * cn * 16);
  l.edges = take(n * ce * sizeof(Edge));
  l.edges_b = take(n * ce * sizeof(Edge));
  l.ebkt = take((size_t)n * (NBKT + 1) * 4);
  l.nkey_b = take(n * cn * 8);
  l.nbkt = take((size_t)n * (NBKT + 1) * 4);
  l.st = take((size_t)n * sizeof(SampleState));
  l.seeds = take((size_t)n * 8);
  l.counters = take(64);
  l.work = take(4 * WORK_SLOTS * 8);
  l.keys = take(with_keys ? 2 * LL * 8 : 0);
  // scratch blocks are indexed by (sample, block) in the kernels
  l.scratch = take(bits ? 0 : G.scratch_words * 8 * n);
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

// The thread's error message, set by the other translation units of the
// library (rsa_mix.cu) as well.
namespace rsa_detail {
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace rsa_detail

enum Kind {
  KD_INIT, KD_ROW_CMIN, KD_COL_CMIN, KD_ROW_ACCEPT, KD_COL_ACCEPT, KD_TILE_CMIN, KD_TILE_ACCEPT,
  KD_LINE_CMIN_H, KD_LINE_CMIN_V, KD_LINE_COMBINE, KD_LINE_ACCEPT_H, KD_LINE_ACCEPT_V,
  KD_LINE_CODES, KD_LWIN_H, KD_LWIN_V, KD_LCOMB, KD_LACC_H, KD_LACC_V,
  KD_ROUND_END, KD_EDGES, KD_BUCKET, KD_SEARCH_INIT, KD_PROBE_COPY, KD_PROBE, KD_DECIDE, KD_COUNT
};
const char* const kKindNames[KD_COUNT] = {
    "k_init",         "k_row_cmin",    "k_col_cmin",   "k_row_accept", "k_col_accept",
    "k_tile_cmin",    "k_tile_accept", "k_line_cmin_h", "k_line_cmin_v", "k_line_combine",
    "k_line_accept_h", "k_line_accept_v", "k_line_codes", "k_lwin_h", "k_lwin_v", "k_lcomb",
    "k_lacc_h",       "k_lacc_v",      "k_round_end",  "k_edges",      "k_bucket",     "k_search_init",
    "k_probe_copy",   "k_probe",       "k_search_decide"};

// Optional per-kernel timing with CUDA events recorded around each launch
// on the launch stream, plus launch counts (always kept).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;  // kind of record i uses events 2i, 2i+1
  unsigned long long launches[KD_COUNT] = {};
  double ms[KD_COUNT] = {};
};

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
  u32* h_counter = nullptr;  // pinned, 64 bytes: loop counters, configuration bits
  unsigned long long work[4] = {0, 0, 0, 0};  // accumulated round-pass work
  int device = -1;
  int sm_count = 0;
  int tile_blocks[2] = {0, 0};  // resident blocks per SM: cmin, accept
  Prof prof;
  // CUDA graphs of a chunk of greedy rounds and of bisection probes, captured
  // once per (workspace, batch size, key source) on a private stream and
  // replayed on the run's stream
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  // chunks the previous run needed before its samples were done: the next
  // run launches that many before its first device->host check
  u32 round_chunks_hint = 1, probe_chunks_hint = 1;
  u32 round_check = ROUND_CHECK;  // greedy rounds per graph chunk / host check
  u32 lw_threads = 256;           // CTA size of the long-k window pass (256 or 128;
                                  // rsa_create sets default_window_threads)
  // test-only lowered caps of the device loops (0 = default; rsa_test_caps)
  u32 t_round = 0, t_uf = 0, t_probe = 0, t_edges = 0;
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    const void* ws = nullptr;
    u32 n = 0;
    bool keys = false;
    u32 caps[6] = {0, 0, 0, 0, 0, 0};  // caps, rounds per chunk, window CTA size in the graph
    unsigned long long launches[32] = {};
  } g_round, g_probe;
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
  g.uf_cap = h->t_uf ? h->t_uf : UF_CAP;
  g.edge_limit = h->t_edges ? std::min(h->t_edges, g.cap_edges) : g.cap_edges;
  g.LL = (u64)h->L * h->L;
  g.occ = reinterpret_cast<u8*>(b + l.occ);
  g.owner = reinterpret_cast<u32*>(b + l.owner);
  g.cmin = reinterpret_cast<u64*>(b + l.cmin);
  g.base = reinterpret_cast<u64*>(b + l.base);
  g.keys = h->with_keys ? reinterpret_cast<const u64*>(b + l.keys) : nullptr;
  g.node_key = reinterpret_cast<u64*>(b + l.node_key);
  g.node_idx = reinterpret_cast<u32*>(b + l.node_idx);
  g.node_pos = reinterpret_cast<u32*>(b + l.node_pos);
  g.edges_b = reinterpret_cast<Edge*>(b + l.edges_b);
  g.ebkt = reinterpret_cast<u32*>(b + l.ebkt);
  g.nkey_b = reinterpret_cast<u64*>(b + l.nkey_b);
  g.nbkt = reinterpret_cast<u32*>(b + l.nbkt);
  g.uf = reinterpret_cast<u64*>(b + l.uf);
  g.edges = reinterpret_cast<Edge*>(b + l.edges);
  g.st = reinterpret_cast<SampleState*>(b + l.st);
  g.scratch = reinterpret_cast<u64*>(b + l.scratch);
  g.work = reinterpret_cast<u64*>(b + l.work);
  return g;
}

cudaEvent_t prof_event(Prof& p, size_t i) {
  while (p.pool.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p.pool.push_back(e);
  }
  return p.pool[i];
}

// Launch wrapper: counts launches and, when profiling is on, brackets the
// launch with two events on its stream.
template <typename K, typename... Args>
void launch(rsa_t* h, int kind, K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
            Args... args) {
  Prof& p = h->prof;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p.on) {
    size_t i = p.kinds.size();
    e0 = prof_event(p, 2 * i);
    e1 = prof_event(p, 2 * i + 1);
    if (e0 && e1) {
      cudaEventRecord(e0, st);
      p.kinds.push_back(kind);
    }
  }
  kernel<<<grid, block, smem, st>>>(args...);
  if (e0 && e1) cudaEventRecord(e1, st);
  p.launches[kind] += 1;
}

// As launch(), for a kernel launched in thread-block clusters of
// cluster_x CTAs along x.  Returns the launch's error.
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(rsa_t* h, int kind, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, u32 cluster_x, Args... args) {
  Prof& p = h->prof;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p.on) {
    size_t i = p.kinds.size();
    e0 = prof_event(p, 2 * i);
    e1 = prof_event(p, 2 * i + 1);
    if (e0 && e1) {
      cudaEventRecord(e0, st);
      p.kinds.push_back(kind);
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster_x;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e0 && e1) cudaEventRecord(e1, st);
  p.launches[kind] += 1;
  return e;
}

template <int F, int NT>
cudaError_t launch_lwin_nt(rsa_t* h, Group g, const Geometry& G, const u32* occw, const u32* occT,
                           u16* out, u8* lflag, u32 n, cudaStream_t st) {
  const dim3 grid(g.L * G.lw_cfg.nc, n), block(NT);
  const int kind = F == 0 ? KD_LWIN_H : KD_LWIN_V;
  const u32 nc = G.lw_cfg.nc, C = G.lw_cfg.P / NT;
  if constexpr (NT == 128) {
    if (C == 32) return launch_cluster(h, kind, k_lwin<F, 32, 128>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
    return launch_cluster(h, kind, k_lwin<F, 16, 128>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
  } else {
    switch (C) {
      case 1: return launch_cluster(h, kind, k_lwin<F, 1, 256>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
      case 2: return launch_cluster(h, kind, k_lwin<F, 2, 256>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
      case 4: return launch_cluster(h, kind, k_lwin<F, 4, 256>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
      case 8: return launch_cluster(h, kind, k_lwin<F, 8, 256>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
      default: return launch_cluster(h, kind, k_lwin<F, 16, 256>, grid, block, 0, st, nc, g, G.lw_cfg, occw, occT, out, lflag);
    }
  }
}

// The window pass with the handle's CTA size: 256 threads, or 128 threads
// with twice the cells per thread (spans of 2048 or 4096 cells).
template <int F>
cudaError_t launch_lwin(rsa_t* h, Group g, const Geometry& G, const u32* occw, const u32* occT,
                        u16* out, u8* lflag, u32 n, cudaStream_t st) {
  if (h->lw_threads == 128) return launch_lwin_nt<F, 128>(h, g, G, occw, occT, out, lflag, n, st);
  return launch_lwin_nt<F, 256>(h, g, G, occw, occT, out, lflag, n, st);
}

// Default CTA size of the long-k window pass: 128 threads x 32 cells on
// 4096-cell spans with k >= 512 (measured 3% faster than 256 x 16 at
// L = 8192, k = 512 and L = 32768, k = 4096), 256 threads elsewhere.
u32 default_window_threads(const Geometry& G, u32 k) {
  return G.lw && G.lw_cfg.P == 4096 && k >= 512 ? 128u : 256u;
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

template <int K>
int tile_occ_k(rsa_t* h) {
  // the cell-minimum pass is sized for six resident blocks of ~38 KB static
  // shared memory: ask for the largest shared-memory carveout
  CUDA_TRY(cudaFuncSetAttribute(k_tile_cmin<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->tile_blocks[0], k_tile_cmin<K>, TILE_THREADS, 0));
  CUDA_TRY(
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->tile_blocks[1], k_tile_accept<K>, TILE_THREADS, 0));
  return 0;
}

int tile_occupancy(rsa_t* h) {
  if (h->sm_count) return 0;
  CUDA_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
  int rc = 0;
  switch (h->k) {
    case 1: rc = tile_occ_k<1>(h); break;
    case 2: rc = tile_occ_k<2>(h); break;
    case 4: rc = tile_occ_k<4>(h); break;
    case 8: rc = tile_occ_k<8>(h); break;
    case 16: rc = tile_occ_k<16>(h); break;
    default: rc = tile_occ_k<32>(h); break;
  }
  if (rc) return rc;
  for (int i = 0; i < 2; ++i) h->tile_blocks[i] = std::max(1, h->tile_blocks[i]);
  return 0;
}

template <int K>
void launch_tile_k(rsa_t* h, Group g, TileCfg tc, u32* occw, u8* dead, const u32* tgrid,
                   cudaStream_t stream) {
  launch(h, KD_TILE_CMIN, k_tile_cmin<K>, dim3(tgrid[0]), dim3(TILE_THREADS), 0, stream, g, tc, occw, dead);
  launch(h, KD_TILE_ACCEPT, k_tile_accept<K>, dim3(tgrid[1]), dim3(TILE_THREADS), 0, stream, g, tc, occw,
         (const u8*)dead);
}

int launch_tile(rsa_t* h, Group g, TileCfg tc, u32* occw, u8* dead, const u32* tgrid,
                cudaStream_t stream) {
  switch (h->k) {
    case 1: launch_tile_k<1>(h, g, tc, occw, dead, tgrid, stream); break;
    case 2: launch_tile_k<2>(h, g, tc, occw, dead, tgrid, stream); break;
    case 4: launch_tile_k<4>(h, g, tc, occw, dead, tgrid, stream); break;
    case 8: launch_tile_k<8>(h, g, tc, occw, dead, tgrid, stream); break;
    case 16: launch_tile_k<16>(h, g, tc, occw, dead, tgrid, stream); break;
    case 32: launch_tile_k<32>(h, g, tc, occw, dead, tgrid, stream); break;
    default: return fail(RSA_EINVAL, "tile path needs k in {1,2,4,8,16,32}");
  }
  return 0;
}

void drop_graph(rsa_t::GraphSlot& gs) {
  if (gs.exec) cudaGraphExecDestroy(gs.exec);
  gs.exec = nullptr;
  gs.ws = nullptr;
}

// Run `body(stream)` once, either directly or through a captured graph.
template <typename B>
int run_chunk(rsa_t* h, rsa_t::GraphSlot& gs, cudaStream_t stream, u32 n, B body) {
  if (!h->use_graphs || h->prof.on) {
    body(stream);
    return launch_check("chunk launches");
  }
  const u32 caps[6] = {h->t_round, h->t_uf, h->t_probe, h->t_edges, h->round_check,
                       h->lw_threads};
  if (!(gs.exec && gs.ws == h->ws && gs.n == n && gs.keys == h->with_keys &&
        std::memcmp(gs.caps, caps, sizeof(caps)) == 0)) {
    drop_graph(gs);
    if (!h->cap_stream)
      CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    unsigned long long before[KD_COUNT];
    std::memcpy(before, h->prof.launches, sizeof(before));
    CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    body(h->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RSA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&gs.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      gs.exec = nullptr;
      return fail(RSA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < KD_COUNT; ++i) {
      gs.launches[i] = h->prof.launches[i] - before[i];
      h->prof.launches[i] = before[i];
    }
    gs.ws = h->ws;
    gs.n = n;
    gs.keys = h->with_keys;
    std::memcpy(gs.caps, caps, sizeof(caps));
  }
  CUDA_TRY(cudaGraphLaunch(gs.exec, stream));
  for (int i = 0; i < KD_COUNT; ++i) h->prof.launches[i] += gs.launches[i];
  return 0;
}

int run_impl(rsa_t* h, const uint64_t* seeds, u32 n, const uint64_t* keys, cudaStream_t stream) {
  if (n == 0) return fail(RSA_EINVAL, "n_samples must be >= 1");
  NvtxRange run_range("rsa_run");
  int rc;
  CUDA_TRY(cudaGetDevice(&h->device));
  if (!h->h_counter) CUDA_TRY(cudaMallocHost(&h->h_counter, 64));
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

  // long-k lines made of whole k-blocks run the argmin-offset round for
  // seeded priorities; caller priorities cannot be inverted
  const bool use_lw = G.lw && !h->with_keys;
  const u32 line_nseg = use_lw ? G.lw_cfg.nc : G.lc.nseg;
  CUDA_TRY(cudaMemcpyAsync(d_seeds, seeds, (size_t)n * 8, cudaMemcpyHostToDevice, stream));
  if (keys)
    CUDA_TRY(cudaMemcpyAsync(b + l.keys, keys, 2 * LL * 8, cudaMemcpyHostToDevice, stream));
  if (G.tile) {
    CUDA_TRY(cudaMemsetAsync(b + l.occw, 0, (size_t)n * LL / 8, stream));
    CUDA_TRY(cudaMemsetAsync(b + l.dead, 0, (size_t)n * G.tc.T2, stream));
  } else if (G.line) {
    CUDA_TRY(cudaMemsetAsync(b + l.occw, 0, (size_t)n * LL / 8, stream));
    CUDA_TRY(cudaMemsetAsync(b + l.occT, 0, (size_t)n * LL / 8, stream));
    const size_t ncode = G.tc.T2;
    CUDA_TRY(cudaMemsetAsync(b + l.dead, 0, (size_t)n * (2ull * h->L * line_nseg + ncode),
                             stream));
  } else {
    CUDA_TRY(cudaMemsetAsync(g.occ, 0, (size_t)n * LL, stream));
  }
  CUDA_TRY(cudaMemsetAsync(g.owner, 0xFF, (size_t)n * LL * 4, stream));
  CUDA_TRY(cudaMemsetAsync(b + l.counters, 0, 64, stream));
  CUDA_TRY(cudaMemsetAsync(b + l.work, 0, 4 * WORK_SLOTS * 8, stream));
  launch(h, KD_INIT, k_init, dim3((n + 127) / 128), dim3(128), 0, stream, g,
         (const u64*)d_seeds);
  if ((rc = launch_check("k_init"))) return rc;

  if (G.line) {
    if ((rc = set_smem(k_line_cmin<0>, G.line_smem))) return rc;
    if ((rc = set_smem(k_line_cmin<1>, G.line_smem))) return rc;
    if ((rc = set_smem(k_line_accept<0>, G.line_acc_smem))) return rc;
    if ((rc = set_smem(k_line_accept<1>, G.line_acc_smem))) return rc;
    if ((rc = set_smem(k_line_accept_codes<0>, G.line_codes_smem))) return rc;
    if ((rc = set_smem(k_line_accept_codes<1>, G.line_codes_smem))) return rc;
    if ((rc = set_smem(k_lcomb, sizeof(LcombSmem)))) return rc;
  } else if (!G.tile) {
    if ((rc = set_smem(k_row<0>, G.row_smem))) return rc;
    if ((rc = set_smem(k_row<1>, G.row_smem))) return rc;
    if ((rc = set_smem(k_col<0>, G.col_smem))) return rc;
    if ((rc = set_smem(k_col<1>, G.col_smem))) return rc;
  }
  const dim3 rg(G.row_grid_x.x, n), cg(G.col_grid_x.x, n);
  TileCfg tc = G.tc;
  tc.items = (u64)n * tc.T2;
  u32* occw = reinterpret_cast<u32*>(b + l.occw);
  u8* dead = reinterpret_cast<u8*>(b + l.dead);
  u32 tgrid[2] = {0, 0};
  if (G.tile) {
    if ((rc = tile_occupancy(h))) return rc;
    for (int i = 0; i < 2; ++i)
      tgrid[i] = (u32)std::min<u64>(tc.items, (u64)h->sm_count * h->tile_blocks[i]);
  }
  // every round accepts at least the smallest live key, so n_j + 1 rounds
  // always suffice
  const u32 round_cap = h->t_round ? h->t_round : cap_nodes_of(h->L, h->k) + 2;
  const u32 probe_cap = h->t_probe ? h->t_probe : PROBE_CAP;
  // one chunk = ROUND_CHECK greedy rounds; k_round_end counts the samples
  // still active after each round into d_counter
  u32* occT = reinterpret_cast<u32*>(b + l.occT);
  u64* cB = reinterpret_cast<u64*>(b + l.cB);
  int body_rc = 0;
  auto rounds = [&](cudaStream_t st) {
    for (u32 i = 0; i < h->round_check; ++i) {
      if (cudaMemsetAsync(d_counter, 0, 4, st) != cudaSuccess) body_rc = RSA_ECUDA;
      if (G.tile) {
        if (launch_tile(h, g, tc, occw, dead, tgrid, st)) body_rc = RSA_EINVAL;
      } else if (use_lw) {
        u8* lflag = dead;                                          // [n][2][L][nc]
        u8* cdead = dead + (size_t)n * 2 * h->L * line_nseg;       // [n][T^2]
        u16* cH = reinterpret_cast<u16*>(b + l.cH);
        u16* cV = reinterpret_cast<u16*>(b + l.cV);
        u32* mk = reinterpret_cast<u32*>(b + l.masks);
        const size_t mw = (size_t)n * LL / 32;  // words of one mask array
        const AccMasks mh{mk, mk + mw, mk + 2 * mw}, mv{mk + 3 * mw, mk + 4 * mw, mk + 5 * mw};
        if (launch_lwin<0>(h, g, G, occw, occT, cH, lflag, n, st) != cudaSuccess) body_rc = RSA_ECUDA;
        if (launch_lwin<1>(h, g, G, occw, occT, cV, lflag, n, st) != cudaSuccess) body_rc = RSA_ECUDA;
        launch(h, KD_LCOMB, k_lcomb, dim3((G.tc.T2 + LC_WARPS - 1) / LC_WARPS, n),
               dim3(LC_WARPS * 32), sizeof(LcombSmem), st, g, (const u16*)cH, (const u16*)cV, mh,
               mv, cdead);
        const dim3 ag(h->L * line_nseg, n);
        launch(h, KD_LACC_H, k_lacc<0>, ag, dim3(LW_THREADS), 0, st, g, G.lw_cfg, occw, occT, mh,
               (const u8*)lflag);
        launch(h, KD_LACC_V, k_lacc<1>, ag, dim3(LW_THREADS), 0, st, g, G.lw_cfg, occw, occT, mv,
               (const u8*)lflag);
      } else if (G.line) {
        const dim3 lg(h->L * G.lc.nseg, n), tg(G.tc.T2, n);
        u8* ldead = dead;                                          // [n][2][L][nseg]
        u8* cdead = dead + (size_t)n * 2 * h->L * G.lc.nseg;       // [n][T^2]
        launch(h, KD_LINE_CMIN_H, k_line_cmin<0>, lg, dim3(LINE_THREADS), G.line_smem, st, g,
               G.lc, (const u32*)occw, (const u32*)occT, g.cmin, cB, ldead);
        launch(h, KD_LINE_CMIN_V, k_line_cmin<1>, lg, dim3(LINE_THREADS), G.line_smem, st, g,
               G.lc, (const u32*)occw, (const u32*)occT, g.cmin, cB, ldead);
        if (h->with_keys) {
          // caller-supplied priorities cannot be inverted: compare values
          launch(h, KD_LINE_COMBINE, k_line_combine, tg, dim3(256), 0, st, g, g.cmin, cB);
          launch(h, KD_LINE_ACCEPT_H, k_line_accept<0>, lg, dim3(LINE_THREADS), G.line_acc_smem, st,
                 g, G.lc, occw, occT, (const u64*)g.cmin, (const u64*)cB);
          launch(h, KD_LINE_ACCEPT_V, k_line_accept<1>, lg, dim3(LINE_THREADS), G.line_acc_smem, st,
                 g, G.lc, occw, occT, (const u64*)g.cmin, (const u64*)cB);
        } else {
          u16* c16 = reinterpret_cast<u16*>(b + l.code16);
          u16* c16T = reinterpret_cast<u16*>(b + l.code16T);
          launch(h, KD_LINE_CODES, k_line_codes, tg, dim3(256), 0, st, g, (const u64*)g.cmin,
                 (const u64*)cB, c16, c16T, cdead);
          launch(h, KD_LINE_ACCEPT_H, k_line_accept_codes<0>, lg, dim3(LINE_THREADS),
                 G.line_codes_smem, st, g, G.lc, occw, occT, (const u16*)c16, (const u16*)c16T,
                 (const u8*)ldead);
          launch(h, KD_LINE_ACCEPT_V, k_line_accept_codes<1>, lg, dim3(LINE_THREADS),
                 G.line_codes_smem, st, g, G.lc, occw, occT, (const u16*)c16, (const u16*)c16T,
                 (const u8*)ldead);
        }
      } else {
        launch(h, KD_ROW_CMIN, k_row<0>, rg, dim3(G.row_threads), G.row_smem, st, g, G.row);
        launch(h, KD_COL_CMIN, k_col<0>, cg, dim3(G.col_threads), G.col_smem, st, g, G.col);
        launch(h, KD_ROW_ACCEPT, k_row<1>, rg, dim3(G.row_threads), G.row_smem, st, g, G.row);
        launch(h, KD_COL_ACCEPT, k_col<1>, cg, dim3(G.col_threads), G.col_smem, st, g, G.col);
      }
      launch(h, KD_ROUND_END, k_round_end, dim3((n + 127) / 128), dim3(128), 0, st, g, round_cap,
             d_counter);
    }
  };
  {
  NvtxRange rounds_range("greedy rounds");
  for (u32 chunks = 0;;) {
    const u32 burst = chunks == 0 ? h->round_chunks_hint : 1;
    for (u32 i = 0; i < burst; ++i, ++chunks)
      if ((rc = run_chunk(h, h->g_round, stream, n, rounds))) return rc;
    if (body_rc) return fail(body_rc, "round launches failed");
    u32 active;
    if ((rc = read_counter(h, d_counter, &active))) return rc;
    if (active == 0) {
      h->round_chunks_hint = chunks;
      break;
    }
  }
  }
  NvtxRange wrap_range("contact graph and first-wrap search");
  // contact graph of the jammed lattice
  {
    // rows per sample spread over enough blocks to fill the GPU across the batch
    const u32 bx = (u32)std::min<u64>(h->L, std::max<u64>(1, 65536 / n));
    if (h->L % 4 == 0 && h->L >= 8)
      launch(h, KD_EDGES, k_edges4, dim3(bx, n), dim3(EDGES_THREADS), 0, stream, g);
    else
      launch(h, KD_EDGES, k_edges, dim3(bx, n), dim3(EDGES_THREADS), 0, stream, g);
    if ((rc = launch_check("k_edges"))) return rc;
  }
  launch(h, KD_BUCKET, k_bucket, dim3(n), dim3(1024), 0, stream, g);
  // bisection for the first wrap
  launch(h, KD_SEARCH_INIT, k_search_init, dim3((n + 127) / 128), dim3(128), 0, stream, g);
  {
    u32 bx = (u32)std::min<u64>(((u64)g.cap_nodes + 255) / 256, 1024);
    launch(h, KD_SEARCH_INIT, k_uf_identity, dim3(bx, n), dim3(256), 0, stream, g);
  }
  if ((rc = launch_check("search init"))) return rc;
  // enough blocks per sample to fill the GPU across the batch, no more
  const u64 per_sample = std::max<u64>(8, 16384 / n);
  const u32 copy_bx = (u32)std::min<u64>(((u64)g.cap_nodes + 255) / 256, per_sample);
  const u32 probe_bx = (u32)std::min<u64>(((u64)g.cap_edges + 255) / 256, per_sample);
  auto probes = [&](cudaStream_t st) {
    for (u32 i = 0; i < PROBE_CHECK; ++i) {
      if (cudaMemsetAsync(d_counter + 1, 0, 4, st) != cudaSuccess) body_rc = RSA_ECUDA;
      launch(h, KD_PROBE_COPY, k_probe_copy, dim3(copy_bx, n), dim3(256), 0, st, g);
      launch(h, KD_PROBE, k_probe, dim3(probe_bx, n), dim3(256), 0, st, g);
      launch(h, KD_DECIDE, k_search_decide, dim3(n), dim3(256), 0, st, g, probe_cap,
             d_counter + 1);
    }
  };
  for (u32 chunks = 0; chunks * PROBE_CHECK < probe_cap + PROBE_CHECK;) {
    const u32 burst = chunks == 0 ? h->probe_chunks_hint : 1;
    for (u32 i = 0; i < burst; ++i, ++chunks)
      if ((rc = run_chunk(h, h->g_probe, stream, n, probes))) return rc;
    if (body_rc) return fail(body_rc, "probe launches failed");
    u32 open;
    if ((rc = read_counter(h, d_counter + 1, &open))) return rc;
    if (open == 0) {
      h->probe_chunks_hint = chunks;
      break;
    }
  }
  // round-pass work counters of this run (for throughput accounting)
  unsigned long long wk[4 * WORK_SLOTS];
  CUDA_TRY(cudaMemcpyAsync(wk, b + l.work, sizeof(wk), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  for (u32 i = 0; i < 4 * WORK_SLOTS; ++i) h->work[i / WORK_SLOTS] += wk[i];
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

// ---------------------------------------------------------------------
// Workspace-free runs.  Some callers cannot call cudaMalloc: a process whose
// device memory pool is owned by another allocator (a framework's caching
// allocator that has reserved the whole HBM), or a latency-critical serving
// loop that must not hit the device-wide synchronisation cudaMalloc and
// cudaFree can cause.  rsa_run_static serves them from this fixed array,
// which every GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------
constexpr size_t STATIC_WS_BYTES = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_static_ws[STATIC_WS_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
void* g_static_ptr[MAX_DEVICES] = {};
unsigned long long g_static_ctx[MAX_DEVICES] = {};

// Unique id of the current CUDA context (cuCtxGetId, reached through the
// runtime's driver entry-point table so the library does not link libcuda),
// or 0 if there is none or the driver lacks the call.
unsigned long long current_context_id() {
  typedef int (*ctx_id_fn)(void*, unsigned long long*);
  static ctx_id_fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return reinterpret_cast<ctx_id_fn>(f);
  }();
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != 0) return 0;
  return id;
}

// Device address of g_static_ws on the current device, looked up once per
// device (with that device current) and again whenever that device's context
// has changed since (a context destroyed by cudaDeviceReset and created anew
// may place the array elsewhere).  In host code the symbol itself is only a
// host-side stand-in, never a device address.
int static_workspace(void** out) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(RSA_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_static_ptr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p)
      return fail(RSA_ECUDA, std::string("cudaGetSymbolAddress(static workspace): ") +
                                 cudaGetErrorString(e));
    g_static_ptr[dev] = p;
    g_static_ctx[dev] = current_context_id();  // the lookup made the context current
  }
  *out = g_static_ptr[dev];
  return 0;
}

// The configuration of the first m accepted k-mers of sample `sample` of
// the last run: winding bits into *wdirs, and, if counts is given, the
// cluster-size histogram counts[0 .. m] (cap >= m + 1).
int configuration(rsa_t* h, uint32_t sample, uint32_t m, uint32_t* counts, uint32_t cap,
                  uint32_t* wdirs) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (sample >= h->last_n) return fail(RSA_EINVAL, "sample out of range");
  if (counts && cap < (u64)m + 1) return fail(RSA_EINVAL, "counts needs m + 1 entries");
  std::vector<SampleState> st;
  int rc = fetch_states(h, st);
  if (rc) return rc;
  if ((rc = status_code(st[sample].status))) {
    g_err = "sample " + std::to_string(sample) + " has no valid result";
    return rc;
  }
  const u32 nj = st[sample].n_nodes;
  if (m > nj) return fail(RSA_EINVAL, "m exceeds n_j of the sample");
  if (counts) std::memset(counts, 0, (size_t)cap * sizeof(uint32_t));
  *wdirs = 0;
  if (m == 0) return 0;
  cudaStream_t stream = h->stream;
  Group g = group_of(h, h->last_n);
  const u32 bx = (u32)std::min<u64>(((u64)g.cap_edges + 255) / 256, 2048);
  const u32 nb = (u32)std::min<u64>(((u64)nj + 256) / 256, 1024);
  k_select_key<<<1, 1024, 0, stream>>>(g, sample, m);
  k_cfg_init<<<nb, 256, 0, stream>>>(g, sample);
  k_cfg_union<<<bx, 256, 0, stream>>>(g, sample);
  if (counts) {
    k_cfg_count<<<nb, 256, 0, stream>>>(g, sample);
    k_cfg_hist<<<nb, 256, 0, stream>>>(g, sample);
  }
  CUDA_TRY(cudaGetLastError());
  const char* b = static_cast<const char*>(h->ws);
  const size_t so = h->lay.st + (size_t)sample * sizeof(SampleState);
  CUDA_TRY(cudaMemcpyAsync(h->h_counter + 12, b + so + offsetof(SampleState, wdirs), 4,
                           cudaMemcpyDeviceToHost, stream));
  if (counts)
    CUDA_TRY(cudaMemcpyAsync(counts,
                             b + h->lay.edges + (size_t)sample * g.cap_edges * sizeof(Edge),
                             ((size_t)m + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  const u32 w = h->h_counter[12];
  if (w & CFG_CAPPED) return fail(RSA_ETIMEOUT, "union-find walk cap reached");
  *wdirs = w & 3u;
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
  h->lw_threads = default_window_threads(h->geo, k);
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

int rsa_run_static(uint32_t L, uint32_t k, const uint64_t* seeds, uint32_t n, uint32_t* n_j,
                   uint32_t* n_c, void* stream) {
  if (!seeds || !n_j || !n_c) return fail(RSA_EINVAL, "null seeds or output array");
  if (!(k >= 1 && k <= L && L <= 32768)) return fail(RSA_EINVAL, "need 1 <= k <= L <= 32768");
  if (n == 0) return fail(RSA_EINVAL, "n must be >= 1");
  rsa h;
  h.L = L;
  h.k = k;
  h.seed = 0;
  h.geo = plan(L, k);
  const size_t need = layout_of(L, k, n, false, h.geo).total;
  if (need > STATIC_WS_BYTES)
    return fail(RSA_EINVAL, "rsa_run_static: L=" + std::to_string(L) + " k=" + std::to_string(k) +
                                " n=" + std::to_string(n) + " needs " + std::to_string(need) +
                                " bytes of workspace; the static workspace holds " +
                                std::to_string(STATIC_WS_BYTES));
  void* ws = nullptr;
  int rc = static_workspace(&ws);
  if (rc) return rc;
  h.use_graphs = false;  // plain launches only: nothing is created or allocated
  h.bound_ptr = ws;  // the run's buffers (all re-initialised by the run) live here
  h.bound_bytes = STATIC_WS_BYTES;
  alignas(8) u32 counter[16] = {};  // pageable host words for the loop checks
  h.h_counter = counter;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = run_impl(&h, seeds, n, nullptr, st);
  h.h_counter = nullptr;
  if (rc) return rc;
  // results straight from the per-sample state records (strided copies)
  const char* sts = static_cast<const char*>(ws) + h.lay.st;
  CUDA_TRY(cudaMemcpy2DAsync(n_c, sizeof(u32), sts + offsetof(SampleState, status),
                             sizeof(SampleState), sizeof(u32), n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  int first = 0;
  for (u32 i = 0; i < n && !first; ++i) {
    first = status_code(n_c[i]);
    if (first) g_err = "sample " + std::to_string(i) + " status bits " + std::to_string(n_c[i]);
  }
  CUDA_TRY(cudaMemcpy2DAsync(n_j, sizeof(u32), sts + offsetof(SampleState, n_nodes),
                             sizeof(SampleState), sizeof(u32), n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpy2DAsync(n_c, sizeof(u32), sts + offsetof(SampleState, nc),
                             sizeof(SampleState), sizeof(u32), n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return first;
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

int rsa_contacts(rsa_t* h, uint32_t* n_x, uint32_t* n_y, uint32_t* n_xy, uint32_t n) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (n > h->last_n) return fail(RSA_EINVAL, "n exceeds samples of the last run");
  std::vector<SampleState> st;
  int rc = fetch_states(h, st);
  if (rc) return rc;
  for (u32 i = 0; i < n; ++i) {
    if (n_x) n_x[i] = st[i].contacts_x;
    if (n_y) n_y[i] = st[i].contacts_y;
    if (n_xy) n_xy[i] = st[i].contacts_xy;
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

int rsa_cluster_sizes(rsa_t* h, uint32_t sample, uint32_t m, uint32_t* counts, uint32_t cap) {
  if (!counts) return fail(RSA_EINVAL, "null counts");
  uint32_t w;
  return configuration(h, sample, m, counts, cap, &w);
}

int rsa_wrap_dirs(rsa_t* h, uint32_t sample, uint32_t m, uint32_t* wrap_x, uint32_t* wrap_y) {
  uint32_t w = 0;
  int rc = configuration(h, sample, m, nullptr, 0, &w);
  if (rc) return rc;
  if (wrap_x) *wrap_x = w & 1u;
  if (wrap_y) *wrap_y = (w >> 1) & 1u;
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

int rsa_test_caps(rsa_t* h, uint32_t round_cap, uint32_t uf_steps, uint32_t probe_cap,
                  uint32_t edge_cap) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  h->t_round = round_cap;
  h->t_uf = uf_steps;
  h->t_probe = probe_cap;
  h->t_edges = edge_cap;
  return 0;
}

int rsa_set_rounds_per_check(rsa_t* h, uint32_t rounds) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (rounds < 1 || rounds > 64) return fail(RSA_EINVAL, "rounds per check must be in 1 .. 64");
  if (rounds != h->round_check) h->round_chunks_hint = 1;
  h->round_check = rounds;
  return 0;
}

int rsa_set_window_threads(rsa_t* h, uint32_t threads) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  if (threads == 0) threads = default_window_threads(h->geo, h->k);
  if (threads != 256 && threads != 128) return fail(RSA_EINVAL, "window CTA size must be 128 or 256");
  if (threads == 128 && !(h->geo.lw && (h->geo.lw_cfg.P == 4096 || h->geo.lw_cfg.P == 2048)))
    return fail(RSA_EINVAL, "128-thread windows need the long-k offset path with spans of 2048 or 4096 cells");
  h->lw_threads = threads;
  return 0;
}

int rsa_profile(rsa_t* h, int enable) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  h->prof.on = enable != 0;
  return 0;
}

int rsa_kernel_stats(rsa_t* h, double* ms, unsigned long long* launches, uint32_t n_kinds) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  Prof& p = h->prof;
  if (!p.kinds.empty()) {
    if (h->stream || h->device >= 0) CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < p.kinds.size(); ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.pool[2 * i], p.pool[2 * i + 1]) == cudaSuccess)
        p.ms[p.kinds[i]] += t;
    }
    p.kinds.clear();
  }
  for (uint32_t i = 0; i < n_kinds && i < (uint32_t)KD_COUNT; ++i) {
    if (ms) ms[i] = p.ms[i];
    if (launches) launches[i] = p.launches[i];
    p.ms[i] = 0.0;
    p.launches[i] = 0;
  }
  return 0;
}

int rsa_work_stats(rsa_t* h, unsigned long long* out, uint32_t n) {
  if (!h) return fail(RSA_EINVAL, "null handle");
  for (uint32_t i = 0; i < n && i < 4; ++i) {
    if (out) out[i] = h->work[i];
    h->work[i] = 0;
  }
  return 0;
}

const char* rsa_kernel_name(uint32_t kind) {
  return kind < (uint32_t)KD_COUNT ? kKindNames[kind] : "";
}

void rsa_destroy(rsa_t* h) {
  if (!h) return;
  drop_graph(h->g_round);
  drop_graph(h->g_probe);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  if (h->own_ptr) cudaFree(h->own_ptr);
  if (h->h_counter) cudaFreeHost(h->h_counter);
  delete h;
}

const char* rsa_last_error(void) { return g_err.c_str(); }

}  // extern "C"
