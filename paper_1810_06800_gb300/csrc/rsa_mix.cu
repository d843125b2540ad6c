// rsa_mix.cu -- batching of samples of uneven (L, k) and the autotuner that
// picks how each shape runs (C ABI in include/rsa.h).
//
//   rsa_run_small  small lattices, one CTA per sample (rsa_small.cuh): any
//                  mix of shapes in one persistent launch;
//   rsa_run_mix    a batch of samples of any shapes: the small ones in one
//                  persistent launch, every other shape on its own handle
//                  (graph-replayed rounds) on its own stream, all at once;
//   rsa_tune       per (GPU, L, k, batch size): small mode and its CTA size,
//                  or the global path and its rounds per host check, by
//                  timing each candidate once; kept in a JSON-lines cache.
// Everything here runs the library's own kernels through its public calls;
// results never depend on the choices made (tested).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/rsa.h"
#include "rsa_small.cuh"

using namespace rsak;

namespace rsa_detail {
int set_error(int code, const std::string& msg);
}

namespace {

using rsa_detail::set_error;

#define MIX_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return set_error(RSA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool small_eligible(uint32_t L, uint32_t k) {
  return k >= 1 && k <= L && L <= SMALL_LMAX && (uint64_t)L * L / k <= SMALL_NMAX;
}

int status_to_code(u32 bits) {
  if (bits & ST_NOWRAP) return RSA_ENOWRAP;
  if (bits & (ST_UF_CAP | ST_ROUND_CAP)) return RSA_ETIMEOUT;
  if (bits & ST_NODE_OVF) return RSA_ENOMEM;
  return 0;
}

// k_small launches since the last rsa_mix_launches() call.
std::atomic<unsigned long long> g_small_launches{0};

// Resident CTAs of k_small per SM for a CTA size and lattice bound.
int small_blocks_per_sm(uint32_t threads, uint32_t Lm, int* out) {
  const size_t smem = small_smem_bytes(Lm);
  MIX_CUDA(cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)small_smem_bytes(SMALL_LMAX)));
  MIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_small, (int)threads, smem));
  return 0;
}

}  // namespace

extern "C" int rsa_run_small(const uint32_t* L, const uint32_t* k, const uint64_t* seeds,
                             uint32_t n, uint32_t threads, uint32_t* n_j, uint32_t* n_c,
                             void* stream) {
  if (!L || !k || !seeds || !n_j || !n_c || n == 0)
    return set_error(RSA_EINVAL, "rsa_run_small: null array or n == 0");
  if (threads == 0) threads = 512;
  nvtxRangePushA("rsa_run_small");
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  if (threads % 32 || threads > 1024) return set_error(RSA_EINVAL, "threads must be 32 .. 1024, a multiple of 32");
  std::vector<SmallJob> jobs(n);
  uint32_t Lm = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (!small_eligible(L[i], k[i]))
      return set_error(RSA_EINVAL, "rsa_run_small: sample " + std::to_string(i) + " (L=" +
                                       std::to_string(L[i]) + ", k=" + std::to_string(k[i]) +
                                       ") needs L <= 128 and L^2/k <= 4096");
    jobs[i] = SmallJob{L[i], k[i], seeds[i]};
    Lm = std::max(Lm, L[i]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, bps = 0;
  MIX_CUDA(cudaGetDevice(&dev));
  MIX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int rc = small_blocks_per_sm(threads, Lm, &bps);
  if (rc) return rc;
  if (bps < 1) return set_error(RSA_EINVAL, "rsa_run_small: CTA size does not fit an SM");
  // job table, results and the work counter, stream-ordered
  const size_t jb = sizeof(SmallJob) * n, ob = sizeof(SmallOut) * n;
  char* d = nullptr;
  MIX_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), jb + ob + 256, st));
  SmallJob* djobs = reinterpret_cast<SmallJob*>(d);
  SmallOut* dout = reinterpret_cast<SmallOut*>(d + jb);
  u32* dnext = reinterpret_cast<u32*>(d + jb + ob);
  std::vector<SmallOut> out(n);
  cudaError_t e = cudaMemcpyAsync(djobs, jobs.data(), jb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dnext, 0, 4, st);
  if (e == cudaSuccess) {
    const u32 grid = (u32)std::min<uint64_t>(n, (uint64_t)sms * bps);
    k_small<<<grid, threads, small_smem_bytes(Lm), st>>>(djobs, n, dout, dnext, Lm, UF_CAP);
    e = cudaGetLastError();
    if (e == cudaSuccess) g_small_launches.fetch_add(1);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), dout, ob, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(RSA_ECUDA, std::string("rsa_run_small: ") + cudaGetErrorString(e));
  int first = 0;
  for (uint32_t i = 0; i < n; ++i) {
    n_j[i] = out[i].n_j;
    n_c[i] = out[i].n_c;
    const int c = status_to_code(out[i].status);
    if (c && !first) {
      first = c;
      set_error(c, "sample " + std::to_string(i) + " status bits " + std::to_string(out[i].status));
    }
  }
  return first;
}

// ---------------------------------------------------------------------
// Autotuner.  For one (GPU, L, k, batch size rounded up to a power of two)
// it times every candidate way to run the batch once -- small mode at 256,
// 512 and 1024 threads per CTA when the shape fits it, and the global path
// at 2, 4 and 8 greedy rounds per host check -- on seeds 1 .. n, and keeps
// the fastest.  Results go to a JSON-lines cache ($RSA_TUNE_CACHE, else
// $HOME/.cache/rsa_gb300/tune.jsonl), read back on the next process start.
// ---------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<std::string, uint32_t, uint32_t, uint32_t>, rsa_tune_t> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  const char* p = std::getenv("RSA_TUNE_CACHE");
  if (p && *p) return p;
  const char* home = std::getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/rsa_gb300/tune.jsonl";
}

// Value of "key": in one of our own JSON lines (numbers and plain strings).
bool json_field(const std::string& line, const char* key, std::string* out) {
  const std::string pat = std::string("\"") + key + "\":";
  size_t a = line.find(pat);
  if (a == std::string::npos) return false;
  a += pat.size();
  while (a < line.size() && line[a] == ' ') ++a;
  if (a < line.size() && line[a] == '"') {
    const size_t b = line.find('"', a + 1);
    if (b == std::string::npos) return false;
    *out = line.substr(a + 1, b - a - 1);
  } else {
    size_t b = a;
    while (b < line.size() && line[b] != ',' && line[b] != '}') ++b;
    *out = line.substr(a, b - a);
  }
  return true;
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (!f) return;
  char buf[1024];
  while (std::fgets(buf, sizeof(buf), f)) {
    const std::string line(buf);
    std::string gpu, L, k, n, mode, thr, rpc, ms, wt;
    if (!json_field(line, "gpu", &gpu) || !json_field(line, "L", &L) || !json_field(line, "k", &k) ||
        !json_field(line, "n", &n) || !json_field(line, "mode", &mode) ||
        !json_field(line, "threads", &thr) || !json_field(line, "rounds_per_check", &rpc) ||
        !json_field(line, "ms_per_sample", &ms))
      continue;
    rsa_tune_t c;
    c.mode = mode == "small" ? RSA_MODE_SMALL : RSA_MODE_GLOBAL;
    c.threads = (uint32_t)std::strtoul(thr.c_str(), nullptr, 10);
    c.rounds_per_check = (uint32_t)std::strtoul(rpc.c_str(), nullptr, 10);
    c.ms_per_sample = std::strtod(ms.c_str(), nullptr);
    c.window_threads = json_field(line, "window_threads", &wt)
                           ? (uint32_t)std::strtoul(wt.c_str(), nullptr, 10) : 256u;
    g_tune[std::make_tuple(gpu, (uint32_t)std::strtoul(L.c_str(), nullptr, 10),
                           (uint32_t)std::strtoul(k.c_str(), nullptr, 10),
                           (uint32_t)std::strtoul(n.c_str(), nullptr, 10))] = c;
  }
  std::fclose(f);
}

void tune_store_locked(const std::string& gpu, uint32_t L, uint32_t k, uint32_t nb,
                       const rsa_tune_t& c) {
  const std::string path = tune_path();
  // create the cache directory, one path level at a time (errors ignored:
  // an unwritable cache leaves the in-memory table)
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0)
    for (size_t i = 1; i <= slash; ++i)
      if (i == slash || path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;  // the in-memory table still holds it
  std::fprintf(f,
               "{\"gpu\": \"%s\", \"L\": %u, \"k\": %u, \"n\": %u, \"mode\": \"%s\", "
               "\"threads\": %u, \"rounds_per_check\": %u, \"window_threads\": %u, "
               "\"ms_per_sample\": %.6g}\n",
               gpu.c_str(), L, k, nb, c.mode == RSA_MODE_SMALL ? "small" : "global", c.threads,
               c.rounds_per_check, c.window_threads, c.ms_per_sample);
  std::fclose(f);
}

}  // namespace

namespace {

rsa_tune_t default_config(uint32_t L, uint32_t k) {
  rsa_tune_t c{};
  if (small_eligible(L, k)) {
    c.mode = RSA_MODE_SMALL;
    c.threads = 512;
  } else {
    c.mode = RSA_MODE_GLOBAL;
    c.rounds_per_check = 4;
    c.window_threads = 0;  // the handle's own default
  }
  return c;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Time one way of running nb samples (seeds 1 .. nb) of (L, k); ms per sample.
int time_config(uint32_t L, uint32_t k, uint32_t nb, const rsa_tune_t& c, cudaStream_t st,
                double* ms) {
  std::vector<uint64_t> seeds(nb);
  for (uint32_t i = 0; i < nb; ++i) seeds[i] = i + 1;
  std::vector<uint32_t> nj(nb), nc(nb), Ls(nb, L), ks(nb, k);
  int rc = 0;
  double best = 1e300;
  if (c.mode == RSA_MODE_SMALL) {
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      const double t0 = now_ms();
      rc = rsa_run_small(Ls.data(), ks.data(), seeds.data(), nb, c.threads, nj.data(), nc.data(), st);
      best = std::min(best, now_ms() - t0);
    }
  } else {
    rsa_t* h = nullptr;
    if ((rc = rsa_create(L, k, 1, &h))) return rc;
    rc = rsa_set_rounds_per_check(h, c.rounds_per_check);
    if (!rc && c.window_threads) rc = rsa_set_window_threads(h, c.window_threads);
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      const double t0 = now_ms();
      rc = rsa_run_seeds(h, seeds.data(), nb, st);
      if (!rc) rc = rsa_results(h, nj.data(), nc.data(), nb);
      best = std::min(best, now_ms() - t0);
    }
    rsa_destroy(h);
  }
  *ms = best / nb;
  return rc;
}

}  // namespace

extern "C" int rsa_tune(uint32_t L, uint32_t k, uint32_t n, int measure, rsa_tune_t* out) {
  if (!out || !(k >= 1 && k <= L && L <= 32768) || n == 0)
    return set_error(RSA_EINVAL, "rsa_tune: bad arguments");
  int dev = 0;
  cudaDeviceProp prop;
  MIX_CUDA(cudaGetDevice(&dev));
  MIX_CUDA(cudaGetDeviceProperties(&prop, dev));
  uint32_t nb = 1;
  while (nb < n && nb < (1u << 20)) nb <<= 1;
  const auto key = std::make_tuple(std::string(prop.name), L, k, nb);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *out = it->second;
      return 0;
    }
  }
  *out = default_config(L, k);
  if (!measure) return 0;
  // the tuning batch: nb samples, fewer where their workspaces would pass 8 GB
  uint64_t ws = 0;
  int rc = rsa_workspace_bytes(L, k, 1, &ws);
  if (rc) return rc;
  const uint32_t nt = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nb, (8ull << 30) / std::max<uint64_t>(ws, 1)));
  std::vector<rsa_tune_t> cands;
  if (small_eligible(L, k))
    for (uint32_t t : {256u, 512u, 1024u}) {
      rsa_tune_t c{};
      c.mode = RSA_MODE_SMALL;
      c.threads = t;
      cands.push_back(c);
    }
  // the 128-thread window pass exists only for some shapes: ask a handle
  bool w128 = false;
  {
    rsa_t* h = nullptr;
    if (rsa_create(L, k, 1, &h) == 0) {
      w128 = rsa_set_window_threads(h, 128) == 0;
      rsa_destroy(h);
    }
  }
  for (uint32_t r : {2u, 4u, 8u})
    for (uint32_t wt : {256u, 128u}) {
      if (wt == 128 && !w128) continue;
      rsa_tune_t c{};
      c.mode = RSA_MODE_GLOBAL;
      c.rounds_per_check = r;
      c.window_threads = wt;
      cands.push_back(c);
    }
  cudaStream_t st = nullptr;
  MIX_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  rsa_tune_t best = *out;
  best.ms_per_sample = 1e300;
  for (rsa_tune_t c : cands) {
    double ms = 0;
    if ((rc = time_config(L, k, nt, c, st, &ms))) break;
    if (ms < best.ms_per_sample) {
      best = c;
      best.ms_per_sample = ms;
    }
  }
  cudaStreamDestroy(st);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  tune_store_locked(std::get<0>(key), L, k, nb, best);
  *out = best;
  return 0;
}

// ---------------------------------------------------------------------
// Mixed batches.  Handles and streams of the global-path shapes are kept
// per (device, L, k) between calls (a serving loop reuses them); their
// workspaces grow to the largest group seen.  rsa_mix_release frees them.
// ---------------------------------------------------------------------
namespace {

struct MixSlot {
  std::mutex mu;  // one batch at a time on the handle
  rsa_t* h = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};
std::mutex g_mix_mu;
std::map<std::tuple<int, uint32_t, uint32_t>, std::unique_ptr<MixSlot>> g_mix;
std::map<int, std::pair<cudaStream_t, cudaEvent_t>> g_small_stream;

int mix_slot(int dev, uint32_t L, uint32_t k, MixSlot** out) {
  std::lock_guard<std::mutex> lock(g_mix_mu);
  std::unique_ptr<MixSlot>& p = g_mix[std::make_tuple(dev, L, k)];
  if (!p) p.reset(new MixSlot());
  MixSlot& s = *p;
  if (!s.h) {
    int rc = rsa_create(L, k, 1, &s.h);
    if (rc) return rc;
    MIX_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
    MIX_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  }
  *out = &s;
  return 0;
}

}  // namespace

extern "C" int rsa_run_mix(const uint32_t* L, const uint32_t* k, const uint64_t* seeds, uint32_t n,
                           uint32_t* n_j, uint32_t* n_c, void* stream) {
  if (!L || !k || !seeds || !n_j || !n_c || n == 0)
    return set_error(RSA_EINVAL, "rsa_run_mix: null array or n == 0");
  for (uint32_t i = 0; i < n; ++i)
    if (!(k[i] >= 1 && k[i] <= L[i] && L[i] <= 32768))
      return set_error(RSA_EINVAL, "rsa_run_mix: sample " + std::to_string(i) + " needs 1 <= k <= L <= 32768");
  nvtxRangePushA("rsa_run_mix");
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  int dev = 0;
  MIX_CUDA(cudaGetDevice(&dev));
  const char* at = std::getenv("RSA_AUTOTUNE");
  const bool measure = !(at && at[0] == '0');
  // samples grouped by shape, in order of first appearance
  std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> groups;
  for (uint32_t i = 0; i < n; ++i) groups[{L[i], k[i]}].push_back(i);
  std::vector<uint32_t> small_idx;
  uint32_t small_threads = 512;
  uint64_t small_work = 0;
  struct Job {
    uint32_t L, k, rpc, wt;
    const std::vector<uint32_t>* idx;
  };
  std::vector<Job> global;
  for (auto& gkv : groups) {
    rsa_tune_t c;
    int rc = rsa_tune(gkv.first.first, gkv.first.second, (uint32_t)gkv.second.size(), measure, &c);
    if (rc) return rc;
    if (c.mode == RSA_MODE_SMALL && small_eligible(gkv.first.first, gkv.first.second)) {
      small_idx.insert(small_idx.end(), gkv.second.begin(), gkv.second.end());
      const uint64_t work = (uint64_t)gkv.first.first * gkv.first.first * gkv.second.size();
      if (work > small_work) {
        small_work = work;
        small_threads = c.threads;
      }
    } else {
      global.push_back(Job{gkv.first.first, gkv.first.second, c.rounds_per_check ? c.rounds_per_check : 4u,
                           c.window_threads, &gkv.second});
    }
  }
  // everything already queued on the caller's stream comes first
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEvent_t start = nullptr;
  MIX_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  MIX_CUDA(cudaEventRecord(start, cs));
  std::vector<std::pair<int, std::string>> errs(global.size() + 1, {0, ""});
  std::vector<std::thread> workers;
  std::vector<cudaEvent_t> dones;
  bool setup_failed = false;
  for (size_t g = 0; g < global.size(); ++g) {
    MixSlot* slot = nullptr;
    int rc = mix_slot(dev, global[g].L, global[g].k, &slot);
    if (rc) {
      // the shapes already handed to workers still run; join them below
      errs[g] = {rc, rsa_last_error()};
      setup_failed = true;
      break;
    }
    cudaStreamWaitEvent(slot->st, start, 0);
    dones.push_back(slot->done);
    workers.emplace_back([&, g, slot, dev] {
      cudaSetDevice(dev);
      std::lock_guard<std::mutex> slot_lock(slot->mu);
      const Job& J = global[g];
      const uint32_t m = (uint32_t)J.idx->size();
      std::vector<uint64_t> sd(m);
      std::vector<uint32_t> a(m), b(m);
      for (uint32_t i = 0; i < m; ++i) sd[i] = seeds[(*J.idx)[i]];
      int rc2 = rsa_set_rounds_per_check(slot->h, J.rpc);
      if (rsa_set_window_threads(slot->h, J.wt)) rsa_set_window_threads(slot->h, 0);
      if (!rc2) rc2 = rsa_run_seeds(slot->h, sd.data(), m, slot->st);
      if (!rc2) rc2 = rsa_results(slot->h, a.data(), b.data(), m);
      if (!rc2) cudaEventRecord(slot->done, slot->st);
      for (uint32_t i = 0; i < m; ++i) {
        n_j[(*J.idx)[i]] = a[i];
        n_c[(*J.idx)[i]] = b[i];
      }
      if (rc2) errs[g] = {rc2, rsa_last_error()};
    });
  }
  if (!small_idx.empty() && !setup_failed) {
    cudaStream_t sst = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_mix_mu);
      auto& ss = g_small_stream[dev];
      if (!ss.first) {
        cudaStreamCreateWithFlags(&ss.first, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&ss.second, cudaEventDisableTiming);
      }
      sst = ss.first;
      dones.push_back(ss.second);
    }
    cudaStreamWaitEvent(sst, start, 0);
    const uint32_t m = (uint32_t)small_idx.size();
    std::vector<uint32_t> Ls(m), ks(m), a(m), b(m);
    std::vector<uint64_t> sd(m);
    for (uint32_t i = 0; i < m; ++i) {
      Ls[i] = L[small_idx[i]];
      ks[i] = k[small_idx[i]];
      sd[i] = seeds[small_idx[i]];
    }
    const int rc = rsa_run_small(Ls.data(), ks.data(), sd.data(), m, small_threads, a.data(), b.data(), sst);
    cudaEventRecord(dones.back(), sst);
    for (uint32_t i = 0; i < m; ++i) {
      n_j[small_idx[i]] = a[i];
      n_c[small_idx[i]] = b[i];
    }
    if (rc) errs.back() = {rc, rsa_last_error()};
  }
  for (auto& w : workers) w.join();
  // later work on the caller's stream comes after this batch
  for (cudaEvent_t e : dones) cudaStreamWaitEvent(cs, e, 0);
  cudaEventDestroy(start);
  for (auto& e : errs)
    if (e.first) return set_error(e.first, e.second);
  return 0;
}

extern "C" unsigned long long rsa_mix_launches(void) {
  unsigned long long total = g_small_launches.exchange(0);
  uint32_t nk = 0;
  while (rsa_kernel_name(nk)[0]) ++nk;
  std::vector<double> ms(nk);
  std::vector<unsigned long long> ln(nk);
  std::lock_guard<std::mutex> lock(g_mix_mu);
  for (auto& kv : g_mix) {
    std::lock_guard<std::mutex> slot_lock(kv.second->mu);
    if (!kv.second->h) continue;
    if (rsa_kernel_stats(kv.second->h, ms.data(), ln.data(), nk) == 0)
      for (unsigned long long v : ln) total += v;
  }
  return total;
}

extern "C" void rsa_mix_release(void) {
  std::lock_guard<std::mutex> lock(g_mix_mu);
  for (auto& kv : g_mix) {
    std::lock_guard<std::mutex> slot_lock(kv.second->mu);
    rsa_destroy(kv.second->h);
    if (kv.second->st) cudaStreamDestroy(kv.second->st);
    if (kv.second->done) cudaEventDestroy(kv.second->done);
  }
  g_mix.clear();
  for (auto& kv : g_small_stream) {
    cudaStreamDestroy(kv.second.first);
    cudaEventDestroy(kv.second.second);
  }
  g_small_stream.clear();
}
