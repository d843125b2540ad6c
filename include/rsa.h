/*
 * rsa.h -- C ABI of the GB300 library for random sequential adsorption (RSA)
 * of linear k-mers on an L x L periodic square lattice.
 *
 * Model (arXiv:1810.06800, Sec. I and Sec. II.A): k-mers cover k consecutive
 * cells, horizontal or vertical; deposition is RSA on a torus until jamming.
 * Per sample the library returns
 *   n_j -- the number of k-mers at jamming (p_j = k n_j / L^2, Sec. I), and
 *   n_c -- the number of k-mers on the lattice when a cluster first wraps the
 *          torus in one or both directions (p_c = k n_c / L^2, Sec. II.D).
 *
 * Deposition order: every (orientation o, row y, column x) placement is one
 * candidate, idx = (o*L + y)*L + x (o = 0 horizontal, covering (y, x+i mod L);
 * o = 1 vertical, covering (y+i mod L, x); i < k).  The viable-list form of
 * RSA (Sec. II.B) tries each candidate once in uniformly random order; here
 * that order is the ascending order of the 64-bit priority
 *     key(idx) = mix64(base + 0x9E3779B97F4A7C15 * (idx + 1)),
 *     base     = mix64(seed + 0x9E3779B97F4A7C15),
 * mix64 being the splitmix64 output finaliser (Steele, Lea, Flood 2014).
 * mix64 is a bijection, so the 2 L^2 keys of a sample are distinct.
 *
 * Conventions for every entry point:
 *   - return 0 on success or a negative RSA_E* code; rsa_last_error() then
 *     holds a message (thread-local, valid until the next call on the thread);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default);
 *   - host pointers are caller-owned and only read/written during the call;
 *   - no call traps the GPU: device-side failures are recorded in a status
 *     word per sample and reported by rsa_results().
 *   - 1 <= k <= L <= 32768.
 */
#ifndef RSA_GB300_H
#define RSA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSA_OK        0
#define RSA_EINVAL   (-1)  /* bad argument                                  */
#define RSA_ENOMEM   (-2)  /* device allocation or bound workspace too small */
#define RSA_ECUDA    (-3)  /* a CUDA runtime call failed                     */
#define RSA_ETIMEOUT (-4)  /* a device loop hit its iteration cap            */
#define RSA_ENOWRAP  (-5)  /* no wrapping cluster at jamming (contradicts the
                              Appendix A Proposition; n_c = UINT32_MAX)      */
#define RSA_ESTATE   (-6)  /* call out of order (e.g. results before a run)  */

typedef struct rsa rsa_t;

/* Create a handle for lattice size L, k-mer length k and base seed.  Sample
 * i of rsa_run_batch uses seed + i.  Allocates no device memory yet.
 * Errors: RSA_EINVAL unless 1 <= k <= L <= 32768 and out != NULL. */
int rsa_create(uint32_t L, uint32_t k, uint64_t seed, rsa_t **out);

/* Run n_samples samples (seeds seed .. seed + n_samples - 1) to jamming and
 * find each first-wrap count, on `stream`.  Device memory is allocated on
 * first use (or taken from a bound workspace).  The call returns once the
 * work is enqueued; it synchronises `stream` a few times while running the
 * data-dependent round and bisection loops.  Results stay on the device
 * until rsa_results(). */
int rsa_run_batch(rsa_t *h, uint32_t n_samples, void *stream);

/* As rsa_run_batch with explicit per-sample seeds (host array of n). */
int rsa_run_seeds(rsa_t *h, const uint64_t *seeds, uint32_t n, void *stream);

/* TEST ONLY: one sample whose candidate order is given by the caller:
 * keys[idx] for idx < 2 L^2 (host array), all distinct and != 2^64 - 1
 * (RSA_EINVAL otherwise). */
int rsa_run_keys(rsa_t *h, const uint64_t *keys, void *stream);

/* Workspace-free batched run (the paper has no counterpart; this is an
 * interface for callers that cannot allocate device memory: processes whose
 * device memory pool belongs to another allocator, or latency-critical loops
 * that must not call cudaMalloc/cudaFree, which can synchronise the device).
 * Same computation and results as rsa_run_seeds + rsa_results for the n
 * samples with the given seeds, but all device state lives in one fixed
 * 64 MiB array inside the library (held by every GPU that loads it until the
 * process exits); no handle, no device or pinned allocation.
 *   seeds: host array of n seeds (read);  n_j, n_c: host arrays of n (written).
 * Sizes whose workspace (rsa_workspace_bytes(L, k, n)) exceeds 64 MiB are
 * rejected with RSA_EINVAL.  The first call on a device looks up the array's
 * device address (once per device, with that device current, and again after
 * that device's context has been destroyed and re-created, e.g. by
 * cudaDeviceReset); make that first call before any stream capture starts on
 * the device.  Every call
 * reuses the same array: a call re-initialises what it needs, but two calls
 * whose work overlaps on the GPU (other streams, other threads) race on it.
 * Synchronises `stream` like rsa_run_seeds; returns the first per-sample
 * error code, as rsa_results does. */
int rsa_run_static(uint32_t L, uint32_t k, const uint64_t *seeds, uint32_t n, uint32_t *n_j,
                   uint32_t *n_c, void *stream);

/* ---- batching of uneven shapes (no counterpart in the paper: a way of
 * running many of its samples at once) ---------------------------------- */

/* Small lattices, one CTA per sample: all greedy rounds and the whole
 * first-wrap search of a sample run in one CTA's shared memory, and the n
 * samples -- of any mix of shapes -- run in one persistent launch (each CTA
 * takes the next sample from a work counter).  Sample i has lattice L[i],
 * k-mer length k[i] and seed seeds[i] (host arrays of n, read); n_j, n_c
 * are host arrays of n (written).  Results equal rsa_run_seeds +
 * rsa_results for the same (L, k, seed).  Every sample needs L <= 128 and
 * L^2 / k <= 4096 (RSA_EINVAL otherwise).  threads: CTA size, a multiple of
 * 32 up to 1024 (0 = 512).  Allocates its job table stream-ordered on
 * `stream` and synchronises it; returns the first per-sample error code. */
int rsa_run_small(const uint32_t *L, const uint32_t *k, const uint64_t *seeds, uint32_t n,
                  uint32_t threads, uint32_t *n_j, uint32_t *n_c, void *stream);

/* A batch of samples of uneven shapes (same arrays as rsa_run_small, any
 * 1 <= k <= L <= 32768): samples are grouped by shape, each shape runs the
 * way rsa_tune picks for it, the small-lattice groups together in one
 * persistent launch and every other shape on its own handle and stream, all
 * concurrently (one host thread per such shape).  Work queued on `stream`
 * before the call runs first, work queued after it runs after the batch.
 * Handles and streams of the shapes seen are kept for later calls (their
 * device memory too) until rsa_mix_release().  Results are the same as
 * running each sample alone.  Calls that share a shape run one at a time on
 * it.  Set RSA_AUTOTUNE=0 to use the default choices instead of timing. */
int rsa_run_mix(const uint32_t *L, const uint32_t *k, const uint64_t *seeds, uint32_t n,
                uint32_t *n_j, uint32_t *n_c, void *stream);
void rsa_mix_release(void);
/* Measurement support (no counterpart in the paper): the number of kernel
 * launches made by rsa_run_small and by rsa_run_mix's cached handles since
 * the previous call, then reset.  Synchronises those handles' streams. */
unsigned long long rsa_mix_launches(void);

/* How a shape runs: RSA_MODE_SMALL (one CTA per sample, `threads` per CTA)
 * or RSA_MODE_GLOBAL (the tiled / long-k / general kernels over the whole
 * batch, `rounds_per_check` greedy rounds per captured graph chunk and host
 * check, `window_threads` threads per CTA of the long-k window pass, 0 for
 * the handle's default as rsa_set_window_threads(h, 0) gives it).
 * ms_per_sample is the time measured when the choice was made (0 for an
 * unmeasured default). */
#define RSA_MODE_GLOBAL 0
#define RSA_MODE_SMALL 1
typedef struct {
  uint32_t mode, threads, rounds_per_check, window_threads;
  double ms_per_sample;
} rsa_tune_t;

/* The choice for (L, k) and a batch of n samples on the current GPU.  Looked
 * up in a per-process table backed by a JSON-lines file ($RSA_TUNE_CACHE,
 * else $HOME/.cache/rsa_gb300/tune.jsonl), keyed by (GPU name, L, k, n
 * rounded up to a power of two).  If absent and `measure` is non-zero, every
 * candidate (small mode at 256 / 512 / 1024 threads where the shape fits it;
 * the global path at 2 / 4 / 8 rounds per check) is timed once on seeds
 * 1 .. n (at most 8 GB of workspace) and the fastest is kept and appended
 * to the file; otherwise a default is returned (small mode at 512 threads
 * where it fits, else the global path at 4 rounds per check and 256-thread
 * windows).  The long-k window pass is also timed at 128 threads per CTA
 * (twice the cells per thread) where the shape allows it. */
int rsa_tune(uint32_t L, uint32_t k, uint32_t n, int measure, rsa_tune_t *out);

/* Greedy rounds per captured graph chunk and host check of later runs on
 * this handle (1 .. 64, default 4).  Results do not depend on it. */
int rsa_set_rounds_per_check(rsa_t *h, uint32_t rounds);

/* CTA size of the long-k window pass of later runs on this handle: 256 or
 * 128 threads per CTA, each thread then holding twice as many cells of the
 * span; 0 restores the default (128 on the argmin-offset long-k path with
 * 4096-cell spans and k >= 512, 256 otherwise).  128 needs the argmin-offset long-k path
 * with spans of 2048 or 4096 cells (RSA_EINVAL otherwise).  Results do not
 * depend on it. */
int rsa_set_window_threads(rsa_t *h, uint32_t threads);

/* Copy the last run's results to caller-owned host arrays of length n
 * (n <= samples of the last run; either pointer may be NULL).  Synchronises
 * the run's stream.  Returns the first per-sample error code, if any; a
 * sample without a wrap has n_c = UINT32_MAX. */
int rsa_results(rsa_t *h, uint32_t *n_j, uint32_t *n_c, uint32_t n);

/* Per-sample diagnostics of the last run (any pointer may be NULL, arrays of
 * length n): rounds of the parallel greedy, bisection probes, contact edges
 * of the k-mer graph, and the status code. */
int rsa_sample_stats(rsa_t *h, uint32_t *rounds, uint32_t *probes, uint32_t *edges,
                     int32_t *status, uint32_t n);

/* Interspecific contacts at jamming (Sec. II.A, Eq. nxy: n_xy* =
 * n_xy / (n_x + n_y + n_xy)) for each of the last run's first n samples.
 * A contact is a lattice edge (4-neighbour pair on the torus) whose two
 * sites belong to different k-mers; n_x counts those between two horizontal
 * k-mers, n_y between two vertical ones, n_xy between perpendicular ones.
 * Host arrays of length n (any may be NULL). */
int rsa_contacts(rsa_t *h, uint32_t *n_x, uint32_t *n_y, uint32_t *n_xy, uint32_t n);

/* The configuration of the first m accepted k-mers (in RSA order) of sample
 * `sample` of the last run, 0 <= m <= n_j: m = n_c is the percolating state
 * and m = n_j the jamming state of Sec. III ("Structure of the percolating
 * and jamming states").  Clusters are connected components of occupied
 * sites, 4-neighbours on the torus (Sec. II.C).
 *
 * rsa_cluster_sizes: counts[s] = number of clusters made of exactly s k-mers
 *   (s k sites), s = 0 .. m; counts[0] = 0 and the sum of s counts[s] is m.
 *   n_s of Eq. CSD is counts[s] / L^2 for cluster size s k.  counts is a
 *   caller-owned host array of cap >= m + 1 entries (RSA_EINVAL otherwise);
 *   entries past m are zeroed.
 * rsa_wrap_dirs: *wrap_x (*wrap_y) = 1 iff some cluster winds round the
 *   torus along x (y) (Sec. II.D, "in one or both directions"); either
 *   pointer may be NULL.  The directions are those of the closed cycles'
 *   windings (a, b), decided from a L and b L modulo 2^16: exact whenever
 *   |a|, |b| < 2^16 / 2^v (2^v the largest power of two dividing L), which
 *   covers any cycle shorter than 2^16 L / 2^v lattice steps.
 *
 * Both run on the stream of the last run and return when the result is on
 * the host; they reuse that sample's union-find scratch, so call them after
 * rsa_results.  RSA_EINVAL for a bad sample, m or array; the sample's own
 * error code if it has no valid result; RSA_ETIMEOUT if a union-find walk hit
 * its cap. */
int rsa_cluster_sizes(rsa_t *h, uint32_t sample, uint32_t m, uint32_t *counts, uint32_t cap);
int rsa_wrap_dirs(rsa_t *h, uint32_t sample, uint32_t m, uint32_t *wrap_x, uint32_t *wrap_y);

/* TEST ONLY: the accepted candidates (idx) of sample `sample` of the last run,
 * sorted ascending; *count receives n_j; at most cap values are written. */
int rsa_accepted(rsa_t *h, uint32_t sample, uint32_t *idx, uint32_t cap, uint32_t *count);

/* TEST ONLY (no counterpart in the paper): lower the caps of the device
 * loops for later runs on this handle, so that a test can make each capped
 * loop run out on purpose and check that the run reports it and the GPU
 * stays usable.  0 restores a cap's default.
 *   round_cap  greedy rounds per sample (default n_j bound + 2): a sample
 *              still undecided after that many rounds stops with
 *              RSA_ETIMEOUT from rsa_results;
 *   uf_steps   steps of one union-find walk and retries of one link (default
 *              2^20): a walk that runs out stops its probe, RSA_ETIMEOUT;
 *   probe_cap  bisection probes per sample (default 40), RSA_ETIMEOUT;
 *   edge_cap   contact edges stored per sample (default: the buffer's
 *              capacity, min(2 L^2, 6 L^2/k + 4 L) + 64): more edges than
 *              that stop the sample with RSA_ENOMEM, and nothing is written
 *              past the cap.
 * Every loop ends by its cap; nothing waits without a limit or faults. */
int rsa_test_caps(rsa_t *h, uint32_t round_cap, uint32_t uf_steps, uint32_t probe_cap,
                  uint32_t edge_cap);

/* Measurement support (no counterpart in the paper).  rsa_profile(h, 1)
 * makes later runs record a CUDA event pair around every kernel launch on
 * the run's stream; rsa_kernel_stats() synchronises that stream and returns,
 * per kernel kind i < n_kinds, the summed device time in ms[i] and the
 * number of launches in launches[i] since the previous call, then resets
 * both (launch counts are kept even with profiling off).  rsa_kernel_name(i)
 * names kind i ("" past the last kind). */
int rsa_profile(rsa_t *h, int enable);
int rsa_kernel_stats(rsa_t *h, double *ms, unsigned long long *launches, uint32_t n_kinds);
const char *rsa_kernel_name(uint32_t kind);
/* Work done by the round kernels since the previous call (then reset; n <= 4
 * values are written).  Tile path (power-of-two k <= 32): out[0] cells of live
 * tiles processed by the cell-minimum pass, out[1] live candidates it gave a
 * priority, out[2] / out[3] cells and accepted candidates of the acceptance
 * pass.  Long-k path: out[0] / out[1] cells processed by the horizontal /
 * vertical window-minimum passes, out[2] by the acceptance passes, out[3] by
 * the code pass (segments and tiles without live candidates are skipped and
 * not counted).  Zero on the general path. */
int rsa_work_stats(rsa_t *h, unsigned long long *out, uint32_t n);

/* Bytes of device workspace a run of n_samples needs for (L, k). */
int rsa_workspace_bytes(uint32_t L, uint32_t k, uint32_t n_samples, uint64_t *bytes);

/* Use caller-owned device memory (e.g. a torch tensor) as the workspace;
 * the library never frees it.  dev_ptr must be 256-byte aligned.  A run that
 * needs more than `bytes` fails with RSA_ENOMEM.  Pass NULL to unbind. */
int rsa_bind_workspace(rsa_t *h, void *dev_ptr, uint64_t bytes);

/* Release the handle and any device memory the library allocated. */
void rsa_destroy(rsa_t *h);

/* Message of the last error on this thread ("" if none). */
const char *rsa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSA_GB300_H */
