/*
 * pa_gb300.h -- C ABI of the GB300 (sm_103a) MMH-MH privacy-amplification hash
 * of "An efficient hybrid hash based privacy amplification algorithm for QKD"
 * (arXiv 2105.13678).
 *
 * The library compresses an n-bit partially secure key to r output bits:
 *   Algorithm 1 (Sec. 3.1):  x = <x_1..x_k>, a = <a_1..a_k> (gamma-bit slices),
 *   MMH, Eq. 2:              y = sum_i a_i x_i  mod p,  p = 2^gamma - 1,
 *   MH,  Eq. 4:              z = ((b y + c) mod 2^gamma) >> (gamma - r),
 * with gamma a Mersenne prime exponent and n <= k * gamma (step 0, Sec. 4).
 *
 * Conventions shared by every entry point
 *   - Bit strings are arrays of uint64_t; bit t lives in word t/64 at bit t%64.
 *   - key:  ceil(n/64) words.  Bits at or past n in the last word are ignored.
 *   - seed: ceil((k+2)*gamma/64) words: a_1..a_k, then b, then c, each a
 *           gamma-bit slice in that order.  a_i is taken mod p (the all-ones
 *           slice is p == 0); bit 0 of b is forced to 1 (gcd(b, 2) = 1).
 *   - out:  ceil(r/64) words; bits at or past r are written as 0.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Device pointers are owned by the caller and never freed by the library.
 *     A plan owns the device workspace and tables it allocates.
 *   - Calls are asynchronous on `stream` unless stated otherwise; a plan's
 *     workspace is reused by every call on that plan, so calls that share a
 *     plan must be ordered (same stream, or event-ordered).
 *
 * Return codes: PA_OK (0); PA_RELOAD (1): some key slice x_i equals
 * 2^gamma - 1 (Algorithm 1 reload rule) -- the output is zero-filled and the caller
 * must draw a new key; negative values are errors.
 */
#ifndef PA_GB300_H
#define PA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_OK 0
#define PA_RELOAD 1
#define PA_ERR_INVALID (-1)     /* bad argument: n = 0, r = 0, null pointer, no gamma fits */
#define PA_ERR_NOMEM (-2)       /* device or host allocation failed */
#define PA_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define PA_ERR_TIMEOUT (-4)     /* a bounded wait expired */
#define PA_ERR_BUDGET (-5)      /* job larger than the server's whole HBM budget */
#define PA_ERR_CANCELLED (-6)   /* job cancelled by pa_serve_destroy */
#define PA_ERR_UNSUPPORTED (-7) /* sizes beyond what the kernels implement */
#define PA_ERR_BUSY (-8)        /* server queue full / ticket unknown */

/* Step-0 parameters (Sec. 4).  Pass NULL for the defaults. */
typedef struct pa_params {
    uint32_t gamma;        /* 0: smallest Mersenne exponent >= r + gamma_margin;
                              otherwise a Mersenne exponent > r to use as is   */
    uint32_t gamma_margin; /* default 128: gamma - r >= margin keeps the
                              2^(r - gamma) term of the Sec. 3.2 bounds tiny;
                              with params != NULL, 0 means gamma > r strictly */
    uint32_t tune;         /* 1: time the candidate four-step splits and column
                              tiles of each transform shape on this plan's
                              workspace at pa_plan time and keep the fastest;
                              with backend AUTO also build both backends and
                              keep the one whose hash measured faster.  Cached
                              per process (pa_tune_cache_save / _load carry it
                              across processes); 0: default geometry and the
                              AUTO rule below.  The output bits do not depend
                              on it.                                          */
    uint32_t backend;      /* PA_BACKEND_AUTO (0), PA_BACKEND_GOLDILOCKS or
                              PA_BACKEND_P3; the output bits do not depend on it */
    uint32_t reserved[4];  /* must be zero */
} pa_params;

/* Arithmetic of the exact products (a design choice; the paper fixes only
 * the results of Eq. 2 and Eq. 4):
 *   GOLDILOCKS  one transform over q = 2^64 - 2^32 + 1 with the irrational-
 *               base weighted transform (cyclic mod 2^G - 1 without padding);
 *   P3          zero-padded transforms over three 30-bit primes, the
 *               coefficients recovered by the Chinese remainder theorem
 *               (about half the integer work per transformed element);
 *   AUTO        P3 when it is feasible and its Eq. 2 transform is no longer
 *               than the Goldilocks one, or twice as long but at most 2^20
 *               (where P3 was measured faster); else GOLDILOCKS. */
#define PA_BACKEND_AUTO 0u
#define PA_BACKEND_GOLDILOCKS 1u
#define PA_BACKEND_P3 2u

typedef struct pa_plan_info {
    uint64_t n_bits, r_bits;
    uint32_t gamma;           /* Mersenne exponent, p = 2^gamma - 1           */
    uint32_t backend;         /* PA_BACKEND_GOLDILOCKS or PA_BACKEND_P3          */
    uint64_t k;               /* segments, ceil(n / gamma)                      */
    uint64_t key_words, seed_words, out_words;
    uint64_t mmh_len;         /* transform length for Eq. 2                      */
    uint64_t mh_len;          /* transform length for Eq. 4                      */
    uint64_t workspace_bytes; /* device bytes owned by the plan                 */
} pa_plan_info;

typedef struct pa_plan_s pa_plan_t;

/* Step 0 (Sec. 4, Table 3): choose gamma and k for (n, r) and allocate the
 * plan's device workspace and twiddle/weight tables on the current device.
 * Blocking.  Returns PA_ERR_INVALID if no tabulated exponent fits and
 * PA_ERR_UNSUPPORTED beyond the largest transform the kernels implement. */
int pa_plan(uint64_t n_bits, uint64_t r_bits, const pa_params *params, pa_plan_t **out);
int pa_plan_info_get(const pa_plan_t *plan, pa_plan_info *info);
int pa_plan_destroy(pa_plan_t *plan);

/* Algorithm 1 on device buffers (key, seed, out as above; `status` is an
 * optional device int that receives PA_OK or PA_RELOAD when the work runs).
 * Asynchronous: returns PA_OK once enqueued. */
int pa_hash(pa_plan_t *plan, const uint64_t *key, const uint64_t *seed, uint64_t *out,
            int *status, void *stream);

/* Algorithm 1 on HOST buffers: copies key and seed in (overlapped with the
 * column transforms), runs, copies out and synchronises `stream`.  Returns
 * PA_OK, PA_RELOAD or an error. */
int pa_hash_host(pa_plan_t *plan, const uint64_t *key, const uint64_t *seed, uint64_t *out,
                 void *stream);

/* Asynchronous form of pa_hash_host for streams of blocks: enqueues the copies
 * (on a plan-owned copy stream), the hash and the copy-out on `stream` and
 * returns.  `status` is a HOST int (pinned memory recommended, may be NULL)
 * written with PA_OK / PA_RELOAD when the work completes.  Two staging slots
 * alternate, so the input copies of one call overlap the transforms of the
 * previous call; key, seed, out and status must stay valid until `stream` has
 * passed the call.  Pinned host buffers are needed for the overlap. */
int pa_hash_host_async(pa_plan_t *plan, const uint64_t *key, const uint64_t *seed, uint64_t *out, int *status,
                       void *stream);

/* The MMH value y = sum a_i x_i mod p of Eq. 2 (ceil(gamma/64) device words,
 * canonical in [0, p)), for checking the intermediate.  Asynchronous. */
int pa_debug_mmh(pa_plan_t *plan, const uint64_t *key, const uint64_t *seed, uint64_t *y,
                 int *status, void *stream);

/* Comparison scheme (the prior-art scheme the paper compares against): the
 * modular-arithmetic hash over the whole key, Eq. 4 with alpha = n, beta = r:
 * z = ((b x + c) mod 2^n) >> (n - r), b forced odd.  The plan's seed holds
 * b = bits [0, n) and c = bits [n, 2n) (ceil(2n/64) words; pa_plan_info
 * reports gamma = n, k = 0, mmh_len = 0).  Only pa_hash and pa_hash_batch
 * accept such a plan.  n <= about 1.3e8 bits (one exact n x n-bit product). */
int pa_mh_plan(uint64_t n_bits, uint64_t r_bits, pa_plan_t **out);

/* Comparison scheme: Toeplitz-hashing PA (the other prior-art family the
 * paper compares against, Sec. 1 and Table 1, computed with the key split into
 * segments): z = T x over GF(2), T the r x n Toeplitz matrix
 * T[i][j] = s[i - j + n - 1] of a seed s of n + r - 1 bits
 * (ceil((n + r - 1)/64) words).  Key segments and output blocks of
 * 2^block_log bits (6..22; 0: the smallest power of two >= r, at most 2^22);
 * each block product is an exact integer convolution of 1-bit digits on the
 * three-prime transforms of length 4 * 2^block_log, accumulated over the
 * segments, whose coefficients' parities are the output bits.  Only pa_hash
 * (status always PA_OK) and pa_hash_batch accept such a plan; pa_plan_info
 * reports gamma = 0, k = the number of segments, mmh_len = the transform
 * length.  Device workspace about 96 n bytes. */
int pa_toeplitz_plan(uint64_t n_bits, uint64_t r_bits, uint32_t block_log, pa_plan_t **out);

/* Seed reuse.  When the same hash seed (a, b, c) serves many blocks,
 * pa_seed_prepare transforms a_1..a_k and b once and keeps their spectra (and
 * a copy of the seed) in the plan: k N_mmh + N_mh 64-bit words (GOLDILOCKS) or
 * 3 (k N_mmh + N_mh) 32-bit words (P3) plus the seed, allocated on the first
 * call (blocking).  pa_hash_prepared then runs Algorithm 1 on a
 * key with that seed, transforming only the key slices and y: k + 3 transforms
 * instead of 2k + 4, same output bits as pa_hash with the same seed.  Returns
 * PA_ERR_INVALID if the plan has no prepared seed.  Both are asynchronous on
 * `stream` and use the plan's workspace like pa_hash. */
int pa_seed_prepare(pa_plan_t *plan, const uint64_t *seed, void *stream);
int pa_hash_prepared(pa_plan_t *plan, const uint64_t *key, uint64_t *out, int *status, void *stream);

/* Algorithm 1 without any device allocation, for callers that cannot call
 * cudaMalloc (device memory owned by another allocator or pool, code paths
 * where an allocation and its possible device synchronisation are not
 * allowed, or a device footprint fixed at start-up).  Same result as
 * pa_plan(n, r, params) followed by pa_hash.  All intermediate buffers and
 * tables live in one library-owned static device array of
 * PA_NOALLOC_SCRATCH_BYTES, resident on every GPU that loads the library until
 * the process exits.  Blocks whose workspace does not fit (about n <= 1e7 key
 * bits at r = 0.1 n) return PA_ERR_UNSUPPORTED.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and should be
 * made before any stream capture on that device; the lookup is repeated when
 * the device's context has been re-created (after cudaDeviceReset).  Every call shares the array:
 * calls whose work overlaps on the GPU race, so order them (one stream, or
 * events).  key, seed, out and status are device pointers as for pa_hash.
 * Asynchronous.  This entry point has no counterpart in the paper. */
#define PA_NOALLOC_SCRATCH_BYTES (16ULL << 20)
int pa_hash_noalloc(uint64_t n_bits, uint64_t r_bits, const pa_params *params, const uint64_t *key,
                    const uint64_t *seed, uint64_t *out, int *status, void *stream);

/* Batched Algorithm 1 over `count` independent blocks, each with its own plan
 * (plans must be distinct objects).  keys/seeds/outs are HOST arrays of device
 * pointers; statuses is a device int[count] (may be NULL).  The first call for
 * a given list of plans and buffers captures one CUDA graph whose branches run
 * the blocks concurrently; later calls with the same arguments replay it.
 * Asynchronous. */
int pa_hash_batch(pa_plan_t *const *plans, const uint64_t *const *keys,
                  const uint64_t *const *seeds, uint64_t *const *outs, int *statuses,
                  int count, void *stream);
/* Drop the graphs cached by pa_hash_batch (they are also dropped when one of
 * their plans is destroyed). */
int pa_batch_cache_clear(void);

/* ---- serving: a continuous-batching request loop on one GPU ---------------
 * Jobs are admitted while their device bytes (plan workspace) fit in the HBM
 * budget; admitted jobs run concurrently on `slots` streams; others wait in a
 * FIFO.  key/seed/out are DEVICE pointers owned by the caller and must stay
 * valid until the job completes.  The server's plans use stream-ordered
 * device memory (cudaMallocAsync from the device's default pool), so building
 * and dropping them does not synchronise the device.  Latency is measured
 * from submit to a host function that runs when the job's work is done. */
typedef struct pa_server_s pa_server_t;
typedef struct pa_serve_config {
    uint64_t hbm_budget_bytes; /* admission budget for plan workspaces         */
    uint32_t slots;            /* concurrent jobs on the device (streams)      */
    uint32_t max_queue;        /* pending jobs before submit returns PA_ERR_BUSY */
    pa_params params;          /* step-0 parameters for every job               */
} pa_serve_config;
typedef struct pa_serve_stats {
    uint64_t submitted, completed, failed, cancelled, queued, running;
    uint64_t bits_completed;          /* sum of n over completed jobs          */
    double p50_latency_ms, p99_latency_ms, max_latency_ms; /* submit -> done  */
    double busy_seconds;              /* first submit -> last completion       */
    uint64_t peak_budget_bytes;       /* highest admitted workspace in use     */
} pa_serve_stats;

int pa_serve_create(const pa_serve_config *cfg, pa_server_t **out);
int pa_serve_submit(pa_server_t *srv, uint64_t n_bits, uint64_t r_bits, const uint64_t *key,
                    const uint64_t *seed, uint64_t *out, uint64_t *ticket);
int pa_serve_poll(pa_server_t *srv, uint64_t ticket, int *status);  /* PA_OK if done, PA_ERR_BUSY if not */
int pa_serve_wait(pa_server_t *srv, uint64_t ticket, uint64_t timeout_ns, int *status);
int pa_serve_stats_get(pa_server_t *srv, pa_serve_stats *stats);
/* Start the statistics afresh (counters, latencies, busy time; the peak
 * budget restarts at what is held now).  Jobs in flight are counted when they
 * complete. */
int pa_serve_stats_reset(pa_server_t *srv);
/* Stop the server: later submits return PA_ERR_CANCELLED, queued jobs finish
 * with status PA_ERR_CANCELLED, running jobs complete; returns when none is
 * running.  poll, wait and stats keep working until pa_serve_destroy. */
int pa_serve_shutdown(pa_server_t *srv);
int pa_serve_destroy(pa_server_t *srv); /* pa_serve_shutdown, then frees the server */

/* ---- tracing: per-kernel device time ---------------------------------------
 * pa_trace_enable(1) clears earlier records and brackets every later kernel
 * launch of the library with a CUDA event pair on its launching stream (not
 * while the stream is being captured into a graph); pa_trace_enable(0) stops
 * recording.  pa_trace_collect waits for the recorded events and fills up to
 * max_entries aggregates, one per kernel and stage ("mmh.row_mac", ...);
 * *count receives the number of distinct entries. */
typedef struct pa_trace_entry {
    char name[32];
    uint64_t launches;
    double total_ms;
} pa_trace_entry;
int pa_trace_enable(int on);
int pa_trace_collect(pa_trace_entry *out, int max_entries, int *count);
/* Restrict tracing to the launches named `name` ("mmh.<kernel>" or
 * "mh.<kernel>", as pa_trace_collect reports them), so that one kernel can
 * be timed with two events per launch and nothing between the others;
 * NULL or "" traces every launch again.  Host-only; never fails. */
int pa_trace_select(const char *name);

/* ---- diagnostics for host-side checks (no device work) --------------------
 * pa_plan_estimate_bytes: device bytes pa_plan would allocate for (n, r).
 * pa_field_constants: the primitive 2^log_n-th root of unity omega and the
 *   element theta with theta^(2^log_n) = 2 in F_q, q = 2^64 - 2^32 + 1, that
 *   the weighted transforms use (log_n <= 26).
 * pa_transform_len: log2 of the transform length chosen for a modulus of
 *   2^G - 1 with K accumulated products. */
int pa_plan_estimate_bytes(uint64_t n_bits, uint64_t r_bits, const pa_params *params, uint64_t *bytes);
int pa_field_constants(uint32_t log_n, uint64_t *omega, uint64_t *theta);
int pa_transform_len(uint64_t G, uint64_t K, uint32_t *log_n);
/* Four-step geometry of a plan's transform (stage 0: Eq. 2, stage 1: Eq. 4):
 * N = 2^log_r x 2^log_c, column passes work on tiles of tile_cols columns. */
int pa_plan_geometry(const pa_plan_t *plan, int stage, uint32_t *log_r, uint32_t *log_c, uint32_t *tile_cols);
/* Device check of the F_q arithmetic used inside the transforms: for i < n,
 * out[4i .. 4i+3] = (a[i] + b[i], a[i] - b[i], a[i] * b[i], (a[i] mod 2^32) * b[i])
 * mod q, canonical; a, b, out (4n words) are device arrays, any 64-bit inputs.
 * Asynchronous. */
int pa_selftest_field(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n, void *stream);

/* Tuning results (pa_params.tune): pa_tune_cache_save writes every cached
 * geometry and backend decision of this process to a text file and returns the
 * number of entries; pa_tune_cache_load adds a file's entries to the cache and
 * returns their number, or PA_ERR_INVALID if the file cannot be read or holds
 * a malformed or invalid entry (the valid ones are kept).  Host-only. */
int pa_tune_cache_save(const char *path);
int pa_tune_cache_load(const char *path);

/* ---- tensor-core limb convolution (the alternative arithmetic, measured) ---
 * An exact n-limb product as int8 matrix products costs 2 n^2 multiply-adds
 * (32-limb blocks: Toeplitz(B_q) (64 x 32) times columns A_p); GB300 has no
 * int8 tcgen05.mma kind, so these use the warp-level mma.sync m16n8k32.
 * pa_tc_limbconv_tile: for t < ntiles, out[t] (64 x 8 int32, row-major) =
 *   Toeplitz(bq[t]) x a[t], bq[t] 32 limbs, a[t] 8 columns of 32 limbs
 *   (a[t][c * 32 + j]); device pointers; asynchronous.  Entry i of column c is
 *   the convolution of bq[t] with column c at index i (exact).
 * pa_tc_int8_rate: int8 multiply-add throughput of mma.sync on this device
 *   (ctas_per_sm x SMs CTAs of 8 warps, `iters` rounds of 8 independent
 *   products each, timed with CUDA events); blocking. */
int pa_tc_limbconv_tile(const uint8_t *bq, const uint8_t *a, int32_t *out, int ntiles, void *stream);
int pa_tc_int8_rate(uint64_t iters, uint32_t ctas_per_sm, double *tops, double *ms);

/* Failure injection for tests of the error paths (host side only; no device
 * work fails): of the library's next device and pinned host allocations,
 * `skip` succeed and the following `count` fail as if the memory were
 * exhausted (the call returns PA_ERR_NOMEM).  pa_debug_fail_allocs(0, 0)
 * switches it off.  Not thread-safe; for tests. */
int pa_debug_fail_allocs(uint32_t skip, uint32_t count);

/* Human-readable name of a return code (static string). */
const char *pa_status_string(int code);
/* Library version string. */
const char *pa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PA_GB300_H */
