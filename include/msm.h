/*
 * msm.h -- C ABI of the GB300 epsilon-neighbour-graph library.
 *
 * Method: Uno, Sugiyama and Tsuda, "Efficient Construction of Neighborhood
 * Graphs by the Multiple Sorting Method".  Points are mapped to ell-bit
 * strings by sign random projection (Sec. 3.2, Eq. 3), repeated for Q
 * independent replicates (Sec. 4.1); the multiple sorting method with
 * blockwise masking (Sec. 2.2) enumerates, per replicate, all string pairs
 * within Hamming distance d (Eq. 5); the union of candidates is then checked
 * against the exact distance (Sec. 4.1, last step).
 *
 * General rules for every entry point:
 *   - Pointers documented "device" must be CUDA device (or managed) memory of
 *     the current device; "host" pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls that must read a count back
 *     (documented) synchronise on it before returning.  Such reads go through
 *     a 1 KB host-mapped pinned buffer per calling thread (allocated by its
 *     first read, kept for the life of the process) written by a one-warp
 *     kernel, not through a copy engine, so a device-to-host copy that the
 *     caller keeps running on another stream does not hold them up.
 *   - Inputs are never modified.  Return value is MSM_OK or a negative
 *     MSM_E_* code; msm_last_error() gives a message for the calling thread.
 *   - Pair encoding: (uint64_t)i << 32 | j with 0 <= i < j < n.
 *   - String layout: replicate-major [Q][n][W] uint64 words, W = ceil(ell/64);
 *     bit c of a string is bit (c & 63) of word (c >> 6); bits >= ell are 0.
 *   - Blocks: block b (0-based, b < k) covers bits [floor(b*ell/k),
 *     floor((b+1)*ell/k)).
 *   - Limits: 1 <= ell <= 256, 1 <= k <= min(ell, 32), 0 <= d < k,
 *     2 <= n < 2^31, 1 <= dim <= 4096.
 */
#ifndef MSM_H
#define MSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MSM_OK 0
#define MSM_E_INVAL (-1)     /* argument outside the documented limits */
#define MSM_E_NOMEM (-2)     /* an allocation failed */
#define MSM_E_OVERFLOW (-3)  /* a caller-sized output is too small */
#define MSM_E_CUDA (-4)      /* a CUDA runtime call or launch failed */
#define MSM_E_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define MSM_E_ZERO_NORM (-6) /* cosine metric with an all-zero row */
#define MSM_E_NONFINITE (-7) /* NaN or Inf in the input vectors */

/* ---- element types of X ---- */
#define MSM_DT_F32 0
#define MSM_DT_BF16 1

/* ---- metrics ---- */
#define MSM_COSINE 0    /* Eq. 2: 1 - x_i.x_j / (|x_i| |x_j|) */
#define MSM_EUCLIDEAN 1 /* |x_i - x_j|_2 */

/* ---- output modes of msm_eps_graph ---- */
#define MSM_OUT_PAIRS_DIST 0 /* pairs and float distances */
#define MSM_OUT_PAIRS 1      /* pairs only (dist = NULL) */
#define MSM_OUT_COUNT 2      /* count only (pairs = dist = NULL) */

/* ---- string families (msm_params.hash) ---- */
#define MSM_HASH_SIGN 0  /* sign random projection, Eq. 3 (1 bit per symbol) */
#define MSM_HASH_E2LSH 1 /* E2LSH symbols floor(r^T x / width + u) (Datar et al.) */

/* ---- flags ---- */
#define MSM_FLAG_CANONICAL 1 /* sort output pairs ascending (i, then j) */
#define MSM_FLAG_SIMT_PROJECTION 2 /* project on CUDA cores, not tcgen05 */

/* Device memory provider.  alloc(bytes, stream, ctx) returns device memory
 * usable in stream order on `stream` (NULL on failure); free(ptr, stream,
 * ctx) releases it in stream order.  Scratch memory is freed before the
 * call returns; output buffers (msm_pairs) stay alive and belong to the
 * caller, who releases them with the same allocator (msm_free_pairs).
 * A NULL allocator selects cudaMallocAsync / cudaFreeAsync on `stream`. */
typedef struct msm_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} msm_allocator;

/* A pair list produced by the library (device memory from the allocator). */
typedef struct msm_pairs {
  uint64_t* pairs; /* device [count], (i << 32) | j, i < j; NULL if count 0 */
  float* dist;     /* device [count] or NULL (see output modes)            */
  int64_t count;
} msm_pairs;

/* Counters and per-phase device times of one call (all optional). */
typedef struct msm_stats {
  int64_t Q;              /* replicates used                                  */
  int64_t masks;          /* (replicate, kept-block set) groupings performed  */
  int64_t checks;         /* pairs inspected inside groups of equal keys      */
  int64_t cand;           /* |E| = |E_1 u ... u E_Q| (Sec. 4.1)               */
  int64_t type1;          /* |E| - result size: type-I errors removed (4.2)   */
  int64_t proj_recompute; /* projection signs decided in double precision     */
  int64_t dist_recompute; /* epsilon comparisons decided in double precision  */
  int64_t overflow_retries; /* candidate-buffer regrowths                     */
  float ms[8]; /* device ms: 0 norms+R, 1 projection, 2 grouping sorts,
                  3 group boundaries, 4 in-group checks, 5 recheck,
                  6 canonical sort, 7 whole call                             */
  /* Per kernel class, summed over the call's launches (CUDA events around
   * each launch): 0 projection, 1 radix histogram, 2 radix scatter,
   * 3 scans, 4 group boundaries, 5 in-group pair check, 6 recheck,
   * 7 other (norms, generator, canonical sort). */
  float kernel_ms[8];
  int64_t kernel_launches[8];
  /* String geometry used (chosen by the Sec. 4.3 rule when msm_params.ell
   * was 0) and that rule's output-size estimate S (-1 when not estimated). */
  int ell, k, d, reserved;
  double S_est;
  /* In-group pairs that took the per-pair tests of the pair check: the
   * pairs left by its tile-level reference prefilter (a subset of
   * `checks`; the rest were decided a tile or a row at a time). */
  int64_t evaluated;
} msm_stats;

/* Parameters of msm_eps_graph. */
typedef struct msm_params {
  int ell;  /* string length in bits (Sec. 3.2); 0 = automatic: ell, k,
               d and Q from the Sec. 4.3 rule (msm_choose_params) on an
               output-size estimate (msm_estimate_output, 2^22 samples)  */
  int k;    /* blocks per string (Sec. 2.2)                             */
  int d;    /* Hamming threshold = masked blocks per grouping (Sec. 2.2) */
  int Q;    /* replicates; 0 = smallest Q meeting miss_ratio (Sec. 4.3) */
  uint64_t seed;     /* seed of R when R == NULL (msm_gaussian)         */
  const float* R;    /* optional device [Q][dim][ell] float projection  */
  int out_mode;      /* MSM_OUT_*                                       */
  int flags;         /* MSM_FLAG_*                                      */
  int group_bits;    /* grouping-key width 8..32; 0 = automatic         */
  int check_min_blocks; /* tuning: register budget of the pair check, as
                           resident CTAs per SM: 2, 4 or 5 for count-only
                           output (fused recheck), 6 or 8 otherwise;
                           0 = automatic                                  */
  int64_t cand_capacity; /* initial candidate buffer (pairs); 0 = auto */
  /* Optional projection features (learned form): when Y is non-NULL the
   * strings are the sign projection of Y (device [n][dim_y] of dtype_y)
   * instead of X, and R is [Q][dim_y][ell]; the recheck still uses X. */
  const void* Y;
  int dim_y;
  int dtype_y;
  /* Tuning (results never depend on these; 0 = automatic): */
  int masks_per_batch;   /* kept-block sets grouped per sort batch         */
  int check_ctas_per_sm; /* pair-check grid, CTAs per SM (1..16)           */
  /* String family.  MSM_HASH_E2LSH: ell counts symbols of symbol_bits bits
   * (2 or 4; 0 = 4), the low bits of floor(r^T x / width + u) with R drawn
   * as for Eq. 3 and u by msm_e2lsh_offsets from `seed`; width is the
   * bucket width in the units of X (0 = 4 radii, or the Sec. 4.3 rule when
   * ell == 0); d counts differing symbols; the bound uses msm_e2lsh_p at
   * the radius (Euclidean eps, or sqrt(2 eps) for cosine on unit rows). */
  int hash;
  int symbol_bits;
  float width;
} msm_params;

/* Library version (major * 10000 + minor * 100 + patch). */
int msm_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices); a diagnostic for launch accounting. */
int64_t msm_launch_count(void);

/* Message for a status code, and the last error message of this thread. */
const char* msm_strerror(int status);
const char* msm_last_error(void);

/* Sec. 4.2: non-collision probability of one sign bit at the radius:
 * p = arccos(1 - eps) / pi for MSM_COSINE; for MSM_EUCLIDEAN on unit
 * vectors |x - y|^2 = 2 (cosine distance) (Sec. 5.1), so
 * p = arccos(1 - eps^2 / 2) / pi.  Returns -1 for an invalid eps. */
double msm_collision_p(int metric, double eps);

/* Sec. 4.2 bound on the expected missing-edge ratio,
 * (1 - sum_{t=0}^{d} C(ell, t) p^t (1 - p)^(ell - t))^Q.  Returns -1 on
 * invalid arguments. */
double msm_miss_bound(int ell, int d, double p, int Q);

/* Sec. 4.3: smallest Q >= 1 whose bound is <= gamma, written to *Q.
 * MSM_E_INVAL if gamma <= 0, p outside [0, 1), or no Q <= 2^24 suffices. */
int msm_solve_Q(int ell, int d, double p, double gamma, int* Q);

/* Sec. 4.3 parameter rule (host arithmetic).  Given n, the non-collision
 * probability p at the radius (msm_collision_p), gamma and an estimate S of
 * the output size:
 *   ell = 2 ceil(log2 n) (halved when S < 1), at most 256;
 *   replicate budget Qmax = min(24, max(ceil(30 S / n), 5));
 *   d = the smallest d >= 0 whose bound-minimal Q (msm_solve_Q) is <= Qmax;
 *   k = max(2 d, 1): the fewest blocks for which k - d blocks hold half of
 *   the string, log2 n letters;
 *   Q = that minimal Q.
 * MSM_E_INVAL if no d with k <= min(ell, 32) meets the budget. */
int msm_choose_params(int64_t n, double p, double gamma, double S, int* ell,
                      int* k, int* d, int* Q);

/* Sec. 4.3 output-size estimate: S = (pairs within eps among `samples`
 * uniformly random pairs i != j) / samples * n (n - 1) / 2.  Pair t is
 * drawn from block t of Philox4x64-10 with key {seed, 1}: i = w0 mod n,
 * j = w1 mod (n - 1), then j += 1 if j >= i.  X: device [n][dim].
 * Synchronises. */
int msm_estimate_output(const void* X, int64_t n, int dim, int dtype,
                        int metric, float eps, int64_t samples,
                        uint64_t seed, double* S, void* stream);

/* E2LSH (Sec. 3.1; Datar et al. 2004): non-collision probability of one
 * symbol for a pair at distance c when the bucket width is w c:
 * 2 Phi(-w) + 2 / (sqrt(2 pi) w) (1 - exp(-w^2 / 2)).  -1 if w <= 0. */
double msm_e2lsh_p(double w);

/* E2LSH bucket offsets, `count` floats in [0, 1) to device `out`: element e
 * is (w0 >> 40) 2^-24 with w0 word 0 of Philox4x64-10 block e under key
 * {seed, 2}.  Asynchronous. */
int msm_e2lsh_offsets(uint64_t seed, int64_t count, float* out, void* stream);

/* E2LSH symbol strings: symbol c of replicate q for row i is the low
 * symbol_bits bits (two's complement) of h = floor(t / width + u[q][c]),
 * t = r_{q,c}^T x_i; packed LSB first, symbol c at bits [c sb, (c+1) sb)
 * of strings [Q][n][ceil(ell sb / 64)] (device, caller-owned).  Every h is
 * the one of the double-precision evaluation of that expression with t by
 * sequential fma.  R: device [Q][dim][ell] float; u: device [Q][ell].
 * recomputed (optional host): symbols settled in double.  Synchronises. */
int msm_project_e2lsh(const void* X, int64_t n, int dim, int dtype,
                      const float* R, const float* u, float width, int ell,
                      int Q, int symbol_bits, uint64_t* strings,
                      int64_t* recomputed, void* stream);

/* msm_enumerate over symbol strings of symbol_bits (1, 2 or 4) bits: ell
 * counts symbols, blocks are groups of whole symbols, d counts differing
 * symbols.  Synchronises. */
int msm_enumerate_symbols(const uint64_t* strings, int64_t n, int ell,
                          int symbol_bits, int k, int d, int Q, int flags,
                          const msm_allocator* alloc, msm_pairs* out,
                          msm_stats* stats, void* stream);

/* Step A0' (Sec. 3.2: R has i.i.d. N(0, 1) entries).  Writes `count`
 * standard normal floats to device `out`: element e comes from block e/4 of
 * the counter-based generator Philox4x64-10 (Salmon et al., SC 2011) with
 * counter {e/4, 0, 0, 0} and key {seed, 0}; the block's words (w0, w1) and
 * (w2, w3) feed two Box-Muller pairs, evaluated in double precision and
 * rounded to float.  Asynchronous. */
int msm_gaussian(uint64_t seed, int64_t count, float* out, void* stream);

/* Step A1, Eq. 3: strings[q][i] bit c = 1 iff r_{q,c}^T x_i > 0.
 *   X        device [n][dim], element type `dtype` (row-major, rows packed)
 *   R        device [Q][dim][ell] float, or NULL to draw it with msm_gaussian
 *            from `seed` (R_q is the q-th [dim][ell] block)
 *   strings  device [Q][n][W] uint64, caller-owned, fully overwritten
 *   flags    MSM_FLAG_SIMT_PROJECTION forces the CUDA-core kernel; otherwise
 *            rows of 128/256/384/512 bytes with a 16-byte-aligned X use the
 *            tcgen05 tensor-core kernel
 *   recomputed  optional host pointer: number of signs decided in double
 *            precision because a lower-precision result lay within its
 *            rounding-error bound of zero (synchronises when non-NULL)
 * The sign of every bit equals the sign of the double-precision dot product
 * accumulated by sequential fma over the dim coordinates.
 * Scratch comes from cudaMallocAsync; the call synchronises on `stream`. */
int msm_project(const void* X, int64_t n, int dim, int dtype, const float* R,
                uint64_t seed, int ell, int Q, int flags, uint64_t* strings,
                int64_t* recomputed, void* stream);

/* Steps A3-A7 (Sec. 2.2, Eq. 5, Appendix): every pair (i, j), i < j, whose
 * strings lie within Hamming distance d in at least one of the Q pools,
 * reported once.
 *   strings  device [Q][n][W] uint64 (layout above)
 *   out      receives the pair list (dist = NULL), allocated with `alloc`;
 *            ascending when flags has MSM_FLAG_CANONICAL
 *   stats    optional host pointer
 * Synchronises on `stream` (counts are read back). */
int msm_enumerate(const uint64_t* strings, int64_t n, int ell, int k, int d,
                  int Q, int flags, const msm_allocator* alloc,
                  msm_pairs* out, msm_stats* stats, void* stream);

/* Step A8 (Sec. 4.1, last step): keep the candidate pairs whose distance is
 * <= eps (inclusive, Def. 1.1).
 *   X         device [n][dim] of `dtype`
 *   cand      device [m] candidate pairs (any order, i < j < n)
 *   pairs_out device [m] capacity, caller-owned; dist_out device [m] or NULL
 *   count     host pointer, receives the number kept (synchronises)
 *   recomputed optional host pointer: comparisons decided in double
 * Every decision equals the one made on the double-precision distance of
 * Eq. 2 (cosine) or the Euclidean norm, accumulated by sequential fma;
 * returned distances are within 1e-5 relative of that value.  Output order
 * is unspecified.  MSM_E_ZERO_NORM for a zero row under MSM_COSINE.
 * MSM_E_INVAL when some candidate is not a pair i < j < n: such a candidate
 * is skipped without reading X, and the outputs of that call are then
 * incomplete. */
int msm_recheck(const void* X, int64_t n, int dim, int dtype, int metric,
                float eps, const uint64_t* cand, int64_t m,
                uint64_t* pairs_out, float* dist_out, int64_t* count,
                int64_t* recomputed, void* stream);

/* msm_recheck for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment variant.  It serves code that runs
 * inside a host application owning the whole GPU (for example a serving
 * process whose caching allocator has reserved the device, or a component
 * held to a fixed memory budget), where a cudaMalloc issued from this
 * library would fail or bypass the host's accounting.
 *   Arguments, outputs, results and error codes are those of msm_recheck
 *   (including MSM_E_INVAL for a candidate that is not a pair i < j < n);
 *   the caller still provides X, cand, pairs_out, dist_out and count.
 *   Scratch: a static device array of about 3 MB per GPU that loads the
 *   library (row norms and counters), so n must be <= 262144 (2^18) rows;
 *   larger n returns MSM_E_INVAL with a message.  No cudaMalloc, cudaFree or
 *   allocating library call is made.
 *   The first call on each device looks up the array's device address (make
 *   that first call before any stream capture).  Every call on a device uses
 *   the same array and clears its counters first; calls whose work overlaps
 *   on the GPU (other streams, other threads) race on it and must be
 *   serialised by the caller.  Synchronises on `stream`. */
int msm_recheck_noalloc(const void* X, int64_t n, int dim, int dtype,
                        int metric, float eps, const uint64_t* cand, int64_t m,
                        uint64_t* pairs_out, float* dist_out, int64_t* count,
                        int64_t* recomputed, void* stream);

/* The whole method (Sec. 4.1): projection, blockwise MSM over Q replicates
 * with replicate de-duplication, epsilon recheck.
 *   X          host or device [n][dim] of `dtype` (host memory is copied in)
 *   metric     MSM_COSINE or MSM_EUCLIDEAN; eps the radius
 *   miss_ratio gamma of Sec. 4.3, used only when params->Q == 0
 *   params     string geometry and options (see msm_params)
 *   out        receives the result (see output modes), allocated with
 *              `alloc`; count is always set
 *   stats      optional host pointer
 * Synchronises on `stream`. */
int msm_eps_graph(const void* X, int64_t n, int dim, int dtype, int metric,
                  float eps, double miss_ratio, const msm_params* params,
                  const msm_allocator* alloc, msm_pairs* out,
                  msm_stats* stats, void* stream);

/* ---- Batched form: many independent point sets in one call ----
 * The paper builds one graph per call.  These entry points run the same
 * method on S independent point sets at once: set s is the rows
 * [set_offsets[s], set_offsets[s+1]) of one concatenated pool, and pairs
 * are only formed inside a set (no set sees another).  Every grouping sort
 * covers all sets (one radix segment per kept-block set, split at the set
 * boundaries), so the launch count does not grow with S.
 *   set_offsets  host [nsets + 1]: set_offsets[0] = 0, nondecreasing; the
 *                pool has n = set_offsets[nsets] rows (2 <= n < 2^31);
 *                empty and one-point sets are allowed; 1 <= nsets <= 2^24
 * Pair indices are rows of the concatenated pool. */

/* msm_enumerate over the sets: every pair (i, j), i < j, of one set whose
 * strings lie within Hamming distance d in at least one pool.  Strings are
 * [Q][n][W] over the concatenated rows.  Synchronises. */
int msm_enumerate_sets(const uint64_t* strings, const int64_t* set_offsets,
                       int nsets, int ell, int k, int d, int Q, int flags,
                       const msm_allocator* alloc, msm_pairs* out,
                       msm_stats* stats, void* stream);

/* msm_eps_graph over the sets (X: host or device [n][dim] of dtype, the
 * concatenated rows).  set_counts: optional host [nsets], receives the
 * number of result pairs of every set.  With MSM_OUT_COUNT no pair or
 * candidate list is stored: each candidate is checked against eps as soon
 * as the pair check finds it.  Synchronises. */
int msm_eps_graph_sets(const void* X, const int64_t* set_offsets, int nsets,
                       int dim, int dtype, int metric, float eps,
                       double miss_ratio, const msm_params* params,
                       const msm_allocator* alloc, msm_pairs* out,
                       int64_t* set_counts, msm_stats* stats, void* stream);

/* ---- Reusable count-only plans (batched form, CUDA graph) ----
 * A plan fixes the shape of msm_eps_graph_sets with MSM_OUT_COUNT: the set
 * offsets, dim, dtype, metric, eps and msm_params (Y must be NULL; a given R
 * must stay alive and unchanged while the plan exists).  msm_plan_run then
 * builds the graph counts of any X of that shape.  The whole pipeline
 * (norms, projection, every grouping sort and pair check of every
 * replicate, with the epsilon test fused into the pair check) is issued
 * without a host round trip; the first run executes it directly and keeps
 * its buffers, the second captures it into a CUDA graph, and every later run
 * is a single graph launch plus one read-back of the counts.  Results equal
 * those of msm_eps_graph_sets. */
typedef struct msm_plan msm_plan;

/* Creates a plan (device memory from `alloc`, or cudaMallocAsync when NULL;
 * the allocator must outlive the plan).  *plan receives the handle. */
int msm_plan_create(const int64_t* set_offsets, int nsets, int dim, int dtype,
                    int metric, float eps, double miss_ratio,
                    const msm_params* params, const msm_allocator* alloc,
                    msm_plan** plan);

/* Device buffer [n][dim] of the plan's dtype that every run reads; filling
 * it directly and passing X = NULL (or this pointer) avoids a copy. */
void* msm_plan_input(msm_plan* plan);

/* One run.  X: host or device [n][dim] (copied into the plan's input), or
 * NULL to use the input buffer as it is.  *count receives the number of
 * result pairs, set_counts (optional host [nsets]) the number per set,
 * stats (optional) the counters and ms[7] the device time of the run.
 * Ordered after prior work on `stream`; synchronises on the plan.  When the
 * tensor-core projection cannot settle every sign from its queue, the call
 * is answered on the CUDA-core projection and the plan is rebuilt on it. */
int msm_plan_run(msm_plan* plan, const void* X, int64_t* count,
                 int64_t* set_counts, msm_stats* stats, void* stream);

/* 1 once the plan runs as a captured CUDA graph (from its second run on). */
int msm_plan_is_graph(const msm_plan* plan);

/* Releases the plan and its device memory (synchronises on the plan). */
void msm_plan_destroy(msm_plan* plan, void* stream);

/* Autotuner for count-only runs of one shape (msm_eps_graph_sets or a
 * plan): times candidate values of the launch knobs of msm_params
 * (check_min_blocks, check_ctas_per_sm, masks_per_batch) on X (device or
 * host [n][dim]) with at most 2 replicates per trial, and writes the fastest
 * into *params.  With cache_path (or NULL), a result stored there for the
 * same device, shape and geometry is used without timing, and a new result
 * is appended to the file.  Results never depend on the knobs.
 * Synchronises. */
int msm_autotune(const void* X, const int64_t* set_offsets, int nsets,
                 int dim, int dtype, int metric, float eps,
                 msm_params* params, const char* cache_path,
                 const msm_allocator* alloc, void* stream);

/* ---- Learned projection ----
 * Sec. 6 of the paper proposes combining MSM with non-random hashing.  The
 * learned form feeds the sign projection (Eq. 3) with features
 *   y = W2 gelu(W1 x + b1) + b2      (gelu(h) = h Phi(h), exact erf form)
 * instead of x (msm_params.Y); the epsilon recheck still uses x, so the
 * result never contains a false pair.  Weights W1 [hidden][dim] and
 * W2 [dim_out][hidden] are bf16 (raw 16-bit storage); biases, features and
 * gradients are float; every product accumulates in float.
 * Parameter vector order (float): W1, b1, W2, b2. */

/* y for every row of X (device [n][dim] of dtype) into device Y
 * [n][dim_out].  On tcgen05 tensor cores, both layers fused, when dim <= 128
 * (multiple of 8), hidden is a multiple of 64 and dim_out is 64 or 128: X
 * (float) and the gelu activations are then split into bf16 high and low
 * parts, so every operand carries 16 significant bits and every product
 * accumulates in float; other shapes use a float CUDA-core GEMM.  Scratch
 * from cudaMallocAsync.  Synchronises (tensor-core path: it reads the
 * status of its bounded waits and returns MSM_E_TIMEOUT if one ran out). */
int msm_mlp_forward(const void* X, int64_t n, int dim, int dtype,
                    const void* W1, const float* b1, const void* W2,
                    const float* b2, int hidden, int dim_out, float* Y,
                    void* stream);

/* Training loss of `batch` pairs (pair_i[t], pair_j[t]) with label[t] = 1
 * for an epsilon-neighbour pair and 0 otherwise:
 *   mean of max(0, m_pos - cos(y_i, y_j)) (label 1), max(0, cos - m_neg)
 * and its gradient with respect to (W1, b1, W2, b2), written to device
 * `grads` (hidden*dim + hidden + dim_out*hidden + dim_out floats).
 * *loss (host) receives the loss; synchronises. */
int msm_mlp_grad(const void* X, int64_t n, int dim, int dtype, const void* W1,
                 const float* b1, const void* W2, const float* b2, int hidden,
                 int dim_out, const uint32_t* pair_i, const uint32_t* pair_j,
                 const uint8_t* label, int64_t batch, float m_pos, float m_neg,
                 float* grads, float* loss, void* stream);

/* One Adam step (Kingma and Ba, 2015; step counts from 1) on the float
 * master parameters `params` (device, the order above, `count` floats) with
 * moment buffers m, v, then refresh of the bf16 copies W1_bf16, W2_bf16.
 * Asynchronous. */
int msm_mlp_adam(float* params, const float* grads, float* m, float* v,
                 int64_t count, int step, float lr, float beta1, float beta2,
                 float eps, void* W1_bf16, void* W2_bf16, int hidden, int dim,
                 int dim_out, void* stream);

/* Testing aid, not part of the method: the poll limit of the bounded waits
 * inside the tensor-core projection (every wait also ends after 2 s of
 * device time).  A wait that runs out makes its CTA stop, wait for the copies
 * and MMAs it already issued, release its tensor memory and report it; the
 * call then returns MSM_E_TIMEOUT (msm_project) and nothing faults.  0
 * restores the default of 2^22 polls.  Applies to later calls of every
 * thread; returns the previous limit. */
int msm_set_wait_limit(uint32_t polls);

/* Release the buffers of a msm_pairs returned by this library. */
void msm_free_pairs(msm_pairs* p, const msm_allocator* alloc, void* stream);

/* Measurement aid, not part of the method: the exact number of pairs i < j
 * with distance <= eps (Def. 1.1), by exhaustive comparison on the GPU with
 * the same decision rule as msm_recheck.  Used to measure the missing-edge
 * ratio of msm_eps_graph.  Synchronises. */
int msm_eps_count_exhaustive(const void* X, int64_t n, int dim, int dtype,
                             int metric, float eps, int64_t* count,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MSM_H */
