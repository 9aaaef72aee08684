/*
 * tlrmvn.h - C ABI of the GB300 (sm_103a) tile-low-rank quasi-Monte Carlo library
 * for high-dimensional multivariate normal (MVN) and Student-t (MVT) probabilities.
 *
 * Method: Cao, Genton, Keyes & Turkiyyah, "Exploiting low rank covariance
 * structures for computing high-dimensional normal and Student-t probabilities"
 * (arXiv 2003.11183).  The library computes
 *
 *     log Phi_n(a, b; Sigma)        (eq. 1)      or
 *     log T_n(a, b; Sigma, nu)      (eq. 3 / eq. 4)
 *
 * by the separation-of-variables integrand (eq. 2) on a block-reordered
 * tile-low-rank (TLR) Cholesky factor (Section 3.3, Algorithms 4 and 5),
 * evaluated over randomly shifted Richtmyer lattice points (Section 2.1) by
 * the TLR integrands of Algorithms 6 and 7 (Section 3.4).
 *
 * Conventions for every entry point:
 *  - Return value: TLRMVN_OK (0) or a positive TLRMVN_E_* code; a one-line
 *    description of the last failure on the calling thread is available from
 *    tlrmvn_last_error().  Outputs are written only on success.
 *  - Arrays are plain C arrays.  "host" pointers point to CPU memory,
 *    "device" pointers to memory of the current CUDA device.  The caller owns
 *    every array it passes; the library copies what it needs and keeps no
 *    caller pointer after the call returns.
 *  - Streams: a cudaStream_t passed as void*; NULL selects the library's own
 *    stream.  Calls return after their work on that stream has completed.
 *  - One handle may be used by one call at a time; different handles are
 *    independent.  The library allocates device memory with the CUDA runtime.
 */
#ifndef TLRMVN_H
#define TLRMVN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TLRMVN_OK          0
#define TLRMVN_E_INVAL     1  /* invalid argument: n <= 0, tile <= 0, NaN, a_i > b_i, bad option */
#define TLRMVN_E_NOT_SPD   2  /* a Cholesky pivot was not positive: covariance not positive definite */
#define TLRMVN_E_NOMEM     3  /* device or host allocation failed */
#define TLRMVN_E_CUDA      4  /* CUDA runtime error (no usable device, launch failure, ...) */
#define TLRMVN_E_FORMAT    5  /* tlrmvn_factor_import: buffer is not a factor of this format */
#define TLRMVN_E_NOTSUP    6  /* requested precision / mode not available */
#define TLRMVN_E_TIMEOUT   7  /* a bounded device-side wait (tensor-core pipeline) expired; the kernel
                                 freed its resources and returned, the CUDA context stays usable */
#define TLRMVN_E_RANK      8  /* tlrmvn_factor_*: the rank cap stopped the truncation of an off-diagonal
                                 tile before the tolerance was met, and the options ask for that to fail */
#define TLRMVN_E_BUSY      9  /* tlrmvn_server_submit: admission refused (the request can never fit the
                                 server's memory budget, or the server is shutting down) */

/* ---- option values --------------------------------------------------- */
/* Arithmetic of the integrand (tlrmvn_opts.precision). */
#define TLRMVN_FP64        0  /* everything in float64 */
#define TLRMVN_FP32        1  /* diagonal-tile sweep and low-rank shifts in float32 */
#define TLRMVN_BF16_SHIFT  2  /* float32 sweep; low-rank shifts on tcgen05 tensor cores, bf16 in, fp32 accumulate */
#define TLRMVN_FP16_SHIFT  3  /* as BF16_SHIFT with fp16 operands: U and V scaled per off-diagonal tile by
                                 powers of two into fp16's range, the inverse applied to each projection
                                 before it is stored (TLRMVN_E_NOTSUP if a tile's range cannot be met) */

/* Preconditioner (tlrmvn_factor_opts.reorder), Section 3.3. */
#define TLRMVN_REORDER_NONE       0  /* geometric order only ("tlrmvn") */
#define TLRMVN_REORDER_BLOCK      1  /* Algorithm 4, block reordering ("rtlrmvn") */
#define TLRMVN_REORDER_ITERATIVE  2  /* Algorithm 5, iterative block reordering ("rrtlrmvn") */

/* Arithmetic of the factorisation's Schur complement (tlrmvn_factor_opts.schur), Section 3.3. */
#define TLRMVN_SCHUR_EXACT 0  /* left-looking: every off-diagonal factor tile L_ij is formed from the
                                 exact Schur complement and truncated once by ACA                      */
#define TLRMVN_SCHUR_TLR   1  /* tile-low-rank arithmetic as Algorithm 5 prints it: the covariance is
                                 compressed by ACA first; each product with Sigma_jj^-T and each
                                 Schur subtraction of the right-looking update is truncated by ACA at
                                 tol; diagonal blocks stay dense and exact                            */

/* Covariance kernels of tlrmvn_factor_kernel (Section 3.2; unit variance each). */
#define TLRMVN_KERNEL_EXP          0  /* exp(-d/beta);                          params = {beta}      */
#define TLRMVN_KERNEL_MATERN15     1  /* (1 + sqrt3 d/ell) exp(-sqrt3 d/ell);   params = {ell}       */
#define TLRMVN_KERNEL_EXP_MATERN15 2  /* sum of the two;                        params = {beta, ell} */

typedef struct tlrmvn_factor_s* tlrmvn_factor_t;  /* opaque, library-owned, device-resident */

typedef struct {
  int    tile;      /* tile size m (> 0); the last tile of the geometric order may be shorter   */
  double tol;       /* absolute ACA truncation tolerance of the off-diagonal tiles (>= 0)      */
  int    max_rank;  /* rank cap per off-diagonal tile; 0 = tile size                           */
  int    reorder;   /* TLRMVN_REORDER_*                                                        */
  void*  stream;    /* cudaStream_t or NULL                                                    */
  int    strict_rank; /* 0: a tile whose truncation the rank cap stopped keeps the capped rank
                         (counted in tlrmvn_factor_info's `capped`); nonzero: the factorisation
                         fails with TLRMVN_E_RANK instead                                        */
  int    schur;     /* TLRMVN_SCHUR_*; with TLRMVN_SCHUR_TLR, `capped` counts every truncation
                       (construction, product, subtraction) that the rank cap stopped           */
} tlrmvn_factor_opts;

typedef struct {
  int    precision;        /* TLRMVN_FP64 / TLRMVN_FP32 / TLRMVN_BF16_SHIFT / TLRMVN_FP16_SHIFT      */
  int    n_shifts;         /* M >= 1 random shifts ("batches")                                      */
  int    n_points;         /* N >= 1 lattice points per shift                                       */
  int    periodize;        /* nonzero: tent (baker's) transform of each lattice coordinate          */
  const uint64_t* shifts;  /* host, M x (n + 1) row-major uint64 fractions (shift / 2^64), or NULL:
                              then shift (s, i) = splitmix64 output number s*(n+1)+i from seed     */
  uint64_t seed;           /* used only when shifts == NULL                                         */
  int64_t sample_chunk;    /* samples in flight per pass; 0 = automatic                             */
  void*  stream;           /* cudaStream_t or NULL                                                  */
} tlrmvn_opts;

/* ---- factorisation (Section 3.3) -------------------------------------- */

/* Build the block-reordered TLR Cholesky factor of a covariance given by a kernel
 * on 2-D locations.  Section 3.2: locations are indexed by a cardinality-balanced
 * k-d bisection whose leaves (tile-sized clusters) become the tiles; Section 3.3:
 * the factor is formed in float64 on the GPU, reordered by Algorithm 4 or 5 when
 * requested, with off-diagonal tiles truncated by adaptive cross approximation.
 *   xy      host, n x 2 row-major locations
 *   kernel  TLRMVN_KERNEL_*, params host array (1 or 2 entries), nugget >= 0 on the diagonal
 *   a_ref, b_ref  host, length n, limits that steer the reordering (may be NULL
 *           when reorder == NONE); -INFINITY / +INFINITY allowed, a_ref <= b_ref
 *   out     receives the handle; free with tlrmvn_factor_free. */
int tlrmvn_factor_kernel(const double* xy, int64_t n, int kernel, const double* params, double nugget,
                         const double* a_ref, const double* b_ref, const tlrmvn_factor_opts* opts,
                         tlrmvn_factor_t* out);

/* Same from a dense covariance.  cov: host, column-major n x n with leading
 * dimension ld >= n, symmetric positive definite; tiles are consecutive runs of
 * `tile` indices in the given order. */
int tlrmvn_factor_dense(const double* cov, int64_t n, int64_t ld, const double* a_ref, const double* b_ref,
                        const tlrmvn_factor_opts* opts, tlrmvn_factor_t* out);

/* Post-hoc within-tile reordering of a finished factor for new limits (derived
 * from the factor structure of Section 3.3; not in the paper).  The block
 * reorderings also order the variables within each diagonal block by the limits,
 * which a resident factor meets anew in every request; this returns, without
 * refactoring, the factor of the same covariance with each tile's variables in
 * the univariate-conditioning order of the new limits on the tile's conditional
 * covariance B_j B_j^T: per tile an m x m Cholesky factor of the permuted block
 * becomes the new B_j, the tile's rows of U are permuted and its column blocks of
 * V rotated by an orthogonal m x m matrix, so every off-diagonal rank is kept.
 *   a, b   host, length n, original index order (the request's limits)
 *   out    receives a new handle (free it with tlrmvn_factor_free); f is unchanged.
 * Float64 on the GPU; TLRMVN_E_INVAL for invalid limits, TLRMVN_E_NOT_SPD if a
 * permuted block is not positive definite to float64 precision. */
int tlrmvn_factor_reorder_tiles(tlrmvn_factor_t f, const double* a, const double* b, void* stream,
                                tlrmvn_factor_t* out);

/* Shape of a factor: n, number of tiles r, tile size m, total stored rank
 * K = sum of off-diagonal tile ranks, and the number of tiles whose rank cap
 * stopped ACA before the tolerance.  Any output pointer may be NULL. */
int tlrmvn_factor_info(tlrmvn_factor_t f, int64_t* n, int* r, int* m, int64_t* k_total, int* capped);

/* Ranks of the off-diagonal tiles (Section 3.3: each L_ij ~ U_ij V_ij^T).
 * ranks: caller-owned host array of r * r int32; entry i*r + j is the rank of
 * tile (i, j) for i > j and 0 elsewhere.  TLRMVN_E_INVAL for a null argument. */
int tlrmvn_factor_ranks(tlrmvn_factor_t f, int32_t* ranks);

/* Serialise a factor to host memory (checkpoint; also how tests hand the same
 * factor to an independent implementation).  If buf == NULL, *bytes receives the
 * size needed.  Layout (little-endian):
 *   char magic[8] = "TLRMVN01"; int64 n, r, m, k_total;
 *   int64 tile_off[r + 1]; int64 perm[n]  (perm[position] = original index);
 *   int32 rank[r * r]  (rank[i*r + j] for i > j, else 0);
 *   float64 B[r][m][m]  (diagonal tiles, row-major, zero above the diagonal and
 *                        outside a short last tile);
 *   then for each i > j in row-major (i, j) order: float64 U_ij[m_i][k], V_ij[m_j][k]
 *   (row-major), with L_ij ~ U_ij V_ij^T. */
int tlrmvn_factor_export(tlrmvn_factor_t f, void* buf, size_t* bytes);

/* Load a factor in the export layout (host buffer) onto the current device. */
int tlrmvn_factor_import(const void* buf, size_t bytes, tlrmvn_factor_t* out);

int tlrmvn_factor_free(tlrmvn_factor_t f);

/* ---- probabilities (Algorithms 6 and 7) -------------------------------- */

/* log Phi_n(a, b; Sigma) (nu = INFINITY) or log T_n(a, b; Sigma, nu) (nu > 0).
 *   a, b        host, length n, in the ORIGINAL index order; -INFINITY/+INFINITY allowed
 *   logp        host, receives log of the QMC estimate (mean over shifts of the
 *               per-shift lattice means, Section 2.1)
 *   err         host, receives the standard error of that mean divided by the
 *               mean (the paper's relative error, Section 4), which is also the
 *               standard error of logp to first order; NaN when n_shifts == 1
 *   per_shift   host, length n_shifts or NULL: log of each shift's lattice mean
 *   per_sample  host, length n_shifts * n_points or NULL: log integrand of every
 *               sample, shift-major (sample s*N + k-1 is point k of shift s)
 * Device scratch (tlrmvn_prob_scratch_bytes) comes from the device's default
 * memory pool, whose release threshold the first call raises to the maximum,
 * so that the next call reuses it without mapping it again; the application
 * returns it to the driver with cudaMemPoolTrimTo on that pool. */
int tlrmvn_prob(tlrmvn_factor_t f, const double* a, const double* b, double nu, const tlrmvn_opts* opts,
                double* logp, double* err, double* per_shift, double* per_sample);

/* Same with every array in device memory (inputs already resident; outputs
 * written on the device).  per_shift / per_sample may be NULL. */
int tlrmvn_prob_device(tlrmvn_factor_t f, const double* a, const double* b, double nu,
                       const tlrmvn_opts* opts, double* logp, double* err, double* per_shift,
                       double* per_sample);

/* ---- autotuner -------------------------------------------------------- */

/* Launch choices of the integrand for one factor and precision (no counterpart
 * in the paper; they change how the work is launched, not what is computed):
 *   sub       variables per sub-tile of the float32 sweep (64 or 128) or of the
 *             float64 sweep (32 or 64); the coupling between sub-tiles of a
 *             diagonal tile is a dense product
 *   threads   threads per block of the float32 sweep; 0 = the occupancy rule
 *   chunk     samples in flight per pass; 0 = as many as fit the memory rule
 *             (opts->sample_chunk, when set, still takes precedence)
 *   tc_ctas   whole-tile sweeps of the BF16-/FP16-shift paths sharing an SM (1..6; with spt 2
 *             at most 4 take effect)
 *   spt       samples per thread of the whole-tile sweep: 1 or 2 (two independent chains
 *             per thread, 256 samples per block)
 *   ms        tlrmvn_autotune: device milliseconds per solve of the choice (-1
 *             when it came from the cache); candidates: how many were timed */
typedef struct {
  int sub, threads;
  int64_t chunk;
  int tc_ctas;
  double ms;
  int candidates;
  int spt;
} tlrmvn_tuning;

/* Times each candidate launch choice for opts->precision on solves of this very
 * problem (a, b host, length n, original order; nu; opts as for tlrmvn_prob, whose
 * sample count S = n_shifts * n_points the choice is made for), keeps the fastest
 * on the factor (every later solve of this factor in this precision uses it) and
 * appends it to the text file cache_path (NULL: no cache).  Unless force is
 * nonzero, a cache entry for the same device, precision, n, tile size, total
 * rank (to 2 bits of its logarithm), S (to a factor of 2) and distribution
 * (normal / Student-t) is used instead of timing.  Costs two or three solves per
 * candidate (at most 8 candidates).  out (nullable) receives the choice. */
int tlrmvn_autotune(tlrmvn_factor_t f, const double* a, const double* b, double nu, const tlrmvn_opts* opts,
                    const char* cache_path, int force, tlrmvn_tuning* out);
/* The launch choice a factor uses for a precision; and setting one by hand
 * (TLRMVN_E_INVAL for values outside the ranges above). */
int tlrmvn_get_tuning(tlrmvn_factor_t f, int precision, tlrmvn_tuning* out);
int tlrmvn_set_tuning(tlrmvn_factor_t f, int precision, const tlrmvn_tuning* t);

/* ---- many problems in one launch -------------------------------------- */

/* A batch plan: `count` problems (each its own factor, tile size <= 128 for
 * TLRMVN_FP32, any for TLRMVN_BF16_SHIFT, and
 * its own nu; INFINITY for MVN) solved together by one persistent kernel whose
 * blocks take (problem, 128-sample chunk) work items from a device counter,
 * largest problems first; each item runs Algorithm 6/7 for its chunk over all
 * tiles of its problem.  The launch sequence (limit permutation, persistent
 * integrand, estimator) is captured once in a CUDA graph; tlrmvn_batch_run
 * replays it for new limits.  Needed by likelihood fitting, where the same
 * covariances meet new limits at every step (Section 5 of the paper).
 *   opts: precision TLRMVN_FP32 (float sweep, float SIMT shifts and
 *         projections) or TLRMVN_BF16_SHIFT (every tile through the same
 *         whole-tile tcgen05 sweep as tlrmvn_prob's BF16-shift path, with the
 *         chunk's projections and y in block-private bf16 buffers; results equal
 *         that path's on the same shifts up to the order of its float sums);
 *         opts->shifts must be NULL: problem p draws its shifts from seed
 *         opts->seed + p exactly as tlrmvn_prob does with that seed; n_shifts /
 *         n_points / periodize apply to all problems.  TLRMVN_E_TIMEOUT: a
 *         bounded wait of the tensor-core kernel expired (the plan stays usable).
 *   factors, nu: host arrays of length count; the factors must outlive the plan.
 * tlrmvn_batch_run: a[p], b[p] host arrays of the problem's length (original
 * order); logp / err host arrays of length count. */
typedef struct tlrmvn_batch_s* tlrmvn_batch_t;
int tlrmvn_batch_create(int count, const tlrmvn_factor_t* factors, const double* nu, const tlrmvn_opts* opts,
                        tlrmvn_batch_t* out);
int tlrmvn_batch_run(tlrmvn_batch_t plan, const double* const* a, const double* const* b, double* logp,
                     double* err);
int tlrmvn_batch_free(tlrmvn_batch_t plan);
/* Autotunes a plan (no counterpart in the paper): replays it on these limits
 * (as for tlrmvn_batch_run) with 1, 2, ... CTAs of the persistent integrand per
 * SM, up to all that fit, times each replay with CUDA events and keeps the
 * fastest in the plan's graph; the choice is appended to the text file
 * cache_path (NULL: no cache) and, unless force is nonzero, read back from it
 * for a plan of the same device, problem count, total dimension, total rank
 * and samples.  ctas_per_sm, ms (nullable): the choice and its milliseconds per
 * replay (-1 when it came from the cache). */
int tlrmvn_batch_tune(tlrmvn_batch_t plan, const double* const* a, const double* const* b, const char* cache_path,
                      int force, int* ctas_per_sm, double* ms);
/* create + run + free in one call */
int tlrmvn_prob_batch(int count, const tlrmvn_factor_t* factors, const double* const* a, const double* const* b,
                      const double* nu, const tlrmvn_opts* opts, double* logp, double* err);

/* ---- serving loop ----------------------------------------------------- */

/* A server keeps the given factors resident and answers probability requests
 * with new limits as they arrive (e.g. the likelihood evaluations of Section 5,
 * or an online service).  Requests wait in arrival order; `lanes` worker
 * threads, each with its own CUDA stream, take the oldest request as soon as a
 * lane is free and the request's scratch fits in what is left of
 * `memory_budget` bytes.  Requests that arrive while others run are therefore
 * admitted as lanes and memory free up, and their kernels overlap on the
 * device.  A request's result depends on its own inputs only: it is the same
 * alone and in the mix.  Factors must outlive the server; they may be used by
 * other calls meanwhile.
 *   tlrmvn_server_submit copies a, b (host, length n of the factor) and, when
 *     opts->shifts is set, the shifts; opts->stream is ignored.  Returns an id.
 *     TLRMVN_E_BUSY (admission refused) if the request alone exceeds the budget.
 *   tlrmvn_server_wait blocks until the request is done and returns its logp,
 *     err and latency (submission to completion, milliseconds); an id can be
 *     waited for once.
 *   tlrmvn_server_free waits for every queued request, then stops the lanes. */
typedef struct tlrmvn_server_s* tlrmvn_server_t;
typedef struct {
  int64_t completed, queued;
  int in_flight, peak_in_flight;  /* requests on the device now / at most at once */
  int64_t overlapped;             /* requests admitted while another was running  */
  int64_t peak_bytes;             /* largest admitted scratch at once              */
  double p50_ms, p99_ms;          /* latency percentiles of completed requests     */
} tlrmvn_server_stats_t;
int tlrmvn_server_create(const tlrmvn_factor_t* factors, int n_factors, int lanes, int64_t memory_budget,
                         tlrmvn_server_t* out);
int tlrmvn_server_submit(tlrmvn_server_t server, int factor, const double* a, const double* b, double nu,
                         const tlrmvn_opts* opts, int64_t* request_id);
int tlrmvn_server_wait(tlrmvn_server_t server, int64_t request_id, double* logp, double* err, double* latency_ms);
int tlrmvn_server_stats(tlrmvn_server_t server, tlrmvn_server_stats_t* out);
int tlrmvn_server_free(tlrmvn_server_t server);
/* Device scratch (bytes) one request with these options takes on this factor:
 * what the server charges against its budget (also a tlrmvn_prob call's peak). */
int tlrmvn_prob_scratch_bytes(tlrmvn_factor_t f, const tlrmvn_opts* opts, int64_t* bytes);

/* ---- pooled estimate over replicas -------------------------------------- */

/* The estimate of Section 2.1 from per-shift log lattice means gathered on the
 * host, e.g. from replicas of one problem solved with disjoint shifts on several
 * GPUs or processes (each shift batch is an independent estimate, so the pooled
 * estimate is exactly what one solve over all the shifts would return):
 *   per_shift  host, count >= 1 values ell_s = log of shift s's lattice mean
 *              (the per_shift output of tlrmvn_prob); -INFINITY allowed
 *   logp, err  host, receive log((1/count) sum_s exp(ell_s)) and the standard
 *              error of that mean divided by the mean (NaN when count == 1 or every
 *              ell_s is -INFINITY; logp is then -INFINITY in the latter case)
 * Float64 on the host, no device work.  TLRMVN_E_INVAL for null pointers,
 * count < 1, NaN or +INFINITY values. */
int tlrmvn_estimate_pooled(const double* per_shift, int64_t count, double* logp, double* err);

/* ---- estimator without device allocation ------------------------------ */

/* The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory - a serving loop that reserved its memory up front and
 * must not take the device-wide synchronisation of cudaMalloc/cudaFree, or an
 * application whose device memory belongs to another allocator.
 *
 * Computes the same estimate as tlrmvn_prob from per-sample log integrand
 * values (the per_sample output of tlrmvn_prob / tlrmvn_prob_device):
 *   per_sample  device, n_shifts * n_points doubles, shift-major
 *   out         device, 2 doubles: log p_hat, err (as tlrmvn_prob's logp / err)
 *   per_shift   device, n_shifts doubles, or NULL
 *   stream      cudaStream_t or NULL (library stream); returns after completion.
 * It allocates nothing: its scratch (one double per shift) is a fixed array in
 * the library, TLRMVN_NOALLOC_MAX_SHIFTS doubles, held by every GPU that loads
 * the library until the process exits.  n_shifts above that limit returns
 * TLRMVN_E_INVAL.  The first call on a device looks up the array's device
 * address.  All calls share
 * the array: calls whose work overlaps on the GPU (different streams, or other
 * threads) race on it and must be serialised by the caller. */
#define TLRMVN_NOALLOC_MAX_SHIFTS 65536
int tlrmvn_estimate_noalloc(const double* per_sample, int n_shifts, int64_t n_points, double* out,
                            double* per_shift, void* stream);

/* ---- diagnostics ------------------------------------------------------ */
const char* tlrmvn_strerror(int status);
const char* tlrmvn_last_error(void);   /* thread-local detail of the last failure, "" if none */

/* Exercises the bounded-wait path of the tensor-core kernels (no counterpart in
 * the paper): one thread waits `polls` times (1 .. 2^20) on an mbarrier that
 * nothing arrives at, then gives up and records a code, as those kernels do
 * when a copy or MMA never completes.  Returns TLRMVN_E_TIMEOUT when the wait
 * gave up (the expected outcome; the CUDA context stays usable), TLRMVN_OK if
 * the barrier unexpectedly completed, TLRMVN_E_INVAL for polls out of range,
 * TLRMVN_E_CUDA on a launch failure.  stream: cudaStream_t or NULL. */
int tlrmvn_selftest_wait_timeout(int polls, void* stream);

/* Evaluates, on the GPU, the float32 Phi(-x) that the float sweep uses for
 * one-sided limits (a Mills-ratio fit, no counterpart in the paper) at n host
 * values x >= 0 (1 <= n <= 2^24), writing n host floats to out; for tests of
 * its error bound.  TLRMVN_E_INVAL for bad arguments, TLRMVN_E_CUDA on a
 * device error. */
int tlrmvn_selftest_phi_neg(const float* x, int n, float* out);

/* Evaluates, on the GPU, the float32 normal quantile that the float sweep uses
 * (the library's own polynomial fit in Giles' variable -log(4p(1-p)) for
 * p > 0.0017, Wichura's AS 241 tail forms below; no counterpart in the paper) at
 * n host pairs (p, lp), p in [0, 1/2] and lp = log p (read when p < 1e-30, where
 * it carries the value: p may underflow to 0), writing Phi^-1 to n host floats
 * out (1 <= n <= 2^24); for tests of its error bound.  TLRMVN_E_INVAL for bad
 * arguments, TLRMVN_E_CUDA on a device error. */
int tlrmvn_selftest_ndtri(const float* p, const float* lp, int n, float* out);

/* Measured float32 FMA throughput of the current device (no counterpart in the
 * paper; the denominator beside the derived SMs x 128 lanes x 2 x clock peak of
 * the float sweep's roofline): eight blocks of 256 threads per SM, each thread
 * eight independent fused multiply-add chains, timed with CUDA events on
 * `stream` (NULL: the library's stream) after one untimed launch.  *tflops:
 * flops per second / 1e12.  TLRMVN_E_INVAL for a null output, TLRMVN_E_CUDA on
 * a device error. */
int tlrmvn_measure_fp32_peak(void* stream, double* tflops);

/* Kernel classes of the integrand, for tlrmvn_profile_get.  On the BF16-shift
 * path with tiles of more than 64 variables the shifts, the coupling and the
 * projections are computed inside the diagonal-tile sweep's kernel and are
 * timed as TLRMVN_KC_DIAG. */
#define TLRMVN_KC_SHIFT   0  /* low-rank limit shifts  Delta_i = U_i W_i           */
#define TLRMVN_KC_DIAG    1  /* diagonal-tile SOV sweep (eq. 2 on B_i)              */
#define TLRMVN_KC_VPROJ   2  /* projections  W_col_i = V_i^T y_i                    */
#define TLRMVN_KC_CHI     3  /* Student-t scale chi_nu^-1(w0)/sqrt(nu)              */
#define TLRMVN_KC_REDUCE  4  /* per-shift and cross-shift log-sum reductions        */
#define TLRMVN_KC_COUPLE  5  /* in-tile coupling between sub-tiles of a diagonal tile */
#define TLRMVN_KC_PREP    6  /* limit validation and permutation                    */
#define TLRMVN_KC_COUNT   7

/* Process-wide kernel timing: when enabled, every integrand launch is bracketed
 * by CUDA events on its stream and, once the call has completed, its device
 * time is added to its class.  Enabling costs two event records per launch.
 * tlrmvn_profile_get returns the accumulated milliseconds and launch count of
 * one class; tlrmvn_profile_reset clears all classes. */
int tlrmvn_profile_enable(int on);
int tlrmvn_profile_reset(void);
int tlrmvn_profile_get(int kernel_class, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* TLRMVN_H */
