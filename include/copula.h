/*
 * copula.h -- C ABI of libcopula, a GB300 (sm_103a) implementation of the
 * divide-and-combine maximum pseudo-likelihood copula estimator of
 * Wei, Kim & Conlon, "Parallel Computing for Copula Parameter Estimation with
 * Big Data" (arXiv:1609.05530).
 *
 * The estimator (Section 2.4): the N x 2 data matrix is split by rows into M
 * disjoint contiguous subsets (Eq. 14); on each subset the margins are
 * replaced by their normalised ranks u = r/(m+1) (Eq. 12, ranks taken within
 * the subset), the one-parameter copula density is fitted by maximising the
 * pseudo log-likelihood sum_i log c(u_i, v_i; theta) (Eq. 13), the asymptotic
 * variance of each subset estimate is computed (Section 2.3, after Genest,
 * Ghoudi & Rivest 1995), and the subset estimates are combined by the
 * inverse-variance weighted mean (Eq. 15).
 *
 * Conventions for every call below:
 *   - "device" pointers point to memory of the current CUDA device, owned by
 *     the caller; "host" pointers point to ordinary host memory owned by the
 *     caller.  The library never frees caller memory.
 *   - Calls that take a stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream) enqueue their work on it and return without waiting,
 *     unless stated otherwise.  Host-side arguments are fully consumed before
 *     the call returns.
 *   - Return value: COPULA_SUCCESS (0) or a negative COPULA_ERR_* code.
 *     Argument errors are detected on the host before anything is enqueued.
 *     Per-subset numerical outcomes are reported through status_out.
 *   - A context is not thread-safe: use one per host thread.
 *   - Scratch memory ("workspace") is supplied by the caller; its size comes
 *     from the matching *_workspace_size query.  Its contents need not be
 *     initialised and are overwritten.  Calls that overlap in time on the GPU
 *     must use distinct workspaces.
 */
#ifndef COPULA_H
#define COPULA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Copula families (Section 2.2): Gaussian (Eq. 7-8, theta = rho in (-1,1)),
 * Frank (Eq. 10, theta real, theta = 0 is independence) and
 * Gumbel-Hougaard (Eq. 11, theta >= 1). */
enum { COPULA_GAUSSIAN = 0, COPULA_FRANK = 1, COPULA_GUMBEL = 2 };

/* Storage type of the input pairs. */
enum { COPULA_DTYPE_F32 = 0, COPULA_DTYPE_F64 = 1 };

/* Arithmetic of the likelihood passes: all-FP64, or FP32 per-point terms with
 * compensated FP32 sums inside each warp and FP64 across warps, Newton state
 * and combine in FP64 ("FP32-compensated"). */
enum { COPULA_PREC_F64 = 0, COPULA_PREC_F32C = 1 };

/* Combine weights: inverse asymptotic variance (Eq. 15, the paper's rule),
 * observed Fisher information -sum l_tt, or equal weights. */
enum { COPULA_W_INVVAR = 0, COPULA_W_FISHER = 1, COPULA_W_EQUAL = 2 };

/* Return codes. */
enum {
  COPULA_SUCCESS = 0,
  COPULA_ERR_ARG = -1,         /* invalid argument (see each call) */
  COPULA_ERR_WORKSPACE = -2,   /* workspace missing or too small */
  COPULA_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  COPULA_ERR_UNSUPPORTED = -4  /* size outside what the library handles */
};

/* Per-subset status codes written to status_out.  Only OK and BOUNDARY
 * subsets enter the combine of Eq. 15: the others have no asymptotic variance
 * to weight them by. */
enum {
  COPULA_OK = 0,            /* interior maximiser found */
  COPULA_BOUNDARY = 1,      /* maximiser on the family's own edge: Gumbel theta = 1 */
  COPULA_NOT_CONVERGED = 2, /* Newton iteration cap reached; theta is the last iterate */
  COPULA_DEGENERATE = 3,    /* NaN in the subset's data; theta and var are NaN */
  COPULA_CAPPED = 4         /* the likelihood still rises at a search cap (below);
                               theta is the cap (typical of tiny subsets) */
};

/* Parameter caps of the search (a maximiser on a cap gets COPULA_CAPPED):
 * Gaussian |rho| <= 1 - 1e-9, Frank |theta| <= 50, Gumbel 1 <= theta <= 50.
 *
 * Subset sizes.  Subsets must have 2 <= m.  A subset of up to
 * COPULA_MAX_SUBSET pairs (FP32 storage) or COPULA_MAX_SUBSET_F64 pairs (FP64
 * storage, whose 64-bit sort keys take more shared memory) is ranked and
 * fitted by one thread block from shared memory.  Larger subsets, up to
 * COPULA_MAX_SUBSET_STREAM / COPULA_MAX_SUBSET_STREAM_F64 pairs, take the
 * streaming path: a sample sort over many thread blocks ranks them, and one
 * cooperative kernel runs the Newton passes and the variance of all of them
 * together (the first call that plans such subsets must not be inside CUDA
 * graph capture: it sets kernel attributes).  A sample-sort bucket larger
 * than one thread block orders in shared memory (about 1e-11 per bucket of
 * 3072 pairs for any input order, or an input built against the sampled
 * rows) is ranked by direct pairwise counting instead: exact, but with work
 * quadratic in the bucket's size.  Anything larger is
 * COPULA_ERR_UNSUPPORTED. */
#define COPULA_MAX_SUBSET 20480
#define COPULA_MAX_SUBSET_F64 15000
#define COPULA_MAX_SUBSET_STREAM 3145728
#define COPULA_MAX_SUBSET_STREAM_F64 2097152

typedef struct copula_opts {
  int32_t precision; /* COPULA_PREC_*; default COPULA_PREC_F32C */
  int32_t weight;    /* COPULA_W_*;   default COPULA_W_INVVAR */
  int32_t max_iter;  /* Newton iteration cap; <= 0 selects 64 */
  int32_t block;     /* threads per subset CTA; 0 = autotuned choice */
  double rtol;       /* Newton step tolerance |dtheta| <= rtol max(1,|theta|);
                        <= 0 selects 1e-13 (F64) or 1e-6 (F32C) */
} copula_opts;

/* Fills *opts with the defaults listed above. */
void copula_opts_default(copula_opts* opts);

typedef struct copula_ctx copula_ctx;

/* Creates a context on the current CUDA device.  It holds pinned host
 * staging memory for the small per-call descriptors (subset offsets and the
 * work schedule), the device properties and the start-value tables.
 * Returns COPULA_ERR_ARG if ctx is NULL, COPULA_ERR_CUDA on a CUDA failure. */
int copula_ctx_create(copula_ctx** ctx);

/* Destroys a context; waits for its pending staging copies first. */
int copula_ctx_destroy(copula_ctx* ctx);

/* Workspace bytes that copula_fit needs for this partition.
 *   dtype            COPULA_DTYPE_*
 *   opts             may be NULL (defaults)
 *   subset_offsets   host, K+1 int64 row offsets, off[0] = 0, off[K] = n,
 *                    strictly increasing with every subset size >= 2
 * ctx may be NULL: the query then needs no GPU and assumes the sm_100-class
 * shared-memory limit and the default block sizes; its answer covers calls
 * on any context that uses those block sizes (with a context, the answer is
 * the exact need of calls on that context).  Returns COPULA_ERR_ARG for an
 * invalid partition,
 * COPULA_ERR_UNSUPPORTED if a subset exceeds COPULA_MAX_SUBSET_STREAM(_F64). */
int copula_fit_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts,
                              const int64_t* subset_offsets, int64_t K, size_t* bytes);

/* The whole estimator on one dataset (Section 2.4, Eq. 12-15).
 *   family             COPULA_GAUSSIAN / COPULA_FRANK / COPULA_GUMBEL
 *   dtype              storage type of u and v
 *   u, v               device, n values each: the two columns of X, in row
 *                      order (any real values; only their within-subset
 *                      order matters, -0.0 equals +0.0, ties are broken by
 *                      row index).  NaN marks its subset DEGENERATE.
 *   subset_offsets     host, K+1 int64 row offsets of the M = K subsets
 *                      (Eq. 14): subset k is rows [off[k], off[k+1]).
 *   theta_out          device, K doubles: theta_hat_m (Eq. 13 maximiser)
 *   var_out            device, K doubles or NULL: asymptotic variance of
 *                      theta_hat_m, sigma_m^2 in Eq. 15 (sandwich / m)
 *   status_out         device, K int32 or NULL: COPULA_OK etc.
 *   theta_combined_out device, 1 double or NULL: Eq. 15 with opts->weight
 *                      over the subsets with status OK or BOUNDARY and a
 *                      finite positive weight (NaN if none is left).
 *   workspace          device, >= copula_fit_workspace_size bytes, 256-byte
 *                      aligned.
 * Errors: COPULA_ERR_ARG for a bad family, dtype, n or partition, or NULL
 * required pointers; COPULA_ERR_WORKSPACE if the workspace is too small;
 * COPULA_ERR_UNSUPPORTED if a subset exceeds COPULA_MAX_SUBSET_STREAM(_F64). */
int copula_fit(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v,
               int64_t n, const int64_t* subset_offsets, int64_t K, double* theta_out,
               double* var_out, int32_t* status_out, double* theta_combined_out,
               const copula_opts* opts, void* workspace, size_t workspace_bytes, void* stream);

/* copula_fit with optional per-subset diagnostics (each may be NULL):
 *   info_out    device, K doubles: observed information -sum d2l/dtheta2 at
 *               theta_hat (the FISHER combine weight)
 *   iters_out   device, K int32: likelihood passes the Newton driver took
 *               (0 for the Gaussian family, solved from its score cubic; on
 *               the FP64 path of a shared-memory subset, including the
 *               FP32 search whose root starts the FP64 passes)
 *   phase_ns_out device, 4*K uint64: GPU global-timer stamps per subset at
 *               start, after the rank transform, after the parameter search
 *               and at the end (nanoseconds, for profiling). */
int copula_fit_ex(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v,
                  int64_t n, const int64_t* subset_offsets, int64_t K, double* theta_out,
                  double* var_out, int32_t* status_out, double* theta_combined_out,
                  double* info_out, int32_t* iters_out, uint64_t* phase_ns_out,
                  const copula_opts* opts, void* workspace, size_t workspace_bytes, void* stream);

/* Kernel timing: when on (default off), every fit call records CUDA events
 * on its stream around the per-subset fit kernel(s), and
 * copula_ctx_kernel_ms waits for the last call's end event and returns that
 * span in milliseconds.  copula_ctx_launches returns how many kernels the
 * last call launched. */
int copula_ctx_set_timing(copula_ctx* ctx, int32_t on);
int copula_ctx_kernel_ms(copula_ctx* ctx, double* ms);
int copula_ctx_launches(copula_ctx* ctx, int32_t* launches);

/* Stage spans (ms) of the streaming path in the last timed call: ms[0] ranks
 * of u, ms[1] ranks of v, ms[2] pi and sum r_u r_v, ms[3] the cooperative fit
 * kernel (Newton passes and variance).  Waits for the call's last event.
 * COPULA_ERR_ARG if that call had no subset on the streaming path. */
int copula_ctx_stage_ms(copula_ctx* ctx, double* ms);

/* Phase timestamps of the streaming fit kernel in the last timed call
 * (profiling): ns_out[0] its start, ns_out[j] the release of its j-th grid
 * barrier (device global timer, nanoseconds); *count the number recorded
 * (up to 256), of which the first min(count, cap) are written.  Each chunk
 * sweep of the kernel ends at a barrier, so the differences are the sweeps'
 * spans.  Waits for the call's last event.  COPULA_ERR_ARG if that call had
 * no subset on the streaming path. */
int copula_ctx_stream_stamps(copula_ctx* ctx, uint64_t* ns_out, int32_t cap, int32_t* count);

/* Batched estimator: B independent datasets in one launch sequence.
 *   family                host, B int32 families
 *   u, v                  device, concatenated columns of all datasets
 *                         (sum of n_b values each)
 *   dataset_offsets       host, B+1 int64 row offsets of the datasets
 *   subset_offsets        host, S+1 int64 global row offsets of all subsets,
 *                         S = total subsets; the subsets of dataset b are
 *                         [dataset_subset_start[b], dataset_subset_start[b+1])
 *                         and must tile that dataset's rows exactly.
 *   dataset_subset_start  host, B+1 int64
 *   theta_out, var_out, status_out   device, S entries each (var/status may be NULL)
 *   theta_combined_out    device, B doubles (may be NULL)
 * A subset's result does not depend on which other datasets share the call.
 * The workspace query takes the same families (host, B int32): with
 * per-family block tables (copula_ctx_set_family_blocks) the need depends on
 * them; family may be NULL only when every family uses the same table
 * (COPULA_ERR_ARG otherwise).
 * A context keeps its last plan (the schedule built from a partition, its
 * families, the storage type, options and block tables): a call whose
 * arguments are the same as the previous plan's reuses it without planning
 * again, which also makes a size query followed by the call plan once.
 * Errors as for copula_fit. */
int copula_fit_batch_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts,
                                    int32_t B, const int32_t* family, const int64_t* dataset_offsets,
                                    const int64_t* subset_offsets,
                                    const int64_t* dataset_subset_start, size_t* bytes);
int copula_fit_batch(copula_ctx* ctx, int32_t B, const int32_t* family, int32_t dtype,
                     const void* u, const void* v, const int64_t* dataset_offsets,
                     const int64_t* subset_offsets, const int64_t* dataset_subset_start,
                     double* theta_out, double* var_out, int32_t* status_out,
                     double* theta_combined_out, const copula_opts* opts, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Plans: the batched fit split into a one-off schedule upload and a launch
 * sequence that touches only device memory, so that copula_plan_run can be
 * captured into a CUDA graph and replayed.
 *   copula_plan_create   validates the partition (as copula_fit_batch),
 *                        builds the schedule and returns the workspace size;
 *                        the plan keeps a pinned copy of the schedule
 *   copula_plan_upload   copies the schedule into `workspace` on `stream`;
 *                        do it once per workspace before any run
 *   copula_plan_run      enqueues counter reset, the fit kernels and the
 *                        combine on `stream` (no host transfers; capturable)
 *   copula_plan_destroy  frees the plan (not the workspace)
 * A plan belongs to the context it was made with and uses its block table. */
typedef struct copula_plan copula_plan;
int copula_plan_create(copula_ctx* ctx, copula_plan** plan, int32_t B, const int32_t* family, int32_t dtype,
                       const int64_t* dataset_offsets, const int64_t* subset_offsets,
                       const int64_t* dataset_subset_start, const copula_opts* opts,
                       size_t* workspace_bytes);
int copula_plan_upload(copula_plan* plan, void* workspace, size_t workspace_bytes, void* stream);
int copula_plan_run(copula_plan* plan, const void* u, const void* v, double* theta_out, double* var_out,
                    int32_t* status_out, double* theta_combined_out, void* workspace,
                    size_t workspace_bytes, void* stream);
int copula_plan_destroy(copula_plan* plan);

/* Per-subset diagnostics of the last copula_plan_run on `workspace`,
 * enqueued on `stream` after it (device-to-device copies, capturable):
 *   info_out    device, S doubles or NULL: observed information
 *               -sum d2l/dtheta2 at theta_hat (the FISHER weight)
 *   iters_out   device, S int32 or NULL: likelihood passes of the Newton
 *               driver (as copula_fit_ex's iters_out)
 * COPULA_ERR_WORKSPACE if the workspace is smaller than the plan's. */
int copula_plan_diagnostics(copula_plan* plan, const void* workspace, size_t workspace_bytes, double* info_out,
                            int32_t* iters_out, void* stream);

/* Threads per subset CTA chosen by subset size: subsets with m <= m_max[i]
 * (the first i that holds) use threads[i] (128, 256 or 512); larger subsets
 * and count = 0 fall back to the built-in rule (128 up to m = 1536, 256 up to
 * 6144, else 512).  m_max must increase.  Used by the autotuner; a subset's
 * result depends only on its data and the block it runs with. */
int copula_ctx_set_blocks(copula_ctx* ctx, const int32_t* m_max, const int32_t* threads, int32_t count);

/* Bounded waits of the streaming path.  Its cooperative fit kernel meets at
 * grid-wide barriers; a block that waits longer than `spins` polls (about
 * 256 ns apart; 0 selects the built-in 2^24, a few seconds) gives up, flags
 * the call, and every block returns: the streaming subsets of that call keep
 * their preset results (theta, var NaN; status COPULA_DEGENERATE; the Eq. 15
 * value of their datasets NaN), while shared-memory subsets are unaffected,
 * and the context stays usable.  phantom_arrivals = 1 makes every barrier
 * wait for one block that does not exist, so that the give-up path can be
 * tested without a fault (0 for normal use).  COPULA_ERR_ARG for spins < 0
 * or phantom_arrivals outside {0, 1}. */
int copula_ctx_set_wait_limit(copula_ctx* ctx, int64_t spins, int32_t phantom_arrivals);

/* copula_ctx_set_blocks for one family's subsets only (COPULA_GAUSSIAN,
 * COPULA_FRANK or COPULA_GUMBEL; COPULA_ERR_ARG otherwise): the autotuner
 * tunes each family apart, since their per-pass costs differ. */
int copula_ctx_set_family_blocks(copula_ctx* ctx, int32_t family, const int32_t* m_max, const int32_t* threads,
                                 int32_t count);

/* copula_fit with HOST buffers: u, v (n values of dtype), theta_out, var_out,
 * status_out (K entries, var/status may be NULL) and theta_combined_out
 * (1 double, may be NULL) are host pointers.  The call moves the inputs to
 * the GPU, fits, copies the results back (one copy, through the context's
 * pinned staging, so the output arrays need not be pinned) and waits for the
 * stream before returning.  Inputs in page-locked host memory that the
 * device can address (cudaHostAlloc / cudaHostRegister on a unified-address
 * system) are read by the fit kernel directly, once each, over the host
 * link, when every subset takes the shared-memory path; otherwise (pageable
 * inputs, or streaming subsets, which read their inputs several times) they
 * are first copied into the workspace.  For full speed u and v should be
 * pinned.  workspace must hold copula_fit_host_workspace_size bytes, 256-byte
 * aligned. */
int copula_fit_host_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts,
                                   const int64_t* subset_offsets, int64_t K, size_t* bytes);
int copula_fit_host(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u_host,
                    const void* v_host, int64_t n, const int64_t* subset_offsets, int64_t K,
                    double* theta_out, double* var_out, int32_t* status_out,
                    double* theta_combined_out, const copula_opts* opts, void* workspace,
                    size_t workspace_bytes, void* stream);

/* copula_fit_batch with HOST buffers, the batched counterpart of
 * copula_fit_host: u, v (the concatenated columns of all B datasets, sum of
 * n_b values of dtype each) are read from host memory (in place when pinned
 * and device-addressable and every subset takes the shared-memory path,
 * otherwise copied into the workspace first); theta_out, var_out,
 * status_out (S entries, var/status may be NULL) and theta_combined_out (B
 * doubles, may be NULL) are host arrays filled before the call returns.
 * Partition arguments and errors as for copula_fit_batch; workspace as
 * copula_fit_batch_host_workspace_size says, 256-byte aligned. */
int copula_fit_batch_host_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts, int32_t B,
                                         const int32_t* family, const int64_t* dataset_offsets,
                                         const int64_t* subset_offsets, const int64_t* dataset_subset_start,
                                         size_t* bytes);
int copula_fit_batch_host(copula_ctx* ctx, int32_t B, const int32_t* family, int32_t dtype, const void* u_host,
                          const void* v_host, const int64_t* dataset_offsets, const int64_t* subset_offsets,
                          const int64_t* dataset_subset_start, double* theta_out, double* var_out,
                          int32_t* status_out, double* theta_combined_out, const copula_opts* opts,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Normalised-rank step alone (Eq. 12 within each subset, Section 2.4): writes
 * the within-subset ordinal rank 1..m of every x value (ties by row index,
 * -0.0 == +0.0) to ranks_out (device, n int32).  A subset holding NaN gets
 * rank 0 everywhere.  Same workspace rule as copula_fit (use
 * copula_fit_workspace_size with this partition). */
int copula_ranks(copula_ctx* ctx, int32_t dtype, const void* x, int64_t n,
                 const int64_t* subset_offsets, int64_t K, int32_t* ranks_out, void* workspace,
                 size_t workspace_bytes, void* stream);

/* One likelihood pass (Eq. 13 and its first two theta-derivatives) at given
 * parameters, on pseudo-observations computed from u and v per subset:
 *   theta_in     device, K doubles (one parameter per subset)
 *   l_out, g_out, h_out   device, K doubles: sum log c, sum dl/dtheta,
 *                sum d2l/dtheta2 over each subset (any may be NULL)
 * Workspace as for copula_fit. */
int copula_loglik(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v,
                  int64_t n, const int64_t* subset_offsets, int64_t K, const double* theta_in,
                  double* l_out, double* g_out, double* h_out, const copula_opts* opts,
                  void* workspace, size_t workspace_bytes, void* stream);

/* Sample rank correlations of every subset, the statistics behind the
 * inversion of Kendall's tau and of Spearman's rho that Section 2.3 lists
 * beside the MPL: on each subset's ranks (Eq. 12, within the subset, ties by
 * row index),
 *   tau_out[k] = (concordant - discordant pairs) / (m(m-1)/2),
 *   rho_out[k] = 1 - 6 sum (r_u - r_v)^2 / (m (m^2 - 1)),
 * both exact (integer counts, then one FP64 division).
 *   u, v               device, n values of dtype (as copula_fit)
 *   subset_offsets     host, K+1 int64 row offsets (Eq. 14)
 *   tau_out, rho_out   device, K doubles each; NaN for a subset holding NaN
 *   workspace          device, >= copula_fit_workspace_size bytes, 256-byte
 *                      aligned
 * Subsets up to COPULA_MAX_SUBSET (FP64 storage: COPULA_MAX_SUBSET_F64)
 * rows are done by one thread block each in shared memory (the inversions of
 * pi by a merge sort there); larger ones, up to COPULA_MAX_SUBSET_STREAM
 * (_F64), are ranked by the streaming path's sample sort and their
 * inversions counted chunk by chunk (within each chunk of 16,384 u-ranks by
 * a merge sort in shared memory, across chunks by merge walks over the sorted
 * chunks).  The first call that plans such subsets must not be
 * inside CUDA graph capture (it sets kernel attributes).  Larger subsets give
 * COPULA_ERR_UNSUPPORTED without enqueueing anything.  COPULA_ERR_ARG for a
 * bad dtype or partition or NULL pointers. */
int copula_rank_corr(copula_ctx* ctx, int32_t dtype, const void* u, const void* v, int64_t n,
                     const int64_t* subset_offsets, int64_t K, double* tau_out, double* rho_out,
                     void* workspace, size_t workspace_bytes, void* stream);

/* The rank-correlation inversion estimators that Section 2.3 lists beside
 * the MPL: for each value r[k], the parameter of `family` whose population
 * Kendall's tau (which = 0) or Spearman's rho (which = 1) equals r[k] --
 * applied to the sample values of copula_rank_corr, one estimate per subset.
 * Population maps: Gaussian (2/pi) asin(rho) and (6/pi) asin(rho/2) and
 * Gumbel tau = 1 - 1/theta, inverted in closed form; Frank's Debye-function
 * forms (Section 2.5 prints their values at its parameters) and Gumbel's
 * rho_S = 12 int_0^1 (1 + A(t))^-2 dt - 3 (A its Pickands function),
 * inverted by a bracketed FP64 Newton iteration on Gauss-Legendre sums, one
 * warp per value.
 *   family        COPULA_GAUSSIAN / COPULA_FRANK / COPULA_GUMBEL
 *   which         0 Kendall's tau, 1 Spearman's rho
 *   r             device, K doubles
 *   theta_out     device, K doubles
 *   status_out    device, K int32 or NULL: COPULA_OK; COPULA_BOUNDARY for
 *                 Gumbel at r <= 0 (theta = 1, independence); COPULA_CAPPED
 *                 beyond a search cap (Gaussian |rho| <= 1 - 1e-9, Frank
 *                 |theta| <= 50, Gumbel theta <= 50; theta is the cap);
 *                 COPULA_DEGENERATE for r NaN or outside [-1, 1] (theta NaN);
 *                 COPULA_NOT_CONVERGED if 100 iterations do not settle.
 * Enqueued on `stream`; no context, no workspace, no allocation (the first
 * call builds the quadrature nodes on the host, once per process).
 * COPULA_ERR_ARG for a bad family or which, K < 0, or NULL pointers with
 * K > 0; COPULA_ERR_CUDA if the launch fails. */
int copula_theta_from_rank_corr(int32_t family, int32_t which, const double* r, int64_t K, double* theta_out,
                                int32_t* status_out, void* stream);

/* ------------------------------------------------------------------------
 * The simulation study of Sections 2.5-2.6.
 * ------------------------------------------------------------------------ */

/* The four double integrals behind Eq. 19 and Eq. 20 for K parameter pairs
 * of one family, over the square [delta, 1 - delta]^2:
 *   integrals_out[4k + 0] = int int |c(.; a_k) - c(.; b_k)|
 *   integrals_out[4k + 1] = int int |c(.; a_k)|
 *   integrals_out[4k + 2] = int int (c(.; a_k) - c(.; b_k))^2
 *   integrals_out[4k + 3] = int int c(.; a_k)^2
 *   relative_out[2k] = [0] / [1] (Eq. 19), relative_out[2k + 1] =
 *   sqrt([2] / [3]) (Eq. 20), with c the copula density (Eq. 8, 10, 11),
 *   a_k = theta_a[k] (the full-data estimate) and b_k = theta_b[k] (the
 *   combined one).
 * Quadrature: a product rule of 10-point Gauss-Legendre panels per axis,
 * graded geometrically towards both edges (20 panels from delta, or from
 * 1e-12 when delta = 0, to 0.02; with delta = 0 also 40 panels from 1e-100
 * to 1e-12 for the Gaussian and Frank families; 24 equal panels from 0.02
 * to 1/2), the upper half of each axis mirroring the lower one; FP64.
 * The Gumbel density grows like 1/|(1 - u, 1 - v)| near (1, 1), so its
 * squared integrals diverge as delta -> 0: use delta > 0 for that family.
 *   family                     COPULA_GAUSSIAN / FRANK / GUMBEL
 *   delta                      0 <= delta < 0.02
 *   theta_a, theta_b           device, K doubles each
 *   integrals_out              device, 4K doubles, or NULL
 *   relative_out               device, 2K doubles, or NULL (not both NULL)
 *   workspace                  device, copula_density_distance_workspace_size
 *                              bytes, 256-byte aligned
 * 1 <= K <= 65535.  COPULA_ERR_ARG for bad arguments, COPULA_ERR_WORKSPACE,
 * COPULA_ERR_CUDA.  Stream-ordered; allocates nothing. */
int copula_density_distance_workspace_size(int32_t family, double delta, int64_t K, size_t* bytes);
int copula_density_distance(int32_t family, double delta, int64_t K, const double* theta_a, const double* theta_b,
                            double* integrals_out, double* relative_out, void* workspace, size_t workspace_bytes,
                            void* stream);

/* The summaries of S simulations (Section 2.6) from their per-simulation
 * combined estimates theta_combined[s] (Eq. 16, the Eq. 15 combine of
 * simulation s) and full-data estimates theta_full[s] (device, S doubles
 * each), written to summary_out (device, 10 doubles):
 *   [0] mean combined estimate (Eq. 17)   [1] mean full-data estimate (Eq. 18)
 *   [2] estimated bias [0] - [1]          [3] estimated MSE, mean of (comb - full)^2
 *   [4] relative L1 distance (Eq. 19)     [5] relative L2 distance (Eq. 20)
 *   [6..9] the four integrals of copula_density_distance
 * between the densities at [1] (full) and [0] (combined), over
 * [delta, 1 - delta]^2 as there.  Workspace:
 * copula_simulation_summary_workspace_size bytes, 256-byte aligned.
 * S >= 1.  Errors as copula_density_distance. */
int copula_simulation_summary_workspace_size(int32_t family, double delta, size_t* bytes);
int copula_simulation_summary(int32_t family, double delta, int32_t S, const double* theta_combined,
                              const double* theta_full, double* summary_out, void* workspace,
                              size_t workspace_bytes, void* stream);

/* copula_fit for callers that cannot allocate device memory -- code that
 * runs under a fixed memory budget it owns in full, plugins that are handed
 * only their input and output buffers, or serving loops that must never
 * enter an allocator.  It takes no context and no workspace and allocates
 * nothing (device or host): its scratch (job schedule, counters, per-subset
 * variance / information / pass counts) lives in one fixed array of about
 * 115 KB in the library's device memory, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart:
 * this is a deployment variant of copula_fit.  It always uses the built-in
 * block sizes (it has no context, so no tuned block table), so its results
 * are those of copula_fit on a context with the default block sizes; after
 * copula_ctx_set_blocks the two can differ within the parity tolerances.
 *   Arguments as for copula_fit (u, v, theta_out, var_out, status_out,
 *   theta_combined_out on the device; subset_offsets on the host; opts may
 *   be NULL).
 *   Limits: at most 2048 subsets; every subset takes the shared-memory path
 *   with its per-rank table and scan array in shared memory (FP32C: m <=
 *   COPULA_MAX_SUBSET with FP32 storage, COPULA_MAX_SUBSET_F64 with FP64
 *   storage; FP64 path: m <= 11,889).  Larger requests return
 *   COPULA_ERR_UNSUPPORTED without enqueueing anything; use copula_fit for
 *   them.
 *   The first call on each device looks up the array's device address and
 *   the SM count and builds the start-value tables; make that first call
 *   before any stream capture.
 *   All calls share the one array and a call leaves its contents behind (each
 *   call writes everything it reads, in stream order).  Calls that overlap in
 *   time on the GPU -- on different streams or from different host threads --
 *   race on it and must be serialised by the caller. */
int copula_fit_noalloc(int32_t family, int32_t dtype, const void* u, const void* v, int64_t n,
                       const int64_t* subset_offsets, int64_t K, double* theta_out, double* var_out,
                       int32_t* status_out, double* theta_combined_out, const copula_opts* opts,
                       void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of fit requests (no counterpart in the paper,
 * which fits one dataset at a time; this runs its estimator as a service).
 * ------------------------------------------------------------------------ */

/* Device-memory arena bookkeeping: first-fit allocation of byte offsets in
 * [0, bytes) in 256-byte granules, with coalescing of freed neighbours.  It
 * only manages offsets (no memory is touched), so it also runs without a GPU.
 *   copula_arena_alloc returns COPULA_ERR_WORKSPACE when no free block is
 *   large enough; copula_arena_free takes an offset returned by alloc. */
typedef struct copula_arena copula_arena;
int copula_arena_create(copula_arena** arena, size_t bytes);
int copula_arena_destroy(copula_arena* arena);
int copula_arena_alloc(copula_arena* arena, size_t bytes, size_t* offset);
int copula_arena_free(copula_arena* arena, size_t offset);
int copula_arena_stats(copula_arena* arena, size_t* used, size_t* peak, size_t* largest_free);

enum { COPULA_REQ_PENDING = 0, COPULA_REQ_RUNNING = 1, COPULA_REQ_DONE = 2, COPULA_REQ_ERROR = 3 };

/* One fit request (one dataset).  u, v: host arrays of n values (pinned
 * memory gives full-speed copies) that must stay valid until the request
 * completes; subset_offsets: host, K+1 row offsets (copied at submit);
 * theta_out, var_out, status_out: host arrays of K entries filled at
 * completion (each may be NULL). */
typedef struct copula_request {
  int32_t family;
  int32_t dtype;
  const void* u;
  const void* v;
  int64_t n;
  const int64_t* subset_offsets;
  int64_t K;
  copula_opts opts;
  double* theta_out;
  double* var_out;
  int32_t* status_out;
} copula_request;

typedef struct copula_result {
  int32_t state;         /* COPULA_REQ_* */
  int32_t rc;            /* COPULA_SUCCESS or the error of a failed request */
  double theta_combined; /* Eq. 15 */
  double latency_s;      /* submit to completion */
  double queue_s;        /* submit to admission */
} copula_result;

typedef struct copula_server_statistics {
  int64_t fits_done;
  int64_t errors;
  int64_t batches;
  int64_t pending;
  double mean_batch;          /* requests per launched batch */
  int32_t max_inflight_batches;
  int32_t reserved;
  double fits_per_s;          /* completed fits / (last completion - first arrival) */
  double p50_s, p99_s;        /* latency percentiles (submit to completion) */
  double mean_queue_s;
  size_t arena_peak_bytes;
} copula_server_statistics;

typedef struct copula_server copula_server;

/* Creates a server on the current device.
 *   arena, arena_bytes  device memory the server may use (the HBM budget),
 *                       owned by the caller, >= 1 MiB; all request inputs,
 *                       outputs and workspaces are carved from it
 *   max_slots           most requests in flight at once
 *   streams             most batches in flight at once (1..16), each on its
 *                       own CUDA stream
 * A scheduler thread admits pending requests in arrival order while slots
 * and arena space allow, packs the admitted requests of one kind (dtype and
 * options) into one copula_fit_batch, and overlaps batches on the streams.
 * A subset's result is the same whichever requests share its batch. */
int copula_server_create(copula_server** srv, void* arena, size_t arena_bytes, int32_t max_slots,
                         int32_t streams);
/* Queues a request and returns its ticket at once.  COPULA_ERR_ARG for an
 * invalid request, COPULA_ERR_WORKSPACE if it can never fit the arena. */
int copula_server_submit(copula_server* srv, const copula_request* req, uint64_t* ticket);
/* Non-blocking status; a finished ticket is released after it is reported. */
int copula_server_poll(copula_server* srv, uint64_t ticket, copula_result* result);
/* Waits up to timeout_s (<= 0: no limit) for the ticket to finish. */
int copula_server_wait(copula_server* srv, uint64_t ticket, double timeout_s, copula_result* result);
int copula_server_stats(copula_server* srv, copula_server_statistics* stats);
int copula_server_reset_stats(copula_server* srv);
/* Finishes all queued and running requests, then frees the server. */
int copula_server_destroy(copula_server* srv);

/* Measured issue rates of the GPU units the fit kernels are bound by, for
 * the denominators of their rooflines (not part of the paper's method).
 * Runs one short probe kernel per unit on the current device (each thread
 * keeps 8 independent dependency chains of one instruction) and times it
 * with CUDA events, best of three after a warm-up; takes a few
 * milliseconds, allocates and frees its own small sink buffers, and waits
 * for `stream`.  rates_out[i], for i < count (count <= 5 is filled, further
 * entries are set to 0), in results per second over the whole GPU:
 *   0  ex2.approx.f32   (MUFU)      1  lg2.approx.f32  (MUFU)
 *   2  rcp.approx.f32   (MUFU)      3  FP32 fused multiply-add
 *   4  FP64 fused multiply-add
 * COPULA_ERR_ARG for a NULL pointer or count < 1, COPULA_ERR_CUDA on a CUDA
 * failure. */
int copula_measure_unit_rates(double* rates_out, int32_t count, void* stream);

/* Library version (major*10000 + minor*100 + patch). */
int copula_version(void);

/* Text of the last error recorded by a call on this context ("" if none). */
const char* copula_last_error(copula_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* COPULA_H */
