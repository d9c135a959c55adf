/*
 * ttgbf.h -- C ABI of the tensor-train grid-based (point-mass) filter on GB300.
 *
 * The library runs the Bayesian recursion of arXiv 2501.07942 (Sec. 1,
 * Eqs. asx/asz; Alg. 2 and Alg. 3) for a batch of independent filters that
 * share one grid and one linear-Gaussian dynamic model: each filter's density
 * is a tensor train (Sec. 3, Eq. ttd_exact) over an equidistant,
 * cell-centred grid (Sec. 2, Eq. pdf_pm).  One filter step is
 *     ttgbf_predict  (Chapman-Kolmogorov, Eqs. pdf_predII / tpmconvFFT),
 *     ttgbf_update   (Bayes rule, Eqs. pmf_filtrace_a/b), and
 *     ttgbf_estimate (mean, covariance, log normaliser).
 * Every step of the path runs in the library's own CUDA kernels (sm_103a).
 *
 * Conventions for every entry point:
 *  - Return value 0 (TTGBF_OK) or a negative TTGBF_E* code.
 *  - Arguments are validated on the host before anything is enqueued; on
 *    TTGBF_EINVAL / TTGBF_ENONFINITE / TTGBF_ECAPACITY / TTGBF_ESINGULAR the
 *    filter state is unchanged.
 *  - After a CUDA error the context is poisoned: every later call except
 *    ttgbf_free returns TTGBF_EPOISONED (for a batch split into parts: once
 *    any part is poisoned).
 *  - Fault injection for tests of these paths (no GPU fault is made): the
 *    environment variable TTGBF_FAULT, read by ttgbf_init, set to "cuda:N"
 *    makes the N-th status check after init report a CUDA error (the call
 *    returns TTGBF_ECUDA and poisons the context), set to "alloc" makes
 *    ttgbf_init fail with TTGBF_ENOMEM after validating its arguments.
 *  - Host arrays passed in are owned by the caller and are read (or copied)
 *    before the call returns.  Device pointers passed in are owned by the
 *    caller and must stay valid until the work enqueued on the context's
 *    stream has passed them.
 *  - Work is enqueued asynchronously on the stream given at init.  Calls that
 *    return host data (ttgbf_estimate, ttgbf_ranks, ttgbf_stats,
 *    ttgbf_export_cores) synchronise that stream.
 *  - Thread safety: a context is used by one host thread at a time.
 */
#ifndef TTGBF_H
#define TTGBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTGBF_OK 0
#define TTGBF_EINVAL (-1)     /* bad shape, mode, size or option           */
#define TTGBF_ENONFINITE (-2) /* NaN or Inf in F, Q, R, z, grid or prior   */
#define TTGBF_ENOMEM (-3)     /* device allocation failed or workspace too small */
#define TTGBF_ECUDA (-4)      /* a CUDA call failed; the context is poisoned */
#define TTGBF_ECAPACITY (-5)  /* rank_cap * max_shift_span > 160, or a shear spans more than
                                 max_shift_span^2 shifts (more than max_shift_span pieces) */
#define TTGBF_ESINGULAR (-6)  /* F has no LDU factorisation without pivoting */
#define TTGBF_EPOISONED (-7)  /* an earlier CUDA error poisoned the context */

typedef struct ttgbf_ctx ttgbf_ctx;

/* Equidistant cell-centred grid (Sec. 2, Eq. pdf_pm; Sec. 4, first bullet).
 * Mode m has n[m] cells on [lo[m], hi[m]]; cell i is centred at
 * lo + (i + 1/2) (hi - lo)/n.  All three arrays are host arrays of d entries. */
typedef struct {
  int32_t d;
  const int32_t* n;
  const double* lo;
  const double* hi;
} ttgbf_grid;

/* Gaussian prior with diagonal covariance (Alg. 2 step 1): each filter starts
 * from the rank-1 tensor prod_m N(xi_m; mean[m], var[m]), normalised.
 * Host arrays of d entries. */
typedef struct {
  const double* mean;
  const double* var;
} ttgbf_prior;

typedef struct {
  int32_t batch;          /* number of independent filters (>= 1) */
  int32_t rank_cap;       /* maximal TT rank R^max after rounding (Sec. 3.2); >= 1 */
  double eps;             /* rounding tolerance: ||A - round(A)||_F <= eps ||A||_F when the cap does not bind */
  int32_t max_shift_span; /* widest rank expansion S applied at once (0 = 10); rank_cap * S must
                             not exceed 160.  A shear spanning more shifts is applied in pieces
                             (see ttgbf_predict), up to max_shift_span^2 shifts */
  void* stream;           /* cudaStream_t for all work; NULL = legacy default stream */
  void* workspace;        /* caller-owned device memory of ttgbf_workspace_bytes() bytes, 256-byte
                             aligned, or NULL to let the library cudaMalloc it (freed by ttgbf_free) */
  size_t workspace_bytes; /* size of `workspace` when it is given */
  int32_t precision;      /* TTGBF_PRECISION_FP32 (0, default) or TTGBF_PRECISION_FP64; see below */
  int32_t conv;           /* TTGBF_CONV_AUTO (0, default), TTGBF_CONV_DENSE or TTGBF_CONV_FFT */
  /* Launch configuration (0 = default; ttgbf_autotune chooses them from measured step times):
   * parts: sub-batches on their own streams, 1..8 (default one per 12 filters, at most 8; the
   *        environment variable TTGBF_PARTS overrides the default);
   * tsqr_slice_blocks: 128-row blocks per CTA slice of a tall R factor, 2, 4, 8 (default) or 16;
   * svd_threads: CTA width of the truncating SVD stages, 512 (default) or 1024. */
  int32_t parts;
  int32_t tsqr_slice_blocks;
  int32_t svd_threads;
  /* Likelihood factors that couple several modes (ttgbf_meas_comp with three
   * or more modes, or two modes other than (0, 1)) are applied by a
   * deterministic TT cross of rank cross_rank (see ttgbf_update).  0 (the
   * default): no workspace for it, and such components are TTGBF_EINVAL.
   * Otherwise max(rank_cap, 2) <= cross_rank <= min(64, rank_cap * max_shift_span);
   * the workspace grows by about batch * (2 cross_rank^2 N_max + 2 (d + 1)
   * cross_rank^2) floats. */
  int32_t cross_rank;
  /* (left-to-right, right-to-left) pairs of cross sweeps before the final
   * left-to-right sweep; 0 = 1. */
  int32_t cross_sweeps;
  int32_t contraction;    /* TTGBF_CONTRACT_FP32 (0, default), _TF32 or _TF32X3; see below */
} ttgbf_opts;

/* How the Gaussian kernel of the predictive step (Eq. tpmconvFFT, applied to
 * the grid index of every core) is computed:
 *  DENSE: the N x N Toeplitz matrix (fused with the mode's cloud-in-cell
 *         scaling when one precedes it) as a GEMM over the core's fibres.
 *  FFT:   the linear convolution of every fibre through zero-padded cyclic
 *         FFTs of length M = 2^m >= 2N - 1 (float32; the kernel's spectrum is
 *         computed in float64 on the host); a preceding scaling is applied as
 *         its cloud-in-cell gather while the fibres are loaded.  Taken for
 *         modes with N <= 512 whose scaling has at most 3 source cells per
 *         target cell; other modes use DENSE.
 *  AUTO:  FFT for modes with N >= 256, DENSE below (the faster of the two on
 *         GB300 at those sizes). */
#define TTGBF_CONV_AUTO 0
#define TTGBF_CONV_DENSE 1
#define TTGBF_CONV_FFT 2

/* Arithmetic of the TT rounding (Sec. 4.1 "round").  The cores, the shears,
 * the per-mode operators and the likelihood are float32 in both modes, and
 * the log normaliser and the moments are accumulated in float64.
 *  FP32: every stage forms the R factor of its tall unfolding (Householder)
 *        and the SVD of R (pivoted QR, then one-sided Jacobi) in float32.
 *  FP64: the stages that decide a truncation (the left-to-right sweep and the
 *        split of the merged 2-site core) form R and its SVD in float64, so
 *        the singular values compared with eps ||A|| / sqrt(d - 1) are those
 *        of the float32 cores to float64 accuracy; the orthogonalisation
 *        sweep, which truncates nothing, stays float32.  GB300 issues float64
 *        at a small fraction of its float32 rate: this mode is slower.
 *        The float64 SVD keeps at most min(rank_cap + 16, 80) leading rows of
 *        the pivoted QR for its Jacobi sweeps; what the pivoted QR leaves is
 *        counted in the discarded tail. */
#define TTGBF_PRECISION_FP32 0
#define TTGBF_PRECISION_FP64 1

/* Arithmetic of the core contractions (the grouped products that apply the
 * rounding's factors to the cores, the per-mode operators of the predictive
 * step and the 2-site merge of the update):
 *  FP32:   float32 fused multiply-adds on the CUDA cores.
 *  TF32:   the tensor cores (tcgen05.mma, kind::tf32): operands rounded to
 *          TF32 (10-bit mantissa, round to nearest), float32 accumulation.
 *          A product's relative error is about 2^-11 per term, which can
 *          exceed eps-level rounding tolerances: the TT's error against the
 *          float32 path grows accordingly.
 *  TF32X3: the tensor cores with each operand split into a TF32 part and a
 *          TF32-rounded remainder, three products (hi*hi + hi*lo + lo*hi):
 *          float32-level products (about 2^-21 relative) at three times the
 *          tensor work.
 * A tensor-core product whose completion wait exceeds one second is written
 * as NaN and makes the next ttgbf_stats return TTGBF_ECUDA. */
#define TTGBF_CONTRACT_FP32 0
#define TTGBF_CONTRACT_TF32 1
#define TTGBF_CONTRACT_TF32X3 2

/* One measurement component z_c = h_c(x_...) + v_c (Sec. 4, fourth bullet: the
 * likelihood tensor).  htab is a caller-owned DEVICE array with h_c evaluated
 * at the grid points, row-major over the component's modes:
 *  nmodes = 1: modes[0] = m, n[m] floats; the factor scales core m exactly.
 *  nmodes = 2, modes = (0, 1): n[0]*n[1] floats [i_0][i_1]; the factor
 *         multiplies the merged first two cores exactly (their left TT rank
 *         is 1; several such components multiply them one after the other),
 *         n[0] <= 160.
 *  nmodes = 2, any other pair modes = (m, n), m != n: n[m]*n[n] floats
 *         [i_m][i_n]; applied by the TT cross over the block of cores
 *         min(m, n)..max(m, n) (opts.cross_rank > 0).
 *  nmodes = k >= 3: the consecutive modes modes[0] .. modes[1], with
 *         modes[1] = modes[0] + k - 1; n[modes[0]] * ... * n[modes[1]] floats
 *         [i_modes[0]]...[i_modes[1]], at most 2^31 - 1; applied by the TT
 *         cross over that block (opts.cross_rank > 0).
 * The library cannot check the size of a device array: a shorter table is
 * read out of bounds. */
typedef struct {
  int32_t nmodes;
  int32_t modes[2];
  const float* htab;
  /* 0 for an ordinary component.  > 0 for an angle-like one (the bearing of
   * the radar study of Sec. 5, in degrees: 360): the residual z_c - h_c is
   * taken modulo period into [-period/2, period/2] before it enters the
   * Gaussian, so that a bearing near the +-180 cut is compared with the
   * nearer branch.  Negative or non-finite: TTGBF_EINVAL. */
  double period;
} ttgbf_meas_comp;

typedef struct {
  int32_t b;                   /* number of components */
  const ttgbf_meas_comp* comp; /* host array of b components */
} ttgbf_meas;

/* Per-filter diagnostics of the most recent step. */
typedef struct {
  double tail_sum;     /* sum over roundings of the discarded relative Frobenius tail */
  double tail_max;     /* largest single discarded relative tail */
  double mass_pred;    /* mass of the predictive density before normalisation */
  double log_c;        /* log of the normaliser c of Eq. pmf_filtrace_b, this step */
  double log_lik;      /* cumulative sum of log c */
  int32_t max_rank;    /* largest TT rank after the step */
  int32_t cap_hits;    /* roundings in which the rank cap bound */
} ttgbf_step_stats;

/* Bytes of device workspace needed by ttgbf_init for this grid and options. */
size_t ttgbf_workspace_bytes(const ttgbf_grid* grid, const ttgbf_opts* opts);

/* Create a context holding `opts->batch` filters, each initialised to the
 * prior.  Copies grid, prior and options.  *out is set on success only.
 *
 * A batch of 24 filters or more runs as up to 8 sub-batches ("parts", one
 * per 12 filters; environment TTGBF_PARTS=1..8 overrides), each on a stream
 * the library creates; the workspace then holds the parts' arenas back to
 * back (ttgbf_workspace_bytes accounts for this).  Every call keeps the
 * stream contract below for caller memory: the parts start after the work
 * already on `opts->stream` when a call reads caller device memory, and
 * `opts->stream` waits for them when a call reads or writes caller memory.
 * Calls that touch only the filters' own state (predict, shear, scale,
 * convolve, round, normalise) let the parts run on without a join, so an
 * event recorded on `opts->stream` right after them does not cover their
 * work; the next call that returns results (estimate, estimate_dev, ranks,
 * stats, export) does. */
int ttgbf_init(ttgbf_ctx** out, const ttgbf_grid* grid, const ttgbf_prior* prior,
               const ttgbf_opts* opts);

/* Predictive step with the re-gridded transition (Eq. pdf_predII through the
 * FFT-form of Eq. tpmconvFFT on a fixed grid): x+ = F x + w, w ~ N(0, Q).
 * F: host d*d row-major; Q: host d*d row-major, must be diagonal and
 * positive.  F = L D U (LDU without pivoting) is applied as elementary
 * shears and axis scalings with hat weights, each shear followed by TT
 * rounding, then the per-mode Gaussian convolution with
 * kappa_m(t) = D_m N(D_m t; 0, Q_mm) over each core's grid index, then
 * normalisation (Alg. 2 step 4).  Same F and Q for every filter.
 * A shear whose hat weights span S > max_shift_span integer shifts is
 * applied as the TT sum of ceil(S / max_shift_span) pieces of consecutive
 * shifts, each expanded and rounded on its own, and the sum rounded again
 * (its discarded tails are reported like any rounding's); TTGBF_ECAPACITY
 * when that takes more than max_shift_span pieces. */
int ttgbf_predict(ttgbf_ctx* ctx, const double* F, const double* Q);

/* Predictive step with the textbook transition (Eq. pdf_predII with the
 * transition matrix of Eq. TPMmat, T[j, i] = N(x_j; F x_i, Q) delta, then
 * normalisation), without the re-gridding's hat and cloud-in-cell
 * interpolation of ttgbf_predict: for an upper bidiagonal F (couplings of
 * adjacent modes only, F[m][n] = 0 unless n == m or n == m + 1) and a
 * diagonal positive Q the transition's Gaussian factorises over the modes,
 * K_m(j, i, i') = D_m N(x_{m,j} - F_mm x_{m,i} - F_{m,m+1} x_{m+1,i'}; 0, Q_mm),
 * and the factors apply in the order m = 0, 1, ... (each sums out i_m while
 * i_{m+1} is still the old index).  A coupled factor acts on the 2-site block
 * of cores (m, m+1): its product with the block is built by the TT cross of
 * rank opts.cross_rank (see ttgbf_update; the entries it needs are sums over
 * i_m of K times the block), the block's link rounded; an uncoupled factor
 * and the last mode's are dense N x N matrices on their core.  Needs
 * opts.cross_rank > 0.  TTGBF_EINVAL for other F, a non-diagonal Q or
 * cross_rank 0.  Not recorded by the adjoint (ttgbf_adj_backward then
 * returns TTGBF_ECAPACITY).  Same F and Q for every filter. */
int ttgbf_predict_exact(ttgbf_ctx* ctx, const double* F, const double* Q);

/* Bayes update (Eqs. pmf_filtrace_a/b; Alg. 2 step 2): P <- L P / c with the
 * likelihood L(i) = prod_c N(z_c; h_c(x_i), R_cc), then TT rounding and
 * normalisation; log c is accumulated into the log-likelihood.
 * R: host b*b row-major, diagonal and positive.  z: HOST array [batch][b]
 * (float64), one measurement vector per filter, copied to the device.
 * The one-mode and (0, 1) components are applied first (exactly), with log
 * c, rounding and normalisation.  Then every other component ("block"
 * component, see ttgbf_meas_comp) in turn, as its own Bayes update: the TT
 * is put in mixed canonical form with its center in the component's block
 * of cores lo..hi; the product of the factor with that block is built by a
 * deterministic TT cross of rank opts.cross_rank (Sec. 3, Eq. matrixDecomp:
 * skeletons whose rows and columns are chosen by maximum volume -- Gaussian
 * elimination with partial pivoting on a fiber matrix (the rows of the same
 * elimination on an orthonormal basis of its columns), then row exchanges
 * while an entry of B = Q Q[rows]^-1 exceeds 1.05; start index sets from the
 * density block, opts.cross_sweeps refinement pairs, a final left-to-right
 * sweep), which evaluates the factor only on the fibers it visits; log c of the product is added; the block's links are
 * rounded and the TT normalised.  The adjoint (ttgbf_adj_*) does not record
 * block components: a recorded update with one makes ttgbf_adj_backward
 * return TTGBF_ECAPACITY, as for any step the tape cannot hold. */
int ttgbf_update(ttgbf_ctx* ctx, const ttgbf_meas* h, const double* R, const double* z);

/* Same as ttgbf_update with z a DEVICE array [batch][b] of float32. */
int ttgbf_update_dev(ttgbf_ctx* ctx, const ttgbf_meas* h, const double* R, const float* z_dev);

/* Point-mass moments of every filter's current density by TT contraction
 * (Alg. 2 step 3, "power, dot"): mean [batch][d], cov [batch][d][d],
 * log_c [batch] (this step's log normaliser), log_lik [batch] (cumulative).
 * HOST outputs (any may be NULL); synchronises the stream. */
int ttgbf_estimate(ttgbf_ctx* ctx, double* mean, double* cov, double* log_c, double* log_lik);

/* Same with DEVICE outputs (float64), asynchronous. */
int ttgbf_estimate_dev(ttgbf_ctx* ctx, double* mean, double* cov, double* log_c, double* log_lik);

/* Release the context and any memory the library allocated. NULL is a no-op. */
int ttgbf_free(ttgbf_ctx* ctx);

/* Static message for an error code. */
const char* ttgbf_strerror(int code);

/* ---- diagnostics, checkpoint / resume and single-operation hooks ---------- */

/* Current TT ranks, host [batch][d+1] (r_0 = r_d = 1). Synchronises. */
int ttgbf_ranks(ttgbf_ctx* ctx, int32_t* ranks);

/* Per-filter statistics of the last step, host [batch]. Synchronises. */
int ttgbf_stats(ttgbf_ctx* ctx, ttgbf_step_stats* out);

/* Cell-centre coordinates, host array of n[0] + ... + n[d-1] doubles. */
int ttgbf_grid_axes(const ttgbf_ctx* ctx, double* axes);

/* Copy filter f's cores to host memory: concatenated cores, each row-major
 * [r_{k-1}][n_k][r_k] (float32).  ranks_out: host int32[d+1].  cap is the size
 * of buf in floats; TTGBF_ENOMEM if too small.  Synchronises. */
int ttgbf_export_cores(ttgbf_ctx* ctx, int32_t f, float* buf, size_t cap, int32_t* ranks_out);

/* Filter f's TT contracted into its full tensor on the device, float64
 * accumulation of the float32 cores: host out[n_0][n_1]...[n_{d-1}] row-major
 * (the last mode fastest), the density's values at the cell centres (summing
 * to 1 / cell volume after a step's normalisation).  For small grids only: it
 * allocates and frees two device buffers of at most max_k n_0...n_k r_{k+1}
 * doubles.  cap is the size of out in doubles; TTGBF_ENOMEM if n_0...n_{d-1}
 * exceeds it or 2^32, or if the device buffers cannot be allocated.
 * Synchronises. */
int ttgbf_densify(ttgbf_ctx* ctx, int32_t f, double* out, size_t cap);

/* Replace filter f's cores (same layout as export); ranks[k] <= rank_cap for
 * interior links.  Resets f's log-likelihood to log_lik. */
int ttgbf_import_cores(ttgbf_ctx* ctx, int32_t f, const float* buf, const int32_t* ranks,
                       double log_lik);

/* Apply one elementary re-gridding shear x_m += a x_n (m != n) with hat
 * weights to every filter, then round if do_round != 0.  Without rounding the
 * ranks of links between m and n grow by the shift span S (TTGBF_ECAPACITY
 * when S > max_shift_span); with rounding a wider shear is applied in pieces
 * as in ttgbf_predict. */
int ttgbf_shear(ttgbf_ctx* ctx, int32_t m, int32_t n, double a, int32_t do_round);

/* Apply x_m <- lam x_m (cloud-in-cell) to every filter; ranks unchanged. */
int ttgbf_scale(ttgbf_ctx* ctx, int32_t m, double lam);

/* Apply the separable Gaussian convolution with variances q[0..d-1] (host)
 * over every core's grid index; ranks unchanged; no normalisation. */
int ttgbf_convolve(ttgbf_ctx* ctx, const double* q);

/* TT rounding (right-to-left orthogonalisation, left-to-right truncated SVD)
 * of every filter at the context's eps and rank cap. */
int ttgbf_round(ttgbf_ctx* ctx);

/* Normalise every filter to unit mass (sum(P) * cell volume = 1). */
int ttgbf_normalise(ttgbf_ctx* ctx);

/* ---- profiling ------------------------------------------------------------ */

/* Per kernel class: launches, device time between CUDA events recorded on the
 * context's stream around each launch group, and the algorithmic floating-point
 * work the kernels counted on the device (0 for classes that do not count). */
typedef struct {
  char name[24];
  int64_t launches;
  double ms;
  double flops;
} ttgbf_kernel_prof;

/* enable != 0: reset the counters and record events from now on; 0: stop. */
int ttgbf_profile(ttgbf_ctx* ctx, int32_t enable);

/* Copy up to cap class records to out; *count receives the number of classes.
 * Synchronises the stream. */
int ttgbf_profile_read(ttgbf_ctx* ctx, ttgbf_kernel_prof* out, int32_t cap, int32_t* count);

/* Kernel launches made by the library in this process so far. */
uint64_t ttgbf_launch_count(void);

/* ---- groups of uneven batches, CUDA graphs, autotuning -------------------- */

/* A group steps several contexts together: batches of filters of different
 * d, N, rank cap or model (Alg. 3 for each), one context per shape.  A step
 * enqueues predict -> update -> estimate of every context with their
 * operations interleaved (every context's, and every part's, stream starts
 * after the work already on the group's stream and the group's stream waits
 * for all of them at the end), so the contexts' kernels overlap on the GPU.
 * Because one step touches only these streams and synchronises nothing on the
 * host, a horizon of steps can be recorded once into a CUDA graph and
 * launched as a whole.  Contexts used by a group should have distinct streams
 * (contexts sharing a stream run one after another).  The group does not own
 * the contexts; free it before them. */
typedef struct ttgbf_group ttgbf_group;

/* Per context, one step's inputs and outputs (same meaning as ttgbf_predict,
 * ttgbf_update_dev and ttgbf_estimate_dev): F, Q host d*d; h, R as
 * ttgbf_update; z_dev DEVICE float32 [batch][b]; mean [batch][d], cov
 * [batch][d][d], log_c [batch], log_lik [batch] DEVICE float64 (any may be
 * NULL).  For ttgbf_group_capture the device arrays hold a whole horizon:
 * step t reads z_dev + t batch b and writes mean + t batch d, cov +
 * t batch d^2, log_c + t batch, log_lik + t batch. */
typedef struct {
  const double* F;
  const double* Q;
  const ttgbf_meas* h;
  const double* R;
  const float* z_dev;
  double* mean;
  double* cov;
  double* log_c;
  double* log_lik;
} ttgbf_group_step_args;

/* ctxs: host array of n distinct contexts (n >= 1); stream: the group's
 * cudaStream_t (NULL = legacy default stream). */
int ttgbf_group_create(ttgbf_group** out, ttgbf_ctx* const* ctxs, int32_t n, void* stream);

/* One step of every context (args: host array of n).  On TTGBF_EINVAL /
 * TTGBF_ENONFINITE nothing was enqueued.  Asynchronous on the group's stream. */
int ttgbf_group_step(ttgbf_group* g, const ttgbf_group_step_args* args);

/* Record `steps` consecutive steps of every context into a CUDA graph
 * (replacing any earlier one) without running them; ttgbf_group_launch runs
 * it.  The transition operators of each context's F, Q are prepared on the
 * host first (outside the recording).  Every pointer in args is baked into
 * the graph: a launch reads the measurements and writes the estimates at
 * those addresses, so a caller replays a horizon by refilling z_dev.
 * The group's stream and every context's stream must be created streams (the
 * legacy default stream cannot be recorded): TTGBF_EINVAL otherwise.  The
 * recorded steps must bring every context back to the state it started from
 * (which ping-pong buffer holds each core, the canonical form), so that the
 * graph can be launched again: step once before recording and record an
 * even number of steps; TTGBF_EINVAL (nothing recorded) otherwise. */
int ttgbf_group_capture(ttgbf_group* g, const ttgbf_group_step_args* args, int32_t steps);

/* Launch the recorded graph on the group's stream (asynchronous). */
int ttgbf_group_launch(ttgbf_group* g);

/* Kernel launches one launch of the recorded graph makes. */
uint64_t ttgbf_group_graph_kernels(const ttgbf_group* g);

/* Per context (host array of n floats): milliseconds from the start of the
 * last ttgbf_group_step to the end of that context's work in it, every filter
 * of the context finishing then (the per-filter step latency of a batch step).
 * Synchronises; TTGBF_EINVAL when no step was timed (graph launches are not). */
int ttgbf_group_times(ttgbf_group* g, float* ms);

/* Per step of the recorded horizon and per context (host array of steps x n
 * floats, step-major): milliseconds from the start of that step in the last
 * launch of the graph to the end of that context's work in it (the GPU's
 * global timer, written by a one-thread kernel recorded with the graph at
 * every step's start and after every context's step).  Synchronises;
 * TTGBF_EINVAL when no graph was launched. */
int ttgbf_group_graph_times(ttgbf_group* g, float* ms);

int ttgbf_group_free(ttgbf_group* g);

/* Launch-configuration autotuner.  For the batch shape of *base (grid,
 * batch, rank cap, span, precision, conv) and the model F, Q, times `steps`
 * predictive steps (after one untimed step) of every candidate launch
 * configuration: parts 1, 2, 4, 8 (at most the batch), tsqr_slice_blocks 4,
 * 8, 16 and svd_threads 512, 1024; the predictive step is where the
 * rounding's QR and SVD kernels run.  Writes base with the fastest
 * configuration to *best and its time per step (ms) to *best_ms.  Each
 * candidate allocates its own device workspace (cudaMalloc) for the timing.
 * cache_path (may be NULL): a text file of earlier results, one line per
 * shape and GPU; a shape found there is returned without timing (*best_ms
 * then holds the recorded time), a new result is appended.  steps = 0 looks
 * the shape up in cache_path only: TTGBF_EINVAL when it is not there. */
int ttgbf_autotune(const ttgbf_grid* grid, const ttgbf_prior* prior, const ttgbf_opts* base,
                   const double* F, const double* Q, int32_t steps, const char* cache_path,
                   ttgbf_opts* best, double* best_ms);

/* ---- plain full-grid point-mass filter ------------------------------------ */

/* The dense filter of Sec. 2 (Eqs. pdf_pm, pdf_predII, tpmconvFFT,
 * pmf_filtrace_a/b) for ONE filter on the same grid and with the same
 * re-gridded transition as the TT path: the comparison the TT filter is
 * measured against, and the GPU form of the oracle's arithmetic.  The density
 * is held densely (n[0]*...*n[d-1] values, d <= 6) in float32 (precision 32)
 * or float64 (precision 64).  Same conventions as above. */
typedef struct ttgbf_fg ttgbf_fg;

/* Bytes of device workspace for a full-grid filter; 0 on invalid input. */
size_t ttgbf_fg_workspace_bytes(const ttgbf_grid* grid, int32_t precision);

/* Create a full-grid filter initialised to the (diagonal Gaussian) prior.
 * workspace: caller-owned device memory or NULL (the library allocates). */
int ttgbf_fg_init(ttgbf_fg** out, const ttgbf_grid* grid, const ttgbf_prior* prior, int32_t precision,
                  void* stream, void* workspace, size_t workspace_bytes);

/* Predictive step with the re-gridded transition (diagonal Q), as ttgbf_predict. */
int ttgbf_fg_predict(ttgbf_fg* fg, const double* F, const double* Q);

/* Predictive step by the textbook direct sum of Eqs. pdf_predII / TPMmat:
 * P'(j) = sum_i N(xi_j; F xi_i, Q) P(i) delta, normalised; any positive
 * definite Q.  O(N^2) work: at most 2^22 grid points (TTGBF_ECAPACITY). */
int ttgbf_fg_predict_direct(ttgbf_fg* fg, const double* F, const double* Q);

/* Bayes update with one measurement vector z (HOST, b doubles).  The htab
 * pointers of h are DEVICE arrays of float (precision 32) or double
 * (precision 64); components may use any one or two modes, or three or more
 * consecutive ones (the layouts of ttgbf_meas_comp), applied exactly at every
 * grid point. */
int ttgbf_fg_update(ttgbf_fg* fg, const ttgbf_meas* h, const double* R, const double* z);

/* Mean [d], covariance [d][d], this step's log c and the cumulative log
 * likelihood (HOST outputs, any may be NULL).  Synchronises. */
int ttgbf_fg_estimate(ttgbf_fg* fg, double* mean, double* cov, double* log_c, double* log_lik);

/* Copy the density (converted to float64) to host memory of cap doubles. */
int ttgbf_fg_density(ttgbf_fg* fg, double* out, size_t cap);

int ttgbf_fg_free(ttgbf_fg* fg);

/* ---- allocation-free moments ---------------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc (code recorded into a CUDA graph by a framework
 * that forbids allocation while capturing, serving loops with a fixed memory
 * budget, plugins living inside another framework's memory pool).
 *
 * Mass, mean and covariance of `batch` TT densities already in device memory:
 * the same point-mass moments as ttgbf_estimate (its own kernel, float64
 * per-term sums; equal to the oracle's moments of the densified TT within
 * the moment tolerance of the GPU tests), without a context: no memory is
 * allocated.  Its float64 scratch is one static device array of
 * TTGBF_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 * the process exits.
 *   grid        host; the cell-centred grid the cores live on
 *   cores       host array of d DEVICE pointers; core k of filter b is at
 *               cores[k] + b * core_stride[k], row-major [r_k][n_k][r_{k+1}]
 *   core_stride host array of d element strides between filters
 *   ranks       DEVICE int32 [batch][d+1] with r_0 = r_d = 1
 *   rank_max    bound on every rank, 1..TTGBF_NOALLOC_MAX_RANK; a filter whose
 *               ranks break it gets NaN outputs
 *   mass, mean, cov   DEVICE float64 outputs [batch], [batch][d], [batch][d][d]
 *   stream      cudaStream_t or NULL
 * Returns TTGBF_ECAPACITY when batch * d * 3 * rank_max^2 doubles exceed the
 * scratch array (or rank_max > TTGBF_NOALLOC_MAX_RANK), TTGBF_EINVAL /
 * TTGBF_ENONFINITE on bad arguments, TTGBF_ECUDA if the launch fails.
 * Every call looks the array's device address up with cudaGetSymbolAddress
 * (with the caller's device current), so the address stays right after a
 * context reset; the first call on a device also loads the library's device
 * code there, so make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the
 * GPU (different streams, no ordering) race.  Nothing in the array needs to
 * start at zero: every entry a call reads, that call has written first.
 * Asynchronous on `stream`. */
#define TTGBF_NOALLOC_SCRATCH_BYTES (16u << 20)
#define TTGBF_NOALLOC_MAX_RANK 64
int ttgbf_moments_noalloc(int32_t batch, const ttgbf_grid* grid, const float* const* cores,
                          const int64_t* core_stride, const int32_t* ranks, int32_t rank_max,
                          double* mass, double* mean, double* cov, void* stream);

/* ------------------------------------------------------- grid re-design
 * Alg. 4 with linear dynamics, for a batch that shares one grid.
 * ttgbf_design_grid (host only): from each filter's filtering mean (host
 * [batch][d]) and covariance ([batch][d][d]), the predictive moments
 * F m, F C F^T + Q, the corners of the box F m +- kappa sqrt(diag(F C F^T + Q))
 * and the same corners mapped back by F^{-1}; lo, hi (host [d]) receive the
 * axis-aligned box around all corners of all filters (the step maps the grid
 * onto itself, so it must hold the filtering and the predictive density).
 * TTGBF_ESINGULAR if F is singular, TTGBF_EINVAL if the box is degenerate.
 * ttgbf_regrid: every filter's density onto the grid [lo, hi] with the same
 * cell counts: separable piecewise-linear interpolation of the density values
 * at the new cell centres from the old ones (the density zero at points
 * beyond the old grid), then renormalisation on the new grid (one N x N
 * operator per mode on each core; ranks unchanged).  The axes, the cell
 * volume and the transition operators of the next predict follow the new
 * grid; measurement tables passed to the next update must be evaluated on the
 * new axes (ttgbf_grid_axes).  A recording for the reverse pass fails when
 * it meets a regrid.  Asynchronous after one host synchronisation (the new
 * axes' upload). */
int ttgbf_design_grid(int32_t d, int32_t batch, const double* F, const double* Q, const double* mean,
                      const double* cov, double kappa, double* lo, double* hi);
int ttgbf_regrid(ttgbf_ctx* ctx, const double* lo, const double* hi);

/* ---------------------------------------------------------------- adjoint
 * Gradient of the log-likelihood l_b = sum_k log c_k (Eq. pmf_filtrace_b) of
 * every filter b of a context with respect to F, the diagonal of Q and the
 * diagonal of R.  A reverse pass over recorded steps runs the adjoint
 * recursion of the filter equations (transposed shears, scalings, kernels and
 * likelihood products; the adjoints of the normalisations and of log c) with
 * the adjoint density held as a tensor train of the same rank cap and eps,
 * rounded like the forward density, and takes every gradient as an inner
 * product of the adjoint with a derivative operator applied to the recorded
 * forward cores.  Use:
 *   ttgbf_adj_create(&a, ctx, S, n)         S steps per recorded segment, n checkpoints
 *   forward: before every segment s, ttgbf_adj_save(a, s); run the steps
 *   reverse: ttgbf_adj_reset(a); for s = n-1 .. 0:
 *              ttgbf_adj_load(a, s); ttgbf_adj_record(a, 1); run segment s
 *              again (same F, Q, R, z); ttgbf_adj_record(a, 0);
 *              ttgbf_adj_backward(a)
 *   ttgbf_adj_grads(a, dF, dQ, dR, b)
 * The context must be a single part (opts.parts = 1) with d >= 2, F and Q
 * stay fixed over the run, and the single-operation hooks (ttgbf_scale,
 * ttgbf_convolve, an unrounded ttgbf_shear, ttgbf_import_cores) are not used
 * while recording (the recording fails: ttgbf_adj_backward returns
 * TTGBF_ECAPACITY).  Coefficients of L and U that are exactly 0 and scalings
 * exactly 1 are not applied by the filter, so their gradient entries carry no
 * contribution from them.  Device memory: a second context of the same shape
 * for the adjoint density, and about d^2 + 2 d + 3 compact snapshots of the
 * batch per recorded step. */
typedef struct ttgbf_adj ttgbf_adj;

/* steps: most steps recorded between ttgbf_adj_record(1) and (0); slots:
 * checkpoints.  TTGBF_EINVAL for a split context or d < 2. */
int ttgbf_adj_create(ttgbf_adj** out, ttgbf_ctx* ctx, int32_t steps, int32_t slots);
int ttgbf_adj_free(ttgbf_adj* a);
/* Zero the adjoint state and the accumulated gradients (synchronises). */
int ttgbf_adj_reset(ttgbf_adj* a);
/* Save / restore the context's filter state (cores, ranks, log-likelihood,
 * canonical form) in checkpoint slot `slot` (asynchronous). */
int ttgbf_adj_save(ttgbf_adj* a, int32_t slot);
int ttgbf_adj_load(ttgbf_adj* a, int32_t slot);
/* on = 1: record the context's next predict / update calls (clears the
 * recording); on = 0: stop. */
int ttgbf_adj_record(ttgbf_adj* a, int32_t on);
/* Run the recording backwards, carrying the adjoint state from the later
 * segment (asynchronous after a short host upload of the operator tables). */
int ttgbf_adj_backward(ttgbf_adj* a);
/* Accumulated gradients per filter (host arrays): dF [batch][d][d],
 * dQ [batch][d] (dl/dQ_mm), dR [batch][nR] (dl/dR_cc for measurement
 * components 0..nR-1).  Synchronises; TTGBF_ECAPACITY if a rank of the
 * reverse pass outgrew its bound. */
int ttgbf_adj_grads(ttgbf_adj* a, double* dF, double* dQ, double* dR, int32_t nR);
/* Host-only: G_F = dl/dF from the gradients with respect to the strictly
 * lower part of L (GL, d x d), the diagonal D (GD, d) and the strictly upper
 * part of U (GU, d x d) of F = L D U (no pivoting).  TTGBF_ESINGULAR if F has
 * no such factorisation. */
int ttgbf_ldu_adjoint(int32_t d, const double* F, const double* GL, const double* GD, const double* GU,
                      double* GF);

#ifdef __cplusplus
}
#endif
#endif /* TTGBF_H */
