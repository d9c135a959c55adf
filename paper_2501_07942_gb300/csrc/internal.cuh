// internal.cuh -- shared declarations of the ttgbf CUDA path (not part of the C ABI).
//
// Data layout in HBM (float32 unless noted):
//   * TT core k of filter b lives in one of two ping-pong buffers per core,
//     at buf[s][k] + b * core_cap[k], row-major [r_k][n_k][r_{k+1}] with the
//     filter's ACTUAL ranks packed at the start of its capacity slot.
//   * ranks: int32 [batch][d+1] on the device.  Every kernel reads the ranks
//     it needs from there, so a filter step needs no host synchronisation and
//     can be captured in a CUDA graph.
//   * Small dense factors (SVD output P1/P2) use leading dimension kMaxN.
//
// The rounding of Sec. 4.1 ("round") is built from three generic pieces
// driven by device-side work lists: a tall-skinny QR (TSQR) that returns only
// the R factor of a tall matrix, an SVD of that R (pivoted QR, then one-sided
// Jacobi), and a grouped GEMM that applies the resulting small factors to the
// cores.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ttgbf {

constexpr int kMaxN = 160;          // largest column count of a TSQR / SVD problem
constexpr int kTsqrTileRows = 128;  // rows per register block of the TSQR kernel
constexpr int kTsqrMaxSlices = 64;  // row slices (CTAs) per TSQR problem
constexpr int kJacobiSmemFloats = 2 * kMaxN * kMaxN + 8 * kMaxN;  // SVD kernel
constexpr int kMaxD = 16;           // largest state dimension
constexpr int kTile = 64;           // GEMM square tile edge

// Residual r = z - h of a measurement component.  An angle-like component
// (period > 0) has its residual taken modulo the period into [-period/2,
// period/2]: the nearer branch of the angle (the square of the two ends is
// the same).
template <typename T>
__host__ __device__ __forceinline__ T wrap_residual(T r, T period) {
  return period > T(0) ? r - period * floor(r / period + T(0.5)) : r;
}

// A strided matrix view: element (i, j) at p[i * rs + j * cs], i < M, j < n.
struct MatView {
  const float* p;
  long long rs, cs;
  int M, n;
};

// One TSQR problem: the R factor of a tall matrix.  Its rows are cut into
// nslice slices of `slice` rows, one CTA each; with one slice the R factor is
// written to stack0, otherwise the slice factors are stacked in stack0 and
// their R factor is written to stack1 (nlev = 1 or 2: R ends in
// stack[(nlev-1)&1]).
struct TsqrProblem {
  MatView src;
  int slice;
  int nslice;
  int nlev;
  float* stack0;
  float* stack1;
};

struct TsqrWork {
  TsqrProblem* prob;  // [B]
  int* offset;        // [B+1] exclusive prefix of slice counts
  int* counter;       // [B] slices finished (reset by the plan kernel)
};

// Rows per slice of a TSQR problem: `blocks` register blocks of 128 rows
// (8 unless a context's options say otherwise).
constexpr int kTsqrSliceBlocks = 8;
__host__ __device__ inline long long tsqr_slice_rows(int blocks) {
  return (long long)blocks * kTsqrTileRows;
}

// Row-major GEMM C (m x n) = A (m x k) * B (k x n).  `shape` (the tile
// shape) is chosen by the tile scan from m and n.
struct GemmDesc {
  const float* A;
  const float* B;
  float* C;
  int m, n, k, lda, ldb, ldc;
  int shape;
};

struct GemmWork {
  GemmDesc* desc;  // [ndesc]
  int* tiles;      // [ndesc + 1] exclusive prefix of tile counts
  int ndesc;
  int tc;          // kContract*: SIMT float32 tiles, or tensor-core tiles
  int* status;     // set to 1 by a tensor-core tile that gave up waiting
};

// Contraction arithmetic of the grouped GEMM.
enum ContractMode : int { kContractFp32 = 0, kContractTf32 = 1, kContractTf32x3 = 2 };
// Tensor-core tiles: 128 along C's longer side, 32 along the shorter;
// shape kTcShapeN = rows of C along the 128, kTcShapeT = columns of C.
constexpr int kTcTileM = 128;
constexpr int kTcTileN = 32;
constexpr int kTcShapeN = 3;
constexpr int kTcShapeT = 4;

enum StageMode : int { kStageRight = 0, kStageLeft = 1, kStageSplit = 2 };

// Per-filter state of the rounding in progress.
struct RoundState {
  double* normA;     // [B] ||A||_F at the start of the truncation sweep
  double* tail_sum;  // [B] sum of discarded relative tails
  double* tail_max;  // [B]
  int* cap_hits;     // [B]
  int* newrank;      // [B] rank chosen by the last Jacobi stage
};

// Geometry of the TT shared by all filters.
struct TTGeom {
  int d;
  int n[kMaxD];
  long long cap[kMaxD];  // floats per filter per core
};

// ------------------------------------------------------------ launchers
// linalg.cu
// elem: 4-byte words per stack element (1: float32 slice factors, 2: float64);
// slice_blocks: 128-row register blocks per TSQR slice
void launch_plan_stage(cudaStream_t st, int B, int mode, int k, const TTGeom& g, const int* ranks,
                       const float* core_k, const float* W, long long W_cap, int N0, int N1,
                       TsqrWork w, float* stack0, float* stack1, long long stack_cap, int slots,
                       int elem, int slice_blocks);
// tsqr.cu
void launch_tsqr(cudaStream_t st, TsqrWork w, int B, int grid, double* flops);
// left_threads: CTA width of the truncating left-sweep stages (512 or 1024)
void launch_svd(cudaStream_t st, TsqrWork w, int B, int mode, int rank_cap, double eps, int d,
                   int first, RoundState rs, float* P1, float* P2, float* core0_out,
                   long long core0_cap, double* flops, int left_threads);
void launch_plan_gemm_stage(cudaStream_t st, int B, int mode, int k, const TTGeom& g, int* ranks,
                            const int* newrank, const float* cur_a, float* alt_a,
                            const float* cur_b, float* alt_b, const float* P1, const float* P2,
                            const float* W, long long W_cap, int N1, GemmWork gw, int vS,
                            int dstride);
void launch_gemm(cudaStream_t st, GemmWork gw, int grid, double* flops);
void launch_gemm_tc(cudaStream_t st, GemmWork gw, int grid, double* flops);
// Tile prefix for descriptors already written to gw.desc (ndesc entries).
void launch_scan_tiles(cudaStream_t st, GemmWork gw);

// fftconv.cu: the Gaussian kernel of one mode as batched FFT convolutions of
// the fibres of core k (length N, zero padded to M = 2^m >= 2N - 1), with an
// optional cloud-in-cell gather (kCicTaps sources per target cell) on load.
constexpr int kCicTaps = 3;
constexpr int kMaxFftM = 1024;  // N <= 512
struct FftMode {
  int M;
  const float2* khat;  // [M] FFT of the zero-padded kernel, divided by M
  const float2* tw;    // [M / 2] exp(-2 pi i t / M)
  const int* gsrc;     // [N][kCicTaps] source cells (-1: none), or nullptr
  const float* gw;     // [N][kCicTaps] cloud-in-cell weights
};
void launch_conv_fft(cudaStream_t st, int B, int k, const TTGeom& g, const int* ranks, int* off,
                     const float* cur, float* alt, const FftMode& md, int grid, double* flops);
void set_fft_attributes();
// rsvd64.cu: float64 R factor and SVD of the truncating stages (left, split)
void launch_tsqr64(cudaStream_t st, TsqrWork w, int B, int grid, double* flops);
void launch_svd64(cudaStream_t st, TsqrWork w, int B, int mode, int rank_cap, double eps, int d,
                  int first, RoundState rs, float* P1, float* P2, float* core0_out,
                  long long core0_cap, double* flops);
// ttops.cu
void launch_prior(cudaStream_t st, int B, const TTGeom& g, float* const* cores, int* ranks,
                  const double* axes, const double* mean, const double* var);
void launch_shear_expand(cudaStream_t st, int B, const TTGeom& g, int m, int n, int S, int tmin,
                         const float* weights, float* const* cur, float* const* alt,
                         const int* ranks, int virt);
void launch_rank_scale(cudaStream_t st, int B, int d, int* ranks, int lo, int hi, int S);
// A shear applied in pieces of its shift range: save the block, accumulate
// each rounded piece (offsets on the inner links), pack the TT sum.
void launch_block_copy(cudaStream_t st, int B, const TTGeom& g, int lo, int hi,
                       float* const* src, float* const* dst, const int* ranks);
void launch_acc_piece(cudaStream_t st, int B, const TTGeom& g, int lo, int hi, int p, int maxp,
                      int capr, float* const* cur, float* const* acc, const int* ranks,
                      int* acc_rank, int* piece_off);
void launch_acc_sum(cudaStream_t st, int B, const TTGeom& g, int lo, int hi, int np, int maxp,
                    int capr, float* const* acc, float* const* alt, int* ranks,
                    const int* acc_rank, const int* piece_off);
void launch_plan_mode_apply(cudaStream_t st, int B, int k, const TTGeom& g, const int* ranks,
                            const float* M, const float* cur, float* alt, GemmWork gw, int cap_in);
void launch_plan_supercore(cudaStream_t st, int B, const TTGeom& g, const int* ranks,
                           const float* c0, const float* c1, float* W, long long W_cap,
                           GemmWork gw);
// Likelihood factors (ttops.cu).  period: 0, or the period of an angle-like
// component whose residual is wrapped (wrap_residual).
void launch_lik_offset(cudaStream_t st, int B, const float* htab, int ntab, const float* z,
                       int zstride, int zc, double R, float period, float* off, double* logoff);
void launch_lik_apply_2d(cudaStream_t st, int B, float* W, long long W_cap, int N0, int N1,
                         const int* ranks, int d, const float* htab, const float* z, int zstride,
                         int zc, double R, float period, const float* off);
void launch_lik_apply_1d(cudaStream_t st, int B, float* core, long long cap, int N, int k, int d,
                         const int* ranks, const float* htab, const float* z, int zstride, int zc,
                         double R, float period, const float* off);
void launch_logc(cudaStream_t st, int B, const double* mass, const double* logoff, double* log_c,
                 double* log_lik, int add);
void launch_densify_stage(cudaStream_t st, const double* X, long long P, int ra, const float* G, int n, int rb,
                          double* Y);
// Moments of a TT given by per-core base pointers (filter stride cap[kk]) and
// rank indices: core kk has ranks (ranks[b][ridx[kk]], ranks[b][ridx[kk+1]]).
struct MomentArgs {
  int ncores;
  int n[kMaxD + 1];
  int ridx[kMaxD + 2];
  const float* core[kMaxD + 1];
  long long cap[kMaxD + 1];
  const double* axes[kMaxD + 1];  // per-core coordinates (nullptr when mass only)
  double centre[kMaxD + 1];
  double delta;       // cell volume
  int with_moments;   // 0: mass only
  float* scale_core;  // core scaled by 1/mass after the moments (nullptr: none)
  long long scale_cap;
  int scale_idx;      // index kk of scale_core
};
void launch_moments(cudaStream_t st, int B, const MomentArgs& a, const int* ranks, int rstride,
                    double* Awork, long long awork_stride, double* mass, double* mean, double* cov);
// adjoint.cu: kernels of the reverse pass (adjoint recursion in TT form).  Tensor
// trains are given per core as (pointer, per-filter stride) with ranks
// [B][rstride]; environments are rx x ry float matrices at phi_stride.
void launch_env_step(cudaStream_t st, int B, int k, int n, const float* X, long long xcap, const int* xr,
                     const float* Y, long long ycap, const int* yr, int rstride, const float* Phi,
                     long long phi_stride, float* part, int chunks, int phi_max, int* err);
void launch_env_reduce(cudaStream_t st, int B, int k, const int* xr, const int* yr, int rstride,
                       const float* part, int chunks, int phi_max, float* Phi_out, long long phi_stride,
                       double* scal, double mul, int accumulate);
void launch_copy_cores(cudaStream_t st, int B, int k0, int k1, const float* const* src, const long long* scap,
                       const int* n, const int* sr, int rstride, float* const* dst, const long long* dcap);
void launch_mode(cudaStream_t st, int B, int k, int N, const float* M, const float* in, long long icap,
                 float* out, long long ocap, const int* ranks, int rstride);
void launch_add_ones(cudaStream_t st, int B, int d, const float* const* src, const long long* scap,
                     const int* n, float* const* dst, const long long* dcap, int* ranks, int rstride,
                     const double* sc, const double* coef);
void launch_lik1(cudaStream_t st, int B, int k, int N, const float* src, long long scap, float* dst,
                 long long dcap, const int* ranks, int rstride, const float* htab, const float* zv,
                 const float* off, double R, float period, int which);
void launch_lik2_split(cudaStream_t st, int B, int N0, int N1, const float* g0, long long g0cap,
                       const float* g1, long long g1cap, float* o0, long long o0cap, float* o1,
                       long long o1cap, int* ranks, int rstride, const float* htab, const float* zv,
                       const float* off, double R, float period, int which);
void launch_scalars(cudaStream_t st, int B, int op, const double* m, const double* val, double delta,
                    double* sc, double* coef, double* grad, int gstride, int gi, double mul);
void set_adjoint_attributes();

// cross.cu: deterministic TT cross of the product of a likelihood factor with
// the block of cores lo..lo+k-1 of every filter (one CTA per filter per step).
constexpr int kCrossMaxS = 64;  // largest cross rank
enum CrossKind : int { kCrossStart = 0, kCrossLR = 1, kCrossRL = 2, kCrossFinal = 3 };
struct CrossArgs {
  int B, d, lo, k, s;
  int* ranks;                  // [B][d+1]: read during the cross, the block's links written last
  const float* core[kMaxD];    // block cores q = 0..k-1 (current buffers), filter stride cap[q]
  float* out[kMaxD];           // the result's cores (the other buffers)
  long long cap[kMaxD];
  int N[kMaxD];                // grid sizes of the block's modes
  long long stride[kMaxD];     // offset in the table of one step along each block mode (0: not used)
  const float* htab;           // the component's table
  const float* z;              // z[b * zstride + zc]
  int zstride, zc;
  double R;
  float period;
  const float* off;            // [B] likelihood offsets (k_lik_offset)
  float* F;                    // [B][fcap] fiber matrix / B = Q Q[rows]^-1 (column-major)
  float* Qb;                   // [B][fcap] orthonormal basis
  float* rn;                   // [B][mcap] row norms of the start matrices
  unsigned* mask;              // [B][mcap / 32 + 1] rows taken (elimination)
  long long fcap, mcap;
  long long* offI;             // [B][d+1][s] table offsets of the left index sets
  long long* offJ;             // [B][d+1][s] ... of the right index sets
  float* U;                    // [B][d+1][s][s] left interfaces (row vectors)
  float* V;                    // [B][d+1][s][s] right interfaces
  int* sz;                     // [B][2][d+1] sizes of the left and right sets
  int* status;                 // [B] nonzero: a rank of the block exceeded s (the step was skipped)
  // trans != 0: the block is the 2-site block (lo, lo+1) after the mode-lo
  // factor of the textbook transition, T(a, j, i', b) = sum_i K(j, i, i')
  // [G_lo(i) G_lo+1(i')](a, b), K(j, i, i') = dx0 N(xi0_j - F0 xi0_i - F1
  // xi1_i'; 0, q) (no likelihood table); the index sets then hold the raw
  // virtual indices (a, j) and (i', b) instead of table offsets
  int trans;
  float tF0, tF1, tiq, tkc;    // F_lo,lo, F_lo,lo+1, 1 / q, dx0 / sqrt(2 pi q)
  float tlo0, tdx0, tlo1, tdx1;  // axes: xi = lo + (i + 1/2) dx
  float twin;                  // half-width in cells of the old-index window of a sum (beyond it
                               // K < exp(-32) of its peak); <= 0: the whole axis
};
void launch_cross_step(cudaStream_t st, const CrossArgs& a, int q, int kind);
void launch_cross_last(cudaStream_t st, const CrossArgs& a);
// Process-wide count of kernel launches made by the library (capi.cu).
void count_launches(int n);
// Function attributes (large dynamic shared memory); call once per process.
void set_kernel_attributes();
void set_ttops_attributes();
void set_tsqr_attributes();
void set_rsvd64_attributes();

}  // namespace ttgbf
