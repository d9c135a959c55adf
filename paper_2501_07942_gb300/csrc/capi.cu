// capi.cu -- host orchestration of the TT point-mass filter and the C ABI
// declared in include/ttgbf.h.
//
// Step structure (arXiv 2501.07942, Alg. 3 on a fixed axis-aligned grid):
//   predict: F = L D U (no pivoting) -> U's shears (each: TT-operator
//            expansion + rounding) -> D's scalings fused with the Gaussian
//            kernel per mode (when L = I) -> L's shears -> normalise
//   update : one-mode likelihood factors scale core slices; a two-mode
//            component on modes (0,1) multiplies the 2-site supercore, which
//            is then split by a truncated SVD inside the TT rounding sweep;
//            log c is taken before the rounding; normalise afterwards
//   estimate: moments by TT contraction
// All data-dependent sizes (TT ranks) stay on the device; the host enqueues a
// fixed sequence of kernels per call.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "ttgbf.h"

using namespace ttgbf;

namespace {

constexpr int kMaxComps = 16;

enum ProfClass : int { kPTsqr = 0, kPSvd, kPGemm, kPShear, kPMoments, kPLik, kPPlan, kPOther, kPFft,
                       kPCross, kPClasses };
const char* const kProfNames[kPClasses] = {"tsqr", "svd", "gemm", "shear_expand", "moments",
                                           "likelihood", "plan", "other", "fft_conv", "cross"};

// Smallest power of two >= 2N - 1: the length of the zero-padded cyclic
// convolution that equals the linear one on the grid.
int fft_len(int N) {
  int M = 1;
  while (M < 2 * N - 1) M <<= 1;
  return M;
}

std::atomic<unsigned long long> g_launches{0};

struct Arena {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    const size_t at = (off + 255) & ~size_t(255);
    off = at + count * sizeof(T);
    return at;
  }
};

// Offsets of every device buffer inside the workspace.
struct Layout {
  size_t core[2][kMaxD];
  size_t piece_core[2][kMaxD];  // saved block, accumulated pieces (wide shears)
  size_t saved_ranks, acc_rank, piece_off;
  size_t ranks, axes, pmean, pvar;
  size_t normA, tail_sum, tail_max, mass, mass_pred, log_c, log_lik, logoff, mean, cov;
  size_t cap_hits, newrank, lik_off;
  size_t tsqr_prob, tsqr_off, tsqr_cnt, stack[2];
  size_t P1, P2, gdesc, gtiles, awork, W, opmats, zbuf, prof_flops, fft_off;
  size_t xF, xQ, xrn, xmask, xoffI, xoffJ, xU, xV, xsz, xstatus;  // the cross (cross_rank > 0)
  long long x_fcap = 0, x_mcap = 0;
  size_t total;
  long long core_cap[kMaxD];
  long long stack_cap, W_cap, opmats_floats, awork_stride;
  int gdesc_cap, capr;
};

// An NVTX range over one API call (host time; tools such as ncu can filter
// kernels by it, e.g. --nvtx --nvtx-include "ttgbf_update/").
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
};

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Floats of the per-filter TSQR stack for an M x n problem: one n x n R
// factor per row slice.
long long tsqr_stack_for(long long M, int n, int slice_blocks) {
  long long nsl = (M + tsqr_slice_rows(slice_blocks) - 1) / tsqr_slice_rows(slice_blocks);
  nsl = std::max<long long>(1, std::min<long long>(nsl, kTsqrMaxSlices));
  return nsl * (long long)n * n;
}

int validate_grid(const ttgbf_grid* g) {
  if (!g || g->d < 1 || g->d > kMaxD || !g->n || !g->lo || !g->hi) return TTGBF_EINVAL;
  for (int k = 0; k < g->d; ++k) {
    if (g->n[k] < 2 || g->n[k] > 4096) return TTGBF_EINVAL;
    if (!std::isfinite(g->lo[k]) || !std::isfinite(g->hi[k])) return TTGBF_ENONFINITE;
    if (!(g->hi[k] > g->lo[k])) return TTGBF_EINVAL;
  }
  return TTGBF_OK;
}

int validate_opts(const ttgbf_opts* o) {
  if (!o || o->batch < 1 || o->rank_cap < 1) return TTGBF_EINVAL;
  if (o->precision != TTGBF_PRECISION_FP32 && o->precision != TTGBF_PRECISION_FP64) return TTGBF_EINVAL;
  if (o->contraction < TTGBF_CONTRACT_FP32 || o->contraction > TTGBF_CONTRACT_TF32X3) return TTGBF_EINVAL;
  if (o->conv < TTGBF_CONV_AUTO || o->conv > TTGBF_CONV_FFT) return TTGBF_EINVAL;
  if (o->parts < 0 || o->parts > 8) return TTGBF_EINVAL;
  if (o->tsqr_slice_blocks != 0 && o->tsqr_slice_blocks != 2 && o->tsqr_slice_blocks != 4 &&
      o->tsqr_slice_blocks != 8 && o->tsqr_slice_blocks != 16)
    return TTGBF_EINVAL;
  if (o->svd_threads != 0 && o->svd_threads != 512 && o->svd_threads != 1024) return TTGBF_EINVAL;
  if (!std::isfinite(o->eps)) return TTGBF_ENONFINITE;
  if (o->eps < 0.0) return TTGBF_EINVAL;
  const int smax = o->max_shift_span > 0 ? o->max_shift_span : 10;
  if ((long long)o->rank_cap * smax > kMaxN || smax < 2) return TTGBF_ECAPACITY;
  if (o->cross_sweeps < 0 || o->cross_rank < 0) return TTGBF_EINVAL;
  if (o->cross_rank > 0 && (o->cross_rank < o->rank_cap || o->cross_rank < 2 || o->cross_rank > kCrossMaxS ||
                            o->cross_rank > o->rank_cap * smax))
    return TTGBF_EINVAL;
  return TTGBF_OK;
}

Layout make_layout(const ttgbf_grid* g, const ttgbf_opts* o) {
  Layout L{};
  Arena a;
  const int d = g->d, B = o->batch;
  const int smax = o->max_shift_span > 0 ? o->max_shift_span : 10;
  const int capr = o->rank_cap * smax;
  L.capr = capr;
  int nmax = 0;
  long long nsum = 0;
  for (int k = 0; k < d; ++k) {
    nmax = std::max(nmax, (int)g->n[k]);
    nsum += g->n[k];
    const long long cl = (k == 0) ? 1 : capr, cr = (k == d - 1) ? 1 : capr;
    L.core_cap[k] = std::max<long long>(cl * g->n[k] * cr, 1);
  }
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < d; ++k) L.core[s][k] = a.take<float>((size_t)B * L.core_cap[k]);
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < d; ++k) L.piece_core[s][k] = a.take<float>((size_t)B * L.core_cap[k]);
  L.saved_ranks = a.take<int>((size_t)B * (d + 1));
  L.acc_rank = a.take<int>((size_t)B * (d + 1));
  L.piece_off = a.take<int>((size_t)B * smax * (d + 1));
  L.ranks = a.take<int>((size_t)B * (d + 1));
  L.axes = a.take<double>(nsum);
  L.pmean = a.take<double>(d);
  L.pvar = a.take<double>(d);
  L.normA = a.take<double>(B);
  L.tail_sum = a.take<double>(B);
  L.tail_max = a.take<double>(B);
  L.mass = a.take<double>(B);
  L.mass_pred = a.take<double>(B);
  L.log_c = a.take<double>(B);
  L.log_lik = a.take<double>(B);
  L.logoff = a.take<double>(B);
  L.mean = a.take<double>((size_t)B * d);
  L.cov = a.take<double>((size_t)B * d * d);
  L.cap_hits = a.take<int>(B);
  L.newrank = a.take<int>(B);
  L.lik_off = a.take<float>(B);
  L.tsqr_prob = a.take<TsqrProblem>(B);
  L.tsqr_off = a.take<int>((size_t)B + 1);
  L.tsqr_cnt = a.take<int>((size_t)B);
  // tall matrices: rows <= capr * nmax, columns <= max(capr, n0)
  const long long Mmax = (long long)capr * nmax;
  const int nsplit = (d >= 2) ? std::min<int>(g->n[0], kMaxN) : 1;
  long long stack = 0;
  const int sblocks = o->tsqr_slice_blocks > 0 ? o->tsqr_slice_blocks : kTsqrSliceBlocks;
  for (int n = 1; n <= std::max(capr, nsplit); ++n)
    stack = std::max(stack, tsqr_stack_for(Mmax, n, sblocks));
  // float64 slice factors take two words per entry
  if (o->precision == TTGBF_PRECISION_FP64) stack *= 2;
  L.stack_cap = stack;
  L.stack[0] = a.take<float>((size_t)B * stack);
  L.stack[1] = a.take<float>((size_t)B * stack);
  L.P1 = a.take<float>((size_t)B * kMaxN * kMaxN);
  L.P2 = a.take<float>((size_t)B * kMaxN * kMaxN);
  L.gdesc_cap = std::max(2 * B, B * (capr + 1));
  L.gdesc = a.take<GemmDesc>(L.gdesc_cap);
  L.gtiles = a.take<int>(L.gdesc_cap + 2);  // + the tensor-core status word
  L.awork_stride = (long long)(d + 1) * 3 * kMaxN * kMaxN;
  L.awork = a.take<double>((size_t)B * L.awork_stride);
  L.W_cap = (d >= 2) ? (long long)g->n[0] * g->n[1] * o->rank_cap : 1;
  L.W = a.take<float>((size_t)B * L.W_cap);
  long long nn = 0;
  for (int k = 0; k < d; ++k) nn += (long long)g->n[k] * g->n[k];
  // shear tables, per-mode matrices, and per-mode FFT tables (spectrum,
  // twiddles, cloud-in-cell gather: 2M + M + 6N words, 8-byte aligned)
  L.opmats_floats = 2 * nn + (long long)d * d * (smax * smax + 2) * nmax +
                    (long long)d * (3 * fft_len(nmax) + 6 * nmax + 8);
  L.fft_off = a.take<int>((size_t)B + 1);
  L.opmats = a.take<float>(L.opmats_floats);
  L.zbuf = a.take<float>((size_t)B * kMaxComps);
  L.prof_flops = a.take<double>(kPClasses);
  if (o->cross_rank > 0) {
    // fiber matrices: rows <= s * N_max (the block's boundary ranks are at
    // most the rank cap <= s), columns <= s
    const long long s = o->cross_rank;
    L.x_mcap = s * nmax;
    L.x_fcap = L.x_mcap * s;
    L.xF = a.take<float>((size_t)B * L.x_fcap);
    L.xQ = a.take<float>((size_t)B * L.x_fcap);
    L.xrn = a.take<float>((size_t)B * L.x_mcap);
    L.xmask = a.take<unsigned>((size_t)B * (L.x_mcap / 32 + 1));
    L.xoffI = a.take<long long>((size_t)B * (d + 1) * s);
    L.xoffJ = a.take<long long>((size_t)B * (d + 1) * s);
    L.xU = a.take<float>((size_t)B * (d + 1) * s * s);
    L.xV = a.take<float>((size_t)B * (d + 1) * s * s);
    L.xsz = a.take<int>((size_t)B * 2 * (d + 1));
    L.xstatus = a.take<int>((size_t)B);
  }
  L.total = a.off + 256;
  return L;
}

// One elementary re-gridding operation (the order of application is fixed).
struct Op {
  int kind;  // 0 shear, 1 scale
  int m, n;
  double a;
};

}  // namespace

struct ttgbf_adj;

struct ttgbf_ctx {
  int B = 0, d = 0;
  std::vector<int> n;
  std::vector<double> lo, hi, dx, axes;
  std::vector<int> axoff;
  int rank_cap = 0, smax = 0, capr = 0;
  // the cross of block likelihood components: rank (0: not available),
  // refinement sweeps, and its workspace (per-call fields filled in later)
  int cross_s = 0, cross_sweeps = 1;
  CrossArgs x{};
  int precision = TTGBF_PRECISION_FP32;
  int contract = kContractFp32;  // arithmetic of the grouped GEMM (opts.contraction)
  int* tc_status = nullptr;      // set by a tensor-core tile that gave up waiting
  int slice_blocks = kTsqrSliceBlocks, svd_threads = 512;
  double eps = 0.0, delta = 1.0;
  cudaStream_t st = nullptr;
  Layout L{};
  char* base = nullptr;
  bool owns = false;
  TTGeom geom{};
  float* buf[2][kMaxD] = {};
  int cur[kMaxD] = {};
  // a shear wider than smax shifts: saved block cores, accumulated pieces
  float* save[kMaxD] = {};
  float* acc[kMaxD] = {};
  int *saved_ranks = nullptr, *acc_rank = nullptr, *piece_off = nullptr;
  int* ranks = nullptr;
  double *axes_d = nullptr, *pmean = nullptr, *pvar = nullptr;
  double *normA, *tail_sum, *tail_max, *mass, *mass_pred, *log_c, *log_lik, *logoff, *mean, *cov;
  int *cap_hits, *newrank;
  float* lik_off;
  TsqrWork tw{};
  float* stack[2];
  float *P1, *P2;
  GemmDesc* gdesc;
  int* gtiles;
  double* awork;
  float* W;
  float* opmats;
  float* zbuf;
  // pinned host staging
  float* stage_ops = nullptr;
  float* stage_z = nullptr;
  double* stage_est = nullptr;  // mean, cov, log c, log-likelihood read back by estimate
  cudaEvent_t ev_ops = nullptr, ev_z = nullptr;
  bool ev_ops_used = false, ev_z_used = false;
  // cached predict operators
  std::vector<double> lastF, lastQ;
  std::vector<Op> ops;
  std::vector<int> op_S, op_tmin;
  std::vector<long long> op_woff;  // float offsets of shear weight tables in opmats
  std::vector<long long> mat_off;  // per mode: fused (or conv) matrix offset
  std::vector<long long> scale_off;  // per mode: CIC matrix (only used when L != I), -1 if none
  bool fuse = true;
  // the Gaussian kernel of mode k as an FFT convolution (opts.conv): the
  // mode's tables in the operator area (offsets in words, -1: none)
  int conv_mode = TTGBF_CONV_AUTO;
  bool mode_fft[kMaxD] = {};
  long long fft_khat[kMaxD] = {}, fft_tw[kMaxD] = {}, fft_gsrc[kMaxD] = {}, fft_gw[kMaxD] = {};
  int fft_M[kMaxD] = {};
  int* fft_off = nullptr;
  bool poisoned = false;
  bool expanded = false;  // ranks may exceed rank_cap (after an unrounded shear or import)
  // virt_S[k] > 0: core k is a middle core of the shear block being rounded
  // and still holds its unexpanded data (its expanded form is G (x) I_S)
  int virt_S[kMaxD] = {};
  // Mixed canonical form: when canon is true, cores < center are left-
  // orthonormal and cores > center right-orthonormal (the center holds the norm).
  bool canon = false;
  int center = 0;
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool[kPClasses];
  size_t ev_used[kPClasses] = {};
  long long prof_launches[kPClasses] = {};
  double* prof_flops = nullptr;
  bool debug_stages = false;
  // Host-side fault injection (TTGBF_FAULT=cuda:N): the N-th status check
  // after init reports a CUDA error, as a failed call would; 0 = off.
  long long fault_after = 0;
  int sms = 148;
  // A batch split into independent sub-batches ("parts"), each a full
  // context on its own stream: the parts' kernels overlap on the GPU (one
  // part's SVD on part of the SMs while another's QR or GEMM fills the rest).
  // The parent owns no device arena; calls fan out to the parts between a
  // fork and a join on the caller's stream.
  std::vector<ttgbf_ctx*> parts;
  std::vector<int> part_base;  // first filter of each part; part_base[nparts] = B
  std::vector<cudaStream_t> part_st;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  // of a part: the share of the GPU's resident QR CTAs it plans for
  double slot_share = 1.0;
  // reverse pass: while set, predict and update record their steps here
  ttgbf_adj* tape = nullptr;
  int tape_op = -1;  // index in ops of the shear being enqueued
};

namespace {

int cuda_fail(ttgbf_ctx* c) {
  c->poisoned = true;
  return TTGBF_ECUDA;
}

int check(ttgbf_ctx* c) {
  if (c->fault_after > 0 && --c->fault_after == 0) return cuda_fail(c);  // injected
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(c);
  }
  return TTGBF_OK;
}

// Records CUDA events around a group of launches of one kernel class while
// profiling is enabled.
struct Prof {
  ttgbf_ctx* c;
  int cls;
  Prof(ttgbf_ctx* cc, int k, int nlaunch) : c(cc), cls(k) {
    c->prof_launches[k] += nlaunch;
    if (c->prof) record();
  }
  ~Prof() {
    if (c->prof) record();
  }
  void record() {
    auto& pool = c->ev_pool[cls];
    if (c->ev_used[cls] == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    cudaEventRecord(pool[c->ev_used[cls]++], c->st);
  }
};

double* flops_of(ttgbf_ctx* c, int cls) { return c->prof_flops + cls; }

float* curp(ttgbf_ctx* c, int k) { return c->buf[c->cur[k]][k]; }
float* altp(ttgbf_ctx* c, int k) { return c->buf[c->cur[k] ^ 1][k]; }

RoundState round_state(ttgbf_ctx* c) {
  return RoundState{c->normA, c->tail_sum, c->tail_max, c->cap_hits, c->newrank};
}

GemmWork gemm_work(ttgbf_ctx* c, int ndesc) {
  return GemmWork{c->gdesc, c->gtiles, ndesc, c->contract, c->tc_status};
}

// Diagnostic (environment TTGBF_DEBUG_STAGES=1): after each rounding stage,
// synchronise and report filter 0's ranks and whether the two cores the
// stage wrote are finite.  Off by default; it serialises the step.
void debug_stage_report(ttgbf_ctx* c, int mode, int k, int ka, int kb) {
  std::vector<int> rk(c->d + 1);
  cudaStreamSynchronize(c->st);
  cudaMemcpy(rk.data(), c->ranks, sizeof(int) * (c->d + 1), cudaMemcpyDeviceToHost);
  bool fin = true;
  float amax = 0.f;
  for (int kk : {ka, kb}) {
    const size_t cnt = (size_t)rk[kk] * c->n[kk] * rk[kk + 1];
    std::vector<float> h(cnt);
    cudaMemcpy(h.data(), curp(c, kk), sizeof(float) * cnt, cudaMemcpyDeviceToHost);
    for (float v : h) {
      if (!std::isfinite(v)) fin = false;
      else amax = std::max(amax, std::fabs(v));
    }
  }
  std::fprintf(stderr, "[ttgbf stage] mode=%d k=%d ranks=", mode, k);
  for (int v : rk) std::fprintf(stderr, "%d ", v);
  std::fprintf(stderr, "finite=%d absmax=%.3e\n", (int)fin, amax);
}

// One stage of the rounding sweep: R factor, SVD, rank choice, factor application.
// With float64 precision the truncating stages (left, split) form R and its
// SVD in float64 (one TSQR CTA per SM: its shared memory holds a float64 R).
// Recording of the forward pass for the reverse pass (no-ops unless
// c->tape is set; defined with the adjoint below).
enum TapeModeKind : int { kModeConv = 0, kModeScale = 1, kModeConvScale = 2 };
void tape_shear(ttgbf_ctx* c, int m, int n);
void tape_mode(ttgbf_ctx* c, int k, int kind);
void tape_norm(ttgbf_ctx* c, const double* mass);
void tape_upd_in(ttgbf_ctx* c);
void tape_lik(ttgbf_ctx* c, int comp, const ttgbf_meas_comp& cp, const float* z, int zstride, double R);
void tape_logc(ttgbf_ctx* c, const double* mass);
void tape_fail(ttgbf_ctx* c);

void stage(ttgbf_ctx* c, int mode, int k, int first) {
  const int B = c->B;
  const float* src = (mode == kStageSplit) ? c->W : curp(c, k);
  const bool fp64 = c->precision == TTGBF_PRECISION_FP64 && mode != kStageRight;
  {
    Prof p(c, kPPlan, 1);
    const int per_sm = fp64 ? 1 : 2;
    launch_plan_stage(c->st, B, mode, k, c->geom, c->ranks, src, c->W, c->L.W_cap, c->n[0],
                      c->d > 1 ? c->n[1] : 1, c->tw, c->stack[0], c->stack[1], c->L.stack_cap,
                      std::max(1, (int)(per_sm * c->sms * c->slot_share)), fp64 ? 2 : 1,
                      c->slice_blocks);
  }
  {
    Prof p(c, kPTsqr, 1);
    if (fp64) launch_tsqr64(c->st, c->tw, B, c->sms, flops_of(c, kPTsqr));
    else launch_tsqr(c->st, c->tw, B, c->sms, flops_of(c, kPTsqr));
  }
  float* core0_alt = (mode == kStageSplit) ? altp(c, 0) : nullptr;
  {
    Prof p(c, kPSvd, 1);
    if (fp64)
      launch_svd64(c->st, c->tw, B, mode, c->rank_cap, c->eps, c->d, first, round_state(c), c->P1,
                   c->P2, core0_alt, c->L.core_cap[0], flops_of(c, kPSvd));
    else
      launch_svd(c->st, c->tw, B, mode, c->rank_cap, c->eps, c->d, first, round_state(c), c->P1,
                 c->P2, core0_alt, c->L.core_cap[0], flops_of(c, kPSvd), c->svd_threads);
  }
  int ka, kb, ndesc = 2 * B, vS = 0;
  if (mode == kStageRight) {
    ka = k;
    kb = k - 1;
    vS = c->virt_S[kb];
    if (vS > 0) ndesc = B * (c->capr + 1);
  } else if (mode == kStageLeft) {
    ka = k;
    kb = k + 1;
  } else {
    ka = 0;
    kb = 1;
    ndesc = B;
  }
  GemmWork gw = gemm_work(c, ndesc);
  {
    Prof p(c, kPPlan, 2);
    launch_plan_gemm_stage(c->st, B, mode, k, c->geom, c->ranks, c->newrank, curp(c, ka), altp(c, ka),
                           curp(c, kb), altp(c, kb), c->P1, c->P2, c->W, c->L.W_cap,
                           c->d > 1 ? c->n[1] : 1, gw, vS, c->capr + 1);
  }
  c->virt_S[kb] = 0;  // written densely by this stage's second product
  {
    Prof p(c, kPGemm, 1);
    launch_gemm(c->st, gw, c->sms * 8, flops_of(c, kPGemm));
  }
  c->cur[ka] ^= 1;
  c->cur[kb] ^= 1;
  if (c->debug_stages) debug_stage_report(c, mode, k, ka, kb);
}

// TT rounding: right-to-left orthogonalisation, left-to-right truncation.
void enqueue_round(ttgbf_ctx* c) {
  if (c->d < 2) return;
  for (int k = c->d - 1; k >= 1; --k) stage(c, kStageRight, k, 0);
  for (int k = 0; k <= c->d - 2; ++k) stage(c, kStageLeft, k, k == 0);
  c->expanded = false;
  c->canon = true;
  c->center = c->d - 1;
}

// Bring the TT into mixed canonical form with its center inside [lo, hi]:
// cores < lo left-orthonormal, cores > hi right-orthonormal.
void enqueue_center_into(ttgbf_ctx* c, int lo, int hi) {
  if (!c->canon) {
    for (int k = c->d - 1; k >= 1; --k) stage(c, kStageRight, k, 0);
    c->canon = true;
    c->center = 0;
  }
  while (c->center > hi) {
    stage(c, kStageRight, c->center, 0);
    --c->center;
  }
  bool first = true;
  while (c->center < lo) {
    stage(c, kStageLeft, c->center, first);
    first = false;
    ++c->center;
  }
}

MomentArgs tt_moment_args(ttgbf_ctx* c, int with_moments, int scale) {
  MomentArgs a{};
  a.ncores = c->d;
  for (int k = 0; k < c->d; ++k) {
    a.n[k] = c->n[k];
    a.core[k] = curp(c, k);
    a.cap[k] = c->L.core_cap[k];
    a.axes[k] = c->axes_d + c->axoff[k];
    a.centre[k] = 0.5 * (c->lo[k] + c->hi[k]);
  }
  for (int k = 0; k <= c->d; ++k) a.ridx[k] = k;
  a.delta = c->delta;
  a.with_moments = with_moments;
  if (scale) {
    a.scale_core = curp(c, c->d - 1);
    a.scale_cap = c->L.core_cap[c->d - 1];
    a.scale_idx = c->d - 1;
  }
  return a;
}

// Normalise to unit mass by scaling one core: the center of the canonical
// form when there is one (scaling it keeps the other cores orthonormal).
void enqueue_normalise(ttgbf_ctx* c, double* mass_out) {
  MomentArgs a = tt_moment_args(c, 0, 1);
  const int k = c->canon ? c->center : c->d - 1;
  a.scale_core = curp(c, k);
  a.scale_cap = c->L.core_cap[k];
  a.scale_idx = k;
  {
    Prof p(c, kPMoments, 1);
    launch_moments(c->st, c->B, a, c->ranks, c->d + 1, c->awork, c->L.awork_stride, mass_out, nullptr,
                   nullptr);
  }
  tape_norm(c, mass_out);
}

void mode_apply(ttgbf_ctx* c, int k, const float* M) {
  GemmWork gw = gemm_work(c, c->B * c->capr);
  {
    Prof p(c, kPPlan, 2);
    launch_plan_mode_apply(c->st, c->B, k, c->geom, c->ranks, M, curp(c, k), altp(c, k), gw, c->capr);
  }
  {
    Prof p(c, kPGemm, 1);
    launch_gemm(c->st, gw, c->sms * 8, flops_of(c, kPGemm));
  }
  c->cur[k] ^= 1;
  if (!(c->canon && c->center == k)) c->canon = false;
}

// Mode k's Gaussian kernel as batched FFT convolutions of the core's fibres,
// from the tables fft_tables put in the operator area.
void mode_conv_fft(ttgbf_ctx* c, int k) {
  FftMode md{};
  md.M = c->fft_M[k];
  md.khat = reinterpret_cast<const float2*>(c->opmats + c->fft_khat[k]);
  md.tw = reinterpret_cast<const float2*>(c->opmats + c->fft_tw[k]);
  md.gsrc = c->fft_gsrc[k] >= 0 ? reinterpret_cast<const int*>(c->opmats + c->fft_gsrc[k]) : nullptr;
  md.gw = c->fft_gw[k] >= 0 ? c->opmats + c->fft_gw[k] : nullptr;
  {
    Prof p(c, kPFft, 2);
    launch_conv_fft(c->st, c->B, k, c->geom, c->ranks, c->fft_off, curp(c, k), altp(c, k), md,
                    c->sms * 2, flops_of(c, kPFft));
  }
  c->cur[k] ^= 1;
  if (!(c->canon && c->center == k)) c->canon = false;
}

bool conv_uses_fft(const ttgbf_ctx* c, int m) {
  const int N = c->n[m];
  if (N < 2 || fft_len(N) > kMaxFftM) return false;
  if (c->conv_mode == TTGBF_CONV_FFT) return true;
  if (c->conv_mode == TTGBF_CONV_DENSE) return false;
  return N >= 256;
}

double hatf(double t) { return std::max(0.0, 1.0 - std::fabs(t)); }

// Shear x_m += a x_n: integer shift range and hat-weight table.
void shear_table(ttgbf_ctx* c, int m, int n, double a, int* S, int* tmin, std::vector<float>* w) {
  const int Nn = c->n[n];
  std::vector<double> s(Nn);
  int lo = 1 << 30, hi = -(1 << 30);
  for (int i = 0; i < Nn; ++i) {
    s[i] = a * c->axes[c->axoff[n] + i] / c->dx[m];
    const int f = (int)std::floor(s[i]);
    lo = std::min(lo, f);
    hi = std::max(hi, f);
  }
  *tmin = lo;
  *S = hi - lo + 2;
  w->assign((size_t)(*S) * Nn, 0.f);
  for (int u = 0; u < *S; ++u)
    for (int i = 0; i < Nn; ++i) (*w)[(size_t)u * Nn + i] = (float)hatf(lo + u - s[i]);
}

void cic_matrix(ttgbf_ctx* c, int m, double lam, std::vector<double>* W) {
  const int N = c->n[m];
  W->assign((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) {
    const double u = (lam * c->axes[c->axoff[m] + i] - c->lo[m]) / c->dx[m] - 0.5;
    for (int j = 0; j < N; ++j) (*W)[(size_t)j * N + i] = hatf(j - u);
  }
}

void conv_matrix(ttgbf_ctx* c, int m, double q, std::vector<double>* K) {
  const int N = c->n[m];
  const double D = c->dx[m];
  K->assign((size_t)N * N, 0.0);
  const double norm = D / std::sqrt(2.0 * M_PI * q);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      const double t = (double)(j - i) * D;
      (*K)[(size_t)j * N + i] = norm * std::exp(-0.5 * t * t / q);
    }
}

// FFT tables of mode m's kernel with variance q, appended to host at *at
// (4-byte words, 8-byte aligned): the spectrum of kappa zero-padded to M
// (float64 DFT, divided by M so the inverse transform needs no scaling),
// the twiddles exp(-2 pi i t / M), and, when lam != 1, the cloud-in-cell
// gather of the scaling x_m <- lam x_m (kCicTaps sources per target).
// Returns false (and appends nothing) when the scaling needs more taps.
bool fft_tables(ttgbf_ctx* c, int m, double q, double lam, std::vector<float>* host, long long* at) {
  const int N = c->n[m];
  const int M = fft_len(N);
  const double D = c->dx[m];
  std::vector<int> gsrc;
  std::vector<float> gw;
  if (lam != 1.0) {
    gsrc.assign((size_t)N * kCicTaps, -1);
    gw.assign((size_t)N * kCicTaps, 0.f);
    std::vector<int> cnt(N, 0);
    for (int i = 0; i < N; ++i) {
      const double u = (lam * c->axes[c->axoff[m] + i] - c->lo[m]) / D - 0.5;
      const int j0 = (int)std::floor(u);
      for (int j = j0; j <= j0 + 1; ++j) {
        const double w = hatf(j - u);
        if (j < 0 || j >= N || w == 0.0) continue;
        if (cnt[j] == kCicTaps) return false;
        gsrc[(size_t)j * kCicTaps + cnt[j]] = i;
        gw[(size_t)j * kCicTaps + cnt[j]] = (float)w;
        ++cnt[j];
      }
    }
  }
  long long a = (*at + 1) & ~1LL;
  const long long need = 2LL * M + M + (lam != 1.0 ? 2LL * N * kCicTaps : 0);
  if (a + need > (long long)host->size()) return false;
  // spectrum of kappa(t), t = -(N-1)..N-1, placed at t mod M
  const double norm = D / std::sqrt(2.0 * M_PI * q);
  std::vector<double> kap(M, 0.0);
  for (int t = -(N - 1); t <= N - 1; ++t) {
    const double x = t * D;
    kap[(t % M + M) % M] = norm * std::exp(-0.5 * x * x / q);
  }
  c->fft_khat[m] = a;
  for (int u = 0; u < M; ++u) {
    double re = 0.0, im = 0.0;
    for (int t = 0; t < M; ++t) {
      if (kap[t] == 0.0) continue;
      const double ph = -2.0 * M_PI * (double)(((long long)u * t) % M) / M;
      re += kap[t] * std::cos(ph);
      im += kap[t] * std::sin(ph);
    }
    (*host)[a + 2 * u] = (float)(re / M);
    (*host)[a + 2 * u + 1] = (float)(im / M);
  }
  a += 2LL * M;
  c->fft_tw[m] = a;
  for (int t = 0; t < M / 2; ++t) {
    const double ph = -2.0 * M_PI * t / M;
    (*host)[a + 2 * t] = (float)std::cos(ph);
    (*host)[a + 2 * t + 1] = (float)std::sin(ph);
  }
  a += M;
  c->fft_gsrc[m] = c->fft_gw[m] = -1;
  if (lam != 1.0) {
    c->fft_gsrc[m] = a;
    std::memcpy(host->data() + a, gsrc.data(), sizeof(int) * gsrc.size());
    a += (long long)gsrc.size();
    c->fft_gw[m] = a;
    std::memcpy(host->data() + a, gw.data(), sizeof(float) * gw.size());
    a += (long long)gw.size();
  }
  c->fft_M[m] = M;
  *at = a;
  return true;
}

int ldu(const double* F, int d, std::vector<double>* Lm, std::vector<double>* D, std::vector<double>* U) {
  Lm->assign((size_t)d * d, 0.0);
  U->assign((size_t)d * d, 0.0);
  D->assign(d, 0.0);
  double scale = 1.0;
  for (int i = 0; i < d * d; ++i) scale = std::max(scale, std::fabs(F[i]));
  for (int k = 0; k < d; ++k) {
    (*Lm)[(size_t)k * d + k] = 1.0;
    (*U)[(size_t)k * d + k] = 1.0;
  }
  for (int k = 0; k < d; ++k) {
    double s = F[(size_t)k * d + k];
    for (int j = 0; j < k; ++j) s -= (*Lm)[(size_t)k * d + j] * (*D)[j] * (*U)[(size_t)j * d + k];
    (*D)[k] = s;
    if (std::fabs(s) <= 1e-12 * scale) return TTGBF_ESINGULAR;
    for (int i = k + 1; i < d; ++i) {
      double sl = F[(size_t)i * d + k], su = F[(size_t)k * d + i];
      for (int j = 0; j < k; ++j) {
        sl -= (*Lm)[(size_t)i * d + j] * (*D)[j] * (*U)[(size_t)j * d + k];
        su -= (*Lm)[(size_t)k * d + j] * (*D)[j] * (*U)[(size_t)j * d + i];
      }
      (*Lm)[(size_t)i * d + k] = sl / s;
      (*U)[(size_t)k * d + i] = su / s;
    }
  }
  return TTGBF_OK;
}

void wait_stage(cudaEvent_t ev, bool* used) {
  if (*used) cudaEventSynchronize(ev);
  *used = false;
}

// Build and upload every operator of a predict call with this F and Q.
int prepare_predict(ttgbf_ctx* c, const double* F, const double* Q) {
  const int d = c->d;
  std::vector<double> Lm, D, U;
  const int rc = ldu(F, d, &Lm, &D, &U);
  if (rc != TTGBF_OK) return rc;
  std::vector<Op> ops;
  for (int m = 0; m < d; ++m)
    for (int n = m + 1; n < d; ++n)
      if (U[(size_t)m * d + n] != 0.0) ops.push_back({0, m, n, U[(size_t)m * d + n]});
  for (int m = 0; m < d; ++m)
    if (D[m] != 1.0) ops.push_back({1, m, m, D[m]});
  bool lower = false;
  for (int m = d - 1; m >= 0; --m)
    for (int n = 0; n < m; ++n)
      if (Lm[(size_t)m * d + n] != 0.0) {
        ops.push_back({0, m, n, Lm[(size_t)m * d + n]});
        lower = true;
      }
  std::vector<float> host((size_t)c->L.opmats_floats, 0.f);
  long long at = 0;
  std::vector<int> S_list, t_list;
  std::vector<long long> woff;
  for (const Op& op : ops) {
    if (op.kind != 0) {
      S_list.push_back(0);
      t_list.push_back(0);
      woff.push_back(-1);
      continue;
    }
    int S, tmin;
    std::vector<float> w;
    shear_table(c, op.m, op.n, op.a, &S, &tmin, &w);
    if (S > c->smax * c->smax) return TTGBF_ECAPACITY;  // more pieces than the sum's rank room
    if (at + (long long)w.size() > c->L.opmats_floats) return TTGBF_ECAPACITY;
    std::copy(w.begin(), w.end(), host.begin() + at);
    S_list.push_back(S);
    t_list.push_back(tmin);
    woff.push_back(at);
    at += (long long)w.size();
  }
  std::vector<long long> moff(d), soff(d, -1);
  for (int m = 0; m < d; ++m) {
    std::vector<double> K, Wc;
    const int N = c->n[m];
    const bool has_scale = D[m] != 1.0;
    c->mode_fft[m] = false;
    if (conv_uses_fft(c, m)) {
      // the kernel by FFT convolution; a scaling that precedes it on this
      // mode (L = I) is its load-time gather, otherwise its own dense pass
      long long at2 = at;
      if (fft_tables(c, m, Q[(size_t)m * d + m], (has_scale && !lower) ? D[m] : 1.0, &host, &at2)) {
        c->mode_fft[m] = true;
        at = at2;
        moff[m] = -1;
        if (has_scale && lower) {
          cic_matrix(c, m, D[m], &Wc);
          soff[m] = at;
          for (size_t t = 0; t < Wc.size(); ++t) host[at + t] = (float)Wc[t];
          at += (long long)Wc.size();
        }
        continue;
      }
    }
    conv_matrix(c, m, Q[(size_t)m * d + m], &K);
    if (has_scale) cic_matrix(c, m, D[m], &Wc);
    if (has_scale && !lower) {
      // fused operator K_m W_m (the scaling precedes the kernel on this mode)
      std::vector<double> M((size_t)N * N, 0.0);
      for (int j = 0; j < N; ++j)
        for (int l = 0; l < N; ++l) {
          const double kjl = K[(size_t)j * N + l];
          if (kjl == 0.0) continue;
          for (int i = 0; i < N; ++i) M[(size_t)j * N + i] += kjl * Wc[(size_t)l * N + i];
        }
      K.swap(M);
    } else if (has_scale) {
      soff[m] = at;
      for (size_t t = 0; t < Wc.size(); ++t) host[at + t] = (float)Wc[t];
      at += (long long)Wc.size();
    }
    moff[m] = at;
    for (size_t t = 0; t < K.size(); ++t) host[at + t] = (float)K[t];
    at += (long long)K.size();
  }
  wait_stage(c->ev_ops, &c->ev_ops_used);
  std::memcpy(c->stage_ops, host.data(), sizeof(float) * at);
  cudaMemcpyAsync(c->opmats, c->stage_ops, sizeof(float) * at, cudaMemcpyHostToDevice, c->st);
  cudaEventRecord(c->ev_ops, c->st);
  c->ev_ops_used = true;
  c->ops = ops;
  c->op_S = S_list;
  c->op_tmin = t_list;
  c->op_woff = woff;
  c->mat_off = moff;
  c->scale_off = soff;
  c->fuse = !lower;
  c->lastF.assign(F, F + (size_t)d * d);
  c->lastQ.assign(Q, Q + (size_t)d * d);
  return TTGBF_OK;
}

void enqueue_shear(ttgbf_ctx* c, int m, int n, int S, int tmin, const float* wts, bool do_round);

// A shear whose operator spans S > smax shifts: the sum over shifts is cut
// into np <= smax pieces of consecutive shifts (at most smax each).  Every
// piece is expanded from a saved copy of the block and rounded on the block;
// the rounded pieces (ranks <= rank_cap each) are added as tensor trains and
// the sum (ranks <= np * rank_cap <= capr) is rounded on the block again.  The
// result differs from the rounding of the whole expansion only by the pieces'
// own truncations, which the discarded tails report.
void enqueue_shear_pieces(ttgbf_ctx* c, int m, int n, int S, int tmin, const float* wts) {
  const int lo = std::min(m, n), hi = std::max(m, n);
  const int np = (S + c->smax - 1) / c->smax;
  const int Nn = c->n[n];
  enqueue_center_into(c, lo, hi);
  tape_shear(c, m, n);
  float* curv[kMaxD];
  float* altv[kMaxD];
  for (int k = 0; k < c->d; ++k) curv[k] = curp(c, k);
  {
    Prof p(c, kPShear, 1);
    launch_block_copy(c->st, c->B, c->geom, lo, hi, curv, c->save, c->ranks);
  }
  cudaMemcpyAsync(c->saved_ranks, c->ranks, sizeof(int) * (size_t)c->B * (c->d + 1),
                  cudaMemcpyDeviceToDevice, c->st);
  int u0 = 0;
  for (int p = 0; p < np; ++p) {
    const int Sp = (int)((long long)S * (p + 1) / np - (long long)S * p / np);
    if (p > 0)
      cudaMemcpyAsync(c->ranks, c->saved_ranks, sizeof(int) * (size_t)c->B * (c->d + 1),
                      cudaMemcpyDeviceToDevice, c->st);
    for (int k = 0; k < c->d; ++k) altv[k] = altp(c, k);
    {
      Prof pr(c, kPShear, 1);
      launch_shear_expand(c->st, c->B, c->geom, m, n, Sp, tmin + u0, wts + (size_t)u0 * Nn, c->save,
                          altv, c->ranks, 0);
    }
    {
      Prof pr(c, kPOther, 1);
      launch_rank_scale(c->st, c->B, c->d, c->ranks, lo, hi, Sp);
    }
    for (int k = lo; k <= hi; ++k) c->cur[k] ^= 1;
    for (int k = hi; k >= lo + 1; --k) stage(c, kStageRight, k, 0);
    for (int k = lo; k <= hi - 1; ++k) stage(c, kStageLeft, k, k == lo);
    for (int k = 0; k < c->d; ++k) curv[k] = curp(c, k);
    {
      Prof pr(c, kPShear, 1);
      launch_acc_piece(c->st, c->B, c->geom, lo, hi, p, c->smax, c->capr, curv, c->acc, c->ranks,
                       c->acc_rank, c->piece_off);
    }
    u0 += Sp;
  }
  for (int k = 0; k < c->d; ++k) altv[k] = altp(c, k);
  {
    Prof pr(c, kPShear, 1);
    launch_acc_sum(c->st, c->B, c->geom, lo, hi, np, c->smax, c->capr, c->acc, altv, c->ranks,
                   c->acc_rank, c->piece_off);
  }
  for (int k = lo; k <= hi; ++k) c->cur[k] ^= 1;
  // cores outside [lo, hi] are still orthonormal: round the sum on the block
  for (int k = hi; k >= lo + 1; --k) stage(c, kStageRight, k, 0);
  for (int k = lo; k <= hi - 1; ++k) stage(c, kStageLeft, k, k == lo);
  c->canon = true;
  c->center = hi;
}

// Shear x_m += a x_n as a rank-S TT operator on the links between lo and hi,
// followed (do_round) by a rounding restricted to that block: the TT is first
// put in canonical form with its center inside [lo, hi], so the cores outside
// the block are orthonormal and the block's truncations are the ones the full
// TT rounding would make on these links.
void enqueue_shear(ttgbf_ctx* c, int m, int n, int S, int tmin, const float* wts, bool do_round) {
  if (do_round && S > c->smax) {
    enqueue_shear_pieces(c, m, n, S, tmin, wts);
    return;
  }
  const int lo = std::min(m, n), hi = std::max(m, n);
  if (do_round) {
    enqueue_center_into(c, lo, hi);
    tape_shear(c, m, n);
  } else {
    tape_fail(c);
  }
  float* curv[kMaxD];
  float* altv[kMaxD];
  for (int k = 0; k < c->d; ++k) {
    curv[k] = curp(c, k);
    altv[k] = altp(c, k);
  }
  // With rounding, the middle cores (G (x) I_S) are never written out: the
  // right-to-left sweep's products with them use their structure.
  const int virt = do_round ? 1 : 0;
  {
    Prof p(c, kPShear, 1);
    launch_shear_expand(c->st, c->B, c->geom, m, n, S, tmin, wts, curv, altv, c->ranks, virt);
  }
  {
    Prof p(c, kPOther, 1);
    launch_rank_scale(c->st, c->B, c->d, c->ranks, lo, hi, S);
  }
  for (int k = lo; k <= hi; ++k) {
    if (virt && k > lo && k < hi) {
      c->virt_S[k] = S;
    } else {
      c->cur[k] ^= 1;
    }
  }
  if (!do_round) {
    c->expanded = true;
    c->canon = false;
    return;
  }
  for (int k = hi; k >= lo + 1; --k) stage(c, kStageRight, k, 0);
  for (int k = lo; k <= hi - 1; ++k) stage(c, kStageLeft, k, k == lo);
  c->canon = true;
  c->center = hi;
}

int guard(ttgbf_ctx* c) {
  if (!c) return TTGBF_EINVAL;
  if (c->poisoned) return TTGBF_EPOISONED;
  return TTGBF_OK;
}

// A component applied by the cross: three or more modes, or a pair other
// than (0, 1).
bool is_block_comp(const ttgbf_meas_comp& cp) {
  return cp.nmodes >= 3 || (cp.nmodes == 2 && !(cp.modes[0] == 0 && cp.modes[1] == 1));
}

// The modes of a component in the order of its table's indices.
std::vector<int> comp_modes(const ttgbf_meas_comp& cp) {
  std::vector<int> m;
  if (cp.nmodes <= 2) {
    for (int t = 0; t < cp.nmodes; ++t) m.push_back(cp.modes[t]);
  } else {
    for (int t = 0; t < cp.nmodes; ++t) m.push_back(cp.modes[0] + t);
  }
  return m;
}

int validate_meas(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, int* two_mode) {
  if (!h || h->b < 1 || h->b > kMaxComps || !h->comp || !R) return TTGBF_EINVAL;
  if (!finite_all(R, (size_t)h->b * h->b)) return TTGBF_ENONFINITE;
  *two_mode = -1;
  for (int i = 0; i < h->b; ++i) {
    for (int j = 0; j < h->b; ++j)
      if (i != j && R[(size_t)i * h->b + j] != 0.0) return TTGBF_EINVAL;
    if (!(R[(size_t)i * h->b + i] > 0.0)) return TTGBF_EINVAL;
    const ttgbf_meas_comp& cp = h->comp[i];
    if (!cp.htab) return TTGBF_EINVAL;
    if (!(cp.period >= 0.0) || !std::isfinite(cp.period)) return TTGBF_EINVAL;
    if (cp.nmodes < 1 || cp.nmodes > c->d) return TTGBF_EINVAL;
    for (int t = 0; t < std::min(cp.nmodes, 2); ++t)
      if (cp.modes[t] < 0 || cp.modes[t] >= c->d) return TTGBF_EINVAL;
    if (cp.nmodes >= 2 && cp.modes[0] == cp.modes[1]) return TTGBF_EINVAL;
    if (cp.nmodes >= 3 && cp.modes[1] != cp.modes[0] + cp.nmodes - 1) return TTGBF_EINVAL;
    if (is_block_comp(cp)) {
      if (c->cross_s <= 0) return TTGBF_EINVAL;
      long long ntab = 1;
      for (const int m : comp_modes(cp)) ntab *= c->n[m];
      if (ntab > 2147483647LL) return TTGBF_EINVAL;
    } else if (cp.nmodes == 2) {
      if (c->n[0] > kMaxN) return TTGBF_ECAPACITY;
      if (*two_mode < 0) *two_mode = i;  // the first (0, 1) component
    }
  }
  return TTGBF_OK;
}

// The update as a sequence of enqueue steps, so that a split batch can issue
// its parts' steps interleaved (all parts start at once and end together).
// Every step captures what it needs by value; host-side state (ranks
// bookkeeping, canonical center) changes in step order.
using EnqueueOps = std::vector<std::function<void()>>;

// One block component as its own Bayes update: canonical form centred in the
// block, the cross of the factor times the block (cross.cu), log c of the
// product added, the block's links rounded, normalisation.
void enqueue_block_update(ttgbf_ctx* c, const ttgbf_meas_comp& cp, int comp, double r, const float* z,
                          int zstride) {
  const int B = c->B, d = c->d;
  const std::vector<int> modes = comp_modes(cp);
  const int lo = *std::min_element(modes.begin(), modes.end());
  const int hi = *std::max_element(modes.begin(), modes.end());
  const int k = hi - lo + 1;
  tape_fail(c);  // not recordable by the adjoint
  enqueue_center_into(c, lo, hi);
  long long ntab = 1;
  for (const int m : modes) ntab *= c->n[m];
  CrossArgs a = c->x;
  a.B = B;
  a.d = d;
  a.lo = lo;
  a.k = k;
  a.s = c->cross_s;
  a.ranks = c->ranks;
  for (int q = 0; q < k; ++q) {
    a.core[q] = curp(c, lo + q);
    a.out[q] = altp(c, lo + q);
    a.cap[q] = c->L.core_cap[lo + q];
    a.N[q] = c->n[lo + q];
    a.stride[q] = 0;
  }
  // table strides: row-major over the component's modes in their order
  long long st = 1;
  for (int t = (int)modes.size() - 1; t >= 0; --t) {
    a.stride[modes[t] - lo] = st;
    st *= c->n[modes[t]];
  }
  a.htab = cp.htab;
  a.z = z;
  a.zstride = zstride;
  a.zc = comp;
  a.R = r;
  a.period = (float)cp.period;
  a.off = c->lik_off;
  cudaMemsetAsync(c->logoff, 0, sizeof(double) * B, c->st);
  {
    Prof p(c, kPLik, 1);
    launch_lik_offset(c->st, B, cp.htab, (int)ntab, z, zstride, comp, r, (float)cp.period, c->lik_off,
                      c->logoff);
  }
  {
    Prof p(c, kPCross, (k - 1) * (2 * c->cross_sweeps + 2) + 1);
    for (int q = k - 1; q >= 1; --q) launch_cross_step(c->st, a, q, kCrossStart);
    for (int sw = 0; sw < c->cross_sweeps; ++sw) {
      for (int q = 0; q <= k - 2; ++q) launch_cross_step(c->st, a, q, kCrossLR);
      for (int q = k - 1; q >= 1; --q) launch_cross_step(c->st, a, q, kCrossRL);
    }
    for (int q = 0; q <= k - 2; ++q) launch_cross_step(c->st, a, q, kCrossFinal);
    launch_cross_last(c->st, a);
  }
  for (int q = lo; q <= hi; ++q) c->cur[q] ^= 1;
  c->canon = false;
  {
    MomentArgs m = tt_moment_args(c, 0, 0);
    Prof p(c, kPMoments, 1);
    launch_moments(c->st, B, m, c->ranks, d + 1, c->awork, c->L.awork_stride, c->mass, nullptr, nullptr);
  }
  {
    Prof p(c, kPOther, 1);
    launch_logc(c->st, B, c->mass, c->logoff, c->log_c, c->log_lik, 1);
  }
  // round the block's links (the cores outside it are still orthonormal)
  for (int q = hi; q >= lo + 1; --q) stage(c, kStageRight, q, 0);
  for (int q = lo; q <= hi - 1; ++q) stage(c, kStageLeft, q, q == lo);
  c->canon = true;
  c->center = hi;
  enqueue_normalise(c, c->mass);
}

void update_ops(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const float* z, int zstride,
                int two_mode, EnqueueOps* ops) {
  const int B = c->B, d = c->d;
  ops->push_back([=] {
    if (c->expanded) enqueue_round(c);
    cudaMemsetAsync(c->logoff, 0, sizeof(double) * B, c->st);
    tape_upd_in(c);
  });
  for (int i = 0; i < h->b; ++i) {
    const ttgbf_meas_comp cp = h->comp[i];
    if (cp.nmodes != 1) continue;
    const int k = cp.modes[0];
    const double r = R[(size_t)i * h->b + i];
    ops->push_back([=] {
      Prof p(c, kPLik, 2);
      launch_lik_offset(c->st, B, cp.htab, c->n[k], z, zstride, i, r, (float)cp.period, c->lik_off,
                        c->logoff);
      launch_lik_apply_1d(c->st, B, curp(c, k), c->L.core_cap[k], c->n[k], k, d, c->ranks, cp.htab,
                          z, zstride, i, r, (float)cp.period, c->lik_off);
      if (!(c->canon && c->center == k)) c->canon = false;
      tape_lik(c, i, cp, z, zstride, r);
    });
  }
  if (two_mode >= 0) {
    // every two-mode component (all on modes (0, 1)) multiplies the merged core
    struct Two {
      int i;
      ttgbf_meas_comp cp;
      double r;
    };
    std::vector<Two> twos;
    for (int i = 0; i < h->b; ++i)
      if (h->comp[i].nmodes == 2 && !is_block_comp(h->comp[i]))
        twos.push_back({i, h->comp[i], R[(size_t)i * h->b + i]});
    for (int k = d - 1; k >= 2; --k) ops->push_back([=] { stage(c, kStageRight, k, 0); });
    ops->push_back([=] {
      GemmWork gw = gemm_work(c, B);
      {
        Prof p(c, kPPlan, 2);
        launch_plan_supercore(c->st, B, c->geom, c->ranks, curp(c, 0), curp(c, 1), c->W, c->L.W_cap, gw);
      }
      {
        Prof p(c, kPGemm, 1);
        launch_gemm(c->st, gw, c->sms * 8, flops_of(c, kPGemm));
      }
      for (const Two& t : twos) {
        {
          Prof p(c, kPLik, 2);
          launch_lik_offset(c->st, B, t.cp.htab, c->n[0] * c->n[1], z, zstride, t.i, t.r,
                            (float)t.cp.period, c->lik_off, c->logoff);
          launch_lik_apply_2d(c->st, B, c->W, c->L.W_cap, c->n[0], c->n[1], c->ranks, d, t.cp.htab, z,
                              zstride, t.i, t.r, (float)t.cp.period, c->lik_off);
        }
        tape_lik(c, t.i, t.cp, z, zstride, t.r);
      }
      // log c before rounding: mass of the TT [W (modes 0,1 merged), core 2, ...]
      MomentArgs a{};
      a.ncores = d - 1;
      a.n[0] = c->n[0] * c->n[1];
      a.core[0] = c->W;
      a.cap[0] = c->L.W_cap;
      a.ridx[0] = 0;
      for (int k = 2; k < d; ++k) {
        a.n[k - 1] = c->n[k];
        a.core[k - 1] = curp(c, k);
        a.cap[k - 1] = c->L.core_cap[k];
      }
      for (int kk = 1; kk <= d - 1; ++kk) a.ridx[kk] = kk + 1;
      a.delta = c->delta;
      {
        Prof p(c, kPMoments, 1);
        launch_moments(c->st, B, a, c->ranks, d + 1, c->awork, c->L.awork_stride, c->mass, nullptr, nullptr);
      }
      {
        Prof p(c, kPOther, 1);
        launch_logc(c->st, B, c->mass, c->logoff, c->log_c, c->log_lik, 0);
      }
      tape_logc(c, c->mass);
    });
    ops->push_back([=] { stage(c, kStageSplit, 0, 1); });
    for (int k = 1; k <= d - 2; ++k) ops->push_back([=] { stage(c, kStageLeft, k, 0); });
    ops->push_back([=] {
      c->canon = true;
      c->center = d - 1;
    });
  } else {
    ops->push_back([=] {
      MomentArgs a = tt_moment_args(c, 0, 0);
      {
        Prof p(c, kPMoments, 1);
        launch_moments(c->st, B, a, c->ranks, d + 1, c->awork, c->L.awork_stride, c->mass, nullptr,
                       nullptr);
      }
      {
        Prof p(c, kPOther, 1);
        launch_logc(c->st, B, c->mass, c->logoff, c->log_c, c->log_lik, 0);
      }
      tape_logc(c, c->mass);
    });
  }
  ops->push_back([=] { enqueue_normalise(c, c->mass); });
  for (int i = 0; i < h->b; ++i) {
    const ttgbf_meas_comp cp = h->comp[i];
    if (!is_block_comp(cp)) continue;
    const double r = R[(size_t)i * h->b + i];
    ops->push_back([=] { enqueue_block_update(c, cp, i, r, z, zstride); });
  }
}

int enqueue_update(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const float* z, int zstride,
                   int two_mode) {
  EnqueueOps ops;
  update_ops(c, h, R, z, zstride, two_mode, &ops);
  for (auto& op : ops) op();
  return check(c);
}

}  // namespace

// =================================================================== C ABI
extern "C" {

const char* ttgbf_strerror(int code) {
  switch (code) {
    case TTGBF_OK: return "ok";
    case TTGBF_EINVAL: return "invalid argument";
    case TTGBF_ENONFINITE: return "non-finite input";
    case TTGBF_ENOMEM: return "out of device memory or workspace too small";
    case TTGBF_ECUDA: return "CUDA error (context poisoned)";
    case TTGBF_ECAPACITY: return "rank expansion beyond capacity (rank_cap * max_shift_span > 160, or a shear wider than max_shift_span^2 shifts)";
    case TTGBF_ESINGULAR: return "F has no LDU factorisation without pivoting";
    case TTGBF_EPOISONED: return "context poisoned by an earlier CUDA error";
    default: return "unknown error";
  }
}

// Number of parts of a batch: opts.parts when set, else one per 12 filters,
// at most 8 (environment TTGBF_PARTS overrides the default, 1..8).
// Measured on 100 filters of the 128^4
// workload: 1 part 32.8 ms per step, 2 parts 30.9, 4 parts 28.2, 8 parts
// 27.4.
static int choose_parts(const ttgbf_opts* opts) {
  int np = std::min(8, std::max(1, (int)opts->batch / 12));
  if (const char* e = std::getenv("TTGBF_PARTS")) {
    const int v = std::atoi(e);
    if (v >= 1 && v <= 8) np = v;
  }
  if (opts->parts > 0) np = opts->parts;
  return std::max(1, std::min(np, (int)opts->batch));
}

size_t ttgbf_workspace_bytes(const ttgbf_grid* grid, const ttgbf_opts* opts) {
  if (validate_grid(grid) != TTGBF_OK || validate_opts(opts) != TTGBF_OK) return 0;
  const int np = choose_parts(opts);
  if (np == 1) return make_layout(grid, opts).total;
  // the parts' arenas back to back, each starting on a 256-byte boundary
  size_t total = 0;
  for (int p = 0; p < np; ++p) {
    ttgbf_opts po = *opts;
    po.batch = (int)((long long)opts->batch * (p + 1) / np - (long long)opts->batch * p / np);
    total += (make_layout(grid, &po).total + 255) & ~(size_t)255;
  }
  return total;
}

static int init_single(ttgbf_ctx** out, const ttgbf_grid* grid, const ttgbf_prior* prior,
                       const ttgbf_opts* opts) {
  if (!out) return TTGBF_EINVAL;
  int rc = validate_grid(grid);
  if (rc != TTGBF_OK) return rc;
  rc = validate_opts(opts);
  if (rc != TTGBF_OK) return rc;
  if (!prior || !prior->mean || !prior->var) return TTGBF_EINVAL;
  const int d = grid->d;
  if (!finite_all(prior->mean, d) || !finite_all(prior->var, d)) return TTGBF_ENONFINITE;
  for (int k = 0; k < d; ++k)
    if (!(prior->var[k] > 0.0)) return TTGBF_EINVAL;
  // kernel attributes (large dynamic shared memory), once per process even
  // when several threads create contexts at the same time
  static std::once_flag attrs;
  std::call_once(attrs, [] {
    set_kernel_attributes();
    set_ttops_attributes();
    set_tsqr_attributes();
    set_rsvd64_attributes();
    set_fft_attributes();
    set_adjoint_attributes();
  });
  ttgbf_ctx* c = new (std::nothrow) ttgbf_ctx();
  if (!c) return TTGBF_ENOMEM;
  c->B = opts->batch;
  c->d = d;
  c->rank_cap = opts->rank_cap;
  c->smax = opts->max_shift_span > 0 ? opts->max_shift_span : 10;
  c->capr = c->rank_cap * c->smax;
  c->precision = opts->precision;
  c->contract = opts->contraction;
  c->conv_mode = opts->conv;
  c->slice_blocks = opts->tsqr_slice_blocks > 0 ? opts->tsqr_slice_blocks : kTsqrSliceBlocks;
  c->svd_threads = opts->svd_threads > 0 ? opts->svd_threads : 512;
  c->eps = opts->eps;
  c->cross_s = opts->cross_rank;
  c->cross_sweeps = opts->cross_sweeps > 0 ? opts->cross_sweeps : 1;
  c->st = (cudaStream_t)opts->stream;
  {
    const char* dbg = std::getenv("TTGBF_DEBUG_STAGES");
    c->debug_stages = dbg != nullptr && dbg[0] == '1';
  }
  // TTGBF_FAULT=alloc: the device allocation "fails" (after validation)
  const char* fault = std::getenv("TTGBF_FAULT");
  if (fault != nullptr && std::strcmp(fault, "alloc") == 0) {
    delete c;
    return TTGBF_ENOMEM;
  }
  c->n.assign(grid->n, grid->n + d);
  c->lo.assign(grid->lo, grid->lo + d);
  c->hi.assign(grid->hi, grid->hi + d);
  c->dx.resize(d);
  c->axoff.resize(d);
  int off = 0;
  for (int k = 0; k < d; ++k) {
    c->dx[k] = (c->hi[k] - c->lo[k]) / c->n[k];
    c->delta *= c->dx[k];
    c->axoff[k] = off;
    for (int i = 0; i < c->n[k]; ++i) c->axes.push_back(c->lo[k] + (i + 0.5) * c->dx[k]);
    off += c->n[k];
  }
  c->L = make_layout(grid, opts);
  if (opts->workspace) {
    if (opts->workspace_bytes < c->L.total || ((uintptr_t)opts->workspace & 255)) {
      delete c;
      return TTGBF_ENOMEM;
    }
    c->base = (char*)opts->workspace;
  } else {
    if (cudaMalloc(&c->base, c->L.total) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return TTGBF_ENOMEM;
    }
    c->owns = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  const Layout& L = c->L;
  char* b = c->base;
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < d; ++k) c->buf[s][k] = (float*)(b + L.core[s][k]);
  for (int k = 0; k < d; ++k) {
    c->save[k] = (float*)(b + L.piece_core[0][k]);
    c->acc[k] = (float*)(b + L.piece_core[1][k]);
  }
  c->saved_ranks = (int*)(b + L.saved_ranks);
  c->acc_rank = (int*)(b + L.acc_rank);
  c->piece_off = (int*)(b + L.piece_off);
  c->geom.d = d;
  for (int k = 0; k < d; ++k) {
    c->geom.n[k] = c->n[k];
    c->geom.cap[k] = L.core_cap[k];
  }
  c->ranks = (int*)(b + L.ranks);
  c->axes_d = (double*)(b + L.axes);
  c->pmean = (double*)(b + L.pmean);
  c->pvar = (double*)(b + L.pvar);
  c->normA = (double*)(b + L.normA);
  c->tail_sum = (double*)(b + L.tail_sum);
  c->tail_max = (double*)(b + L.tail_max);
  c->mass = (double*)(b + L.mass);
  c->mass_pred = (double*)(b + L.mass_pred);
  c->log_c = (double*)(b + L.log_c);
  c->log_lik = (double*)(b + L.log_lik);
  c->logoff = (double*)(b + L.logoff);
  c->mean = (double*)(b + L.mean);
  c->cov = (double*)(b + L.cov);
  c->cap_hits = (int*)(b + L.cap_hits);
  c->newrank = (int*)(b + L.newrank);
  c->lik_off = (float*)(b + L.lik_off);
  c->tw.prob = (TsqrProblem*)(b + L.tsqr_prob);
  c->tw.offset = (int*)(b + L.tsqr_off);
  c->tw.counter = (int*)(b + L.tsqr_cnt);
  c->stack[0] = (float*)(b + L.stack[0]);
  c->stack[1] = (float*)(b + L.stack[1]);
  c->P1 = (float*)(b + L.P1);
  c->P2 = (float*)(b + L.P2);
  c->gdesc = (GemmDesc*)(b + L.gdesc);
  c->gtiles = (int*)(b + L.gtiles);
  c->tc_status = c->gtiles + L.gdesc_cap + 1;
  c->awork = (double*)(b + L.awork);
  c->W = (float*)(b + L.W);
  c->opmats = (float*)(b + L.opmats);
  c->zbuf = (float*)(b + L.zbuf);
  c->prof_flops = (double*)(b + L.prof_flops);
  c->fft_off = (int*)(b + L.fft_off);
  if (c->cross_s > 0) {
    c->x.F = (float*)(b + L.xF);
    c->x.Qb = (float*)(b + L.xQ);
    c->x.rn = (float*)(b + L.xrn);
    c->x.mask = (unsigned*)(b + L.xmask);
    c->x.offI = (long long*)(b + L.xoffI);
    c->x.offJ = (long long*)(b + L.xoffJ);
    c->x.U = (float*)(b + L.xU);
    c->x.V = (float*)(b + L.xV);
    c->x.sz = (int*)(b + L.xsz);
    c->x.status = (int*)(b + L.xstatus);
    c->x.fcap = L.x_fcap;
    c->x.mcap = L.x_mcap;
  }
  if (cudaMallocHost(&c->stage_ops, sizeof(float) * L.opmats_floats) != cudaSuccess ||
      cudaMallocHost(&c->stage_z, sizeof(float) * (size_t)c->B * kMaxComps) != cudaSuccess ||
      cudaMallocHost(&c->stage_est, sizeof(double) * (size_t)c->B * (d + d * d + 2)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_ops, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_z, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ttgbf_free(c);
    return TTGBF_ENOMEM;
  }
  // constants and the prior
  cudaMemcpyAsync(c->axes_d, c->axes.data(), sizeof(double) * c->axes.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->pmean, prior->mean, sizeof(double) * d, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->pvar, prior->var, sizeof(double) * d, cudaMemcpyHostToDevice, c->st);
  cudaMemsetAsync(c->log_lik, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->log_c, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->tail_sum, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->tail_max, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->cap_hits, 0, sizeof(int) * c->B, c->st);
  cudaMemsetAsync(c->mass_pred, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->prof_flops, 0, sizeof(double) * kPClasses, c->st);
  cudaMemsetAsync(c->tc_status, 0, sizeof(int), c->st);
  launch_prior(c->st, c->B, c->geom, c->buf[0], c->ranks, c->axes_d, c->pmean, c->pvar);
  enqueue_normalise(c, c->mass);
  // synchronous: prior values come from host memory the caller may free
  if (cudaStreamSynchronize(c->st) != cudaSuccess || check(c) != TTGBF_OK) {
    cudaGetLastError();
    ttgbf_free(c);
    return TTGBF_ECUDA;
  }
  *out = c;
  if (fault != nullptr && std::strncmp(fault, "cuda:", 5) == 0)
    c->fault_after = std::max(0L, std::strtol(fault + 5, nullptr, 10));
  return TTGBF_OK;
}

int ttgbf_free(ttgbf_ctx* c);

int ttgbf_init(ttgbf_ctx** out, const ttgbf_grid* grid, const ttgbf_prior* prior, const ttgbf_opts* opts) {
  if (!out) return TTGBF_EINVAL;
  int rc = validate_grid(grid);
  if (rc != TTGBF_OK) return rc;
  rc = validate_opts(opts);
  if (rc != TTGBF_OK) return rc;
  const int np = choose_parts(opts);
  if (np == 1) return init_single(out, grid, prior, opts);
  ttgbf_ctx* c = new (std::nothrow) ttgbf_ctx();
  if (!c) return TTGBF_ENOMEM;
  c->B = opts->batch;
  c->d = grid->d;
  c->st = (cudaStream_t)opts->stream;
  if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TTGBF_ENOMEM;
  }
  for (int p = 0; p <= np; ++p) c->part_base.push_back((int)((long long)c->B * p / np));
  size_t ws_off = 0;
  for (int p = 0; p < np; ++p) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ttgbf_ctx* part = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (st) cudaStreamDestroy(st);
      ttgbf_free(c);
      return TTGBF_ENOMEM;
    }
    c->part_st.push_back(st);
    c->ev_join.push_back(ev);
    ttgbf_opts po = *opts;
    po.batch = c->part_base[p + 1] - c->part_base[p];
    po.stream = st;
    if (opts->workspace) {
      // a caller workspace holds the parts' arenas back to back (the layout
      // ttgbf_workspace_bytes sized)
      const size_t need = (make_layout(grid, &po).total + 255) & ~(size_t)255;
      if (ws_off + need > opts->workspace_bytes) {
        ttgbf_free(c);
        return TTGBF_ENOMEM;
      }
      po.workspace = (char*)opts->workspace + ws_off;
      po.workspace_bytes = need;
      ws_off += need;
    }
    rc = init_single(&part, grid, prior, &po);
    if (rc != TTGBF_OK) {
      ttgbf_free(c);
      return rc;
    }
    part->slot_share = 1.0;
    c->parts.push_back(part);
  }
  *out = c;
  return TTGBF_OK;
}

}  // extern "C"

namespace {

bool split(const ttgbf_ctx* c) { return c != nullptr && !c->parts.empty(); }

// The parts start after the work already on the caller's stream ...
void fork_parts(ttgbf_ctx* c) {
  cudaEventRecord(c->ev_fork, c->st);
  for (cudaStream_t st : c->part_st) cudaStreamWaitEvent(st, c->ev_fork, 0);
}

// ... and the caller's stream continues after all of them.
void join_parts(ttgbf_ctx* c) {
  for (size_t p = 0; p < c->parts.size(); ++p) {
    cudaEventRecord(c->ev_join[p], c->part_st[p]);
    cudaStreamWaitEvent(c->st, c->ev_join[p], 0);
  }
}

// Apply fn(part, p) to every part; stops at the first error (identical
// arguments fail alike on every part, before any launch).  A call that reads
// caller device memory first makes the parts wait for the caller's stream
// (fork); a call that reads or writes caller device memory makes the
// caller's stream wait for the parts at its end (join).  Calls on the
// filters' own state only (predict, shear, scale, convolve, round,
// normalise) do neither, so the parts drift apart and different parts' QR,
// SVD and GEMM phases overlap; the next joining call (or free) waits for
// them.
// A poisoned part poisons the whole batch: only ttgbf_free is valid then.
int parts_guard(const ttgbf_ctx* c) {
  for (const ttgbf_ctx* q : c->parts)
    if (q->poisoned) return TTGBF_EPOISONED;
  return TTGBF_OK;
}

template <typename Fn>
int fan_out(ttgbf_ctx* c, Fn fn, bool join = true, bool fork = true) {
  if (const int rc = parts_guard(c)) return rc;
  if (fork) fork_parts(c);
  int rc = TTGBF_OK;
  for (size_t p = 0; p < c->parts.size() && rc == TTGBF_OK; ++p) rc = fn(c->parts[p], (int)p);
  if (join) join_parts(c);
  return rc;
}

// The part holding filter f and the index of f within it.
int part_of(const ttgbf_ctx* c, int f, int* local) {
  int p = 0;
  while (p + 1 < (int)c->parts.size() && c->part_base[p + 1] <= f) ++p;
  *local = f - c->part_base[p];
  return p;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// The predict step in three parts (validation and setup; elementary
// operation i of the re-gridding; per-mode kernels and normalisation), so
// that a split batch can enqueue its parts operation by operation.
int predict_begin(ttgbf_ctx* c, const double* F, const double* Q) {
  int rc = guard(c);
  if (rc) return rc;
  if (!F || !Q) return TTGBF_EINVAL;
  const int d = c->d;
  if (!finite_all(F, (size_t)d * d) || !finite_all(Q, (size_t)d * d)) return TTGBF_ENONFINITE;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      if (i != j && Q[(size_t)i * d + j] != 0.0) return TTGBF_EINVAL;
      if (i == j && !(Q[(size_t)i * d + j] > 0.0)) return TTGBF_EINVAL;
    }
  const bool same = c->lastF.size() == (size_t)d * d &&
                    std::equal(c->lastF.begin(), c->lastF.end(), F) &&
                    std::equal(c->lastQ.begin(), c->lastQ.end(), Q);
  if (!same) {
    rc = prepare_predict(c, F, Q);
    if (rc) return rc;
  }
  if (c->expanded) enqueue_round(c);
  cudaMemsetAsync(c->tail_sum, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->tail_max, 0, sizeof(double) * c->B, c->st);
  cudaMemsetAsync(c->cap_hits, 0, sizeof(int) * c->B, c->st);
  return TTGBF_OK;
}

void predict_op(ttgbf_ctx* c, size_t i) {
  const Op& op = c->ops[i];
  if (op.kind == 0) {
    c->tape_op = (int)i;
    enqueue_shear(c, op.m, op.n, c->op_S[i], c->op_tmin[i], c->opmats + c->op_woff[i], true);
    c->tape_op = -1;
  } else if (!c->fuse) {
    tape_mode(c, op.m, kModeScale);
    mode_apply(c, op.m, c->opmats + c->scale_off[op.m]);
  }
}

void predict_mode(ttgbf_ctx* c, int k) {
  bool scaled = false;
  for (const Op& op : c->ops) scaled = scaled || (op.kind == 1 && op.m == k);
  tape_mode(c, k, (c->fuse && scaled) ? kModeConvScale : kModeConv);
  if (c->mode_fft[k]) mode_conv_fft(c, k);
  else mode_apply(c, k, c->opmats + c->mat_off[k]);
}

int predict_end(ttgbf_ctx* c) {
  enqueue_normalise(c, c->mass_pred);
  return check(c);
}

}  // namespace

extern "C" {

int ttgbf_predict(ttgbf_ctx* c, const double* F, const double* Q) {
  ApiRange range("ttgbf_predict");
  if (split(c)) {
    if (const int rc = parts_guard(c)) return rc;
    // every part validates the same arguments: a failure can only come
    // from the first part, before anything is enqueued
    for (ttgbf_ctx* q : c->parts) {
      const int rc = predict_begin(q, F, Q);
      if (rc) return rc;
    }
    const size_t nops = c->parts[0]->ops.size();
    for (size_t i = 0; i < nops; ++i)
      for (ttgbf_ctx* q : c->parts) predict_op(q, i);
    for (int k = 0; k < c->d; ++k)
      for (ttgbf_ctx* q : c->parts) predict_mode(q, k);
    int rc = TTGBF_OK;
    for (ttgbf_ctx* q : c->parts) {
      const int r = predict_end(q);
      if (r && !rc) rc = r;
    }
    return rc;
  }
  const int rc = predict_begin(c, F, Q);
  if (rc) return rc;
  for (size_t i = 0; i < c->ops.size(); ++i) predict_op(c, i);
  for (int k = 0; k < c->d; ++k) predict_mode(c, k);
  return predict_end(c);
}

// Host-side checks and the measurement's device copy for one (part) context;
// *zq receives the device measurement pointer and *two the two-mode
// component (-1 if none).
static int update_prepare(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const double* z_host,
                          const float* z_dev, const float** zq, int* two) {
  int rc = guard(c);
  if (rc) return rc;
  *two = -1;
  rc = validate_meas(c, h, R, two);
  if (rc) return rc;
  if (z_dev) {
    *zq = z_dev;
    return TTGBF_OK;
  }
  if (!z_host) return TTGBF_EINVAL;
  if (!finite_all(z_host, (size_t)c->B * h->b)) return TTGBF_ENONFINITE;
  wait_stage(c->ev_z, &c->ev_z_used);
  for (size_t i = 0; i < (size_t)c->B * h->b; ++i) c->stage_z[i] = (float)z_host[i];
  cudaMemcpyAsync(c->zbuf, c->stage_z, sizeof(float) * (size_t)c->B * h->b, cudaMemcpyHostToDevice,
                  c->st);
  cudaEventRecord(c->ev_z, c->st);
  c->ev_z_used = true;
  *zq = c->zbuf;
  return TTGBF_OK;
}

// A split batch: every part prepares (identical arguments fail alike on
// every part, so only the first can fail, before any launch), then the
// parts' enqueue steps are issued interleaved between a fork and a join.
static int update_split(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const double* z_host,
                        const float* z_dev) {
  if (const int rc = parts_guard(c)) return rc;
  if (!h || (!z_host && !z_dev)) return TTGBF_EINVAL;
  const size_t np = c->parts.size();
  std::vector<EnqueueOps> lists(np);
  fork_parts(c);
  int rc = TTGBF_OK;
  for (size_t p = 0; p < np && rc == TTGBF_OK; ++p) {
    ttgbf_ctx* q = c->parts[p];
    const size_t off = (size_t)c->part_base[p] * (size_t)(h->b);
    const float* zq = nullptr;
    int two = -1;
    rc = update_prepare(q, h, R, z_host ? z_host + off : nullptr, z_dev ? z_dev + off : nullptr, &zq,
                        &two);
    if (rc == TTGBF_OK) update_ops(q, h, R, zq, h->b, two, &lists[p]);
  }
  if (rc == TTGBF_OK) {
    size_t nmax = 0;
    for (const EnqueueOps& l : lists) nmax = std::max(nmax, l.size());
    for (size_t i = 0; i < nmax; ++i)
      for (const EnqueueOps& l : lists)
        if (i < l.size()) l[i]();
    for (ttgbf_ctx* q : c->parts) {
      const int r = check(q);
      if (r && !rc) rc = r;
    }
  }
  join_parts(c);
  return rc;
}

int ttgbf_update(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const double* z) {
  ApiRange range("ttgbf_update");
  if (split(c)) return update_split(c, h, R, z, nullptr);
  const float* zq = nullptr;
  int two = -1;
  const int rc = update_prepare(c, h, R, z, nullptr, &zq, &two);
  if (rc) return rc;
  return enqueue_update(c, h, R, zq, h->b, two);
}

int ttgbf_update_dev(ttgbf_ctx* c, const ttgbf_meas* h, const double* R, const float* z_dev) {
  ApiRange range("ttgbf_update");
  if (split(c)) {
    if (!z_dev) return TTGBF_EINVAL;
    return update_split(c, h, R, nullptr, z_dev);
  }
  const float* zq = nullptr;
  int two = -1;
  const int rc = update_prepare(c, h, R, nullptr, z_dev, &zq, &two);
  if (rc) return rc;
  return enqueue_update(c, h, R, zq, h->b, two);
}

static int estimate_common(ttgbf_ctx* c) {
  MomentArgs a = tt_moment_args(c, 1, 0);
  Prof p(c, kPMoments, 1);
  launch_moments(c->st, c->B, a, c->ranks, c->d + 1, c->awork, c->L.awork_stride, c->mass, c->mean,
                 c->cov);
  return check(c);
}

// Moments of every filter, copied to the pinned staging area (no wait).
static int estimate_to_stage(ttgbf_ctx* c) {
  int rc = guard(c);
  if (rc) return rc;
  rc = estimate_common(c);
  if (rc) return rc;
  const size_t B = (size_t)c->B, d = (size_t)c->d;
  double* h = c->stage_est;
  cudaMemcpyAsync(h, c->mean, sizeof(double) * B * d, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(h + B * d, c->cov, sizeof(double) * B * d * d, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(h + B * (d + d * d), c->log_c, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(h + B * (d + d * d + 1), c->log_lik, sizeof(double) * B, cudaMemcpyDeviceToHost,
                  c->st);
  return check(c);
}

// Staged moments of filters [b0, b0 + B) to the caller's host arrays.
static void estimate_from_stage(const ttgbf_ctx* c, size_t b0, double* mean, double* cov,
                                double* log_c, double* log_lik) {
  const size_t B = (size_t)c->B, d = (size_t)c->d;
  const double* h = c->stage_est;
  if (mean) std::memcpy(mean + b0 * d, h, sizeof(double) * B * d);
  if (cov) std::memcpy(cov + b0 * d * d, h + B * d, sizeof(double) * B * d * d);
  if (log_c) std::memcpy(log_c + b0, h + B * (d + d * d), sizeof(double) * B);
  if (log_lik) std::memcpy(log_lik + b0, h + B * (d + d * d + 1), sizeof(double) * B);
}

int ttgbf_estimate(ttgbf_ctx* c, double* mean, double* cov, double* log_c, double* log_lik) {
  ApiRange range("ttgbf_estimate");
  if (split(c)) {
    // every part enqueues its moments and read-back before anything waits,
    // so the parts finish concurrently; the caller's stream joins them
    const int rc = fan_out(c, [&](ttgbf_ctx* q, int) { return estimate_to_stage(q); });
    if (rc) return rc;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
    for (size_t p = 0; p < c->parts.size(); ++p)
      estimate_from_stage(c->parts[p], (size_t)c->part_base[p], mean, cov, log_c, log_lik);
    return check(c);
  }
  const int rc = estimate_to_stage(c);
  if (rc) return rc;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  estimate_from_stage(c, 0, mean, cov, log_c, log_lik);
  return check(c);
}

int ttgbf_estimate_dev(ttgbf_ctx* c, double* mean, double* cov, double* log_c, double* log_lik) {
  ApiRange range("ttgbf_estimate");
  if (split(c)) {
    const int d = c->d;
    return fan_out(c, [&](ttgbf_ctx* q, int p) {
      const size_t b0 = (size_t)c->part_base[p];
      return ttgbf_estimate_dev(q, mean ? mean + b0 * d : nullptr, cov ? cov + b0 * d * d : nullptr,
                                log_c ? log_c + b0 : nullptr, log_lik ? log_lik + b0 : nullptr);
    }, true, false);
  }
  int rc = guard(c);
  if (rc) return rc;
  rc = estimate_common(c);
  if (rc) return rc;
  const int B = c->B, d = c->d;
  if (mean) cudaMemcpyAsync(mean, c->mean, sizeof(double) * B * d, cudaMemcpyDeviceToDevice, c->st);
  if (cov) cudaMemcpyAsync(cov, c->cov, sizeof(double) * B * d * d, cudaMemcpyDeviceToDevice, c->st);
  if (log_c) cudaMemcpyAsync(log_c, c->log_c, sizeof(double) * B, cudaMemcpyDeviceToDevice, c->st);
  if (log_lik) cudaMemcpyAsync(log_lik, c->log_lik, sizeof(double) * B, cudaMemcpyDeviceToDevice, c->st);
  return check(c);
}

int ttgbf_free(ttgbf_ctx* c) {
  if (!c) return TTGBF_OK;
  if (!c->part_st.empty() || c->ev_fork) {
    for (ttgbf_ctx* q : c->parts) ttgbf_free(q);
    for (cudaStream_t st : c->part_st) cudaStreamDestroy(st);
    for (cudaEvent_t e : c->ev_join) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    cudaGetLastError();
    delete c;
    return TTGBF_OK;
  }
  if (c->st || c->base) cudaStreamSynchronize(c->st);
  if (c->owns && c->base) cudaFree(c->base);
  if (c->stage_ops) cudaFreeHost(c->stage_ops);
  if (c->stage_z) cudaFreeHost(c->stage_z);
  if (c->stage_est) cudaFreeHost(c->stage_est);
  if (c->ev_ops) cudaEventDestroy(c->ev_ops);
  if (c->ev_z) cudaEventDestroy(c->ev_z);
  for (int k = 0; k < kPClasses; ++k)
    for (cudaEvent_t e : c->ev_pool[k]) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
  return TTGBF_OK;
}

int ttgbf_ranks(ttgbf_ctx* c, int32_t* ranks) {
  if (split(c)) {
    if (!ranks) return TTGBF_EINVAL;
    return fan_out(c, [&](ttgbf_ctx* q, int p) {
      return ttgbf_ranks(q, ranks + (size_t)c->part_base[p] * (c->d + 1));
    });
  }
  int rc = guard(c);
  if (rc) return rc;
  if (!ranks) return TTGBF_EINVAL;
  cudaMemcpyAsync(ranks, c->ranks, sizeof(int) * (size_t)c->B * (c->d + 1), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  return check(c);
}

int ttgbf_stats(ttgbf_ctx* c, ttgbf_step_stats* out) {
  if (split(c)) {
    if (!out) return TTGBF_EINVAL;
    return fan_out(c, [&](ttgbf_ctx* q, int p) { return ttgbf_stats(q, out + c->part_base[p]); });
  }
  int rc = guard(c);
  if (rc) return rc;
  if (!out) return TTGBF_EINVAL;
  const int B = c->B, d = c->d;
  std::vector<double> ts(B), tm(B), mp(B), lc(B), ll(B);
  std::vector<int> ch(B), rk((size_t)B * (d + 1));
  int tcs = 0;
  cudaMemcpyAsync(&tcs, c->tc_status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(ts.data(), c->tail_sum, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(tm.data(), c->tail_max, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(mp.data(), c->mass_pred, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(lc.data(), c->log_c, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(ll.data(), c->log_lik, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(ch.data(), c->cap_hits, sizeof(int) * B, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(rk.data(), c->ranks, sizeof(int) * rk.size(), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  for (int b = 0; b < B; ++b) {
    int mr = 0;
    for (int k = 0; k <= d; ++k) mr = std::max(mr, rk[(size_t)b * (d + 1) + k]);
    out[b] = ttgbf_step_stats{ts[b], tm[b], mp[b], lc[b], ll[b], mr, ch[b]};
  }
  if (tcs != 0) return cuda_fail(c);  // a tensor-core product was given up (written as NaN)
  return check(c);
}

int ttgbf_grid_axes(const ttgbf_ctx* c, double* axes) {
  if (split(c)) return ttgbf_grid_axes(c->parts[0], axes);
  if (!c || !axes) return TTGBF_EINVAL;
  std::copy(c->axes.begin(), c->axes.end(), axes);
  return TTGBF_OK;
}

int ttgbf_export_cores(ttgbf_ctx* c, int32_t f, float* buf, size_t cap, int32_t* ranks_out) {
  if (split(c)) {
    if (f < 0 || f >= c->B) return TTGBF_EINVAL;
    int local = 0;
    const int p = part_of(c, f, &local);
    return fan_out(c, [&](ttgbf_ctx* q, int pp) {
      return pp == p ? ttgbf_export_cores(q, local, buf, cap, ranks_out) : TTGBF_OK;
    });
  }
  int rc = guard(c);
  if (rc) return rc;
  if (!buf || !ranks_out || f < 0 || f >= c->B) return TTGBF_EINVAL;
  const int d = c->d;
  cudaMemcpyAsync(ranks_out, c->ranks + (size_t)f * (d + 1), sizeof(int) * (d + 1), cudaMemcpyDeviceToHost,
                  c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  size_t need = 0;
  for (int k = 0; k < d; ++k) need += (size_t)ranks_out[k] * c->n[k] * ranks_out[k + 1];
  if (need > cap) return TTGBF_ENOMEM;
  size_t at = 0;
  for (int k = 0; k < d; ++k) {
    const size_t cnt = (size_t)ranks_out[k] * c->n[k] * ranks_out[k + 1];
    cudaMemcpyAsync(buf + at, curp(c, k) + (size_t)f * c->L.core_cap[k], sizeof(float) * cnt,
                    cudaMemcpyDeviceToHost, c->st);
    at += cnt;
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  return check(c);
}

int ttgbf_densify(ttgbf_ctx* c, int32_t f, double* out, size_t cap) {
  if (split(c)) {
    if (f < 0 || f >= c->B) return TTGBF_EINVAL;
    int local = 0;
    const int p = part_of(c, f, &local);
    return fan_out(c, [&](ttgbf_ctx* q, int pp) { return pp == p ? ttgbf_densify(q, local, out, cap) : TTGBF_OK; });
  }
  int rc = guard(c);
  if (rc) return rc;
  if (!out || f < 0 || f >= c->B) return TTGBF_EINVAL;
  const int d = c->d;
  std::vector<int32_t> r(d + 1);
  cudaMemcpyAsync(r.data(), c->ranks + (size_t)f * (d + 1), sizeof(int) * (d + 1), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  // Sizes of the stages' results n_0 ... n_k r_{k+1}; the last is the tensor.
  const long long kMaxElems = 1LL << 32;
  long long P = 1, most = 1;
  for (int k = 0; k < d; ++k) {
    P *= c->n[k];
    if (P > kMaxElems) return TTGBF_ENOMEM;
    most = std::max(most, P * r[k + 1]);
    if (most > kMaxElems) return TTGBF_ENOMEM;
  }
  if ((size_t)P > cap) return TTGBF_ENOMEM;
  double* buf[2] = {nullptr, nullptr};
  if (cudaMalloc(&buf[0], sizeof(double) * most) != cudaSuccess ||
      cudaMalloc(&buf[1], sizeof(double) * most) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf[0]);
    return TTGBF_ENOMEM;
  }
  long long rows = 1;
  for (int k = 0; k < d; ++k) {
    launch_densify_stage(c->st, k ? buf[(k + 1) & 1] : nullptr, rows, r[k], curp(c, k) + (size_t)f * c->L.core_cap[k],
                         c->n[k], r[k + 1], buf[k & 1]);
    rows *= c->n[k];
  }
  cudaMemcpyAsync(out, buf[(d - 1) & 1], sizeof(double) * P, cudaMemcpyDeviceToHost, c->st);
  const bool ok = cudaStreamSynchronize(c->st) == cudaSuccess;
  cudaFree(buf[0]);
  cudaFree(buf[1]);
  if (!ok) return cuda_fail(c);
  return check(c);
}

int ttgbf_import_cores(ttgbf_ctx* c, int32_t f, const float* buf, const int32_t* ranks, double log_lik) {
  if (c) tape_fail(c);
  if (split(c)) {
    if (f < 0 || f >= c->B) return TTGBF_EINVAL;
    int local = 0;
    const int p = part_of(c, f, &local);
    return fan_out(c, [&](ttgbf_ctx* q, int pp) {
      return pp == p ? ttgbf_import_cores(q, local, buf, ranks, log_lik) : TTGBF_OK;
    });
  }
  int rc = guard(c);
  if (rc) return rc;
  const int d = c->d;
  if (!buf || !ranks || f < 0 || f >= c->B) return TTGBF_EINVAL;
  if (ranks[0] != 1 || ranks[d] != 1) return TTGBF_EINVAL;
  if (!std::isfinite(log_lik)) return TTGBF_ENONFINITE;
  bool over = false;
  for (int k = 1; k < d; ++k) {
    if (ranks[k] < 1 || ranks[k] > c->capr) return TTGBF_EINVAL;
    if (ranks[k] > c->rank_cap) over = true;
  }
  size_t at = 0;
  for (int k = 0; k < d; ++k) {
    const size_t cnt = (size_t)ranks[k] * c->n[k] * ranks[k + 1];
    for (size_t t = 0; t < cnt; ++t)
      if (!std::isfinite(buf[at + t])) return TTGBF_ENONFINITE;
    at += cnt;
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  at = 0;
  for (int k = 0; k < d; ++k) {
    const size_t cnt = (size_t)ranks[k] * c->n[k] * ranks[k + 1];
    cudaMemcpy(curp(c, k) + (size_t)f * c->L.core_cap[k], buf + at, sizeof(float) * cnt, cudaMemcpyHostToDevice);
    at += cnt;
  }
  cudaMemcpy(c->ranks + (size_t)f * (d + 1), ranks, sizeof(int) * (d + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(c->log_lik + f, &log_lik, sizeof(double), cudaMemcpyHostToDevice);
  if (over) c->expanded = true;
  c->canon = false;
  return check(c);
}

int ttgbf_shear(ttgbf_ctx* c, int32_t m, int32_t n, double a, int32_t do_round) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_shear(q, m, n, a, do_round); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  if (m < 0 || n < 0 || m >= c->d || n >= c->d || m == n) return TTGBF_EINVAL;
  if (!std::isfinite(a)) return TTGBF_ENONFINITE;
  int S, tmin;
  std::vector<float> w;
  shear_table(c, m, n, a, &S, &tmin, &w);
  if (S > (do_round ? c->smax * c->smax : c->smax)) return TTGBF_ECAPACITY;
  if (c->expanded) enqueue_round(c);
  wait_stage(c->ev_ops, &c->ev_ops_used);
  std::copy(w.begin(), w.end(), c->stage_ops);
  cudaMemcpyAsync(c->opmats, c->stage_ops, sizeof(float) * w.size(), cudaMemcpyHostToDevice, c->st);
  cudaEventRecord(c->ev_ops, c->st);
  c->ev_ops_used = true;
  c->lastF.clear();  // the operator area no longer holds a predict's operators
  enqueue_shear(c, m, n, S, tmin, c->opmats, do_round != 0);
  return check(c);
}

static int upload_mats(ttgbf_ctx* c, const std::vector<std::vector<double>>& mats) {
  size_t tot = 0;
  for (const auto& m : mats) tot += m.size();
  if ((long long)tot > c->L.opmats_floats) return TTGBF_ECAPACITY;
  wait_stage(c->ev_ops, &c->ev_ops_used);
  size_t at = 0;
  for (const auto& m : mats)
    for (double v : m) c->stage_ops[at++] = (float)v;
  cudaMemcpyAsync(c->opmats, c->stage_ops, sizeof(float) * tot, cudaMemcpyHostToDevice, c->st);
  cudaEventRecord(c->ev_ops, c->st);
  c->ev_ops_used = true;
  c->lastF.clear();
  return TTGBF_OK;
}

int ttgbf_scale(ttgbf_ctx* c, int32_t m, double lam) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_scale(q, m, lam); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  tape_fail(c);  // single-operation hooks are not part of a recorded step
  if (m < 0 || m >= c->d) return TTGBF_EINVAL;
  if (!std::isfinite(lam)) return TTGBF_ENONFINITE;
  std::vector<std::vector<double>> mats(1);
  cic_matrix(c, m, lam, &mats[0]);
  rc = upload_mats(c, mats);
  if (rc) return rc;
  mode_apply(c, m, c->opmats);
  return check(c);
}

int ttgbf_convolve(ttgbf_ctx* c, const double* q) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* x, int) { return ttgbf_convolve(x, q); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  tape_fail(c);
  if (!q) return TTGBF_EINVAL;
  if (!finite_all(q, c->d)) return TTGBF_ENONFINITE;
  for (int k = 0; k < c->d; ++k)
    if (!(q[k] > 0.0)) return TTGBF_EINVAL;
  // per mode: FFT tables or the dense Toeplitz matrix (opts.conv)
  std::vector<float> host((size_t)c->L.opmats_floats, 0.f);
  std::vector<long long> off(c->d, -1);
  long long at = 0;
  for (int k = 0; k < c->d; ++k) {
    c->mode_fft[k] = conv_uses_fft(c, k) && fft_tables(c, k, q[k], 1.0, &host, &at);
    if (c->mode_fft[k]) continue;
    std::vector<double> K;
    conv_matrix(c, k, q[k], &K);
    if (at + (long long)K.size() > c->L.opmats_floats) return TTGBF_ECAPACITY;
    off[k] = at;
    for (size_t t = 0; t < K.size(); ++t) host[at + t] = (float)K[t];
    at += (long long)K.size();
  }
  wait_stage(c->ev_ops, &c->ev_ops_used);
  std::memcpy(c->stage_ops, host.data(), sizeof(float) * at);
  cudaMemcpyAsync(c->opmats, c->stage_ops, sizeof(float) * at, cudaMemcpyHostToDevice, c->st);
  cudaEventRecord(c->ev_ops, c->st);
  c->ev_ops_used = true;
  c->lastF.clear();  // the operator area no longer holds a predict's operators
  for (int k = 0; k < c->d; ++k) {
    if (c->mode_fft[k]) mode_conv_fft(c, k);
    else mode_apply(c, k, c->opmats + off[k]);
  }
  return check(c);
}

// The predictive step with the textbook transition (Eqs. pdf_predII,
// TPMmat) for an upper bidiagonal F and a diagonal Q.  The transition's
// Gaussian then factorises over the modes, K_m(j, i, i') = D_m N(xi_{m,j} -
// F_mm xi_{m,i} - F_{m,m+1} xi_{m+1,i'}; 0, Q_mm), and the factors apply in
// the order m = 0, 1, ..., each summing out i_m while i_{m+1} is still the
// old index.  From the canonical form centred at core 0: a coupled factor
// acts on the 2-site block (m, m+1), built by the cross of the transition
// block (cross.cu, no supercore is formed), and the block's link is rounded
// (the center moves to m + 1); an uncoupled factor is a dense matrix on core
// m followed by the truncating left step; the last mode's factor is a matrix
// on the last core; then normalisation.
int ttgbf_predict_exact(ttgbf_ctx* c, const double* F, const double* Q) {
  ApiRange range("ttgbf_predict_exact");
  if (split(c))
    return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_predict_exact(q, F, Q); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  const int d = c->d;
  if (!F || !Q) return TTGBF_EINVAL;
  if (!finite_all(F, (size_t)d * d) || !finite_all(Q, (size_t)d * d)) return TTGBF_ENONFINITE;
  for (int m = 0; m < d; ++m)
    for (int n = 0; n < d; ++n) {
      const double f = F[(size_t)m * d + n], q = Q[(size_t)m * d + n];
      if (f != 0.0 && n != m && n != m + 1) return TTGBF_EINVAL;
      if (m == n ? !(q > 0.0) : q != 0.0) return TTGBF_EINVAL;
    }
  if (c->cross_s <= 0) return TTGBF_EINVAL;
  tape_fail(c);  // not recordable by the adjoint
  // dense factors of the uncoupled modes and of the last mode
  std::vector<std::vector<double>> mats;
  std::vector<long long> off(d, -1);
  long long at = 0;
  for (int m = 0; m < d; ++m) {
    if (m + 1 < d && F[(size_t)m * d + m + 1] != 0.0) continue;
    const int N = c->n[m];
    const double D = c->dx[m], q = Q[(size_t)m * d + m], f = F[(size_t)m * d + m];
    const double norm = D / std::sqrt(2.0 * M_PI * q);
    std::vector<double> K((size_t)N * N);
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const double x = (c->lo[m] + (j + 0.5) * D) - f * (c->lo[m] + (i + 0.5) * D);
        K[(size_t)j * N + i] = norm * std::exp(-0.5 * x * x / q);
      }
    off[m] = at;
    at += (long long)K.size();
    mats.push_back(std::move(K));
  }
  rc = upload_mats(c, mats);
  if (rc) return rc;
  if (c->expanded) enqueue_round(c);
  enqueue_center_into(c, 0, 0);
  for (int m = 0; m + 1 < d; ++m) {
    if (F[(size_t)m * d + m + 1] != 0.0) {
      CrossArgs a = c->x;
      a.B = c->B;
      a.d = d;
      a.lo = m;
      a.k = 2;
      a.s = c->cross_s;
      a.ranks = c->ranks;
      for (int q = 0; q < 2; ++q) {
        a.core[q] = curp(c, m + q);
        a.out[q] = altp(c, m + q);
        a.cap[q] = c->L.core_cap[m + q];
        a.N[q] = c->n[m + q];
        a.stride[q] = 0;
      }
      a.htab = nullptr;
      a.z = nullptr;
      a.off = nullptr;
      a.R = 1.0;
      a.trans = 1;
      const double q = Q[(size_t)m * d + m];
      a.tF0 = (float)F[(size_t)m * d + m];
      a.tF1 = (float)F[(size_t)m * d + m + 1];
      a.tiq = (float)(1.0 / q);
      a.tkc = (float)(c->dx[m] / std::sqrt(2.0 * M_PI * q));
      a.tlo0 = (float)c->lo[m];
      a.tdx0 = (float)c->dx[m];
      a.tlo1 = (float)c->lo[m + 1];
      a.tdx1 = (float)c->dx[m + 1];
      // sums over the old index skip the cells where K < exp(-32) of its
      // peak (8 standard deviations; below float32's resolution); two cells
      // of margin for the rounding of the window's centre
      const double f0 = std::fabs(F[(size_t)m * d + m]);
      a.twin = f0 > 0.0 ? (float)std::min(8.0 * std::sqrt(q) / (f0 * c->dx[m]) + 2.0, 1e6) : 0.f;
      {
        Prof p(c, kPCross, 2 * c->cross_sweeps + 3);
        launch_cross_step(c->st, a, 1, kCrossStart);
        for (int sw = 0; sw < c->cross_sweeps; ++sw) {
          launch_cross_step(c->st, a, 0, kCrossLR);
          launch_cross_step(c->st, a, 1, kCrossRL);
        }
        launch_cross_step(c->st, a, 0, kCrossFinal);
        launch_cross_last(c->st, a);
      }
      c->cur[m] ^= 1;
      c->cur[m + 1] ^= 1;
      stage(c, kStageRight, m + 1, 0);
      stage(c, kStageLeft, m, 1);
    } else {
      mode_apply(c, m, c->opmats + off[m]);
      stage(c, kStageLeft, m, 1);
    }
    c->canon = true;
    c->center = m + 1;
  }
  mode_apply(c, d - 1, c->opmats + off[d - 1]);
  enqueue_normalise(c, c->mass_pred);
  return check(c);
}

// Grid re-design, interpolation step (Alg. 4 step 5): every filter's density
// values onto a new axis-aligned grid of the same cell counts, by separable
// piecewise-linear interpolation (the value at a new point from the two old
// points around it; the density is zero at points beyond the old grid, as
// in the filter's boundary reading: one N x N matrix per mode with at most
// two entries per row), then renormalised on the new grid.  The transition
// operators of the next predict are rebuilt for the new spacing.
int ttgbf_regrid(ttgbf_ctx* c, const double* lo, const double* hi) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_regrid(q, lo, hi); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  if (!lo || !hi) return TTGBF_EINVAL;
  const int d = c->d;
  if (!finite_all(lo, d) || !finite_all(hi, d)) return TTGBF_ENONFINITE;
  for (int k = 0; k < d; ++k)
    if (!(hi[k] > lo[k])) return TTGBF_EINVAL;
  tape_fail(c);
  std::vector<std::vector<double>> mats(d);
  std::vector<double> axes;
  for (int k = 0; k < d; ++k) {
    const int N = c->n[k];
    const double dxn = (hi[k] - lo[k]) / N;
    mats[k].assign((size_t)N * N, 0.0);
    for (int j = 0; j < N; ++j) {
      const double x = lo[k] + (j + 0.5) * dxn;
      axes.push_back(x);
      const double u = (x - c->lo[k]) / c->dx[k] - 0.5;  // position among the old points
      const int i0 = (int)std::floor(u);
      for (int i = i0; i <= i0 + 1; ++i)
        if (i >= 0 && i < N) mats[k][(size_t)j * N + i] = hatf(u - i);
    }
  }
  rc = upload_mats(c, mats);
  if (rc) return rc;
  size_t at = 0;
  for (int k = 0; k < d; ++k) {
    mode_apply(c, k, c->opmats + at);
    at += mats[k].size();
  }
  c->delta = 1.0;
  for (int k = 0; k < d; ++k) {
    c->lo[k] = lo[k];
    c->hi[k] = hi[k];
    c->dx[k] = (hi[k] - lo[k]) / c->n[k];
    c->delta *= c->dx[k];
  }
  c->axes = axes;
  cudaMemcpyAsync(c->axes_d, c->axes.data(), sizeof(double) * c->axes.size(), cudaMemcpyHostToDevice, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  enqueue_normalise(c, c->mass);
  c->lastF.clear();
  c->lastQ.clear();
  return check(c);
}

// Grid re-design, steps 1-4 of Alg. 4, for a batch that shares its grid:
// per filter, the predictive moments of the linear model (x = F m,
// P = F C F^T + Q from the filtering mean m and covariance C), the 2^d
// corners of the box x +- kappa sqrt(diag P), the same corners mapped back by
// F^{-1} into the filtering space, and the axis-aligned box around all of
// them; the batch's grid is the box around every filter's.  (The step's
// transition maps the grid onto itself, so the grid holds both the filtering
// density and the predictive one.)
int ttgbf_design_grid(int32_t d, int32_t batch, const double* F, const double* Q, const double* mean,
                      const double* cov, double kappa, double* lo, double* hi) {
  if (d < 1 || d > kMaxD || batch < 1 || !F || !Q || !mean || !cov || !lo || !hi) return TTGBF_EINVAL;
  if (!finite_all(F, (size_t)d * d) || !finite_all(Q, (size_t)d * d) || !finite_all(mean, (size_t)batch * d) ||
      !finite_all(cov, (size_t)batch * d * d) || !std::isfinite(kappa))
    return TTGBF_ENONFINITE;
  if (!(kappa > 0.0)) return TTGBF_EINVAL;
  // LU of F with partial pivoting, for the corners' F^{-1}
  std::vector<double> A(F, F + (size_t)d * d);
  std::vector<int> piv(d);
  for (int k = 0; k < d; ++k) {
    int p = k;
    for (int i = k + 1; i < d; ++i)
      if (std::fabs(A[(size_t)i * d + k]) > std::fabs(A[(size_t)p * d + k])) p = i;
    if (A[(size_t)p * d + k] == 0.0) return TTGBF_ESINGULAR;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < d; ++j) std::swap(A[(size_t)k * d + j], A[(size_t)p * d + j]);
    for (int i = k + 1; i < d; ++i) {
      const double f = A[(size_t)i * d + k] / A[(size_t)k * d + k];
      A[(size_t)i * d + k] = f;
      for (int j = k + 1; j < d; ++j) A[(size_t)i * d + j] -= f * A[(size_t)k * d + j];
    }
  }
  auto solve = [&](std::vector<double> x) {
    for (int k = 0; k < d; ++k) std::swap(x[k], x[piv[k]]);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < i; ++j) x[i] -= A[(size_t)i * d + j] * x[j];
    for (int i = d - 1; i >= 0; --i) {
      for (int j = i + 1; j < d; ++j) x[i] -= A[(size_t)i * d + j] * x[j];
      x[i] /= A[(size_t)i * d + i];
    }
    return x;
  };
  for (int k = 0; k < d; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  std::vector<double> xp(d), w(d), cpred(d);
  for (int b = 0; b < batch; ++b) {
    const double* m = mean + (size_t)b * d;
    const double* C = cov + (size_t)b * d * d;
    for (int i = 0; i < d; ++i) {
      xp[i] = 0.0;
      for (int j = 0; j < d; ++j) xp[i] += F[(size_t)i * d + j] * m[j];
    }
    for (int i = 0; i < d; ++i) {  // (F C F^T + Q)_ii
      double s = Q[(size_t)i * d + i];
      for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) s += F[(size_t)i * d + j] * C[(size_t)j * d + l] * F[(size_t)i * d + l];
      w[i] = kappa * std::sqrt(std::max(s, 0.0));
    }
    for (long long cidx = 0; cidx < (1LL << d); ++cidx) {
      for (int i = 0; i < d; ++i) cpred[i] = xp[i] + (((cidx >> i) & 1) ? w[i] : -w[i]);
      const std::vector<double> cmeas = solve(cpred);
      for (int i = 0; i < d; ++i) {
        lo[i] = std::min(lo[i], std::min(cpred[i], cmeas[i]));
        hi[i] = std::max(hi[i], std::max(cpred[i], cmeas[i]));
      }
    }
  }
  for (int k = 0; k < d; ++k)
    if (!(hi[k] > lo[k]) || !std::isfinite(lo[k]) || !std::isfinite(hi[k])) return TTGBF_EINVAL;
  return TTGBF_OK;
}

int ttgbf_round(ttgbf_ctx* c) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_round(q); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  enqueue_round(c);
  return check(c);
}

int ttgbf_normalise(ttgbf_ctx* c) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_normalise(q); }, false, false);
  int rc = guard(c);
  if (rc) return rc;
  enqueue_normalise(c, c->mass);
  return check(c);
}

int ttgbf_profile(ttgbf_ctx* c, int32_t enable) {
  if (split(c)) return fan_out(c, [&](ttgbf_ctx* q, int) { return ttgbf_profile(q, enable); });
  int rc = guard(c);
  if (rc) return rc;
  if (enable) {
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
    for (int k = 0; k < kPClasses; ++k) {
      c->ev_used[k] = 0;
      c->prof_launches[k] = 0;
    }
    cudaMemsetAsync(c->prof_flops, 0, sizeof(double) * kPClasses, c->st);
  }
  c->prof = enable != 0;
  return check(c);
}

int ttgbf_profile_read(ttgbf_ctx* c, ttgbf_kernel_prof* out, int32_t cap, int32_t* count) {
  if (split(c)) {
    // parts run concurrently: launches and flops add up, time is the
    // longest part's
    if (!out || !count || cap < 0) return TTGBF_EINVAL;
    std::vector<ttgbf_kernel_prof> tmp((size_t)std::max(cap, 0));
    for (size_t p = 0; p < c->parts.size(); ++p) {
      int32_t n = 0;
      const int rc = ttgbf_profile_read(c->parts[p], tmp.data(), cap, &n);
      if (rc) return rc;
      *count = n;
      for (int k = 0; k < n && k < cap; ++k) {
        if (p == 0) {
          out[k] = tmp[k];
        } else {
          out[k].launches += tmp[k].launches;
          out[k].flops += tmp[k].flops;
          out[k].ms = std::max(out[k].ms, tmp[k].ms);
        }
      }
    }
    return TTGBF_OK;
  }
  int rc = guard(c);
  if (rc) return rc;
  if (!out || !count || cap < 0) return TTGBF_EINVAL;
  double fl[kPClasses];
  cudaMemcpyAsync(fl, c->prof_flops, sizeof(fl), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  *count = kPClasses;
  for (int k = 0; k < kPClasses && k < cap; ++k) {
    double ms = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used[k]; i += 2) {
      float e = 0.f;
      if (cudaEventElapsedTime(&e, c->ev_pool[k][i], c->ev_pool[k][i + 1]) == cudaSuccess) ms += e;
    }
    ttgbf_kernel_prof& o = out[k];
    std::memset(&o, 0, sizeof(o));
    std::strncpy(o.name, kProfNames[k], sizeof(o.name) - 1);
    o.launches = c->prof_launches[k];
    o.ms = ms;
    o.flops = fl[k];
  }
  return check(c);
}

uint64_t ttgbf_launch_count(void) { return g_launches.load(); }

}  // extern "C"

// ================================================================ groups
namespace {

// The GPU's global timer (nanoseconds) into *p: the clock of recorded horizons.
__global__ void k_stamp(unsigned long long* p) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *p = t;
}

void launch_stamp(cudaStream_t st, unsigned long long* p) {
  ttgbf::count_launches(1);
  k_stamp<<<1, 1, 0, st>>>(p);
}

}  // namespace

struct ttgbf_group {
  cudaStream_t st = nullptr;
  std::vector<ttgbf_ctx*> ctxs;   // as given
  std::vector<ttgbf_ctx*> leaves;  // every context's parts (or the context itself)
  std::vector<int> owner;          // leaf -> index in ctxs
  std::vector<int> base;           // leaf -> its first filter within the owner
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;  // per leaf
  // timing of the last ttgbf_group_step: its start on the group's stream and
  // the end of every leaf's work (not recorded into graphs)
  cudaEvent_t ev_t0 = nullptr;
  std::vector<cudaEvent_t> ev_tend;
  bool timed = false, capturing = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long graph_kernels = 0;
  // timing of a recorded horizon: the GPU's global timer written by a one-
  // thread kernel at every step's start (group stream) and at the end of
  // every leaf's step, [step][1 + leaf] nanoseconds, read after a launch
  unsigned long long* stamps = nullptr;
  int graph_steps = 0;
  bool graph_ran = false;
};

namespace {

int group_fail(ttgbf_group* g) {
  for (ttgbf_ctx* c : g->leaves) c->poisoned = true;
  return TTGBF_ECUDA;
}

// Host-side validation of one context's step arguments (nothing enqueued).
int group_validate(ttgbf_ctx* c, const ttgbf_group_step_args& a) {
  if (!a.F || !a.Q || !a.h || !a.R || !a.z_dev) return TTGBF_EINVAL;
  const int d = c->d;
  if (!finite_all(a.F, (size_t)d * d) || !finite_all(a.Q, (size_t)d * d)) return TTGBF_ENONFINITE;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      if (i != j && a.Q[(size_t)i * d + j] != 0.0) return TTGBF_EINVAL;
      if (i == j && !(a.Q[(size_t)i * d + j] > 0.0)) return TTGBF_EINVAL;
    }
  ttgbf_ctx* leaf = c->parts.empty() ? c : c->parts[0];
  int two = -1;
  return validate_meas(leaf, a.h, a.R, &two);
}

// Enqueue one step of every leaf, interleaved operation by operation.
// step_off: offset (in steps) into the horizon arrays of args.
int group_enqueue(ttgbf_group* g, const ttgbf_group_step_args* args, long long t) {
  const size_t nl = g->leaves.size();
  if (!g->capturing) cudaEventRecord(g->ev_t0, g->st);
  else launch_stamp(g->st, g->stamps + (size_t)t * (nl + 1));
  cudaEventRecord(g->ev_fork, g->st);
  for (ttgbf_ctx* q : g->leaves) cudaStreamWaitEvent(q->st, g->ev_fork, 0);
  // predict
  size_t nops = 0;
  for (size_t l = 0; l < nl; ++l) {
    const ttgbf_group_step_args& a = args[g->owner[l]];
    const int rc = predict_begin(g->leaves[l], a.F, a.Q);
    if (rc) return rc;
    nops = std::max(nops, g->leaves[l]->ops.size());
  }
  for (size_t i = 0; i < nops; ++i)
    for (ttgbf_ctx* q : g->leaves)
      if (i < q->ops.size()) predict_op(q, i);
  int dmax = 0;
  for (ttgbf_ctx* q : g->leaves) dmax = std::max(dmax, q->d);
  for (int k = 0; k < dmax; ++k)
    for (ttgbf_ctx* q : g->leaves)
      if (k < q->d) predict_mode(q, k);
  for (ttgbf_ctx* q : g->leaves) predict_end(q);
  // update (device measurements of the step)
  std::vector<EnqueueOps> lists(nl);
  size_t nmax = 0;
  for (size_t l = 0; l < nl; ++l) {
    ttgbf_ctx* q = g->leaves[l];
    const ttgbf_group_step_args& a = args[g->owner[l]];
    const ttgbf_ctx* own = g->ctxs[g->owner[l]];
    const long long b = a.h->b;
    const float* z = a.z_dev + (t * own->B + g->base[l]) * b;
    const float* zq = nullptr;
    int two = -1;
    const int rc = update_prepare(q, a.h, a.R, nullptr, z, &zq, &two);
    if (rc) return rc;
    update_ops(q, a.h, a.R, zq, (int)b, two, &lists[l]);
    nmax = std::max(nmax, lists[l].size());
  }
  for (size_t i = 0; i < nmax; ++i)
    for (size_t l = 0; l < nl; ++l)
      if (i < lists[l].size()) lists[l][i]();
  // estimate into the caller's device arrays
  for (size_t l = 0; l < nl; ++l) {
    ttgbf_ctx* q = g->leaves[l];
    const ttgbf_group_step_args& a = args[g->owner[l]];
    const ttgbf_ctx* own = g->ctxs[g->owner[l]];
    const long long B = q->B, d = q->d;
    const long long f0 = t * own->B + g->base[l];
    const int rc = estimate_common(q);
    if (rc) return rc;
    if (a.mean) cudaMemcpyAsync(a.mean + f0 * d, q->mean, sizeof(double) * B * d, cudaMemcpyDeviceToDevice, q->st);
    if (a.cov)
      cudaMemcpyAsync(a.cov + f0 * d * d, q->cov, sizeof(double) * B * d * d, cudaMemcpyDeviceToDevice, q->st);
    if (a.log_c) cudaMemcpyAsync(a.log_c + f0, q->log_c, sizeof(double) * B, cudaMemcpyDeviceToDevice, q->st);
    if (a.log_lik)
      cudaMemcpyAsync(a.log_lik + f0, q->log_lik, sizeof(double) * B, cudaMemcpyDeviceToDevice, q->st);
  }
  for (size_t l = 0; l < nl; ++l) {
    if (!g->capturing) cudaEventRecord(g->ev_tend[l], g->leaves[l]->st);
    else launch_stamp(g->leaves[l]->st, g->stamps + (size_t)t * (nl + 1) + 1 + l);
    cudaEventRecord(g->ev_join[l], g->leaves[l]->st);
    cudaStreamWaitEvent(g->st, g->ev_join[l], 0);
  }
  g->timed = !g->capturing;
  for (ttgbf_ctx* q : g->leaves) {
    const int rc = check(q);
    if (rc) return rc;
  }
  return TTGBF_OK;
}

int group_guard(ttgbf_group* g, const ttgbf_group_step_args* args) {
  if (!g || !args) return TTGBF_EINVAL;
  for (ttgbf_ctx* q : g->leaves)
    if (q->poisoned) return TTGBF_EPOISONED;
  for (size_t i = 0; i < g->ctxs.size(); ++i) {
    const int rc = group_validate(g->ctxs[i], args[i]);
    if (rc) return rc;
  }
  return TTGBF_OK;
}

}  // namespace

extern "C" {

int ttgbf_group_create(ttgbf_group** out, ttgbf_ctx* const* ctxs, int32_t n, void* stream) {
  if (!out || !ctxs || n < 1) return TTGBF_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return TTGBF_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return TTGBF_EINVAL;
  }
  ttgbf_group* g = new (std::nothrow) ttgbf_group();
  if (!g) return TTGBF_ENOMEM;
  g->st = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    ttgbf_ctx* c = ctxs[i];
    g->ctxs.push_back(c);
    if (c->parts.empty()) {
      g->leaves.push_back(c);
      g->owner.push_back(i);
      g->base.push_back(0);
    } else {
      for (size_t p = 0; p < c->parts.size(); ++p) {
        g->leaves.push_back(c->parts[p]);
        g->owner.push_back(i);
        g->base.push_back(c->part_base[p]);
      }
    }
  }
  if (cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return TTGBF_ENOMEM;
  }
  if (cudaEventCreate(&g->ev_t0) != cudaSuccess) {
    cudaGetLastError();
    ttgbf_group_free(g);
    return TTGBF_ENOMEM;
  }
  for (size_t l = 0; l < g->leaves.size(); ++l) {
    cudaEvent_t e = nullptr, et = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&et) != cudaSuccess) {
      cudaGetLastError();
      if (e) cudaEventDestroy(e);
      ttgbf_group_free(g);
      return TTGBF_ENOMEM;
    }
    g->ev_join.push_back(e);
    g->ev_tend.push_back(et);
  }
  *out = g;
  return TTGBF_OK;
}

int ttgbf_group_step(ttgbf_group* g, const ttgbf_group_step_args* args) {
  ApiRange range("ttgbf_group_step");
  const int rc = group_guard(g, args);
  if (rc) return rc;
  return group_enqueue(g, args, 0);
}

// The host-side state a recorded step sequence depends on: which ping-pong
// buffer holds each core, the canonical form, unexpanded middle cores.
struct LeafState {
  int cur[kMaxD];
  int virt_S[kMaxD];
  bool canon, expanded;
  int center;
  bool operator==(const LeafState& o) const {
    return std::equal(cur, cur + kMaxD, o.cur) && std::equal(virt_S, virt_S + kMaxD, o.virt_S) &&
           canon == o.canon && expanded == o.expanded && center == o.center;
  }
};

static LeafState leaf_state(const ttgbf_ctx* c) {
  LeafState s{};
  std::copy(c->cur, c->cur + kMaxD, s.cur);
  std::copy(c->virt_S, c->virt_S + kMaxD, s.virt_S);
  s.canon = c->canon;
  s.expanded = c->expanded;
  s.center = c->center;
  return s;
}

static void group_drop_graph(ttgbf_group* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  g->graph_kernels = 0;
  if (g->stamps) cudaFree(g->stamps);
  g->stamps = nullptr;
  g->graph_steps = 0;
  g->graph_ran = false;
}

int ttgbf_group_capture(ttgbf_group* g, const ttgbf_group_step_args* args, int32_t steps) {
  ApiRange range("ttgbf_group_capture");
  int rc = group_guard(g, args);
  if (rc) return rc;
  if (steps < 1) return TTGBF_EINVAL;
  // the legacy default stream cannot be recorded, nor joined into a recording
  if (g->st == nullptr) return TTGBF_EINVAL;
  for (ttgbf_ctx* q : g->leaves)
    if (q->prof || q->st == nullptr) return TTGBF_EINVAL;  // event timing cannot be replayed
  // operators of F, Q prepared on the host (and uploaded) before recording
  for (size_t l = 0; l < g->leaves.size(); ++l) {
    ttgbf_ctx* q = g->leaves[l];
    const ttgbf_group_step_args& a = args[g->owner[l]];
    const int d = q->d;
    const bool same = q->lastF.size() == (size_t)d * d && std::equal(q->lastF.begin(), q->lastF.end(), a.F) &&
                      std::equal(q->lastQ.begin(), q->lastQ.end(), a.Q);
    if (!same) {
      rc = prepare_predict(q, a.F, a.Q);
      if (rc) return rc;
    }
  }
  for (ttgbf_ctx* q : g->leaves)
    if (cudaStreamSynchronize(q->st) != cudaSuccess) return group_fail(g);
  if (cudaStreamSynchronize(g->st) != cudaSuccess) return group_fail(g);
  group_drop_graph(g);
  if (cudaMalloc(&g->stamps, sizeof(unsigned long long) * (size_t)steps * (g->leaves.size() + 1)) !=
      cudaSuccess) {
    cudaGetLastError();
    g->stamps = nullptr;
    return TTGBF_ENOMEM;
  }
  std::vector<LeafState> before;
  for (ttgbf_ctx* q : g->leaves) before.push_back(leaf_state(q));
  const unsigned long long l0 = g_launches.load();
  if (cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return group_fail(g);
  }
  g->capturing = true;
  for (int t = 0; t < steps && rc == TTGBF_OK; ++t) rc = group_enqueue(g, args, t);
  g->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(g->st, &graph);
  const unsigned long long recorded = g_launches.load() - l0;
  g_launches.fetch_sub(recorded);  // recorded, not run
  bool periodic = true;
  for (size_t l = 0; l < g->leaves.size(); ++l) {
    periodic = periodic && leaf_state(g->leaves[l]) == before[l];
    // nothing ran: the contexts are where they were
    ttgbf_ctx* q = g->leaves[l];
    std::copy(before[l].cur, before[l].cur + kMaxD, q->cur);
    std::copy(before[l].virt_S, before[l].virt_S + kMaxD, q->virt_S);
    q->canon = before[l].canon;
    q->expanded = before[l].expanded;
    q->center = before[l].center;
  }
  if (e != cudaSuccess || rc != TTGBF_OK) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return rc != TTGBF_OK ? rc : group_fail(g);
  }
  if (!periodic) {
    // a relaunch would start from buffers or a canonical form the recording
    // did not leave: step once before recording, record an even number
    cudaGraphDestroy(graph);
    return TTGBF_EINVAL;
  }
  if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return group_fail(g);
  }
  g->graph = graph;
  g->graph_kernels = recorded;
  g->graph_steps = steps;
  return TTGBF_OK;
}

int ttgbf_group_launch(ttgbf_group* g) {
  if (!g || !g->exec) return TTGBF_EINVAL;
  for (ttgbf_ctx* q : g->leaves)
    if (q->poisoned) return TTGBF_EPOISONED;
  if (cudaGraphLaunch(g->exec, g->st) != cudaSuccess) {
    cudaGetLastError();
    return group_fail(g);
  }
  g_launches.fetch_add(g->graph_kernels);
  g->graph_ran = true;
  return TTGBF_OK;
}

uint64_t ttgbf_group_graph_kernels(const ttgbf_group* g) { return g ? g->graph_kernels : 0; }

int ttgbf_group_times(ttgbf_group* g, float* ms) {
  if (!g || !ms) return TTGBF_EINVAL;
  if (!g->timed) return TTGBF_EINVAL;
  for (size_t i = 0; i < g->ctxs.size(); ++i) ms[i] = 0.f;
  for (size_t l = 0; l < g->leaves.size(); ++l) {
    float e = 0.f;
    if (cudaEventSynchronize(g->ev_tend[l]) != cudaSuccess ||
        cudaEventElapsedTime(&e, g->ev_t0, g->ev_tend[l]) != cudaSuccess) {
      cudaGetLastError();
      return group_fail(g);
    }
    ms[g->owner[l]] = std::max(ms[g->owner[l]], e);
  }
  return TTGBF_OK;
}

int ttgbf_group_graph_times(ttgbf_group* g, float* ms) {
  if (!g || !ms || !g->exec || !g->graph_ran || !g->stamps) return TTGBF_EINVAL;
  const size_t nl = g->leaves.size(), nc = g->ctxs.size();
  std::vector<unsigned long long> st((size_t)g->graph_steps * (nl + 1));
  if (cudaStreamSynchronize(g->st) != cudaSuccess ||
      cudaMemcpy(st.data(), g->stamps, sizeof(unsigned long long) * st.size(), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return group_fail(g);
  }
  for (int t = 0; t < g->graph_steps; ++t) {
    const unsigned long long* row = st.data() + (size_t)t * (nl + 1);
    for (size_t i = 0; i < nc; ++i) ms[(size_t)t * nc + i] = 0.f;
    for (size_t l = 0; l < nl; ++l) {
      const float e = row[1 + l] > row[0] ? (float)((double)(row[1 + l] - row[0]) * 1e-6) : 0.f;
      float& m = ms[(size_t)t * nc + g->owner[l]];
      m = std::max(m, e);
    }
  }
  return TTGBF_OK;
}

int ttgbf_group_free(ttgbf_group* g) {
  if (!g) return TTGBF_OK;
  if (g->st) cudaStreamSynchronize(g->st);
  group_drop_graph(g);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_t0) cudaEventDestroy(g->ev_t0);
  for (cudaEvent_t e : g->ev_join) cudaEventDestroy(e);
  for (cudaEvent_t e : g->ev_tend) cudaEventDestroy(e);
  cudaGetLastError();
  delete g;
  return TTGBF_OK;
}

}  // extern "C"

// ============================================================ autotuning
namespace {

// Cache key of a batch shape: grid, batch, rank cap, span, precision, conv,
// the span of every elementary shear of F on this grid (which sets the rank
// expansions), the GPU's name, and a contraction mode other than float32.
std::string tune_key(const ttgbf_grid* g, const ttgbf_opts* o, const double* F) {
  const int d = g->d;
  std::string k = "d=" + std::to_string(d) + ";n=";
  for (int m = 0; m < d; ++m) k += std::to_string(g->n[m]) + (m + 1 < d ? "," : "");
  k += ";batch=" + std::to_string(o->batch) + ";cap=" + std::to_string(o->rank_cap) +
       ";span=" + std::to_string(o->max_shift_span > 0 ? o->max_shift_span : 10) +
       ";prec=" + std::to_string(o->precision) + ";conv=" + std::to_string(o->conv) + ";shears=";
  std::vector<double> Lm, D, U;
  if (ldu(F, d, &Lm, &D, &U) == TTGBF_OK) {
    for (int m = 0; m < d; ++m)
      for (int n = 0; n < d; ++n) {
        const double a = m < n ? U[(size_t)m * d + n] : (m > n ? Lm[(size_t)m * d + n] : 0.0);
        if (a == 0.0) continue;
        const double dm = (g->hi[m] - g->lo[m]) / g->n[m], dn = (g->hi[n] - g->lo[n]) / g->n[n];
        int lo = 1 << 30, hi = -(1 << 30);
        for (int i = 0; i < g->n[n]; ++i) {
          const int f = (int)std::floor(a * (g->lo[n] + (i + 0.5) * dn) / dm);
          lo = std::min(lo, f);
          hi = std::max(hi, f);
        }
        k += std::to_string(m) + "." + std::to_string(n) + ":" + std::to_string(hi - lo + 2) + ",";
      }
  }
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    std::string name(prop.name);
    for (char& ch : name)
      if (ch == ' ' || ch == '\t') ch = '_';
    k += ";gpu=" + name;
  }
  cudaGetLastError();
  // the tensor-core contraction modes key their own entries (float32
  // contractions keep the key they always had)
  if (o->contraction != TTGBF_CONTRACT_FP32) k += ";contract=" + std::to_string(o->contraction);
  return k;
}

// ms per predictive step of one candidate configuration (its own context,
// stream and workspace); a negative code when it cannot be created.
int tune_time(const ttgbf_grid* grid, const ttgbf_prior* prior, const ttgbf_opts* o, const double* F,
              const double* Q, int steps, double* ms) {
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return TTGBF_ECUDA;
  }
  ttgbf_opts oo = *o;
  oo.stream = st;
  oo.workspace = nullptr;
  oo.workspace_bytes = 0;
  ttgbf_ctx* c = nullptr;
  int rc = ttgbf_init(&c, grid, prior, &oo);
  cudaEvent_t a = nullptr, b = nullptr;
  if (rc == TTGBF_OK) rc = ttgbf_predict(c, F, Q);  // untimed: operators, first rounding
  if (rc == TTGBF_OK) {
    if (split(c)) join_parts(c);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    if (split(c)) fork_parts(c);
    for (int t = 0; t < steps && rc == TTGBF_OK; ++t) rc = ttgbf_predict(c, F, Q);
    if (split(c)) join_parts(c);
    cudaEventRecord(b, st);
    float e = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&e, a, b) != cudaSuccess) {
      cudaGetLastError();
      if (rc == TTGBF_OK) rc = TTGBF_ECUDA;
    }
    *ms = (double)e / steps;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (c) ttgbf_free(c);
  cudaStreamDestroy(st);
  cudaGetLastError();
  return rc;
}

}  // namespace

extern "C" {

int ttgbf_autotune(const ttgbf_grid* grid, const ttgbf_prior* prior, const ttgbf_opts* base,
                   const double* F, const double* Q, int32_t steps, const char* cache_path,
                   ttgbf_opts* best, double* best_ms) {
  if (!grid || !prior || !base || !F || !Q || !best || !best_ms || steps < 0) return TTGBF_EINVAL;
  if (steps == 0 && !cache_path) return TTGBF_EINVAL;
  int rc = validate_grid(grid);
  if (rc) return rc;
  rc = validate_opts(base);
  if (rc) return rc;
  const std::string key = tune_key(grid, base, F);
  if (cache_path) {
    if (FILE* fh = std::fopen(cache_path, "r")) {
      char line[2048];
      while (std::fgets(line, sizeof(line), fh)) {
        char* tab = std::strchr(line, '\t');
        if (!tab || std::string(line, tab - line) != key) continue;
        int parts = 0, sb = 0, sv = 0;
        double ms = 0.0;
        if (std::sscanf(tab + 1, "%d %d %d %lf", &parts, &sb, &sv, &ms) == 4) {
          *best = *base;
          best->parts = parts;
          best->tsqr_slice_blocks = sb;
          best->svd_threads = sv;
          *best_ms = ms;
          std::fclose(fh);
          return TTGBF_OK;
        }
      }
      std::fclose(fh);
    }
  }
  if (steps == 0) return TTGBF_EINVAL;  // cache lookup only, and the shape is not there
  double bms = 1e300;
  ttgbf_opts bo = *base;
  int last = TTGBF_EINVAL;
  for (int parts : {1, 2, 4, 8}) {
    if (parts > base->batch) continue;
    for (int sb : {4, 8, 16})
      for (int sv : {512, 1024}) {
        ttgbf_opts o = *base;
        o.parts = parts;
        o.tsqr_slice_blocks = sb;
        o.svd_threads = sv;
        double ms = 0.0;
        last = tune_time(grid, prior, &o, F, Q, steps, &ms);
        if (last == TTGBF_OK && ms < bms) {
          bms = ms;
          bo = o;
        }
      }
  }
  if (bms == 1e300) return last;
  *best = bo;
  *best_ms = bms;
  if (cache_path) {
    if (FILE* fh = std::fopen(cache_path, "a")) {
      std::fprintf(fh, "%s\t%d %d %d %.6f\n", key.c_str(), bo.parts, bo.tsqr_slice_blocks, bo.svd_threads,
                   bms);
      std::fclose(fh);
    }
  }
  return TTGBF_OK;
}

}  // extern "C"

namespace ttgbf {
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }
}  // namespace ttgbf

// ================================================================ adjoint
// The reverse pass of a run of filter steps: the gradient of the
// log-likelihood l = sum_k log c_k (Eq. pmf_filtrace_b) with respect to the
// elementary operators of F = L D U (shear coefficients and scalings), the
// variances Q_mm and R_cc.  It runs the adjoint recursion of the filter
// equations (the operators the TT step applies, transposed) with the adjoint
// density lambda held as a tensor train in a second context of the same grid
// and rounded there like a forward density, and takes the gradients as inner
// products of lambda with the derivative operators applied to the forward
// pass's cores.  The forward pass's roundings do not enter: it is the
// gradient of the filter equations, evaluated with the TT densities of the
// forward pass.  (Differentiating the roundings with their bases held fixed
// would drop the first-order change of a kept subspace that turns to follow
// its input: a rank-r truncation of A + dA at an A of rank r returns
// A + dA to first order, not U U^T (A + dA).)
//
// While a tape is attached, predict and update record (compact snapshots:
// ranks are at most rank_cap at every recorded point):
//   kTShear  the input y of a shear x_m += a x_n
//   kTMode   the input of a per-mode operator (kernel, scaling or both)
//   kTNorm   a normalisation x = y / m: its output and m
//   kTUpdIn  the input w of the update
//   kTLik    a likelihood factor (component, table, z, offset)
//   kTLogc   the mass c of the update's product (before its rounding)
// and the reverse pass runs the records backwards:
//   norm:  lambda <- (lambda - delta <lambda, x> 1) / m
//   logc:  lambda <- lambda + (delta / c) 1
//   lik:   lambda <- Lambda (.) lambda; dl/dR_c = <g_c (.) lambda, w> at the
//          update's input w, g_c = d log Lambda_c / dR_c
//   mode:  dl/dtheta = <lambda, (dM/dtheta) y>; lambda <- M^T lambda
//   shear: dl/da = <lambda, (dS/da) y>; lambda <- S(-a) lambda (S^T = S(-a))
// and the chain rule through the LDU factorisation gives dl/dF.
namespace {

enum TapeKind : int { kTShear = 0, kTMode, kTNorm, kTUpdIn, kTLik, kTLogc };

struct TapeEntry {
  int kind = 0;
  int k = 0;        // mode: the mode; shear: m
  int n = 0;        // shear: n
  int op = -1;      // shear: index in ops
  int mkind = 0;    // mode: TapeModeKind
  size_t snap = 0;  // byte offset of the snapshot in the tape
  size_t scal = 0;  // byte offset of per-filter doubles (norm, logc) or floats z, off (lik)
  int comp = -1, nmodes = 0, mode0 = 0;
  const float* htab = nullptr;
  double R = 0.0;
  float period = 0.f;
};

struct CkptHost {
  bool valid = false;
  bool canon = false, expanded = false;
  int center = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct ttgbf_adj {
  ttgbf_ctx* c = nullptr;   // the filter batch
  ttgbf_ctx* lc = nullptr;  // holds the adjoint density lambda (same grid and batch)
  int B = 0, d = 0, RS = 0, RL = 0, phi_max = 0, chunks = 16, nparams = 0;
  long long scap[kMaxD] = {};     // snapshot floats per filter per core (rank_cap bound)
  long long lcap[kMaxD] = {};     // scratch floats per filter per core
  size_t snap_cores[kMaxD] = {};  // byte offsets of the cores in a snapshot
  size_t snap_ranks = 0, snap_bytes = 0, scal_bytes = 0;
  char* base = nullptr;
  char* tape = nullptr;
  size_t tape_cap = 0, tape_used = 0;
  std::vector<TapeEntry> entries;
  bool recording = false, failed = false;
  int nslots = 0;
  char* ckpt = nullptr;
  size_t ckpt_bytes = 0;
  std::vector<CkptHost> ckh;
  float* sA[kMaxD] = {};
  float* sB[kMaxD] = {};
  int* sranks = nullptr;
  float* phi[2] = {};
  float* part = nullptr;
  int* err = nullptr;
  double *val = nullptr, *sc = nullptr, *coef = nullptr, *grad = nullptr;
  float* mats = nullptr;
  long long mats_floats = 0;
};

namespace {

// ---- recording
char* tape_take(ttgbf_adj* a, size_t bytes, size_t* off) {
  if (a->failed || a->tape_used + bytes > a->tape_cap) {
    a->failed = true;
    return nullptr;
  }
  *off = a->tape_used;
  a->tape_used += align256(bytes);
  return a->tape + *off;
}

// Snapshot of the context's TT (compact cores, ranks) at dst.
void snap_state(ttgbf_adj* a, char* dst) {
  ttgbf_ctx* c = a->c;
  for (int k = 0; k < a->d; ++k)
    cudaMemcpy2DAsync(dst + a->snap_cores[k], sizeof(float) * a->scap[k], curp(c, k),
                      sizeof(float) * c->L.core_cap[k], sizeof(float) * a->scap[k], a->B,
                      cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(dst + a->snap_ranks, c->ranks, sizeof(int) * (size_t)a->B * (a->d + 1),
                  cudaMemcpyDeviceToDevice, c->st);
}

void tape_push(ttgbf_ctx* c, TapeEntry e, bool with_snap) {
  ttgbf_adj* a = c->tape;
  if (with_snap) {
    char* p = tape_take(a, a->snap_bytes, &e.snap);
    if (!p) return;
    snap_state(a, p);
  }
  a->entries.push_back(e);
}

void tape_fail(ttgbf_ctx* c) {
  if (c->tape) c->tape->failed = true;
}

void tape_shear(ttgbf_ctx* c, int m, int n) {
  if (!c->tape) return;
  if (c->tape_op < 0) {
    tape_fail(c);
    return;
  }
  TapeEntry e;
  e.kind = kTShear;
  e.k = m;
  e.n = n;
  e.op = c->tape_op;
  tape_push(c, e, true);
}

void tape_mode(ttgbf_ctx* c, int k, int kind) {
  if (!c->tape) return;
  TapeEntry e;
  e.kind = kTMode;
  e.k = k;
  e.mkind = kind;
  tape_push(c, e, true);
}

void tape_norm(ttgbf_ctx* c, const double* mass) {
  if (!c->tape) return;
  ttgbf_adj* a = c->tape;
  TapeEntry e;
  e.kind = kTNorm;
  char* p = tape_take(a, a->scal_bytes, &e.scal);
  if (!p) return;
  cudaMemcpyAsync(p, mass, sizeof(double) * a->B, cudaMemcpyDeviceToDevice, c->st);
  tape_push(c, e, true);
}

void tape_upd_in(ttgbf_ctx* c) {
  if (!c->tape) return;
  TapeEntry e;
  e.kind = kTUpdIn;
  tape_push(c, e, true);
}

void tape_lik(ttgbf_ctx* c, int comp, const ttgbf_meas_comp& cp, const float* z, int zstride, double R) {
  if (!c->tape) return;
  ttgbf_adj* a = c->tape;
  TapeEntry e;
  e.kind = kTLik;
  e.comp = comp;
  e.nmodes = cp.nmodes;
  e.mode0 = cp.modes[0];
  e.htab = cp.htab;
  e.R = R;
  e.period = (float)cp.period;
  char* p = tape_take(a, a->scal_bytes, &e.scal);
  if (!p) return;
  // z of this component and the factor's offset, per filter (floats)
  cudaMemcpy2DAsync(p, sizeof(float), z + comp, sizeof(float) * (size_t)zstride, sizeof(float), a->B,
                    cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(p + sizeof(float) * a->B, c->lik_off, sizeof(float) * a->B, cudaMemcpyDeviceToDevice,
                  c->st);
  tape_push(c, e, false);
}

void tape_logc(ttgbf_ctx* c, const double* mass) {
  if (!c->tape) return;
  ttgbf_adj* a = c->tape;
  TapeEntry e;
  e.kind = kTLogc;
  char* p = tape_take(a, a->scal_bytes, &e.scal);
  if (!p) return;
  cudaMemcpyAsync(p, mass, sizeof(double) * a->B, cudaMemcpyDeviceToDevice, c->st);
  tape_push(c, e, false);
}

// ---- tensor-train views of the reverse pass
struct TTv {
  const float* p[kMaxD];
  long long cap[kMaxD];
  const int* ranks;
};

TTv snap_view(const ttgbf_adj* a, size_t snap) {
  TTv v{};
  for (int k = 0; k < a->d; ++k) {
    v.p[k] = reinterpret_cast<const float*>(a->tape + snap + a->snap_cores[k]);
    v.cap[k] = a->scap[k];
  }
  v.ranks = reinterpret_cast<const int*>(a->tape + snap + a->snap_ranks);
  return v;
}

TTv lam_view(ttgbf_adj* a) {
  TTv v{};
  for (int k = 0; k < a->d; ++k) {
    v.p[k] = curp(a->lc, k);
    v.cap[k] = a->lc->L.core_cap[k];
  }
  v.ranks = a->lc->ranks;
  return v;
}

// Left environments of X and Y over all cores: <X, Y> per filter into a->val.
void inner(ttgbf_adj* a, const TTv& X, const TTv& Y) {
  ttgbf_ctx* c = a->c;
  int cur = 0;
  for (int k = 0; k < a->d; ++k) {
    launch_env_step(c->st, a->B, k, c->n[k], X.p[k], X.cap[k], X.ranks, Y.p[k], Y.cap[k], Y.ranks, a->d + 1,
                    a->phi[cur], a->phi_max, a->part, a->chunks, a->phi_max, a->err);
    launch_env_reduce(c->st, a->B, k, X.ranks, Y.ranks, a->d + 1, a->part, a->chunks, a->phi_max,
                      a->phi[cur ^ 1], a->phi_max, k == a->d - 1 ? a->val : nullptr, 1.0, 0);
    cur ^= 1;
  }
}

void add_grad(ttgbf_adj* a, int gi) {
  launch_scalars(a->c->st, a->B, 2, nullptr, a->val, 0.0, nullptr, nullptr, a->grad, a->nparams, gi, 1.0);
}

// lambda <- sc lambda + coef 1 (per-filter sc, coef in a->sc, a->coef).
void lam_add_ones(ttgbf_adj* a) {
  ttgbf_ctx* l = a->lc;
  const float* src[kMaxD];
  float* dst[kMaxD];
  for (int k = 0; k < a->d; ++k) {
    src[k] = curp(l, k);
    dst[k] = altp(l, k);
  }
  launch_add_ones(l->st, a->B, a->d, src, l->L.core_cap, l->n.data(), dst, l->L.core_cap, l->ranks, a->d + 1,
                  a->sc, a->coef);
  for (int k = 0; k < a->d; ++k) l->cur[k] ^= 1;
  l->canon = false;
  l->expanded = true;
}

void lam_bound(ttgbf_adj* a) {
  if (a->lc->expanded) enqueue_round(a->lc);
}

// Operator tables of the reverse pass (float, uploaded at every backward call).
struct AdjMats {
  long long convT[kMaxD], convDq[kMaxD], convDl[kMaxD], scaleT[kMaxD], scaleD[kMaxD];
  std::vector<long long> wT, wD;  // per op: weights of S(-a), of dS/da
  std::vector<int> ST, tT;        // per op: span and first shift of S(-a)
};

void cic_derivative(ttgbf_ctx* c, int m, double lam, std::vector<double>* W) {
  const int N = c->n[m];
  W->assign((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) {
    const double xi = c->axes[c->axoff[m] + i];
    const double u = (lam * xi - c->lo[m]) / c->dx[m] - 0.5;
    for (int j = 0; j < N; ++j) {
      const double t = j - u;
      if (std::fabs(t) < 1.0 && t != 0.0) (*W)[(size_t)j * N + i] = (t > 0 ? 1.0 : -1.0) * xi / c->dx[m];
    }
  }
}

void conv_derivative(ttgbf_ctx* c, int m, double q, std::vector<double>* K) {
  conv_matrix(c, m, q, K);
  const int N = c->n[m];
  const double D = c->dx[m];
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      const double t = (double)(j - i) * D;
      (*K)[(size_t)j * N + i] *= -0.5 / q + 0.5 * t * t / (q * q);
    }
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int N) {
  std::vector<double> C((size_t)N * N, 0.0);
  for (int j = 0; j < N; ++j)
    for (int l = 0; l < N; ++l) {
      const double x = A[(size_t)j * N + l];
      if (x == 0.0) continue;
      for (int i = 0; i < N; ++i) C[(size_t)j * N + i] += x * B[(size_t)l * N + i];
    }
  return C;
}

int build_mats(ttgbf_adj* a, AdjMats* M) {
  ttgbf_ctx* c = a->c;
  const int d = c->d;
  std::vector<float> host;
  auto put = [&](const std::vector<double>& X, bool transpose, int N) -> long long {
    const long long at = (long long)host.size();
    host.resize(host.size() + (size_t)N * N);
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i)
        host[at + (size_t)j * N + i] = (float)(transpose ? X[(size_t)i * N + j] : X[(size_t)j * N + i]);
    return at;
  };
  std::vector<double> Dm(d, 1.0);
  for (const Op& op : c->ops)
    if (op.kind == 1) Dm[op.m] = op.a;
  for (int m = 0; m < d; ++m) {
    const int N = c->n[m];
    const double q = c->lastQ[(size_t)m * d + m];
    std::vector<double> K, dK, W, dW;
    conv_matrix(c, m, q, &K);
    conv_derivative(c, m, q, &dK);
    cic_matrix(c, m, Dm[m], &W);
    cic_derivative(c, m, Dm[m], &dW);
    if (c->fuse && Dm[m] != 1.0) {
      M->convT[m] = put(matmul(K, W, N), true, N);
      M->convDq[m] = put(matmul(dK, W, N), false, N);
      M->convDl[m] = put(matmul(K, dW, N), false, N);
    } else {
      M->convT[m] = put(K, true, N);
      M->convDq[m] = put(dK, false, N);
      M->convDl[m] = -1;
    }
    M->scaleT[m] = put(W, true, N);
    M->scaleD[m] = put(dW, false, N);
  }
  M->wT.assign(c->ops.size(), -1);
  M->wD.assign(c->ops.size(), -1);
  M->ST.assign(c->ops.size(), 0);
  M->tT.assign(c->ops.size(), 0);
  for (size_t i = 0; i < c->ops.size(); ++i) {
    const Op& op = c->ops[i];
    if (op.kind != 0) continue;
    int S, tmin;
    std::vector<float> w;
    shear_table(c, op.m, op.n, -op.a, &S, &tmin, &w);
    if (S > a->lc->smax * a->lc->smax) return TTGBF_ECAPACITY;
    M->ST[i] = S;
    M->tT[i] = tmin;
    M->wT[i] = (long long)host.size();
    host.insert(host.end(), w.begin(), w.end());
    // derivative of the forward weights hat(t - s_i), s_i = a xi_{n,i} / D_m
    const int Nn = c->n[op.n], Sf = c->op_S[i], tf = c->op_tmin[i];
    M->wD[i] = (long long)host.size();
    for (int u = 0; u < Sf; ++u)
      for (int j = 0; j < Nn; ++j) {
        const double xi = c->axes[c->axoff[op.n] + j];
        const double t = (tf + u) - op.a * xi / c->dx[op.m];
        host.push_back(std::fabs(t) < 1.0 && t != 0.0 ? (float)((t > 0 ? 1.0 : -1.0) * xi / c->dx[op.m]) : 0.f);
      }
  }
  if ((long long)host.size() > a->mats_floats) return TTGBF_ECAPACITY;
  if (cudaMemcpyAsync(a->mats, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice, c->st) !=
      cudaSuccess)
    return TTGBF_ECUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return TTGBF_ECUDA;  // host is freed on return
  return TTGBF_OK;
}

TTGeom scratch_geom(const ttgbf_adj* a) {
  TTGeom g{};
  g.d = a->d;
  for (int k = 0; k < a->d; ++k) {
    g.n[k] = a->c->n[k];
    g.cap[k] = a->lcap[k];
  }
  return g;
}

const float* lik_z(const ttgbf_adj* a, const TapeEntry& e) {
  return reinterpret_cast<const float*>(a->tape + e.scal);
}
const float* lik_off(const ttgbf_adj* a, const TapeEntry& e) { return lik_z(a, e) + a->B; }

// ---- the reverse steps
void back_norm(ttgbf_adj* a, const TapeEntry& e) {
  ttgbf_ctx* c = a->c;
  lam_bound(a);  // ranks back to the cap before they grow again
  inner(a, snap_view(a, e.snap), lam_view(a));
  launch_scalars(c->st, a->B, 0, reinterpret_cast<const double*>(a->tape + e.scal), a->val, c->delta, a->sc,
                 a->coef, nullptr, 0, 0, 0.0);
  lam_add_ones(a);
}

void back_logc(ttgbf_adj* a, const TapeEntry& e) {
  ttgbf_ctx* c = a->c;
  launch_scalars(c->st, a->B, 1, reinterpret_cast<const double*>(a->tape + e.scal), nullptr, c->delta, a->sc,
                 a->coef, nullptr, 0, 0, 0.0);
  lam_add_ones(a);
}

// lambda <- Lambda (.) lambda with the factor as the forward pass applied it:
// a one-mode factor scales a core's slices, the two-mode factor multiplies
// the merged cores 0, 1, which the split of the rounding then separates.
void back_lik(ttgbf_adj* a, const TapeEntry& e) {
  ttgbf_ctx* l = a->lc;
  const int B = a->B, d = a->d;
  if (e.nmodes == 1) {
    const int k = e.mode0;
    launch_lik_apply_1d(l->st, B, curp(l, k), l->L.core_cap[k], l->n[k], k, d, l->ranks, e.htab, lik_z(a, e), 1,
                        0, e.R, e.period, lik_off(a, e));
    if (!(l->canon && l->center == k)) l->canon = false;
    return;
  }
  lam_bound(a);  // the merged core holds ranks up to the cap only
  for (int k = d - 1; k >= 2; --k) stage(l, kStageRight, k, 0);
  GemmWork gw = gemm_work(l, B);
  launch_plan_supercore(l->st, B, l->geom, l->ranks, curp(l, 0), curp(l, 1), l->W, l->L.W_cap, gw);
  launch_gemm(l->st, gw, l->sms * 8, flops_of(l, kPGemm));
  launch_lik_apply_2d(l->st, B, l->W, l->L.W_cap, l->n[0], l->n[1], l->ranks, d, e.htab, lik_z(a, e), 1, 0, e.R,
                      e.period, lik_off(a, e));
  stage(l, kStageSplit, 0, 1);
  for (int k = 1; k <= d - 2; ++k) stage(l, kStageLeft, k, 0);
  l->canon = true;
  l->center = d - 1;
  l->expanded = false;
}

// dl/dR_c = <g_c (.) lambda, w> for every likelihood factor of the update
// (lambda the adjoint of the update's input, w that input).
void back_upd_in(ttgbf_adj* a, const TapeEntry& e, const std::vector<TapeEntry>& liks) {
  ttgbf_ctx* l = a->lc;
  const int B = a->B, d = a->d;
  const TTv w = snap_view(a, e.snap);
  for (const TapeEntry& f : liks) {
    TTv Y = lam_view(a);
    if (f.nmodes == 1) {
      const int k = f.mode0;
      launch_lik1(l->st, B, k, l->n[k], curp(l, k), l->L.core_cap[k], a->sB[k], a->lcap[k], l->ranks, d + 1,
                  f.htab, lik_z(a, f), lik_off(a, f), f.R, f.period, 1);
      Y.p[k] = a->sB[k];
      Y.cap[k] = a->lcap[k];
    } else {
      cudaMemcpyAsync(a->sranks, l->ranks, sizeof(int) * (size_t)B * (d + 1), cudaMemcpyDeviceToDevice, l->st);
      launch_lik2_split(l->st, B, l->n[0], l->n[1], curp(l, 0), l->L.core_cap[0], curp(l, 1), l->L.core_cap[1],
                        a->sA[0], a->lcap[0], a->sB[1], a->lcap[1], a->sranks, d + 1, f.htab, lik_z(a, f),
                        lik_off(a, f), f.R, f.period, 1);
      Y.p[0] = a->sA[0];
      Y.p[1] = a->sB[1];
      Y.cap[0] = a->lcap[0];
      Y.cap[1] = a->lcap[1];
      Y.ranks = a->sranks;
    }
    inner(a, w, Y);
    add_grad(a, d * d + d + f.comp);
  }
}

void back_mode(ttgbf_adj* a, const TapeEntry& e, const AdjMats& M) {
  ttgbf_ctx* c = a->c;
  const int k = e.k, d = a->d, N = c->n[k];
  const TTv y = snap_view(a, e.snap);
  auto grad_of = [&](long long moff, int gi) {
    launch_mode(c->st, a->B, k, N, a->mats + moff, y.p[k], a->scap[k], a->sB[k], a->lcap[k], y.ranks, d + 1);
    TTv X = y;
    X.p[k] = a->sB[k];
    X.cap[k] = a->lcap[k];
    inner(a, X, lam_view(a));
    add_grad(a, gi);
  };
  long long mt;
  if (e.mkind == kModeScale) {
    grad_of(M.scaleD[k], k * d + k);
    mt = M.scaleT[k];
  } else {
    grad_of(M.convDq[k], d * d + k);
    if (e.mkind == kModeConvScale) grad_of(M.convDl[k], k * d + k);
    mt = M.convT[k];
  }
  mode_apply(a->lc, k, a->mats + mt);
}

void back_shear(ttgbf_adj* a, const TapeEntry& e, const AdjMats& M) {
  ttgbf_ctx* c = a->c;
  const int m = e.k, n = e.n, d = a->d, lo = std::min(m, n), hi = std::max(m, n);
  const TTv y = snap_view(a, e.snap);
  const TTGeom g = scratch_geom(a);
  // <lambda, (dS/da) y>, the shifts taken in pieces of at most smax (dS/da is
  // a sum over the shifts): the block of y at scratch strides, expanded with
  // the derivative weights of the piece
  launch_copy_cores(c->st, a->B, lo, hi + 1, y.p, y.cap, c->n.data(), y.ranks, d + 1, a->sA, a->lcap);
  const int Sf = c->op_S[e.op], tf = c->op_tmin[e.op], Nn = c->n[n];
  for (int u0 = 0; u0 < Sf; u0 += c->smax) {
    const int Sp = std::min(c->smax, Sf - u0);
    cudaMemcpyAsync(a->sranks, y.ranks, sizeof(int) * (size_t)a->B * (d + 1), cudaMemcpyDeviceToDevice, c->st);
    launch_shear_expand(c->st, a->B, g, m, n, Sp, tf + u0, a->mats + M.wD[e.op] + (long long)u0 * Nn, a->sA,
                        a->sB, a->sranks, 0);
    launch_rank_scale(c->st, a->B, d, a->sranks, lo, hi, Sp);
    TTv Y = y;
    for (int k = lo; k <= hi; ++k) {
      Y.p[k] = a->sB[k];
      Y.cap[k] = a->lcap[k];
    }
    Y.ranks = a->sranks;
    inner(a, lam_view(a), Y);
    add_grad(a, m * d + n);
  }
  // lambda <- S(-a) lambda, rounded on the block as the forward shear is
  lam_bound(a);
  enqueue_shear(a->lc, m, n, M.ST[e.op], M.tT[e.op], a->mats + M.wT[e.op], true);
}

// Gradient with respect to F from the gradients with respect to the
// strictly lower L, diagonal D and strictly upper U of F = L D U: with
// X = L^{-1} dF U^{-1} one has dL = L tril(X) D^{-1}, dD = diag(X),
// dU = D^{-1} triu(X) U, so G_X = tril(L^T G_L D^{-1}) + diag(G_D) +
// triu(D^{-1} G_U U^T) and G_F = L^{-T} G_X U^{-T}.
int ldu_adjoint(int d, const double* F, const double* GL, const double* GD, const double* GU, double* GF) {
  std::vector<double> L, D, U;
  const int rc = ldu(F, d, &L, &D, &U);
  if (rc) return rc;
  auto at = [d](std::vector<double>& A, int i, int j) -> double& { return A[(size_t)i * d + j]; };
  std::vector<double> GX((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      if (i > j) {
        for (int l = 0; l < d; ++l) s += L[(size_t)l * d + i] * GL[(size_t)l * d + j];  // (L^T G_L)_ij
        s /= D[j];
      } else if (i < j) {
        for (int l = 0; l < d; ++l) s += GU[(size_t)i * d + l] * U[(size_t)j * d + l];  // (G_U U^T)_ij
        s /= D[i];
      } else {
        s = GD[i];
      }
      at(GX, i, j) = s;
    }
  std::vector<double> Li((size_t)d * d, 0.0), Ui((size_t)d * d, 0.0);  // L^{-1}, U^{-1}
  for (int j = 0; j < d; ++j) {
    at(Li, j, j) = 1.0;
    for (int i = j + 1; i < d; ++i) {
      double s = 0.0;
      for (int l = j; l < i; ++l) s += L[(size_t)i * d + l] * at(Li, l, j);
      at(Li, i, j) = -s;
    }
  }
  for (int i = 0; i < d; ++i) {
    at(Ui, i, i) = 1.0;
    for (int j = i + 1; j < d; ++j) {
      double s = 0.0;
      for (int l = i; l < j; ++l) s += at(Ui, i, l) * U[(size_t)l * d + j];
      at(Ui, i, j) = -s;
    }
  }
  std::vector<double> T((size_t)d * d, 0.0);  // G_X U^{-T}
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int l = 0; l < d; ++l) s += at(GX, i, l) * at(Ui, j, l);
      at(T, i, j) = s;
    }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int l = 0; l < d; ++l) s += at(Li, l, i) * at(T, l, j);
      GF[(size_t)i * d + j] = s;
    }
  return TTGBF_OK;
}

int adj_guard(ttgbf_adj* a) {
  if (!a || !a->c || !a->lc) return TTGBF_EINVAL;
  if (a->c->poisoned || a->lc->poisoned) return TTGBF_EPOISONED;
  return TTGBF_OK;
}

}  // namespace

extern "C" {

int ttgbf_adj_create(ttgbf_adj** out, ttgbf_ctx* c, int32_t steps, int32_t slots) {
  if (!out) return TTGBF_EINVAL;
  *out = nullptr;
  int rc = guard(c);
  if (rc) return rc;
  if (!c->parts.empty() || c->d < 2 || steps < 1 || slots < 0) return TTGBF_EINVAL;
  ttgbf_adj* a = new (std::nothrow) ttgbf_adj;
  if (!a) return TTGBF_ENOMEM;
  const int d = c->d, B = c->B, cap = c->rank_cap, smax = c->smax;
  a->c = c;
  a->B = B;
  a->d = d;
  // the adjoint density: a context of the same grid, batch, rank cap and eps
  {
    std::vector<int32_t> n(c->n.begin(), c->n.end());
    std::vector<double> mean(d, 0.0), var(d, 1.0);
    ttgbf_grid g{d, n.data(), c->lo.data(), c->hi.data()};
    ttgbf_prior p{mean.data(), var.data()};
    ttgbf_opts o{};
    o.batch = B;
    o.rank_cap = cap;
    o.eps = c->eps;
    o.max_shift_span = smax;
    o.stream = c->st;
    o.precision = c->precision;
    o.contraction = c->contract;
    o.conv = TTGBF_CONV_DENSE;
    o.parts = 1;
    o.tsqr_slice_blocks = c->slice_blocks;
    o.svd_threads = c->svd_threads;
    rc = init_single(&a->lc, &g, &p, &o);
    if (rc) {
      delete a;
      return rc;
    }
  }
  a->RS = cap + 2;
  a->RL = std::max(c->n[0] + 2, cap * smax + 2);
  a->phi_max = a->RS * a->RL;
  a->nparams = d * d + d + kMaxComps;
  int nmax = 0;
  for (int k = 0; k < d; ++k) {
    nmax = std::max(nmax, c->n[k]);
    a->scap[k] = (long long)(k == 0 ? 1 : cap) * c->n[k] * (k == d - 1 ? 1 : cap);
    a->lcap[k] = (long long)(k == 0 ? 1 : a->RL) * c->n[k] * (k == d - 1 ? 1 : a->RL);
  }
  size_t off = 0;
  for (int k = 0; k < d; ++k) {
    a->snap_cores[k] = off;
    off += align256(sizeof(float) * (size_t)B * a->scap[k]);
  }
  a->snap_ranks = off;
  off += align256(sizeof(int) * (size_t)B * (d + 1));
  a->snap_bytes = off;
  a->scal_bytes = align256(sizeof(double) * (size_t)B);
  // per step: the shears' inputs, the per-mode operators' inputs (scalings
  // and kernels), two normalisations and the update's input
  const size_t snaps_per_step = (size_t)d * (d - 1) + 2 * (size_t)d + 3;
  a->tape_cap = (size_t)steps * (snaps_per_step * a->snap_bytes + (3 + kMaxComps) * a->scal_bytes);
  a->nslots = slots;
  a->ckpt_bytes = a->snap_bytes + a->scal_bytes;
  a->ckh.assign((size_t)slots, CkptHost{});
  a->mats_floats = 0;
  for (int k = 0; k < d; ++k) a->mats_floats += 5LL * c->n[k] * c->n[k];
  a->mats_floats += (long long)d * (d - 1) * (smax * smax + smax + 2) * nmax;
  Arena ar;
  const size_t o_tape = ar.take<char>(a->tape_cap);
  const size_t o_ckpt = ar.take<char>((size_t)slots * a->ckpt_bytes);
  size_t o_sA[kMaxD], o_sB[kMaxD];
  for (int k = 0; k < d; ++k) o_sA[k] = ar.take<float>((size_t)B * a->lcap[k]);
  for (int k = 0; k < d; ++k) o_sB[k] = ar.take<float>((size_t)B * a->lcap[k]);
  const size_t o_sr = ar.take<int>((size_t)B * (d + 1));
  const size_t o_phi0 = ar.take<float>((size_t)B * a->phi_max);
  const size_t o_phi1 = ar.take<float>((size_t)B * a->phi_max);
  const size_t o_part = ar.take<float>((size_t)B * a->chunks * a->phi_max);
  const size_t o_err = ar.take<int>(1);
  const size_t o_val = ar.take<double>(B), o_sc = ar.take<double>(B), o_coef = ar.take<double>(B);
  const size_t o_grad = ar.take<double>((size_t)B * a->nparams);
  const size_t o_mats = ar.take<float>((size_t)a->mats_floats);
  if (cudaMalloc(&a->base, ar.off + 256) != cudaSuccess) {
    cudaGetLastError();
    ttgbf_free(a->lc);
    delete a;
    return TTGBF_ENOMEM;
  }
  char* b = a->base;
  a->tape = b + o_tape;
  a->ckpt = b + o_ckpt;
  for (int k = 0; k < d; ++k) {
    a->sA[k] = reinterpret_cast<float*>(b + o_sA[k]);
    a->sB[k] = reinterpret_cast<float*>(b + o_sB[k]);
  }
  a->sranks = reinterpret_cast<int*>(b + o_sr);
  a->phi[0] = reinterpret_cast<float*>(b + o_phi0);
  a->phi[1] = reinterpret_cast<float*>(b + o_phi1);
  a->part = reinterpret_cast<float*>(b + o_part);
  a->err = reinterpret_cast<int*>(b + o_err);
  a->val = reinterpret_cast<double*>(b + o_val);
  a->sc = reinterpret_cast<double*>(b + o_sc);
  a->coef = reinterpret_cast<double*>(b + o_coef);
  a->grad = reinterpret_cast<double*>(b + o_grad);
  a->mats = reinterpret_cast<float*>(b + o_mats);
  *out = a;
  rc = ttgbf_adj_reset(a);
  if (rc) {
    ttgbf_adj_free(a);
    *out = nullptr;
  }
  return rc;
}

int ttgbf_adj_free(ttgbf_adj* a) {
  if (!a) return TTGBF_OK;
  if (a->c && a->c->tape == a) a->c->tape = nullptr;
  if (a->c && a->c->st) cudaStreamSynchronize(a->c->st);
  if (a->base) cudaFree(a->base);
  if (a->lc) ttgbf_free(a->lc);
  cudaGetLastError();
  delete a;
  return TTGBF_OK;
}

int ttgbf_adj_reset(ttgbf_adj* a) {
  int rc = adj_guard(a);
  if (rc) return rc;
  ttgbf_ctx* c = a->c;
  ttgbf_ctx* l = a->lc;
  // lambda = 0: rank-1 cores of zeros
  for (int k = 0; k < a->d; ++k)
    cudaMemset2DAsync(curp(l, k), sizeof(float) * l->L.core_cap[k], 0, sizeof(float) * l->n[k], a->B, c->st);
  std::vector<int> ones((size_t)a->B * (a->d + 1), 1);
  cudaMemcpyAsync(l->ranks, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemsetAsync(a->grad, 0, sizeof(double) * (size_t)a->B * a->nparams, c->st);
  cudaMemsetAsync(a->err, 0, sizeof(int), c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);  // ones is freed on return
  l->canon = false;
  l->expanded = false;
  l->center = 0;
  for (int k = 0; k < kMaxD; ++k) l->virt_S[k] = 0;
  a->entries.clear();
  a->tape_used = 0;
  a->failed = false;
  return check(c);
}

int ttgbf_adj_save(ttgbf_adj* a, int32_t slot) {
  int rc = adj_guard(a);
  if (rc) return rc;
  ttgbf_ctx* c = a->c;
  if (slot < 0 || slot >= a->nslots || a->recording || c->expanded) return TTGBF_EINVAL;
  char* dst = a->ckpt + (size_t)slot * a->ckpt_bytes;
  snap_state(a, dst);
  cudaMemcpyAsync(dst + a->snap_bytes, c->log_lik, sizeof(double) * a->B, cudaMemcpyDeviceToDevice, c->st);
  CkptHost& h = a->ckh[slot];
  h.valid = true;
  h.canon = c->canon;
  h.expanded = c->expanded;
  h.center = c->center;
  return check(c);
}

int ttgbf_adj_load(ttgbf_adj* a, int32_t slot) {
  int rc = adj_guard(a);
  if (rc) return rc;
  ttgbf_ctx* c = a->c;
  if (slot < 0 || slot >= a->nslots || a->recording || !a->ckh[slot].valid) return TTGBF_EINVAL;
  const char* src = a->ckpt + (size_t)slot * a->ckpt_bytes;
  for (int k = 0; k < a->d; ++k)
    cudaMemcpy2DAsync(curp(c, k), sizeof(float) * c->L.core_cap[k], src + a->snap_cores[k],
                      sizeof(float) * a->scap[k], sizeof(float) * a->scap[k], a->B, cudaMemcpyDeviceToDevice,
                      c->st);
  cudaMemcpyAsync(c->ranks, src + a->snap_ranks, sizeof(int) * (size_t)a->B * (a->d + 1),
                  cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->log_lik, src + a->snap_bytes, sizeof(double) * a->B, cudaMemcpyDeviceToDevice, c->st);
  const CkptHost& h = a->ckh[slot];
  c->canon = h.canon;
  c->expanded = h.expanded;
  c->center = h.center;
  for (int k = 0; k < kMaxD; ++k) c->virt_S[k] = 0;
  return check(c);
}

int ttgbf_adj_record(ttgbf_adj* a, int32_t on) {
  int rc = adj_guard(a);
  if (rc) return rc;
  if (on) {
    if (a->c->tape && a->c->tape != a) return TTGBF_EINVAL;
    a->entries.clear();
    a->tape_used = 0;
    a->failed = false;
    a->recording = true;
    a->c->tape = a;
  } else {
    a->recording = false;
    if (a->c->tape == a) a->c->tape = nullptr;
  }
  return TTGBF_OK;
}

int ttgbf_adj_backward(ttgbf_adj* a) {
  int rc = adj_guard(a);
  if (rc) return rc;
  if (a->recording) return TTGBF_EINVAL;
  if (a->failed) {
    a->entries.clear();
    a->tape_used = 0;
    return TTGBF_ECAPACITY;
  }
  ttgbf_ctx* c = a->c;
  AdjMats M;
  rc = build_mats(a, &M);
  if (rc) return rc == TTGBF_ECUDA ? cuda_fail(c) : rc;
  std::vector<TapeEntry> liks;
  for (size_t i = a->entries.size(); i-- > 0;) {
    const TapeEntry& e = a->entries[i];
    switch (e.kind) {
      case kTNorm: back_norm(a, e); break;
      case kTLogc: back_logc(a, e); break;
      case kTLik:
        back_lik(a, e);
        liks.push_back(e);
        break;
      case kTUpdIn:
        back_upd_in(a, e, liks);
        liks.clear();
        break;
      case kTMode: back_mode(a, e, M); break;
      case kTShear: back_shear(a, e, M); break;
      default: break;
    }
  }
  a->entries.clear();
  a->tape_used = 0;
  rc = check(a->lc);
  return rc ? rc : check(c);
}

int ttgbf_adj_grads(ttgbf_adj* a, double* dF, double* dQ, double* dR, int32_t nR) {
  int rc = adj_guard(a);
  if (rc) return rc;
  if (!dF || !dQ || (nR > 0 && !dR) || nR < 0 || nR > kMaxComps) return TTGBF_EINVAL;
  ttgbf_ctx* c = a->c;
  const int d = a->d, B = a->B;
  if (c->lastF.size() != (size_t)d * d) return TTGBF_EINVAL;
  std::vector<double> g((size_t)B * a->nparams);
  int err = 0;
  cudaMemcpyAsync(g.data(), a->grad, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(&err, a->err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c);
  if (err) return TTGBF_ECAPACITY;
  for (int b = 0; b < B; ++b) {
    const double* gb = g.data() + (size_t)b * a->nparams;
    std::vector<double> GL((size_t)d * d, 0.0), GU((size_t)d * d, 0.0), GD(d, 0.0);
    for (int m = 0; m < d; ++m)
      for (int n = 0; n < d; ++n) {
        if (m > n) GL[(size_t)m * d + n] = gb[m * d + n];
        else if (m < n) GU[(size_t)m * d + n] = gb[m * d + n];
        else GD[m] = gb[m * d + m];
      }
    rc = ldu_adjoint(d, c->lastF.data(), GL.data(), GD.data(), GU.data(), dF + (size_t)b * d * d);
    if (rc) return rc;
    for (int m = 0; m < d; ++m) dQ[(size_t)b * d + m] = gb[d * d + m];
    for (int k = 0; k < nR; ++k) dR[(size_t)b * nR + k] = gb[d * d + d + k];
  }
  return TTGBF_OK;
}

int ttgbf_ldu_adjoint(int32_t d, const double* F, const double* GL, const double* GD, const double* GU,
                      double* GF) {
  if (d < 1 || d > kMaxD || !F || !GL || !GD || !GU || !GF) return TTGBF_EINVAL;
  if (!finite_all(F, (size_t)d * d)) return TTGBF_ENONFINITE;
  return ldu_adjoint(d, F, GL, GD, GU, GF);
}

}  // extern "C"
