// adjoint.cu -- kernels of the reverse pass of the filter (the gradient of
// the log-likelihood l = sum_k log c_k, Eq. pmf_filtrace_b, with respect to
// the model F, Q, R).
//
// The reverse pass runs the adjoint recursion of the filter equations
// (transposed transition operators, transposed likelihood product, the
// adjoints of the normalisations and of log c) with the adjoint density held
// as a tensor train and rounded like the forward density; the gradients are
// inner products of the adjoint with the derivative operators applied to the
// forward pass's recorded cores.  The pieces here:
//   * environments: Phi_{k+1} = sum_i X_k(:,i,:)^T Phi_k Y_k(:,i,:), the left
//     contraction of two tensor trains (an inner product), split over the
//     grid index into chunks and reduced;
//   * a dense operator on one core's grid index (the derivatives of the
//     Gaussian kernel and of the cloud-in-cell scaling);
//   * the TT sum with the all-ones tensor (the adjoints of normalisation and
//     of log c);
//   * the likelihood factors (and their derivative in R) on one core or on
//     the merged cores 0, 1 (written as an exact split with an identity core).
// The transposed shear is the shear with the opposite coefficient; it and the
// transposed kernels use the forward kernels.
#include <math.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

// ----------------------------------------------------------- environments
// One chunk of grid indices of core k: part[b][chunk] = sum over i in the
// chunk of X_k(:,i,:)^T Phi Y_k(:,i,:), with Phi (rx x ry) the environment
// before core k ([1] when k = 0).  Ranks: rx = xr[k], rx' = xr[k+1], ry, ry'
// likewise.  Every product is held to phi_max floats; a larger one sets *err
// and leaves its chunk zero.
__global__ void k_env_step(int B, int k, int n, const float* __restrict__ X, long long xcap,
                           const int* __restrict__ xr, const float* __restrict__ Y, long long ycap,
                           const int* __restrict__ yr, int rstride, const float* __restrict__ Phi,
                           long long phi_stride, float* __restrict__ part, int chunks, int phi_max,
                           int* err) {
  extern __shared__ float sm[];
  const int b = blockIdx.y, ch = blockIdx.x;
  if (b >= B || ch >= chunks) return;
  const int rx = xr[(long long)b * rstride + k], rx1 = xr[(long long)b * rstride + k + 1];
  const int ry = yr[(long long)b * rstride + k], ry1 = yr[(long long)b * rstride + k + 1];
  float* out = part + ((long long)b * chunks + ch) * phi_max;
  float* P = sm;                // rx x ry
  float* T = sm + phi_max;      // rx x ry1
  float* A = sm + 2 * phi_max;  // rx1 x ry1 accumulator
  const bool fits = (long long)rx * ry <= phi_max && (long long)rx * ry1 <= phi_max &&
                    (long long)rx1 * ry1 <= phi_max;
  if (!fits) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    for (int e = threadIdx.x; e < phi_max; e += blockDim.x) out[e] = 0.f;
    return;
  }
  const float* Xb = X + (long long)b * xcap;
  const float* Yb = Y + (long long)b * ycap;
  if (k == 0) {
    if (threadIdx.x == 0) P[0] = 1.f;
  } else {
    for (int e = threadIdx.x; e < rx * ry; e += blockDim.x) P[e] = Phi[(long long)b * phi_stride + e];
  }
  for (int e = threadIdx.x; e < rx1 * ry1; e += blockDim.x) A[e] = 0.f;
  __syncthreads();
  const int i0 = (int)((long long)n * ch / chunks), i1 = (int)((long long)n * (ch + 1) / chunks);
  for (int i = i0; i < i1; ++i) {
    // T = Phi Y_i   (Y_i(alpha, alpha') = Y[(alpha n + i) ry1 + alpha'])
    for (int e = threadIdx.x; e < rx * ry1; e += blockDim.x) {
      const int be = e / ry1, ap = e - be * ry1;
      const float* pr = P + be * ry;
      const float* yc = Yb + (long long)i * ry1 + ap;
      const long long ys = (long long)n * ry1;
      float acc = 0.f;
      for (int al = 0; al < ry; ++al) acc = fmaf(pr[al], __ldg(yc + al * ys), acc);
      T[e] = acc;
    }
    __syncthreads();
    // A += X_i^T T   (X_i(beta, beta') = X[(beta n + i) rx1 + beta'])
    for (int e = threadIdx.x; e < rx1 * ry1; e += blockDim.x) {
      const int bp = e / ry1, ap = e - bp * ry1;
      const float* xc = Xb + (long long)i * rx1 + bp;
      const long long xs = (long long)n * rx1;
      float acc = A[e];
      for (int be = 0; be < rx; ++be) acc = fmaf(__ldg(xc + be * xs), T[be * ry1 + ap], acc);
      A[e] = acc;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rx1 * ry1; e += blockDim.x) out[e] = A[e];
}

// Phi'[b] = sum over chunks of part[b][.] (rx' x ry' entries).  At the last
// core (both ranks 1) the scalar is also written to scal[b] (times mul, added
// when accumulate).
__global__ void k_env_reduce(int B, int k, const int* __restrict__ xr, const int* __restrict__ yr,
                             int rstride, const float* __restrict__ part, int chunks, int phi_max,
                             float* __restrict__ Phi_out, long long phi_stride, double* scal, double mul,
                             int accumulate) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int rx1 = xr[(long long)b * rstride + k + 1], ry1 = yr[(long long)b * rstride + k + 1];
  const long long cnt = (long long)rx1 * ry1;
  if (cnt > phi_max) return;  // flagged by the step kernel
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[((long long)b * chunks + c) * phi_max + e];
    Phi_out[(long long)b * phi_stride + e] = (float)s;
    if (scal != nullptr && cnt == 1) {
      if (accumulate) scal[b] += mul * s;
      else scal[b] = mul * s;
    }
  }
}

// ------------------------------------------------------ core copies, ranks
struct PtrSet {
  const float* p[kMaxD];
  long long cap[kMaxD];
  int n[kMaxD];
};
struct MutPtrSet {
  float* p[kMaxD];
  long long cap[kMaxD];
};

// dst core k <- src core k for k in [k0, k1) (the used part, from src's ranks).
__global__ void k_copy_cores(int B, int k0, PtrSet src, const int* sr, int rstride, MutPtrSet dst) {
  const int b = blockIdx.z, k = k0 + blockIdx.y;
  if (b >= B) return;
  const long long cnt = (long long)sr[(long long)b * rstride + k] * src.n[k] * sr[(long long)b * rstride + k + 1];
  if (cnt > dst.cap[k]) return;
  const float* s = src.p[k] + (long long)b * src.cap[k];
  float* t = dst.p[k] + (long long)b * dst.cap[k];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x)
    t[e] = s[e];
}

// ---------------------------------------------------- per-mode operator
// out(a, j, c) = sum_i M[j][i] in(a, i, c) on core k (M row-major N x N).
__global__ void k_mode(int B, int k, int N, const float* __restrict__ M, const float* __restrict__ in,
                       long long icap, float* __restrict__ out, long long ocap, const int* __restrict__ ranks,
                       int rstride) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int ra = ranks[(long long)b * rstride + k], rb = ranks[(long long)b * rstride + k + 1];
  const long long total = (long long)ra * N * rb;
  if (total > ocap) return;
  const float* ib = in + (long long)b * icap;
  float* ob = out + (long long)b * ocap;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / ((long long)N * rb);
    const long long rem = e - a * N * rb;
    const int j = (int)(rem / rb), c = (int)(rem - (long long)j * rb);
    const float* mr = M + (long long)j * N;
    const float* col = ib + a * N * rb + c;
    float acc = 0.f;
    for (int i = 0; i < N; ++i) acc = fmaf(__ldg(mr + i), col[(long long)i * rb], acc);
    ob[e] = acc;
  }
}

// ------------------------------------------------ TT sum with all-ones
// out = sc[b] * A  (+)  coef[b] * 1: core 0 = [sc A_0, coef 1], middle cores
// block diagonal diag(A_k, 1), last core = [A_{d-1}; 1].  Ranks of the
// output: r_k + 1 on the inner links (updated by k_ranks_add).
__global__ void k_add_ones(int B, int d, PtrSet src, MutPtrSet dst, const int* __restrict__ ranks,
                           int rstride, const double* __restrict__ sc, const double* __restrict__ coef) {
  const int b = blockIdx.z, k = blockIdx.y;
  if (b >= B || k >= d) return;
  const int ra = ranks[(long long)b * rstride + k], rb = ranks[(long long)b * rstride + k + 1];
  const int N = src.n[k];
  const int oa = k == 0 ? 1 : ra + 1, ob = k == d - 1 ? 1 : rb + 1;
  const long long total = (long long)oa * N * ob;
  if (total > dst.cap[k]) return;
  const float* s = src.p[k] + (long long)b * src.cap[k];
  float* t = dst.p[k] + (long long)b * dst.cap[k];
  const float scb = k == 0 ? (float)sc[b] : 1.f;
  const float cb = (float)coef[b];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long long)N * ob));
    const long long rem = e - (long long)a * N * ob;
    const int i = (int)(rem / ob), c = (int)(rem - (long long)i * ob);
    float v;
    if (k == 0) {
      v = c < rb ? scb * s[(long long)i * rb + c] : cb;
    } else if (k == d - 1) {
      v = a < ra ? s[(long long)a * N + i] : 1.f;
    } else if (a < ra && c < rb) {
      v = s[((long long)a * N + i) * rb + c];
    } else {
      v = (a == ra && c == rb) ? 1.f : 0.f;
    }
    t[e] = v;
  }
}

__global__ void k_set_link(int B, int* ranks, int rstride, int j, int v) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    ranks[(long long)b * rstride + j] = v;
}

__global__ void k_ranks_add(int B, int d, int* ranks, int rstride, int delta) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    for (int j = 1; j < d; ++j) ranks[(long long)b * rstride + j] += delta;
}

// --------------------------------------------------------- likelihoods
// Likelihood factor of one component as the forward pass applies it
// (exp(-((z - h)^2 - off) / (2R)), off the per-filter offset), or
// (which = 1) the derivative of the log of the true likelihood in R,
// -1/(2R) + (z - h)^2 / (2R^2); the residual wrapped for an angle-like
// component (period > 0).
__device__ __forceinline__ float lik_weight(float z, float h, float off, double R, float period, int which) {
  const float df = wrap_residual(z - h, period);
  if (which == 0) return expf(-(df * df - off) * (float)(0.5 / R));
  return (float)(-0.5 / R + (double)df * df * (0.5 / (R * R)));
}

// dst core k = weight(i) * src core k (in place when dst == src).
__global__ void k_lik1(int B, int k, int N, const float* src, long long scap, float* dst, long long dcap,
                       const int* __restrict__ ranks, int rstride, const float* __restrict__ htab,
                       const float* __restrict__ zv, const float* __restrict__ off, double R, float period,
                       int which) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int ra = ranks[(long long)b * rstride + k], rb = ranks[(long long)b * rstride + k + 1];
  const long long total = (long long)ra * N * rb;
  if (total > dcap) return;
  const float zb = zv[b], ob = off[b];
  const float* s = src + (long long)b * scap;
  float* t = dst + (long long)b * dcap;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)((e / rb) % N);
    t[e] = lik_weight(zb, htab[i], ob, R, period, which) * s[e];
  }
}

// The two-mode factor on modes (0, 1) (which as in lik_weight) applied to
// the TT (cores 0, 1 of ranks (1, r1), (r1, r2)), written exactly as core 0 =
// identity (1 x N0 x N0) and core 1 (N0 x N1 x r2) = weight(i0, i1) sum_a
// G0(i0, a) G1(a, i1, :).
__global__ void k_lik2_split(int B, int N0, int N1, const float* __restrict__ g0, long long g0cap,
                             const float* __restrict__ g1, long long g1cap, float* __restrict__ o0,
                             long long o0cap, float* __restrict__ o1, long long o1cap,
                             const int* __restrict__ ranks, int rstride, const float* __restrict__ htab,
                             const float* __restrict__ zv, const float* __restrict__ off, double R,
                             float period, int which) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int r1 = ranks[(long long)b * rstride + 1], r2 = ranks[(long long)b * rstride + 2];
  if ((long long)N0 * N0 > o0cap || (long long)N0 * N1 * r2 > o1cap) return;
  const float zb = zv[b], ob = off[b];
  const float* G0 = g0 + (long long)b * g0cap;
  const float* G1 = g1 + (long long)b * g1cap;
  float* O0 = o0 + (long long)b * o0cap;
  float* O1 = o1 + (long long)b * o1cap;
  const long long total = (long long)N0 * N1 * r2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / r2;  // i0 N1 + i1
    const int c = (int)(e - t * r2);
    const int i0 = (int)(t / N1), i1 = (int)(t - (long long)i0 * N1);
    float acc = 0.f;
    for (int a = 0; a < r1; ++a) acc = fmaf(G0[(long long)i0 * r1 + a], G1[((long long)a * N1 + i1) * r2 + c], acc);
    O1[e] = lik_weight(zb, htab[t], ob, R, period, which) * acc;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N0 * N0;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / N0, j = e - i * N0;
    O0[e] = i == j ? 1.f : 0.f;
  }
}

// ------------------------------------------------------------ scalars
// Per-filter coefficients of the adjoint steps:
//   op 0 (normalisation x = y / m):  sc = 1 / m,  coef = -delta <lambda, x> / m
//   op 1 (log c):                    sc = 1,      coef = delta / c
//   op 2 (gradient):                 grad[b * gstride + gi] += mul * val[b]
__global__ void k_scalars(int B, int op, const double* __restrict__ m, const double* __restrict__ val,
                          double delta, double* sc, double* coef, double* grad, int gstride, int gi,
                          double mul) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    if (op == 0) {
      sc[b] = 1.0 / m[b];
      coef[b] = -delta * val[b] / m[b];
    } else if (op == 1) {
      sc[b] = 1.0;
      coef[b] = delta / m[b];
    } else {
      grad[(long long)b * gstride + gi] += mul * val[b];
    }
  }
}

}  // namespace

// ================================================================ launchers
void launch_env_step(cudaStream_t st, int B, int k, int n, const float* X, long long xcap, const int* xr,
                     const float* Y, long long ycap, const int* yr, int rstride, const float* Phi,
                     long long phi_stride, float* part, int chunks, int phi_max, int* err) {
  count_launches(1);
  const size_t sm = sizeof(float) * 3 * (size_t)phi_max;
  k_env_step<<<dim3(chunks, B), 256, sm, st>>>(B, k, n, X, xcap, xr, Y, ycap, yr, rstride, Phi, phi_stride,
                                               part, chunks, phi_max, err);
}

void launch_env_reduce(cudaStream_t st, int B, int k, const int* xr, const int* yr, int rstride,
                       const float* part, int chunks, int phi_max, float* Phi_out, long long phi_stride,
                       double* scal, double mul, int accumulate) {
  count_launches(1);
  k_env_reduce<<<dim3(8, B), 256, 0, st>>>(B, k, xr, yr, rstride, part, chunks, phi_max, Phi_out, phi_stride,
                                           scal, mul, accumulate);
}

void launch_copy_cores(cudaStream_t st, int B, int k0, int k1, const float* const* src, const long long* scap,
                       const int* n, const int* sr, int rstride, float* const* dst, const long long* dcap) {
  if (k1 <= k0) return;
  PtrSet s{};
  MutPtrSet t{};
  for (int k = k0; k < k1; ++k) {
    s.p[k] = src[k];
    s.cap[k] = scap[k];
    s.n[k] = n[k];
    t.p[k] = dst[k];
    t.cap[k] = dcap[k];
  }
  count_launches(1);
  k_copy_cores<<<dim3(32, k1 - k0, B), 256, 0, st>>>(B, k0, s, sr, rstride, t);
}

void launch_mode(cudaStream_t st, int B, int k, int N, const float* M, const float* in, long long icap,
                 float* out, long long ocap, const int* ranks, int rstride) {
  count_launches(1);
  k_mode<<<dim3(64, B), 256, 0, st>>>(B, k, N, M, in, icap, out, ocap, ranks, rstride);
}

void launch_add_ones(cudaStream_t st, int B, int d, const float* const* src, const long long* scap,
                     const int* n, float* const* dst, const long long* dcap, int* ranks, int rstride,
                     const double* sc, const double* coef) {
  PtrSet s{};
  MutPtrSet t{};
  for (int k = 0; k < d; ++k) {
    s.p[k] = src[k];
    s.cap[k] = scap[k];
    s.n[k] = n[k];
    t.p[k] = dst[k];
    t.cap[k] = dcap[k];
  }
  count_launches(2);
  k_add_ones<<<dim3(16, d, B), 256, 0, st>>>(B, d, s, t, ranks, rstride, sc, coef);
  k_ranks_add<<<(B + 127) / 128, 128, 0, st>>>(B, d, ranks, rstride, 1);
}

void launch_lik1(cudaStream_t st, int B, int k, int N, const float* src, long long scap, float* dst,
                 long long dcap, const int* ranks, int rstride, const float* htab, const float* zv,
                 const float* off, double R, float period, int which) {
  count_launches(1);
  k_lik1<<<dim3(16, B), 256, 0, st>>>(B, k, N, src, scap, dst, dcap, ranks, rstride, htab, zv, off, R, period,
                                      which);
}

void launch_lik2_split(cudaStream_t st, int B, int N0, int N1, const float* g0, long long g0cap,
                       const float* g1, long long g1cap, float* o0, long long o0cap, float* o1,
                       long long o1cap, int* ranks, int rstride, const float* htab, const float* zv,
                       const float* off, double R, float period, int which) {
  count_launches(2);
  k_lik2_split<<<dim3(64, B), 256, 0, st>>>(B, N0, N1, g0, g0cap, g1, g1cap, o0, o0cap, o1, o1cap, ranks,
                                            rstride, htab, zv, off, R, period, which);
  // link 1 now carries the grid index of mode 0
  k_set_link<<<(B + 127) / 128, 128, 0, st>>>(B, ranks, rstride, 1, N0);
}

void launch_scalars(cudaStream_t st, int B, int op, const double* m, const double* val, double delta,
                    double* sc, double* coef, double* grad, int gstride, int gi, double mul) {
  count_launches(1);
  k_scalars<<<(B + 127) / 128, 128, 0, st>>>(B, op, m, val, delta, sc, coef, grad, gstride, gi, mul);
}

void set_adjoint_attributes() {
  cudaFuncSetAttribute(k_env_step, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace ttgbf
