// noalloc.cu -- moments of TT densities for callers that cannot allocate.
//
// ttgbf_moments_noalloc computes the mass, mean and covariance of a batch of
// TT densities that the caller already holds in device memory, without a
// context and without any allocation: the float64 reduction scratch lives in
// the file-scope array g_moment_scratch below, which every GPU that loads the
// library holds until the process exits.  It serves code that must not call
// cudaMalloc: work recorded into a CUDA graph by a framework that forbids
// allocation while capturing, serving loops with a fixed memory budget, or
// plugins running inside another framework's pre-reserved memory pool.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.cuh"
#include "ttgbf.h"

namespace {

constexpr long long kNoAllocScratchDoubles = TTGBF_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kNoAllocMaxRank = TTGBF_NOALLOC_MAX_RANK;

static __device__ __align__(256) double g_moment_scratch[kNoAllocScratchDoubles];

struct NoAllocArgs {
  int d;
  int n[ttgbf::kMaxD];
  double lo[ttgbf::kMaxD];
  double dx[ttgbf::kMaxD];
  double centre[ttgbf::kMaxD];
  const float* core[ttgbf::kMaxD];
  long long stride[ttgbf::kMaxD];
  int rmax;
};

// One CTA per filter: A_k^(p)(a, b) = sum_i (xi_{k,i} - c_k)^p G_k(a, i, b),
// p <= 2, in float64 scratch, then the vector chains of the moments.  A
// filter whose ranks exceed rmax gets NaN outputs.
__global__ void k_moments_noalloc(int B, NoAllocArgs a, const int* ranks, double* scratch,
                                  double* mass_out, double* mean_out, double* cov_out) {
  constexpr int R = kNoAllocMaxRank;
  __shared__ double f[(ttgbf::kMaxD + 1) * R];
  __shared__ double u[ttgbf::kMaxD * R];
  __shared__ double e[R], tmp[R], red[32];
  __shared__ double s_mean[ttgbf::kMaxD];
  __shared__ double s_S[ttgbf::kMaxD * ttgbf::kMaxD];
  __shared__ int s_bad;
  const int b = blockIdx.x;
  if (b >= B) return;
  const int d = a.d;
  const int* rk = ranks + (long long)b * (d + 1);
  if (threadIdx.x == 0) {
    int bad = (rk[0] != 1 || rk[d] != 1);
    for (int k = 0; k <= d; ++k) bad |= (rk[k] < 1 || rk[k] > a.rmax);
    s_bad = bad;
  }
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      mass_out[b] = NAN;
      for (int k = 0; k < d; ++k) mean_out[(long long)b * d + k] = NAN;
      for (int k = 0; k < d * d; ++k) cov_out[(long long)b * d * d + k] = NAN;
    }
    return;
  }
  const long long Astride = (long long)a.rmax * a.rmax;
  double* Ab = scratch + (long long)b * d * 3 * Astride;
  for (int k = 0; k < d; ++k) {
    const int r0 = rk[k], r1 = rk[k + 1], N = a.n[k];
    const float* G = a.core[k] + (long long)b * a.stride[k];
    for (int q = threadIdx.x; q < r0 * r1; q += blockDim.x) {
      const int al = q / r1, be = q - al * r1;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int i = 0; i < N; ++i) {
        const double v = (double)G[((long long)al * N + i) * r1 + be];
        const double x = a.lo[k] + (i + 0.5) * a.dx[k] - a.centre[k];
        s0 += v;
        s1 += x * v;
        s2 += x * x * v;
      }
      Ab[((long long)k * 3 + 0) * Astride + q] = s0;
      Ab[((long long)k * 3 + 1) * Astride + q] = s1;
      Ab[((long long)k * 3 + 2) * Astride + q] = s2;
    }
  }
  __syncthreads();
  auto A = [&](int k, int p) { return Ab + ((long long)k * 3 + p) * Astride; };
  auto vecmat = [&](const double* x, const double* M, int r0, int r1, double* y) {
    for (int be = threadIdx.x; be < r1; be += blockDim.x) {
      double s = 0.0;
      for (int al = 0; al < r0; ++al) s += x[al] * M[(long long)al * r1 + be];
      y[be] = s;
    }
    __syncthreads();
  };
  auto dot = [&](const double* x, const double* y, int len) {
    double s = 0.0;
    for (int t = threadIdx.x; t < len; t += blockDim.x) s += x[t] * y[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot;
  };
  if (threadIdx.x == 0) f[d * R] = 1.0;
  __syncthreads();
  for (int k = d - 1; k >= 0; --k) {
    const int r0 = rk[k], r1 = rk[k + 1];
    const double* A0 = A(k, 0);
    for (int al = threadIdx.x; al < r0; al += blockDim.x) {
      double s = 0.0;
      for (int be = 0; be < r1; ++be) s += A0[(long long)al * r1 + be] * f[(k + 1) * R + be];
      f[k * R + al] = s;
    }
    __syncthreads();
  }
  const double mraw = f[0];
  if (threadIdx.x == 0) e[0] = 1.0;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    const int r0 = rk[k], r1 = rk[k + 1];
    const double* fr = f + (k + 1) * R;
    vecmat(e, A(k, 2), r0, r1, tmp);
    const double s2 = dot(tmp, fr, r1);
    for (int m = 0; m < k; ++m) {
      vecmat(u + m * R, A(k, 1), r0, r1, tmp);
      const double sc = dot(tmp, fr, r1);
      if (threadIdx.x == 0) s_S[m * ttgbf::kMaxD + k] = sc;
      vecmat(u + m * R, A(k, 0), r0, r1, tmp);
      for (int t = threadIdx.x; t < r1; t += blockDim.x) u[m * R + t] = tmp[t];
      __syncthreads();
    }
    vecmat(e, A(k, 1), r0, r1, tmp);
    const double s1 = dot(tmp, fr, r1);
    for (int t = threadIdx.x; t < r1; t += blockDim.x) u[k * R + t] = tmp[t];
    __syncthreads();
    vecmat(e, A(k, 0), r0, r1, tmp);
    for (int t = threadIdx.x; t < r1; t += blockDim.x) e[t] = tmp[t];
    if (threadIdx.x == 0) {
      s_mean[k] = s1;
      s_S[k * ttgbf::kMaxD + k] = s2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double delta = 1.0;
    for (int k = 0; k < d; ++k) delta *= a.dx[k];
    mass_out[b] = mraw * delta;
    for (int k = 0; k < d; ++k) mean_out[(long long)b * d + k] = a.centre[k] + s_mean[k] / mraw;
    for (int k = 0; k < d; ++k)
      for (int l = k; l < d; ++l) {
        const double v = s_S[k * ttgbf::kMaxD + l] / mraw - (s_mean[k] / mraw) * (s_mean[l] / mraw);
        cov_out[((long long)b * d + k) * d + l] = v;
        cov_out[((long long)b * d + l) * d + k] = v;
      }
  }
}

}  // namespace

extern "C" {

int ttgbf_moments_noalloc(int32_t batch, const ttgbf_grid* grid, const float* const* cores,
                          const int64_t* core_stride, const int32_t* ranks, int32_t rank_max,
                          double* mass, double* mean, double* cov, void* stream) {
  if (!grid || !cores || !core_stride || !ranks || !mass || !mean || !cov) return TTGBF_EINVAL;
  if (batch < 1 || grid->d < 1 || grid->d > ttgbf::kMaxD || !grid->n || !grid->lo || !grid->hi)
    return TTGBF_EINVAL;
  if (rank_max < 1 || rank_max > kNoAllocMaxRank) return TTGBF_ECAPACITY;
  const int d = grid->d;
  NoAllocArgs a{};
  a.d = d;
  a.rmax = rank_max;
  for (int k = 0; k < d; ++k) {
    if (grid->n[k] < 1 || !cores[k] || core_stride[k] < 0) return TTGBF_EINVAL;
    if (!std::isfinite(grid->lo[k]) || !std::isfinite(grid->hi[k])) return TTGBF_ENONFINITE;
    if (!(grid->hi[k] > grid->lo[k])) return TTGBF_EINVAL;
    a.n[k] = grid->n[k];
    a.lo[k] = grid->lo[k];
    a.dx[k] = (grid->hi[k] - grid->lo[k]) / grid->n[k];
    a.centre[k] = 0.5 * (grid->lo[k] + grid->hi[k]);
    a.core[k] = cores[k];
    a.stride[k] = core_stride[k];
  }
  const long long need = (long long)batch * d * 3 * (long long)rank_max * rank_max;
  if (need > kNoAllocScratchDoubles) return TTGBF_ECAPACITY;
  // The array's device address is looked up on every call, with the
  // caller's device current: it is cheap, allocates nothing, and stays right
  // after the primary context was reset (the module is then loaded again,
  // possibly at another address).  In host code the array's name is only a
  // host-side stand-in and must never be passed to a kernel.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_moment_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return TTGBF_ECUDA;
  }
  double* scratch = static_cast<double*>(p);
  ttgbf::count_launches(1);
  k_moments_noalloc<<<batch, 128, 0, (cudaStream_t)stream>>>(batch, a, ranks, scratch, mass, mean, cov);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return TTGBF_ECUDA;
  }
  return TTGBF_OK;
}

}  // extern "C"
