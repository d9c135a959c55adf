// fftconv.cu -- the Gaussian transition kernel of the predictive step as a
// batched FFT convolution over every fibre of a core's grid index (Eq.
// tpmconvFFT; the TT convolution of Sec. 4: the kernel acts on the grid index
// of each core alone when Q is diagonal).
//
// Core k of a filter, [r_{k-1}][N][r_k], holds r_{k-1} r_k fibres of length N
// (fixed left and right rank indices).  Each fibre x is replaced by its linear
// convolution with kappa(t) = D N(D t; 0, q), t = -(N-1)..N-1, truncated to
// the grid:  y(j) = sum_i kappa(j - i) x(i).  With M >= 2N - 1 (a power of
// two) the cyclic convolution of length M of x padded with zeros equals it on
// j < N, so y = IFFT(FFT(x) . FFT(kappa_M)) / M.  Two real fibres share one
// complex transform (x_a + i x_b): the kernel is real, so the real and the
// imaginary part of the result are the two convolutions.
//
// When the scaling x_m <- lam x_m of the re-gridding precedes the kernel on
// this mode, its cloud-in-cell matrix (at most kCicTaps source cells per
// target cell) is applied while the fibres are loaded.
//
// A CTA takes 16 fibres (8 complex transforms of length M) at a time:
// Stockham radix-2 passes between two shared-memory buffers (autosorting, no
// bit reversal), twiddles from a table computed in float64 on the host.
#include <math.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kFftThreads = 256;
constexpr int kFftFibres = 16;             // real fibres per item
constexpr int kFftPairs = kFftFibres / 2;  // complex transforms per item

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Forward (inverse = false, exp(-2 pi i ...)) or unscaled inverse transform of
// kFftPairs sequences of length M = 2^logM held at stride MS = M + 1 (the pad
// spreads the sequences' equal indices over the banks) in x; y is the other
// buffer.  Returns the buffer that holds the result.
//
// Stockham pass q (L = 2^q, r = M / L): for j < L/2, k < r,
//   t = w^j x[2 j r + r + k],  y[j r + k] = x[2 j r + k] + t,
//   y[(j + L/2) r + k] = x[2 j r + k] - t,  w = exp(-2 pi i / L).
__device__ float2* fft_pass_all(float2* x, float2* y, int M, int logM, const float2* tw,
                                bool inverse) {
  const int half = M >> 1, MS = M + 1;
  for (int q = 1; q <= logM; ++q) {
    const int lstar = 1 << (q - 1);
    const int rlog = logM - q, r = 1 << rlog;
    for (int t = threadIdx.x; t < kFftPairs * half; t += kFftThreads) {
      const int p = t / half, beta = t - p * half;  // sequence, butterfly
      const int j = beta >> rlog, k = beta & (r - 1);
      float2 w = tw[j << rlog];  // exp(-2 pi i j / L) = tw[j M / L]
      if (inverse) w.y = -w.y;
      const float2* xs = x + p * MS;
      float2* ys = y + p * MS;
      const float2 a = xs[2 * j * r + k];
      const float2 b = cmul(w, xs[2 * j * r + r + k]);
      ys[j * r + k] = make_float2(a.x + b.x, a.y + b.y);
      ys[(j + lstar) * r + k] = make_float2(a.x - b.x, a.y - b.y);
    }
    __syncthreads();
    float2* s = x;
    x = y;
    y = s;
  }
  return x;
}

// Per filter: groups of kFftFibres fibres of core k (exclusive prefix).
__global__ void k_plan_fft(int B, int k, int d, const int* ranks, int* off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < B; ++b) {
    const int* rk = ranks + (long long)b * (d + 1);
    const int nf = rk[k] * rk[k + 1];
    off[b] = acc;
    acc += (nf + kFftFibres - 1) / kFftFibres;
  }
  off[B] = acc;
}

__global__ void __launch_bounds__(kFftThreads) k_conv_fft(int B, int k, int d, int N, int M, int logM,
                                                          const int* ranks, const int* off,
                                                          const float* cur, float* alt,
                                                          long long cap, FftMode md,
                                                          double* flops) {
  extern __shared__ float2 fsm[];
  const int MS = M + 1;
  float2* buf0 = fsm;                       // kFftPairs x MS
  float2* buf1 = fsm + kFftPairs * MS;      // kFftPairs x MS
  float2* tws = buf1 + kFftPairs * MS;      // M / 2 twiddles
  for (int t = threadIdx.x; t < (M >> 1); t += kFftThreads) tws[t] = md.tw[t];
  __syncthreads();
  const int total = off[B];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = B;  // off[lo] <= item < off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= item) lo = mid; else hi = mid;
    }
    const int b = lo;
    const int* rk = ranks + (long long)b * (d + 1);
    const int r0 = rk[k], r1 = rk[k + 1];
    const int nf = r0 * r1;
    const int f0 = (item - off[b]) * kFftFibres;
    const float* G = cur + (long long)b * cap;
    float* Y = alt + (long long)b * cap;
    // ---- load (with the cloud-in-cell gather), zero padding to M
    for (int t = threadIdx.x; t < kFftFibres * M; t += kFftThreads) {
      const int i = t / kFftFibres, phi = t - i * kFftFibres;  // consecutive threads: consecutive fibres
      const int f = f0 + phi;
      float v = 0.f;
      if (i < N && f < nf) {
        const int a = f / r1, c = f - a * r1;
        const float* fib = G + (long long)a * N * r1 + c;
        if (md.gsrc != nullptr) {
#pragma unroll
          for (int s = 0; s < kCicTaps; ++s) {
            const int src = md.gsrc[i * kCicTaps + s];
            if (src >= 0) v = fmaf(md.gw[i * kCicTaps + s], __ldg(fib + (long long)src * r1), v);
          }
        } else {
          v = __ldg(fib + (long long)i * r1);
        }
      }
      float* slot = reinterpret_cast<float*>(buf0 + (phi >> 1) * MS + i);
      slot[phi & 1] = v;
    }
    __syncthreads();
    float2* X = fft_pass_all(buf0, buf1, M, logM, tws, false);
    float2* Wk = X == buf0 ? buf1 : buf0;
    for (int t = threadIdx.x; t < kFftPairs * M; t += kFftThreads) {
      const int p = t / M, u = t - p * M;
      X[p * MS + u] = cmul(X[p * MS + u], md.khat[u]);  // khat carries the 1 / M of the inverse
    }
    __syncthreads();
    float2* Z = fft_pass_all(X, Wk, M, logM, tws, true);
    // ---- store the first N entries of every fibre
    for (int t = threadIdx.x; t < kFftFibres * N; t += kFftThreads) {
      const int j = t / kFftFibres, phi = t - j * kFftFibres;
      const int f = f0 + phi;
      if (f < nf) {
        const int a = f / r1, c = f - a * r1;
        const float* slot = reinterpret_cast<const float*>(Z + (phi >> 1) * MS + j);
        Y[(long long)a * N * r1 + (long long)j * r1 + c] = slot[phi & 1];
      }
    }
    if (threadIdx.x == 0 && flops != nullptr) {
      // two complex transforms (5 M log2 M each) and the spectrum product per pair
      const int nfib = min(kFftFibres, nf - f0);
      atomicAdd(flops, ((nfib + 1) / 2) * (10.0 * M * logM + 6.0 * M));
    }
    __syncthreads();
  }
}

}  // namespace

int fft_smem_bytes(int M) { return (int)sizeof(float2) * (2 * kFftPairs * (M + 1) + M / 2); }

void launch_conv_fft(cudaStream_t st, int B, int k, const TTGeom& g, const int* ranks, int* off,
                     const float* cur, float* alt, const FftMode& md, int grid, double* flops) {
  count_launches(2);
  k_plan_fft<<<1, 32, 0, st>>>(B, k, g.d, ranks, off);
  int logM = 0;
  while ((1 << logM) < md.M) ++logM;
  k_conv_fft<<<grid, kFftThreads, fft_smem_bytes(md.M), st>>>(B, k, g.d, g.n[k], md.M, logM, ranks, off,
                                                              cur, alt, g.cap[k], md, flops);
}

void set_fft_attributes() {
  cudaFuncSetAttribute(k_conv_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       fft_smem_bytes(kMaxFftM));
}

}  // namespace ttgbf
