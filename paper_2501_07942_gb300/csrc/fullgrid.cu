// fullgrid.cu -- the plain full-grid point-mass filter on the GPU (float32 or
// float64): the dense density of Sec. 2 (Eq. pdf_pm) on the same grid and with
// the same discrete operators as the TT path, so that both can be compared at
// equal arithmetic.
//
//   predict : F = L D U (no pivoting) -> 2-tap hat shears along one axis with
//             weights depending on another axis -> per-axis N x N operators
//             (cloud-in-cell scaling fused with the Gaussian kernel of
//             Eq. tpmconvFFT), applied over their band of non-negligible
//             entries -> normalise.  Or the textbook direct sum of
//             Eqs. pdf_predII / TPMmat (small grids).
//   update  : P <- L P / c with the likelihood evaluated from h-tables
//             (Eqs. pmf_filtrace_a/b), fused with the reduction of c.
//   estimate: point-mass mean and covariance by one reduction pass.
// Every pass streams the density once: the kernels are bound by HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "ttgbf.h"

namespace {

constexpr int kFgMaxComps = 16;
constexpr int kFgMaxD = 6;  // dense grids beyond d = 6 do not fit in memory
constexpr int kFgAcc = 1 + kFgMaxD + kFgMaxD * kFgMaxD;
constexpr int kFgPredSum = kFgAcc + 1;  // acc slot: sum of the predictive density (fused pass)
constexpr int kFgLikSum = kFgAcc + 2;   // acc slot: sum of L P

// Division by a run-time constant with a multiply-high and a shift
// (Granlund-Montgomery round-up method), exact for every 32-bit dividend.
struct FastDiv {
  uint32_t d, m, l;
};

FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (uint32_t)(((uint64_t)__umulhi(x, f.m) + x) >> f.l);
}

struct FgGeom {
  int d;
  int n[ttgbf::kMaxD];
  long long stride[ttgbf::kMaxD];  // element stride of each axis (C order)
  FastDiv dstride[ttgbf::kMaxD];
  FastDiv dn[ttgbf::kMaxD];
  double lo[ttgbf::kMaxD];
  double dx[ttgbf::kMaxD];
  double centre[ttgbf::kMaxD];
  long long total;  // < 2^31
};

struct FgLik {
  int b;
  const void* htab[kFgMaxComps];
  double z[kFgMaxComps];
  double inv2r[kFgMaxComps];
  double period[kFgMaxComps];  // 0, or the period of an angle-like component
  // offset in the component's table of one step along each axis (0: the
  // component does not depend on it); the table is row-major over its modes
  long long tstride[kFgMaxComps][ttgbf::kMaxD];
};

__device__ __forceinline__ int axis_index(long long e, const FgGeom& g, int m) {
  const uint32_t t = fdiv((uint32_t)e, g.dstride[m]);
  return (int)(t - fdiv(t, g.dn[m]) * (uint32_t)g.n[m]);
}

template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// Compensated (Kahan) running sum in the density's own precision: per-thread
// partial sums stay accurate without float64 arithmetic per element (float64
// runs at 1/61 of the float32 rate on this GPU).
template <typename T>
struct Kahan {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <typename T>
__global__ void k_fg_prior(T* P, FgGeom g, const double* mean, const double* var) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.total;
       e += (long long)gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int m = 0; m < g.d; ++m) {
      const double x = g.lo[m] + (axis_index(e, g, m) + 0.5) * g.dx[m] - mean[m];
      q += x * x / var[m];
    }
    P[e] = (T)exp(-0.5 * q);
  }
}

// Shear x_m += a x_n: out(.., j_m, .., i_n, ..) = (1-f) in(j_m - k) + f in(j_m - k - 1)
// with s = a xi_{n,i_n} / D_m, k = floor(s), f = s - k (hat weights).
template <typename T>
__global__ void k_fg_shear(const T* __restrict__ in, T* __restrict__ out, FgGeom g, int m, int n,
                           const int* __restrict__ kshift, const double* __restrict__ frac) {
  const long long sm = g.stride[m];
  const int Nm = g.n[m];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = axis_index(e, g, m);
    const int in_ = axis_index(e, g, n);
    const int k = kshift[in_];
    const T f = (T)frac[in_];
    const int s1 = j - k, s2 = j - k - 1;
    T v = 0;
    if (s1 >= 0 && s1 < Nm) v += ((T)1 - f) * in[e + (long long)(s1 - j) * sm];
    if (s2 >= 0 && s2 < Nm) v += f * in[e + (long long)(s2 - j) * sm];
    out[e] = v;
  }
}

// out(.., j, ..) = sum_{i in band(j)} M(j, i) in(.., i, ..) along axis m, as a
// register-blocked product of the banded N x N operator with a tile of 64
// fibres of the axis.  Shared memory: the operator transposed (Mt[i][j]) and
// the tile (tile[i][f]).  Thread (tj, tf) computes rows 4 tj .. 4 tj + 3 for
// fibres 8 tf .. 8 tf + 7 over the union of the four rows' bands.  N must be
// a multiple of 4 and at most 128 (256 threads x 4 rows).
constexpr int kAxFib = 64;
constexpr int kAxPad = kAxFib + 4;

// Column of fibre f in a tile row: fibres 32..63 are shifted by 4 words so that
// the eight 8-fibre groups of a warp hit distinct shared-memory banks.
__device__ __forceinline__ int axcol(int f) { return f + ((f >> 5) << 2); }

// Four consecutive values from shared memory (16-byte aligned).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* v);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_fg_axis(const T* __restrict__ in, T* __restrict__ out,
                                                 long long nfib, int N, long long post,
                                                 const T* __restrict__ M, const int* __restrict__ blo,
                                                 const int* __restrict__ bhi) {
  extern __shared__ unsigned char smraw[];
  T* Mt = reinterpret_cast<T*>(smraw);  // [N][N]
  T* tile = Mt + N * N;                 // [N][kAxPad]
  __shared__ long long fbase[kAxFib];   // element offset of each fibre's first entry
  const int tid = threadIdx.x;
  for (int t = tid; t < N * N; t += blockDim.x) {
    const int j = t / N, i = t - j * N;
    Mt[i * N + j] = M[t];
  }
  const int tf = tid & 7, tj = tid >> 3;  // 8 fibre groups x 32 row groups
  const int j0 = tj * 4;
  const bool rows_ok = j0 < N;
  int lo = N, hi = -1;
  if (rows_ok) {
    for (int q = 0; q < 4; ++q) {
      if (blo[j0 + q] <= bhi[j0 + q]) {
        lo = min(lo, blo[j0 + q]);
        hi = max(hi, bhi[j0 + q]);
      }
    }
  }
  __syncthreads();
  for (long long g0 = (long long)blockIdx.x * kAxFib; g0 < nfib; g0 += (long long)gridDim.x * kAxFib) {
    // ---- load the tile
    if (tid < kAxFib) {
      const long long gf = g0 + tid;
      const long long p = gf / post, q = gf - p * post;
      fbase[tid] = gf < nfib ? p * N * post + q : -1;
    }
    __syncthreads();
    // 8 loads in flight per thread before the shared-memory stores
    const int tot = kAxFib * N;
    if (post == 1) {
      // fibres are contiguous rows of N: consecutive threads read consecutive i
      for (int t0 = tid; t0 < tot; t0 += 8 * 256) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * 256;
          const int f = t / N, i = t - f * N;
          const long long gf = g0 + f;
          v[u] = (t < tot && gf < nfib) ? in[gf * N + i] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * 256;
          if (t < tot) {
            const int f = t / N, i = t - f * N;
            tile[i * kAxPad + axcol(f)] = v[u];
          }
        }
      }
    } else {
      for (int t0 = tid; t0 < tot; t0 += 8 * 256) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * 256;
          const int i = t / kAxFib, f = t - i * kAxFib;
          const long long b = t < tot ? fbase[f] : -1;
          v[u] = b >= 0 ? in[b + (long long)i * post] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * 256;
          if (t < tot) {
            const int i = t / kAxFib, f = t - i * kAxFib;
            tile[i * kAxPad + axcol(f)] = v[u];
          }
        }
      }
    }
    __syncthreads();
    T acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0;
    const int c0 = axcol(tf * 8);
    for (int i = lo; i <= hi; ++i) {
      T m4[4], t8[8];
      ld4<T>(Mt + i * N + j0, m4);
      ld4<T>(tile + i * kAxPad + c0, t8);
      ld4<T>(tile + i * kAxPad + c0 + 4, t8 + 4);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] += m4[a] * t8[b];
    }
    __syncthreads();
    // ---- results back into the tile, then out with the load's access pattern
    if (rows_ok) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) tile[(j0 + a) * kAxPad + c0 + b] = acc[a][b];
    }
    __syncthreads();
    if (post == 1) {
      for (int t = tid; t < kAxFib * N; t += blockDim.x) {
        const int f = t / N, j = t - f * N;
        const long long gf = g0 + f;
        if (gf < nfib) out[gf * N + j] = tile[j * kAxPad + axcol(f)];
      }
    } else {
      for (int t = tid; t < kAxFib * N; t += blockDim.x) {
        const int j = t / kAxFib, f = t - j * kAxFib;
        const long long b = fbase[f];
        if (b >= 0) out[b + (long long)j * post] = tile[j * kAxPad + axcol(f)];
      }
    }
    __syncthreads();
  }
}

// ---- fused pass along one axis (upper-triangular F: L = I)
// When F = D U, every operation of the re-gridding and the kernel on axis m
// commutes with every operation on another axis that does not weight by x_m:
// U's shears x_m += a x_n (n > m) act along m with weights from axis n, the
// scaling and the kernel of axis m act along m alone, and the only operations
// weighting by x_m (the shears x_l += a x_m, l < m) come earlier in the
// canonical order.  So the predictive step is one pass per axis m (m
// ascending): load a tile of fibres along m, apply m's shears in order (each
// zero outside the grid, exactly as its own pass would), then m's banded
// operator (cloud-in-cell scaling fused with the Gaussian kernel), store.
constexpr int kPassMaxShears = kFgMaxD;

struct FgShearList {
  int ns;                              // shears along this axis, in order
  int n[kPassMaxShears];               // weight axis of each
  const int* kshift[kPassMaxShears];   // floor of the shift, per index of the weight axis
  const double* frac[kPassMaxShears];  // fractional part
};

// Tiles of FIB fibres along axis m (N <= 128, a multiple of 4): the operator
// transposed in shared memory (Mt[i][j] = M[j][i]), two tile buffers [N][FIB
// + 4] (shears ping-pong between them, the product goes to the free one).
// The next tile's loads are issued into registers before the current tile's
// shears and product, so they are in flight while the SM computes.  s_in
// multiplies the input (a pending normalisation); sum_acc (nullable) receives
// the sum of the output (the mass before normalisation).
template <typename T, int FIB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_fg_pass(const T* __restrict__ in, T* __restrict__ out,
                                                    FgGeom g, long long nfib, int N, long long post,
                                                    const T* __restrict__ M, const int* __restrict__ blo,
                                                    const int* __restrict__ bhi, FgShearList sh, T s_in,
                                                    double* sum_acc) {
  constexpr int PAD = FIB + 4;
  constexpr int FPT = FIB / 8;           // fibres per thread in the product
  constexpr int PER = FIB * 128 / 256;   // tile elements per thread (N <= 128)
  extern __shared__ unsigned char smraw[];
  T* Mt = reinterpret_cast<T*>(smraw);   // [N][N]
  T* A = Mt + N * N;                     // [N][PAD]
  T* Bw = A + N * PAD;                   // [N][PAD]
  __shared__ long long fb[2][FIB];       // element offset of every fibre's first entry
  __shared__ int sk[kPassMaxShears][FIB];
  __shared__ T sfr[kPassMaxShears][FIB];
  __shared__ double red[8];
  const int tid = threadIdx.x;
  for (int t = tid; t < N * N; t += blockDim.x) {
    const int j = t / N, i = t - j * N;
    Mt[i * N + j] = M[t];
  }
  const int tf = tid & 7, tj = tid >> 3;
  const int j0 = tj * 4;
  const bool rows_ok = j0 < N;
  int lo = N, hi = -1;
  if (rows_ok)
    for (int q = 0; q < 4; ++q)
      if (blo[j0 + q] <= bhi[j0 + q]) {
        lo = min(lo, blo[j0 + q]);
        hi = max(hi, bhi[j0 + q]);
      }
  auto fibre_base = [&](long long gf) -> long long {
    const long long p = gf / post, q = gf - p * post;
    return p * N * post + q;
  };
  const long long tstride = (long long)gridDim.x * FIB;
  long long g0 = (long long)blockIdx.x * FIB;
  if (tid < FIB) fb[0][tid] = (g0 + tid < nfib) ? fibre_base(g0 + tid) : -1;
  __syncthreads();
  T v[PER];
  auto load = [&](int sel, long long gb) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u;
      T x = (T)0;
      if (e < FIB * N) {
        if (post == 1) {
          const int f = e / N, i = e - f * N;
          if (gb + f < nfib) x = in[(gb + f) * N + i];
        } else {
          const int i = e / FIB, f = e - i * FIB;
          const long long b = fb[sel][f];
          if (b >= 0) x = in[b + (long long)i * post];
        }
      }
      v[u] = x;
    }
  };
  if (g0 < nfib) load(0, g0);
  Kahan<T> ks;
  int sel = 0;
  for (; g0 < nfib; g0 += tstride) {
    // ---- the current tile (registers) into A, scaled
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u;
      if (e < FIB * N) {
        int i, f;
        if (post == 1) {
          f = e / N;
          i = e - f * N;
        } else {
          i = e / FIB;
          f = e - i * FIB;
        }
        A[i * PAD + axcol(f)] = v[u] * s_in;
      }
    }
    const long long g1 = g0 + tstride;
    if (tid < FIB) fb[sel ^ 1][tid] = (g1 + tid < nfib) ? fibre_base(g1 + tid) : -1;
    for (int t = tid; t < sh.ns * FIB; t += blockDim.x) {
      const int q = t / FIB, f = t - q * FIB;
      const long long b = fb[sel][f];
      int k = 0;
      T fr = (T)0;
      if (b >= 0) {
        const int ia = axis_index(b, g, sh.n[q]);
        k = sh.kshift[q][ia];
        fr = (T)sh.frac[q][ia];
      }
      sk[q][f] = k;
      sfr[q][f] = fr;
    }
    __syncthreads();
    if (g1 < nfib) load(sel ^ 1, g1);  // in flight during the work below
    // ---- shears along the axis (each zero outside the grid)
    T* cur = A;
    T* oth = Bw;
    for (int q = 0; q < sh.ns; ++q) {
      for (int t = tid; t < N * FIB; t += blockDim.x) {
        const int j = t / FIB, f = t - j * FIB;
        const int k = sk[q][f];
        const T fr = sfr[q][f];
        const int s1 = j - k, s2 = j - k - 1;
        T val = (T)0;
        if (s1 >= 0 && s1 < N) val += ((T)1 - fr) * cur[s1 * PAD + axcol(f)];
        if (s2 >= 0 && s2 < N) val += fr * cur[s2 * PAD + axcol(f)];
        oth[j * PAD + axcol(f)] = val;
      }
      __syncthreads();
      T* sw = cur;
      cur = oth;
      oth = sw;
    }
    // ---- banded operator: rows j0..j0+3, fibres FPT tf..FPT tf + FPT - 1
    T acc[4][FPT];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < FPT; ++b) acc[a][b] = 0;
    const int c0 = axcol(tf * FPT);
    for (int i = lo; i <= hi; ++i) {
      T m4[4], tv[FPT];
      ld4<T>(Mt + i * N + j0, m4);
#pragma unroll
      for (int b = 0; b < FPT; b += 4) ld4<T>(cur + i * PAD + c0 + b, tv + b);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < FPT; ++b) acc[a][b] += m4[a] * tv[b];
    }
    if (rows_ok) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < FPT; ++b) {
          oth[(j0 + a) * PAD + c0 + b] = acc[a][b];
          if (sum_acc != nullptr) ks.add(acc[a][b]);
        }
    }
    __syncthreads();
    // ---- store with the load's access pattern
    if (post == 1) {
      for (int t = tid; t < FIB * N; t += blockDim.x) {
        const int f = t / N, j = t - f * N;
        if (g0 + f < nfib) out[(g0 + f) * N + j] = oth[j * PAD + axcol(f)];
      }
    } else {
      for (int t = tid; t < FIB * N; t += blockDim.x) {
        const int j = t / FIB, f = t - j * FIB;
        const long long b = fb[sel][f];
        if (b >= 0) out[b + (long long)j * post] = oth[j * PAD + axcol(f)];
      }
    }
    __syncthreads();
    sel ^= 1;
  }
  if (sum_acc != nullptr) {
    double sv = (double)ks.s - (double)ks.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
    if ((tid & 31) == 0) red[tid >> 5] = sv;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      atomicAdd(sum_acc, t);
    }
  }
}

// Sum of P (float64 accumulation); optionally P *= scale read from *scale_src.
template <typename T>
__global__ void k_fg_sum(const T* __restrict__ P, long long total, double* acc) {
  __shared__ double red[32];
  Kahan<T> k;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    k.add(P[e]);
  double s = (double)k.s - (double)k.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(acc, t);
  }
}

// P *= 1 / (acc[0] * delta)
template <typename T>
__global__ void k_fg_scale(T* P, long long total, const double* acc, double delta) {
  const T s = (T)(1.0 / (acc[0] * delta));
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    P[e] *= s;
}

// P *= s (a pending normalisation known on the host).
template <typename T>
__global__ void k_fg_mul(T* P, long long total, T s) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    P[e] *= s;
}

// Per component: off_c = min over the table of (z_c - h)^2 (the residual
// wrapped for an angle-like component).
template <typename H>
__global__ void k_fg_lik_off(const H* htab, int ntab, double z, double period, double* off) {
  __shared__ double red[32];
  double mn = INFINITY;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) {
    const double e = ttgbf::wrap_residual(z - (double)htab[i], period);
    mn = fmin(mn, e * e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmin(t, red[w]);
    *off = t;
  }
}

// P <- P * prod_c exp(-((z_c - h_c)^2 - off_c) / (2 R_c)); acc += sum of the result.
// One warp per row of the last axis: factors of components that do not use
// the last axis are evaluated once per row.
// Table offset of component c at the point of the row starting at e0, the
// last axis left out.
__device__ __forceinline__ long long lik_row_offset(const FgLik& lk, int c, long long e0, const FgGeom& g,
                                                     int last) {
  long long t = 0;
  for (int m = 0; m < g.d; ++m)
    if (m != last && lk.tstride[c][m] != 0) t += (long long)axis_index(e0, g, m) * lk.tstride[c][m];
  return t;
}

template <typename T>
__device__ __forceinline__ T lik_factor(const FgLik& lk, int c, long long t, const double* off) {
  const T h = (T)static_cast<const T*>(lk.htab[c])[t];
  const T df = ttgbf::wrap_residual((T)lk.z[c] - h, (T)lk.period[c]);
  return exp_t<T>(-(df * df - (T)off[c]) * (T)lk.inv2r[c]);
}

template <typename T>
__global__ void k_fg_lik(T* P, FgGeom g, FgLik lk, const double* off, double* acc) {
  __shared__ double red[32];
  const int d = g.d, last = d - 1;
  const int NL = g.n[last];
  const long long rows = g.total / NL;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  Kahan<T> k;
  for (long long r = warp0; r < rows; r += nwarps) {
    const long long e0 = r * NL;
    T Lrow = 1;
    long long rb[kFgMaxComps];
    for (int c = 0; c < lk.b; ++c) {
      rb[c] = lik_row_offset(lk, c, e0, g, last);
      if (lk.tstride[c][last] == 0) Lrow *= lik_factor<T>(lk, c, rb[c], off);
    }
    for (int il = lane; il < NL; il += 32) {
      T L = Lrow;
      for (int c = 0; c < lk.b; ++c)
        if (lk.tstride[c][last] != 0) L *= lik_factor<T>(lk, c, rb[c] + (long long)il * lk.tstride[c][last], off);
      const T v = P[e0 + il] * L;
      P[e0 + il] = v;
      k.add(v);
    }
  }
  double s = (double)k.s - (double)k.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(acc, t);
  }
}

// The Bayes update and the posterior moments in one pass:
//   v = P * s * prod_c exp(-((z_c - h_c)^2 - off_c) / (2 R_c)),  P <- v,
// with s = host_scale / (dsum[0] delta) (dsum nullable: the predictive mass a
// fused predictive pass left on the device); lik_acc += sum v, and mom (the
// layout of k_fg_moments) += the point-mass sums of v.  One warp per row of
// the last axis, as both passes it replaces.
template <typename T, int D>
__global__ void k_fg_lik_mom(T* P, FgGeom g, FgLik lk, const double* off, const double* dsum,
                             double host_scale, double delta, double* lik_acc, double* mom) {
  constexpr int NA = 1 + D + D * D;
  constexpr int LAST = D - 1;
  constexpr int PER = (NA + 31) / 32;  // accumulators per lane
  __shared__ double red[NA][8];
  const int NL = g.n[LAST];
  const long long rows = g.total / NL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const T sc = (T)(host_scale / (dsum != nullptr ? dsum[0] * delta : 1.0));
  const T lol = (T)(g.lo[LAST] - g.centre[LAST]), dxl = (T)g.dx[LAST];
  // accumulator a (layout of k_fg_moments) is lane a % 32's slot a / 32: the
  // row sum r_p (p = 0, 1, 2: sums of v, x_last v, x_last^2 v) times the row
  // coordinates x_ma, x_mb (-1: none)
  int ap[PER], ama[PER], amb[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int a = lane + 32 * q;
    ap[q] = -1;
    ama[q] = amb[q] = -1;
    if (a == 0) {
      ap[q] = 0;
    } else if (a < 1 + D) {
      const int m = a - 1;
      ap[q] = m == LAST ? 1 : 0;
      ama[q] = m == LAST ? -1 : m;
    } else if (a < NA) {
      const int m = (a - 1 - D) / D, l = (a - 1 - D) % D;
      if (m <= l) {
        if (l < LAST) {
          ap[q] = 0;
          ama[q] = m;
          amb[q] = l;
        } else if (m < LAST) {
          ap[q] = 1;
          ama[q] = m;
        } else {
          ap[q] = 2;
        }
      }
    }
  }
  Kahan<T> s[PER];
  for (long long r = warp0; r < rows; r += nwarps) {
    const long long e0 = r * NL;
    T Lrow = sc;
    long long rb[kFgMaxComps];
    for (int c = 0; c < lk.b; ++c) {
      rb[c] = lik_row_offset(lk, c, e0, g, LAST);
      if (lk.tstride[c][LAST] == 0) Lrow *= lik_factor<T>(lk, c, rb[c], off);
    }
    Kahan<T> a0, a1, a2;
    for (int il = lane; il < NL; il += 32) {
      T L = Lrow;
      for (int c = 0; c < lk.b; ++c)
        if (lk.tstride[c][LAST] != 0) L *= lik_factor<T>(lk, c, rb[c] + (long long)il * lk.tstride[c][LAST], off);
      const T v = P[e0 + il] * L;
      P[e0 + il] = v;
      const T xl = lol + ((T)il + (T)0.5) * dxl;
      a0.add(v);
      a1.add(xl * v);
      a2.add(xl * xl * v);
    }
    T r0 = a0.s - a0.c, r1 = a1.s - a1.c, r2 = a2.s - a2.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r0 += __shfl_xor_sync(0xffffffffu, r0, o);
      r1 += __shfl_xor_sync(0xffffffffu, r1, o);
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    T x[D];
#pragma unroll
    for (int m = 0; m < LAST; ++m)
      x[m] = (T)(g.lo[m] - g.centre[m]) + ((T)axis_index(e0, g, m) + (T)0.5) * (T)g.dx[m];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      if (ap[q] < 0) continue;
      T t = ap[q] == 0 ? r0 : (ap[q] == 1 ? r1 : r2);
#pragma unroll
      for (int m = 0; m < LAST; ++m) {
        if (ama[q] == m) t *= x[m];
        if (amb[q] == m) t *= x[m];
      }
      s[q].add(t);
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int a = lane + 32 * q;
    if (a < NA) red[a][warp] = (double)s[q].s - (double)s[q].c;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < NA; a += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[a][w];
    atomicAdd(mom + a, t);
    if (a == 0) atomicAdd(lik_acc, t);
  }
}

// acc[0] = sum P, acc[1+m] = sum x_m P, acc[1+D+m*D+l] = sum x_m x_l P (centred
// x, l >= m).  D is the state dimension (compile time, so the sums stay in
// registers).  One warp per row of the last axis: per row only sum v, sum x v
// and sum x^2 v over the last axis are formed, then combined with the row's
// other coordinates.
template <typename T, int D>
__global__ void k_fg_moments(const T* __restrict__ P, FgGeom g, double* acc) {
  constexpr int NA = 1 + D + D * D;
  constexpr int LAST = D - 1;
  __shared__ double red[NA][8];
  Kahan<T> s[NA];
  const int NL = g.n[LAST];
  const long long rows = g.total / NL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const T lol = (T)(g.lo[LAST] - g.centre[LAST]), dxl = (T)g.dx[LAST];
  for (long long r = warp0; r < rows; r += nwarps) {
    const long long e0 = r * NL;
    Kahan<T> a0, a1, a2;
    for (int il = lane; il < NL; il += 32) {
      const T v = P[e0 + il];
      const T xl = lol + ((T)il + (T)0.5) * dxl;
      a0.add(v);
      a1.add(xl * v);
      a2.add(xl * xl * v);
    }
    T r0 = a0.s - a0.c, r1 = a1.s - a1.c, r2 = a2.s - a2.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r0 += __shfl_xor_sync(0xffffffffu, r0, o);
      r1 += __shfl_xor_sync(0xffffffffu, r1, o);
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if (lane == 0) {
      T x[D];
#pragma unroll
      for (int m = 0; m < LAST; ++m)
        x[m] = (T)(g.lo[m] - g.centre[m]) + ((T)axis_index(e0, g, m) + (T)0.5) * (T)g.dx[m];
      s[0].add(r0);
#pragma unroll
      for (int m = 0; m < LAST; ++m) {
        s[1 + m].add(x[m] * r0);
#pragma unroll
        for (int l = m; l < LAST; ++l) s[1 + D + m * D + l].add(x[m] * x[l] * r0);
        s[1 + D + m * D + LAST].add(x[m] * r1);
      }
      s[1 + LAST].add(r1);
      s[1 + D + LAST * D + LAST].add(r2);
    }
  }
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    double t = (double)s[a].s - (double)s[a].c;  // non-zero on lane 0 of each warp only
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[a][warp] = t;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < NA; a += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[a][w];
    atomicAdd(acc + a, t);
  }
}

template <typename T>
void launch_fg_moments(int d, int grid, cudaStream_t st, const T* P, const FgGeom& g, double* acc) {
  switch (d) {
    case 1: k_fg_moments<T, 1><<<grid, 256, 0, st>>>(P, g, acc); break;
    case 2: k_fg_moments<T, 2><<<grid, 256, 0, st>>>(P, g, acc); break;
    case 3: k_fg_moments<T, 3><<<grid, 256, 0, st>>>(P, g, acc); break;
    case 4: k_fg_moments<T, 4><<<grid, 256, 0, st>>>(P, g, acc); break;
    case 5: k_fg_moments<T, 5><<<grid, 256, 0, st>>>(P, g, acc); break;
    default: k_fg_moments<T, 6><<<grid, 256, 0, st>>>(P, g, acc); break;
  }
}

template <typename T>
void launch_fg_lik_mom(int d, int grid, cudaStream_t st, T* P, const FgGeom& g, const FgLik& lk,
                       const double* off, const double* dsum, double host_scale, double delta,
                       double* lik_acc, double* mom) {
  switch (d) {
    case 1: k_fg_lik_mom<T, 1><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
    case 2: k_fg_lik_mom<T, 2><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
    case 3: k_fg_lik_mom<T, 3><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
    case 4: k_fg_lik_mom<T, 4><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
    case 5: k_fg_lik_mom<T, 5><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
    default: k_fg_lik_mom<T, 6><<<grid, 256, 0, st>>>(P, g, lk, off, dsum, host_scale, delta, lik_acc, mom); break;
  }
}

// Textbook direct sum: out_j = sum_i exp(-0.5 (xi_j - F xi_i)^T Qinv (xi_j - F xi_i)) P_i
// (the constant factor is removed by the normalisation that follows).
template <typename T>
__global__ void k_fg_direct(const T* __restrict__ in, T* __restrict__ out, FgGeom g, const double* F,
                            const double* Qinv) {
  __shared__ double sfx[256][ttgbf::kMaxD];
  __shared__ double sp[256];
  const int d = g.d;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double xj[ttgbf::kMaxD];
  for (int m = 0; m < d; ++m)
    xj[m] = j < g.total ? g.lo[m] + (axis_index(j, g, m) + 0.5) * g.dx[m] : 0.0;
  double acc = 0.0;
  for (long long i0 = 0; i0 < g.total; i0 += blockDim.x) {
    const long long i = i0 + threadIdx.x;
    if (i < g.total) {
      double xi[ttgbf::kMaxD];
      for (int m = 0; m < d; ++m) xi[m] = g.lo[m] + (axis_index(i, g, m) + 0.5) * g.dx[m];
      for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int l = 0; l < d; ++l) s += F[m * d + l] * xi[l];
        sfx[threadIdx.x][m] = s;
      }
      sp[threadIdx.x] = (double)in[i];
    } else {
      sp[threadIdx.x] = 0.0;
      for (int m = 0; m < d; ++m) sfx[threadIdx.x][m] = 0.0;
    }
    __syncthreads();
    const int cnt = (int)min((long long)blockDim.x, g.total - i0);
    for (int t = 0; t < cnt; ++t) {
      double q = 0.0;
      for (int m = 0; m < d; ++m) {
        const double um = xj[m] - sfx[t][m];
        for (int l = 0; l < d; ++l) q += um * Qinv[m * d + l] * (xj[l] - sfx[t][l]);
      }
      acc += exp(-0.5 * q) * sp[t];
    }
    __syncthreads();
  }
  if (j < g.total) out[j] = (T)acc;
}

}  // namespace

// ======================================================================= host
struct ttgbf_fg {
  int prec = 32;
  int d = 0;
  std::vector<int> n;
  std::vector<double> lo, hi, dx, axes;
  std::vector<int> axoff;
  double delta = 1.0;
  cudaStream_t st = nullptr;
  FgGeom g{};
  char* base = nullptr;
  bool owns = false;
  size_t bytes = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  double* acc = nullptr;      // [kFgAcc + 4] reductions
  double* off = nullptr;      // [kFgMaxComps]
  double* dparams = nullptr;  // prior mean/var, F, Qinv
  void* mats = nullptr;       // per-axis operators (T)
  int* ints = nullptr;        // band bounds, shear shifts
  double* fracs = nullptr;    // shear fractions
  double log_c = 0.0, log_lik = 0.0;
  std::vector<double> lastF, lastQ;
  struct ShearOp {
    int m, n;
    long long ioff, foff;
  };
  std::vector<ShearOp> shears_u, shears_l;
  std::vector<int> scale_axis;  // axes with a separate scaling operator (L != I)
  long long mat_off[ttgbf::kMaxD] = {}, smat_off[ttgbf::kMaxD] = {};
  long long band_off[ttgbf::kMaxD] = {}, sband_off[ttgbf::kMaxD] = {};
  bool fused = true;
  int sms = 148;
  bool poisoned = false;
  // Normalisations not yet applied to the stored density: it equals the
  // normalised density divided by pending (a host scalar, from the last
  // update's mass) and, when dev_pending, by the predictive mass a fused
  // predictive pass left in acc[kFgPredSum] (times the cell volume).
  double pending = 1.0;
  bool dev_pending = false;
  bool mom_valid = false;  // acc[0..kFgAcc) holds the moments of the stored density
};

namespace {

size_t fg_elem(int prec) { return prec == 64 ? 8 : 4; }

struct FgLayout {
  size_t buf0, buf1, acc, off, dparams, mats, ints, fracs, total;
  long long nmats, nints, nfracs;
};

FgLayout fg_layout(const ttgbf_grid* g, int prec) {
  FgLayout L{};
  long long total = 1, nsum = 0, nn = 0;
  int nmax = 0;
  for (int k = 0; k < g->d; ++k) {
    total *= g->n[k];
    nsum += g->n[k];
    nn += (long long)g->n[k] * g->n[k];
    nmax = std::max(nmax, (int)g->n[k]);
  }
  const size_t e = fg_elem(prec);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = (off + 255) & ~size_t(255);
    off = at + bytes;
    return at;
  };
  L.buf0 = take(total * e);
  L.buf1 = take(total * e);
  L.acc = take(sizeof(double) * (kFgAcc + 8));
  L.off = take(sizeof(double) * kFgMaxComps);
  L.dparams = take(sizeof(double) * (2 * ttgbf::kMaxD + 2 * ttgbf::kMaxD * ttgbf::kMaxD));
  L.nmats = 2 * nn;
  L.mats = take(e * L.nmats);
  L.nints = 4 * nsum + (long long)g->d * g->d * nmax;
  L.ints = take(sizeof(int) * L.nints);
  L.nfracs = (long long)g->d * g->d * nmax;
  L.fracs = take(sizeof(double) * L.nfracs);
  L.total = off + 256;
  return L;
}

int fg_check(ttgbf_fg* c) {
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    c->poisoned = true;
    return TTGBF_ECUDA;
  }
  return TTGBF_OK;
}

template <typename T>
void fg_launch_scale_sum(ttgbf_fg* c, void* P) {
  cudaMemsetAsync(c->acc, 0, sizeof(double), c->st);
  ttgbf::count_launches(2);
  k_fg_sum<T><<<c->sms * 8, 256, 0, c->st>>>((const T*)P, c->g.total, c->acc);
  k_fg_scale<T><<<c->sms * 8, 256, 0, c->st>>>((T*)P, c->g.total, c->acc, c->delta);
}

double hatw(double t) { return std::max(0.0, 1.0 - std::fabs(t)); }

// Upload operators for F, Q (same elementary sequence as the TT path).
template <typename T>
int fg_prepare(ttgbf_fg* c, const double* F, const double* Q) {
  const int d = c->d;
  // LDU without pivoting
  std::vector<double> Lm((size_t)d * d, 0.0), U((size_t)d * d, 0.0), D(d, 0.0);
  double scale = 1.0;
  for (int i = 0; i < d * d; ++i) scale = std::max(scale, std::fabs(F[i]));
  for (int k = 0; k < d; ++k) Lm[k * d + k] = U[k * d + k] = 1.0;
  for (int k = 0; k < d; ++k) {
    double s = F[k * d + k];
    for (int j = 0; j < k; ++j) s -= Lm[k * d + j] * D[j] * U[j * d + k];
    D[k] = s;
    if (std::fabs(s) <= 1e-12 * scale) return TTGBF_ESINGULAR;
    for (int i = k + 1; i < d; ++i) {
      double sl = F[i * d + k], su = F[k * d + i];
      for (int j = 0; j < k; ++j) {
        sl -= Lm[i * d + j] * D[j] * U[j * d + k];
        su -= Lm[k * d + j] * D[j] * U[j * d + i];
      }
      Lm[i * d + k] = sl / s;
      U[k * d + i] = su / s;
    }
  }
  bool lower = false;
  for (int m = 0; m < d; ++m)
    for (int n = 0; n < m; ++n)
      if (Lm[m * d + n] != 0.0) lower = true;
  std::vector<int> ints;
  std::vector<double> fracs;
  std::vector<T> mats;
  c->shears_u.clear();
  c->shears_l.clear();
  auto add_shear = [&](int m, int n, double a, std::vector<ttgbf_fg::ShearOp>* list) {
    ttgbf_fg::ShearOp op{m, n, (long long)ints.size(), (long long)fracs.size()};
    for (int i = 0; i < c->n[n]; ++i) {
      const double s = a * c->axes[c->axoff[n] + i] / c->dx[m];
      const double k = std::floor(s);
      ints.push_back((int)k);
      fracs.push_back(s - k);
    }
    list->push_back(op);
  };
  for (int m = 0; m < d; ++m)
    for (int n = m + 1; n < d; ++n)
      if (U[m * d + n] != 0.0) add_shear(m, n, U[m * d + n], &c->shears_u);
  for (int m = d - 1; m >= 0; --m)
    for (int n = 0; n < m; ++n)
      if (Lm[m * d + n] != 0.0) add_shear(m, n, Lm[m * d + n], &c->shears_l);
  // per-axis operators and their bands
  // entries below this fraction of the largest are below the density's
  // rounding resolution and are skipped
  const double band_tol = sizeof(T) == 4 ? 1e-12 : 1e-20;
  auto add_band = [&](const std::vector<double>& M, int N) {
    const long long at = (long long)ints.size();
    double mx = 0.0;
    for (double v : M) mx = std::max(mx, std::fabs(v));
    std::vector<int> los(N), his(N);
    for (int j = 0; j < N; ++j) {
      int lo = N, hi = -1;
      for (int i = 0; i < N; ++i)
        if (std::fabs(M[(size_t)j * N + i]) > band_tol * mx) {
          lo = std::min(lo, i);
          hi = std::max(hi, i);
        }
      if (hi < lo) lo = 0, hi = -1;
      los[j] = lo;
      his[j] = hi;
    }
    ints.insert(ints.end(), los.begin(), los.end());
    ints.insert(ints.end(), his.begin(), his.end());
    return at;
  };
  c->scale_axis.clear();
  for (int m = 0; m < d; ++m) {
    const int N = c->n[m];
    const double Dm = c->dx[m], q = Q[m * d + m];
    std::vector<double> K((size_t)N * N), W((size_t)N * N, 0.0);
    const double nrm = Dm / std::sqrt(2.0 * M_PI * q);
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const double t = (double)(j - i) * Dm;
        K[(size_t)j * N + i] = nrm * std::exp(-0.5 * t * t / q);
      }
    const bool has_scale = D[m] != 1.0;
    if (has_scale)
      for (int i = 0; i < N; ++i) {
        const double u = (D[m] * c->axes[c->axoff[m] + i] - c->lo[m]) / Dm - 0.5;
        for (int j = 0; j < N; ++j) W[(size_t)j * N + i] = hatw(j - u);
      }
    if (has_scale && !lower) {
      std::vector<double> Mf((size_t)N * N, 0.0);
      for (int j = 0; j < N; ++j)
        for (int l = 0; l < N; ++l) {
          const double kjl = K[(size_t)j * N + l];
          if (kjl == 0.0) continue;
          for (int i = 0; i < N; ++i) Mf[(size_t)j * N + i] += kjl * W[(size_t)l * N + i];
        }
      K.swap(Mf);
    } else if (has_scale) {
      c->smat_off[m] = (long long)mats.size();
      for (double v : W) mats.push_back((T)v);
      c->sband_off[m] = add_band(W, N);
      c->scale_axis.push_back(m);
    }
    c->mat_off[m] = (long long)mats.size();
    for (double v : K) mats.push_back((T)v);
    c->band_off[m] = add_band(K, N);
  }
  c->fused = !lower;
  cudaMemcpyAsync(c->mats, mats.data(), sizeof(T) * mats.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->fracs, fracs.data(), sizeof(double) * fracs.size(), cudaMemcpyHostToDevice, c->st);
  cudaStreamSynchronize(c->st);  // host vectors are freed on return
  c->lastF.assign(F, F + (size_t)d * d);
  c->lastQ.assign(Q, Q + (size_t)d * d);
  return TTGBF_OK;
}

// Apply every pending normalisation with one pass (for the paths that read
// the density as stored: the direct sum, the general-F sequence, density()).
template <typename T>
void fg_apply_pending(ttgbf_fg* c) {
  if (c->dev_pending) {
    ttgbf::count_launches(1);
    k_fg_scale<T><<<c->sms * 8, 256, 0, c->st>>>((T*)c->buf[c->cur], c->g.total, c->acc + kFgPredSum,
                                                 c->delta);
    c->dev_pending = false;
  }
  if (c->pending != 1.0) {
    ttgbf::count_launches(1);
    k_fg_mul<T><<<c->sms * 8, 256, 0, c->st>>>((T*)c->buf[c->cur], c->g.total, (T)c->pending);
    c->pending = 1.0;
  }
}

// One fused pass along axis m: its U shears (in order), its banded operator,
// the pending host normalisation s_in on load, the output's sum into sum.
template <typename T>
void fg_pass(ttgbf_fg* c, int m, T s_in, double* sum) {
  // float: tiles of 32 fibres, two CTAs per SM (16 warps hide the shared-
  // memory latency of the shears and the banded product); double: one CTA
  constexpr int FIB = 32;
  constexpr int MINB = sizeof(T) == 4 ? 2 : 1;
  FgShearList sl{};
  for (const auto& op : c->shears_u)
    if (op.m == m) {
      sl.n[sl.ns] = op.n;
      sl.kshift[sl.ns] = c->ints + op.ioff;
      sl.frac[sl.ns] = c->fracs + op.foff;
      ++sl.ns;
    }
  const int N = c->n[m];
  long long post = 1;
  for (int k = m + 1; k < c->d; ++k) post *= c->n[k];
  const long long nfib = c->g.total / N;
  const size_t sm = sizeof(T) * ((size_t)N * N + 2 * (size_t)N * (FIB + 4));
  ttgbf::count_launches(1);
  k_fg_pass<T, FIB, MINB><<<c->sms * MINB, 256, sm, c->st>>>((const T*)c->buf[c->cur], (T*)c->buf[c->cur ^ 1], c->g, nfib,
                                                N, post, (const T*)c->mats + c->mat_off[m],
                                                c->ints + c->band_off[m], c->ints + c->band_off[m] + N, sl,
                                                s_in, sum);
  c->cur ^= 1;
}

template <typename T>
void fg_shear(ttgbf_fg* c, const ttgbf_fg::ShearOp& op) {
  ttgbf::count_launches(1);
  k_fg_shear<T><<<c->sms * 16, 256, 0, c->st>>>((const T*)c->buf[c->cur], (T*)c->buf[c->cur ^ 1], c->g,
                                               op.m, op.n, c->ints + op.ioff, c->fracs + op.foff);
  c->cur ^= 1;
}

template <typename T>
void fg_axis(ttgbf_fg* c, int m, long long moff, long long boff) {
  const int N = c->n[m];
  long long post = 1;
  for (int k = m + 1; k < c->d; ++k) post *= c->n[k];
  const long long nfib = c->g.total / N;
  const size_t sm = sizeof(T) * ((size_t)N * N + (size_t)N * kAxPad);
  ttgbf::count_launches(1);
  k_fg_axis<T><<<c->sms * 2, 256, sm, c->st>>>((const T*)c->buf[c->cur], (T*)c->buf[c->cur ^ 1], nfib, N,
                                              post, (const T*)c->mats + moff, c->ints + boff,
                                              c->ints + boff + N);
  c->cur ^= 1;
}

template <typename T>
int fg_predict(ttgbf_fg* c, const double* F, const double* Q, bool direct) {
  const int d = c->d;
  if (direct) {
    fg_apply_pending<T>(c);
    c->mom_valid = false;
    std::vector<double> Qinv((size_t)d * d);
    // invert Q (symmetric positive definite) by Gauss-Jordan
    std::vector<double> A(Q, Q + (size_t)d * d);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) Qinv[i * d + j] = (i == j);
    for (int k = 0; k < d; ++k) {
      const double p = A[k * d + k];
      if (!(std::fabs(p) > 0.0)) return TTGBF_EINVAL;
      for (int j = 0; j < d; ++j) {
        A[k * d + j] /= p;
        Qinv[k * d + j] /= p;
      }
      for (int i = 0; i < d; ++i)
        if (i != k) {
          const double f = A[i * d + k];
          for (int j = 0; j < d; ++j) {
            A[i * d + j] -= f * A[k * d + j];
            Qinv[i * d + j] -= f * Qinv[k * d + j];
          }
        }
    }
    double* dF = c->dparams + 2 * ttgbf::kMaxD;
    double* dQ = dF + ttgbf::kMaxD * ttgbf::kMaxD;
    cudaMemcpyAsync(dF, F, sizeof(double) * d * d, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(dQ, Qinv.data(), sizeof(double) * d * d, cudaMemcpyHostToDevice, c->st);
    ttgbf::count_launches(1);
    k_fg_direct<T><<<(unsigned)((c->g.total + 255) / 256), 256, 0, c->st>>>(
        (const T*)c->buf[c->cur], (T*)c->buf[c->cur ^ 1], c->g, dF, dQ);
    cudaStreamSynchronize(c->st);  // Qinv lives on this stack frame
    c->cur ^= 1;
  } else {
    const bool same = c->lastF.size() == (size_t)d * d && std::equal(c->lastF.begin(), c->lastF.end(), F) &&
                      std::equal(c->lastQ.begin(), c->lastQ.end(), Q);
    if (!same) {
      const int rc = fg_prepare<T>(c, F, Q);
      if (rc) return rc;
    }
    c->mom_valid = false;
    if (c->fused) {
      // one pass per axis; the pending normalisation rides on the first
      // pass, the predictive mass is summed by the last and applied by the
      // update's pass
      if (c->dev_pending) fg_apply_pending<T>(c);
      cudaMemsetAsync(c->acc + kFgPredSum, 0, sizeof(double), c->st);
      for (int m = 0; m < d; ++m)
        fg_pass<T>(c, m, (T)(m == 0 ? c->pending : 1.0), m == d - 1 ? c->acc + kFgPredSum : nullptr);
      c->pending = 1.0;
      c->dev_pending = true;
      return fg_check(c);
    }
    fg_apply_pending<T>(c);
    for (const auto& op : c->shears_u) fg_shear<T>(c, op);
    for (int m : c->scale_axis) fg_axis<T>(c, m, c->smat_off[m], c->sband_off[m]);
    for (const auto& op : c->shears_l) fg_shear<T>(c, op);
    for (int m = 0; m < d; ++m) fg_axis<T>(c, m, c->mat_off[m], c->band_off[m]);
  }
  fg_launch_scale_sum<T>(c, c->buf[c->cur]);
  return fg_check(c);
}

template <typename T>
int fg_update(ttgbf_fg* c, const ttgbf_meas* h, const double* R, const double* z) {
  FgLik lk{};
  lk.b = h->b;
  double logoff = 0.0;
  std::vector<double> offs(h->b);
  for (int i = 0; i < h->b; ++i) {
    const ttgbf_meas_comp& cp = h->comp[i];
    // the component's modes in its table's order, and their strides
    int modes[ttgbf::kMaxD];
    for (int t = 0; t < cp.nmodes; ++t) modes[t] = cp.nmodes <= 2 ? cp.modes[t] : cp.modes[0] + t;
    long long st = 1;
    for (int t = cp.nmodes - 1; t >= 0; --t) {
      lk.tstride[i][modes[t]] = st;
      st *= c->n[modes[t]];
    }
    const int ntab = (int)st;
    lk.htab[i] = cp.htab;
    lk.z[i] = z[i];
    const double r = R[(size_t)i * h->b + i];
    lk.inv2r[i] = 0.5 / r;
    lk.period[i] = cp.period;
    ttgbf::count_launches(1);
    k_fg_lik_off<T><<<1, 256, 0, c->st>>>(static_cast<const T*>(static_cast<const void*>(cp.htab)), ntab,
                                         z[i], cp.period, c->off + i);
    logoff += -0.5 * std::log(2.0 * M_PI * r);
  }
  // one pass: the pending normalisations, the likelihood, log c's sum and
  // the posterior moments (the posterior's own normalisation stays pending)
  // moment slots and the likelihood sum; the predictive sum (kFgPredSum) is
  // read by this pass
  cudaMemsetAsync(c->acc, 0, sizeof(double) * kFgAcc, c->st);
  cudaMemsetAsync(c->acc + kFgLikSum, 0, sizeof(double), c->st);
  ttgbf::count_launches(1);
  launch_fg_lik_mom<T>(c->d, c->sms * 8, c->st, (T*)c->buf[c->cur], c->g, lk, c->off,
                       c->dev_pending ? c->acc + kFgPredSum : nullptr, c->pending, c->delta,
                       c->acc + kFgLikSum, c->acc);
  double hacc = 0.0;
  cudaMemcpyAsync(offs.data(), c->off, sizeof(double) * h->b, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(&hacc, c->acc + kFgLikSum, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaGetLastError();
    c->poisoned = true;
    return TTGBF_ECUDA;
  }
  for (int i = 0; i < h->b; ++i) logoff += -offs[i] * lk.inv2r[i];
  c->log_c = std::log(hacc * c->delta) + logoff;
  c->log_lik += c->log_c;
  c->pending = 1.0 / (hacc * c->delta);
  c->dev_pending = false;
  c->mom_valid = true;
  return fg_check(c);
}

template <typename T>
int fg_estimate(ttgbf_fg* c, double* mean, double* cov) {
  const int d = c->d;
  // the moments are ratios of sums, so a pending normalisation cancels; the
  // update's pass already formed them
  if (!c->mom_valid) {
    cudaMemsetAsync(c->acc, 0, sizeof(double) * kFgAcc, c->st);
    ttgbf::count_launches(1);
    launch_fg_moments<T>(d, c->sms * 4, c->st, (const T*)c->buf[c->cur], c->g, c->acc);
  }
  double a[kFgAcc];
  cudaMemcpyAsync(a, c->acc, sizeof(a), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fg_check(c);
  const double m0 = a[0];
  std::vector<double> mu(d);
  for (int m = 0; m < d; ++m) mu[m] = a[1 + m] / m0;
  if (mean)
    for (int m = 0; m < d; ++m) mean[m] = c->g.centre[m] + mu[m];
  if (cov)
    for (int m = 0; m < d; ++m)
      for (int l = m; l < d; ++l) {
        const double v = a[1 + d + m * d + l] / m0 - mu[m] * mu[l];
        cov[m * d + l] = cov[l * d + m] = v;
      }
  return fg_check(c);
}

}  // namespace

extern "C" {

size_t ttgbf_fg_workspace_bytes(const ttgbf_grid* grid, int32_t precision) {
  if (!grid || grid->d < 1 || grid->d > kFgMaxD || !grid->n || !grid->lo || !grid->hi) return 0;
  if (precision != 32 && precision != 64) return 0;
  long long total = 1;
  for (int k = 0; k < grid->d; ++k) {
    if (grid->n[k] < 4 || grid->n[k] > 128 || grid->n[k] % 4 || !(grid->hi[k] > grid->lo[k])) return 0;
    total *= grid->n[k];
    if (total >= (1ll << 31)) return 0;  // 32-bit element indices
  }
  return fg_layout(grid, precision).total;
}

int ttgbf_fg_init(ttgbf_fg** out, const ttgbf_grid* grid, const ttgbf_prior* prior, int32_t precision,
                  void* stream, void* workspace, size_t workspace_bytes) {
  if (!out || !prior || !prior->mean || !prior->var) return TTGBF_EINVAL;
  const size_t need = ttgbf_fg_workspace_bytes(grid, precision);
  if (need == 0) return TTGBF_EINVAL;
  const int d = grid->d;
  for (int k = 0; k < d; ++k) {
    if (!std::isfinite(grid->lo[k]) || !std::isfinite(grid->hi[k]) || !std::isfinite(prior->mean[k]) ||
        !std::isfinite(prior->var[k]))
      return TTGBF_ENONFINITE;
    if (!(prior->var[k] > 0.0)) return TTGBF_EINVAL;
  }
  ttgbf_fg* c = new (std::nothrow) ttgbf_fg();
  if (!c) return TTGBF_ENOMEM;
  c->prec = precision;
  c->d = d;
  c->st = (cudaStream_t)stream;
  c->n.assign(grid->n, grid->n + d);
  c->lo.assign(grid->lo, grid->lo + d);
  c->hi.assign(grid->hi, grid->hi + d);
  c->dx.resize(d);
  c->axoff.resize(d);
  c->g.d = d;
  long long total = 1;
  for (int k = d - 1; k >= 0; --k) {
    c->g.stride[k] = total;
    total *= grid->n[k];
  }
  c->g.total = total;
  for (int k = 0; k < d; ++k) {
    c->dx[k] = (c->hi[k] - c->lo[k]) / c->n[k];
    c->delta *= c->dx[k];
    c->axoff[k] = (int)c->axes.size();
    for (int i = 0; i < c->n[k]; ++i) c->axes.push_back(c->lo[k] + (i + 0.5) * c->dx[k]);
    c->g.n[k] = c->n[k];
    c->g.dstride[k] = make_fastdiv((uint32_t)c->g.stride[k]);
    c->g.dn[k] = make_fastdiv((uint32_t)c->n[k]);
    c->g.lo[k] = c->lo[k];
    c->g.dx[k] = c->dx[k];
    c->g.centre[k] = 0.5 * (c->lo[k] + c->hi[k]);
  }
  const FgLayout L = fg_layout(grid, precision);
  if (workspace) {
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 255)) {
      delete c;
      return TTGBF_ENOMEM;
    }
    c->base = (char*)workspace;
  } else {
    if (cudaMalloc(&c->base, L.total) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return TTGBF_ENOMEM;
    }
    c->owns = true;
  }
  c->bytes = L.total;
  c->buf[0] = c->base + L.buf0;
  c->buf[1] = c->base + L.buf1;
  c->acc = (double*)(c->base + L.acc);
  c->off = (double*)(c->base + L.off);
  c->dparams = (double*)(c->base + L.dparams);
  c->mats = c->base + L.mats;
  c->ints = (int*)(c->base + L.ints);
  c->fracs = (double*)(c->base + L.fracs);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaMemcpyAsync(c->dparams, prior->mean, sizeof(double) * d, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->dparams + ttgbf::kMaxD, prior->var, sizeof(double) * d, cudaMemcpyHostToDevice, c->st);
  ttgbf::count_launches(1);
  if (precision == 64) {
    cudaFuncSetAttribute(k_fg_axis<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_fg_pass<double, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 216 * 1024);
    k_fg_prior<double><<<c->sms * 8, 256, 0, c->st>>>((double*)c->buf[0], c->g, c->dparams,
                                                      c->dparams + ttgbf::kMaxD);
    fg_launch_scale_sum<double>(c, c->buf[0]);
  } else {
    cudaFuncSetAttribute(k_fg_axis<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_fg_pass<float, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024);
    cudaFuncSetAttribute(k_fg_pass<float, 32, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    k_fg_prior<float><<<c->sms * 8, 256, 0, c->st>>>((float*)c->buf[0], c->g, c->dparams,
                                                     c->dparams + ttgbf::kMaxD);
    fg_launch_scale_sum<float>(c, c->buf[0]);
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess || fg_check(c) != TTGBF_OK) {
    cudaGetLastError();
    if (c->owns) cudaFree(c->base);
    delete c;
    return TTGBF_ECUDA;
  }
  *out = c;
  return TTGBF_OK;
}

static int fg_guard(ttgbf_fg* c) {
  if (!c) return TTGBF_EINVAL;
  return c->poisoned ? TTGBF_EPOISONED : TTGBF_OK;
}

static int fg_check_FQ(ttgbf_fg* c, const double* F, const double* Q, bool diag_q) {
  if (!F || !Q) return TTGBF_EINVAL;
  const int d = c->d;
  for (int i = 0; i < d * d; ++i)
    if (!std::isfinite(F[i]) || !std::isfinite(Q[i])) return TTGBF_ENONFINITE;
  for (int i = 0; i < d; ++i) {
    if (!(Q[i * d + i] > 0.0)) return TTGBF_EINVAL;
    for (int j = 0; j < d; ++j)
      if (diag_q && i != j && Q[i * d + j] != 0.0) return TTGBF_EINVAL;
  }
  return TTGBF_OK;
}

int ttgbf_fg_predict(ttgbf_fg* c, const double* F, const double* Q) {
  int rc = fg_guard(c);
  if (rc) return rc;
  rc = fg_check_FQ(c, F, Q, true);
  if (rc) return rc;
  return c->prec == 64 ? fg_predict<double>(c, F, Q, false) : fg_predict<float>(c, F, Q, false);
}

int ttgbf_fg_predict_direct(ttgbf_fg* c, const double* F, const double* Q) {
  int rc = fg_guard(c);
  if (rc) return rc;
  rc = fg_check_FQ(c, F, Q, false);
  if (rc) return rc;
  if (c->g.total > (1ll << 22)) return TTGBF_ECAPACITY;
  return c->prec == 64 ? fg_predict<double>(c, F, Q, true) : fg_predict<float>(c, F, Q, true);
}

int ttgbf_fg_update(ttgbf_fg* c, const ttgbf_meas* h, const double* R, const double* z) {
  int rc = fg_guard(c);
  if (rc) return rc;
  if (!h || h->b < 1 || h->b > kFgMaxComps || !h->comp || !R || !z) return TTGBF_EINVAL;
  for (int i = 0; i < h->b; ++i) {
    const ttgbf_meas_comp& cp = h->comp[i];
    if (!cp.htab || cp.nmodes < 1 || cp.nmodes > c->d) return TTGBF_EINVAL;
    if (!(cp.period >= 0.0) || !std::isfinite(cp.period)) return TTGBF_EINVAL;
    for (int k = 0; k < std::min(cp.nmodes, 2); ++k)
      if (cp.modes[k] < 0 || cp.modes[k] >= c->d) return TTGBF_EINVAL;
    if (cp.nmodes >= 2 && cp.modes[0] == cp.modes[1]) return TTGBF_EINVAL;
    if (cp.nmodes >= 3 && cp.modes[1] != cp.modes[0] + cp.nmodes - 1) return TTGBF_EINVAL;
    long long ntab = 1;
    for (int t = 0; t < cp.nmodes; ++t) ntab *= c->n[cp.nmodes <= 2 ? cp.modes[t] : cp.modes[0] + t];
    if (ntab > 2147483647LL) return TTGBF_EINVAL;
    if (!std::isfinite(z[i])) return TTGBF_ENONFINITE;
    for (int j = 0; j < h->b; ++j) {
      if (!std::isfinite(R[i * h->b + j])) return TTGBF_ENONFINITE;
      if (i != j && R[i * h->b + j] != 0.0) return TTGBF_EINVAL;
    }
    if (!(R[i * h->b + i] > 0.0)) return TTGBF_EINVAL;
  }
  return c->prec == 64 ? fg_update<double>(c, h, R, z) : fg_update<float>(c, h, R, z);
}

int ttgbf_fg_estimate(ttgbf_fg* c, double* mean, double* cov, double* log_c, double* log_lik) {
  int rc = fg_guard(c);
  if (rc) return rc;
  rc = c->prec == 64 ? fg_estimate<double>(c, mean, cov) : fg_estimate<float>(c, mean, cov);
  if (log_c) *log_c = c->log_c;
  if (log_lik) *log_lik = c->log_lik;
  return rc;
}

int ttgbf_fg_density(ttgbf_fg* c, double* out, size_t cap) {
  int rc = fg_guard(c);
  if (rc) return rc;
  if (!out || cap < (size_t)c->g.total) return TTGBF_EINVAL;
  if (c->prec == 64) fg_apply_pending<double>(c);
  else fg_apply_pending<float>(c);
  if (c->prec == 64) {
    cudaMemcpyAsync(out, c->buf[c->cur], sizeof(double) * c->g.total, cudaMemcpyDeviceToHost, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return fg_check(c);
  } else {
    std::vector<float> tmp((size_t)c->g.total);
    cudaMemcpyAsync(tmp.data(), c->buf[c->cur], sizeof(float) * c->g.total, cudaMemcpyDeviceToHost, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return fg_check(c);
    for (size_t i = 0; i < tmp.size(); ++i) out[i] = tmp[i];
  }
  return fg_check(c);
}

int ttgbf_fg_free(ttgbf_fg* c) {
  if (!c) return TTGBF_OK;
  cudaStreamSynchronize(c->st);
  if (c->owns && c->base) cudaFree(c->base);
  cudaGetLastError();
  delete c;
  return TTGBF_OK;
}

}  // extern "C"
