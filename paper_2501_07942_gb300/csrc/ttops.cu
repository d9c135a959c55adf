// ttops.cu -- tensor-train operations of one filter step on a batch of filters:
// rank-1 prior (Alg. 2 step 1), re-gridding shear expansion (the hat-weight
// shear x_m += a x_n as an operator of TT rank S), per-mode dense operators
// (cloud-in-cell scaling and the Gaussian transition kernel of Eq.
// tpmconvFFT applied over each core's grid index), the likelihood of Eqs.
// pmf_filtrace_a/b, and moments / normalisation by TT contraction ("sum",
// "dot", "power", Sec. 4.1).
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace ttgbf {
namespace {

struct CorePtrs {
  float* p[kMaxD];
};

// --------------------------------------------------------------- prior
__global__ void k_prior(int B, TTGeom g, CorePtrs cores, int* ranks, const double* axes,
                        const double* mean, const double* var) {
  const int b = blockIdx.x, k = blockIdx.y;
  if (b >= B || k >= g.d) return;
  int off = 0;
  for (int j = 0; j < k; ++j) off += g.n[j];
  float* G = cores.p[k] + (long long)b * g.cap[k];
  for (int i = threadIdx.x; i < g.n[k]; i += blockDim.x) {
    const double x = axes[off + i] - mean[k];
    G[i] = (float)exp(-0.5 * x * x / var[k]);
  }
  if (k == 0 && threadIdx.x == 0) {
    int* rk = ranks + (long long)b * (g.d + 1);
    for (int j = 0; j <= g.d; ++j) rk[j] = 1;
  }
}

// ------------------------------------------------------- shear expansion
// Shear x_m += a x_n (m != n).  With s(i) = a xi_{n,i} / D_m and integer
// shifts t = tmin + u, u < S, the operator is sum_u Shift_t (mode m) x
// diag(hat(t - s)) (mode n) x identity between them: a TT operator of rank S
// on the links between modes lo = min(m,n) and hi = max(m,n).
//   core lo : (r_lo,     N, r_lo+1 S)
//   middle  : (r_l S,    N, r_l+1 S)   = G_l (x) I_S
//   core hi : (r_hi S,   N, r_hi+1)
// The shifted side is mode m, the weighted side mode n.
__global__ void k_shear_expand(int B, TTGeom g, int m, int n, int S, int tmin, const float* wts,
                               CorePtrs cur, CorePtrs alt, const int* ranks, int virt) {
  const int b = blockIdx.z;
  const int lo = m < n ? m : n, hi = m < n ? n : m;
  // virt: the middle cores keep their unexpanded data (G (x) I_S implied)
  const int l = virt ? (blockIdx.y == 0 ? lo : hi) : lo + blockIdx.y;
  if (b >= B || l > hi) return;
  const int* rk = ranks + (long long)b * (g.d + 1);
  const int a0 = rk[l], a1 = rk[l + 1];
  const int N = g.n[l];
  const int o0 = (l == lo) ? a0 : a0 * S;
  const int o1 = (l == hi) ? a1 : a1 * S;
  const int rows = o0 * N;  // < 2^31: at most 160 x 4096 (x 160 columns)
  const float* in = cur.p[l] + (long long)b * g.cap[l];
  float* out = alt.p[l] + (long long)b * g.cap[l];
  const bool shift_side = (l == m);
  const int Nn = g.n[n];
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const float invS = 1.f / (float)S;
  // one warp per output row (x, i); lanes along the row's o1 entries
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += gridDim.x * wpb) {
    const int x = r / N, i = r - x * N;
    float* orow = out + (long long)r * o1;
    if (l == lo) {
      // row x, entries (beta, u): beta < a1, u < S (y < 2^12: the float
      // quotient is exact after truncation)
      for (int y = lane; y < o1; y += 32) {
        const int beta = (int)(((float)y + 0.5f) * invS), u = y - beta * S;
        float v = 0.f;
        if (shift_side) {
          const int src = i - (tmin + u);
          if (src >= 0 && src < N) v = in[((long long)x * N + src) * a1 + beta];
        } else {
          v = wts[u * Nn + i] * in[((long long)x * N + i) * a1 + beta];
        }
        orow[y] = v;
      }
    } else if (l == hi) {
      const int beta = x / S, u = x - beta * S;
      const int src = shift_side ? i - (tmin + u) : i;
      const bool ok = src >= 0 && src < N;
      const float wv = shift_side ? 1.f : wts[u * Nn + i];
      const float* irow = in + ((long long)beta * N + (ok ? src : 0)) * a1;
      for (int y = lane; y < o1; y += 32) orow[y] = ok ? wv * irow[y] : 0.f;
    } else {
      const int alpha = x / S, s0 = x - alpha * S;
      const float* irow = in + ((long long)alpha * N + i) * a1;
      for (int y = lane; y < o1; y += 32) {
        const int beta = (int)(((float)y + 0.5f) * invS), t = y - beta * S;
        orow[y] = (s0 == t) ? irow[beta] : 0.f;
      }
    }
  }
}

__global__ void k_rank_scale(int B, int d, int* ranks, int lo, int hi, int S) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    int* rk = ranks + (long long)b * (d + 1);
    for (int l = lo + 1; l <= hi; ++l) rk[l] *= S;
  }
}

// ------------------------------------------- a wide shear applied in pieces
// A shear's TT operator is a sum over its integer shifts t of E_t (x) H_t
// (shift of mode m, hat weights on mode n).  When that sum is wider than the
// expansion capacity it is split into pieces of consecutive shifts; each
// piece is expanded from a saved copy of the block's cores and rounded, and
// the rounded pieces are added as tensor trains (Sec. 4.1: the TT sum, whose
// end cores concatenate along the inner rank and whose middle cores are
// block diagonal) before a final rounding of the sum.  The accumulator keeps
// every block core at fixed strides [cl][N][cr] (cl = 1 for core 0, else
// capr; cr = 1 for core d-1, else capr), the capacity layout of that core.

// Used part of cores lo..hi copied between two buffer sets of the same layout.
__global__ void k_block_copy(int B, TTGeom g, int lo, CorePtrs src, CorePtrs dst,
                             const int* ranks) {
  const int b = blockIdx.z, l = lo + blockIdx.y;
  if (b >= B) return;
  const int* rk = ranks + (long long)b * (g.d + 1);
  const long long cnt = (long long)rk[l] * g.n[l] * rk[l + 1];
  const float* s = src.p[l] + (long long)b * g.cap[l];
  float* t = dst.p[l] + (long long)b * g.cap[l];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x)
    t[e] = s[e];
}

// Offsets of piece p on the block's inner links lo+1..hi: the accumulated
// ranks of the pieces before it, the sum's rank held to the accumulator's
// capacity capr (never reached: the host allows at most capr / rank_cap
// pieces of rank <= rank_cap).  One thread per filter.
__global__ void k_acc_begin(int B, int d, int lo, int hi, int p, int maxp, int capr,
                            const int* ranks, int* acc_rank, int* piece_off) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int* rk = ranks + (long long)b * (d + 1);
    int* ar = acc_rank + (long long)b * (d + 1);
    int* po = piece_off + ((long long)b * maxp + p) * (d + 1);
    for (int l = lo + 1; l <= hi; ++l) {
      const int o = (p == 0) ? 0 : ar[l];
      po[l] = o;
      ar[l] = min(o + rk[l], capr);
    }
  }
}

__device__ __forceinline__ int acc_stride_left(int l, int capr) { return l == 0 ? 1 : capr; }
__device__ __forceinline__ int acc_stride_right(const TTGeom& g, int l, int capr) {
  return l == g.d - 1 ? 1 : capr;
}

// Piece p's rounded cores (current buffers, current ranks) into the
// accumulator at the piece's offsets.
__global__ void k_acc_scatter(int B, TTGeom g, int lo, int hi, int p, int maxp, int capr,
                              CorePtrs cur, CorePtrs acc, const int* ranks, const int* piece_off) {
  const int b = blockIdx.z, l = lo + blockIdx.y;
  if (b >= B) return;
  const int* rk = ranks + (long long)b * (g.d + 1);
  const int* po = piece_off + ((long long)b * maxp + p) * (g.d + 1);
  const int r0 = rk[l], r1 = rk[l + 1], N = g.n[l];
  const int ro = (l > lo) ? po[l] : 0, co = (l < hi) ? po[l + 1] : 0;
  const int cl = acc_stride_left(l, capr), cr = acc_stride_right(g, l, capr);
  const float* s = cur.p[l] + (long long)b * g.cap[l];
  float* t = acc.p[l] + (long long)b * g.cap[l];
  const long long cnt = (long long)r0 * N * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % r1);
    const long long ai = e / r1;
    const int i = (int)(ai % N), a = (int)(ai / N);
    if (ro + a < cl && co + x < cr) t[((long long)(ro + a) * N + i) * cr + co + x] = s[e];
  }
}

// The piece whose rows (columns) of link l hold index idx.
__device__ __forceinline__ int piece_of(const int* po0, int np, int d, int l, int idx) {
  int p = 0;
  for (int q = 1; q < np; ++q)
    if (po0[(long long)q * (d + 1) + l] <= idx) p = q;
  return p;
}

// The TT sum of the pieces, packed at its ranks into the other buffer set:
// end cores as accumulated, middle cores block diagonal (zero between pieces).
__global__ void k_acc_gather(int B, TTGeom g, int lo, int hi, int np, int maxp, int capr,
                             CorePtrs acc, CorePtrs alt, const int* ranks, const int* acc_rank,
                             const int* piece_off) {
  const int b = blockIdx.z, l = lo + blockIdx.y;
  if (b >= B) return;
  const int* rk = ranks + (long long)b * (g.d + 1);
  const int* ar = acc_rank + (long long)b * (g.d + 1);
  const int* po0 = piece_off + (long long)b * maxp * (g.d + 1);
  const int N = g.n[l];
  const int Rl = (l > lo) ? ar[l] : rk[l], Rr = (l < hi) ? ar[l + 1] : rk[l + 1];
  const int cl = acc_stride_left(l, capr), cr = acc_stride_right(g, l, capr);
  const bool middle = (l > lo && l < hi);
  const float* s = acc.p[l] + (long long)b * g.cap[l];
  float* t = alt.p[l] + (long long)b * g.cap[l];
  const long long cnt = (long long)Rl * N * Rr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % Rr);
    const long long ai = e / Rr;
    const int i = (int)(ai % N), a = (int)(ai / N);
    float v = 0.f;
    if (a < cl && x < cr &&
        (!middle || piece_of(po0, np, g.d, l, a) == piece_of(po0, np, g.d, l + 1, x)))
      v = s[((long long)a * N + i) * cr + x];
    t[e] = v;
  }
}

// The sum's ranks on the inner links (after the gather has read them).
__global__ void k_acc_ranks(int B, int d, int lo, int hi, int* ranks, const int* acc_rank) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    for (int l = lo + 1; l <= hi; ++l) ranks[(long long)b * (d + 1) + l] = acc_rank[(long long)b * (d + 1) + l];
}

// ------------------------------------------------------- per-mode apply
// G'(a, j, b) = sum_i M(j, i) G(a, i, b): one GEMM (N x N) x (N x r_{k+1}) per
// (filter, left index a).
__global__ void k_plan_mode_apply(int B, int k, TTGeom g, const int* ranks, const float* M,
                                  const float* cur, float* alt, GemmWork gw, int cap_in) {
  const int N = g.n[k];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < B * cap_in; q += gridDim.x * blockDim.x) {
    const int b = q / cap_in, a = q - b * cap_in;
    const int* rk = ranks + (long long)b * (g.d + 1);
    const int r0 = rk[k], r1 = rk[k + 1];
    GemmDesc x{M, nullptr, nullptr, 0, 0, 0, N, r1, r1};
    if (a < r0) {
      const long long off = (long long)b * g.cap[k] + (long long)a * N * r1;
      x.B = cur + off;
      x.C = alt + off;
      x.m = N;
      x.n = r1;
      x.k = N;
    }
    gw.desc[q] = x;
  }
}

// W_b = core0 (N0 x r1) * core1 (r1 x N1 r2): the 2-site supercore of modes 0, 1.
__global__ void k_plan_supercore(int B, TTGeom g, const int* ranks, const float* c0, const float* c1,
                                 float* W, long long W_cap, GemmWork gw) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int* rk = ranks + (long long)b * (g.d + 1);
    const int r1 = rk[1], r2 = rk[2];
    const int cols = g.n[1] * r2;
    GemmDesc x{c0 + (long long)b * g.cap[0], c1 + (long long)b * g.cap[1], W + (long long)b * W_cap,
               g.n[0], cols, r1, r1, cols, cols};
    gw.desc[b] = x;
  }
}

// ----------------------------------------------------------- likelihood
// Per filter b: off_b = min_i (z_b - h(i))^2 over the component's table (the
// residual wrapped for an angle-like component, as everywhere below), so that
// the scaled likelihood exp(-((z-h)^2 - off)/(2R)) is <= 1 with maximum 1.
// logoff_b accumulates the dropped factor log(exp(-off/(2R)) / sqrt(2 pi R)).
__global__ void k_lik_offset(int B, const float* htab, int ntab, const float* z, int zstride, int zc,
                             double R, float period, float* off, double* logoff) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const float zb = z[(long long)b * zstride + zc];
  float mn = INFINITY;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) {
    const float e = wrap_residual(zb - htab[i], period);
    mn = fminf(mn, e * e);
  }
  __shared__ float s_m[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = s_m[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fminf(v, s_m[w]);
    off[b] = v;
    logoff[b] += -(double)v / (2.0 * R) - 0.5 * log(2.0 * 3.14159265358979323846 * R);
  }
}

// The same offset for a large table (a factor on three or more modes): a
// grid of chunks per filter, each folding its chunk's minimum into off_b with
// an atomic minimum on the float's bits (non-negative floats order like their
// bit patterns); then k_lik_offset_log adds the dropped factor.
__global__ void k_lik_offset_chunks(int B, const float* htab, long long ntab, const float* z, int zstride,
                                    int zc, float period, float* off) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const float zb = z[(long long)b * zstride + zc];
  float mn = INFINITY;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ntab;
       i += (long long)gridDim.x * blockDim.x) {
    const float e = wrap_residual(zb - htab[i], period);
    mn = fminf(mn, e * e);
  }
  __shared__ float s_m[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = s_m[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fminf(v, s_m[w]);
    atomicMin(reinterpret_cast<unsigned*>(off) + b, __float_as_uint(v));
  }
}

__global__ void k_lik_offset_init(int B, float* off) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) off[b] = INFINITY;
}

__global__ void k_lik_offset_log(int B, double R, const float* off, double* logoff) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    logoff[b] += -(double)off[b] / (2.0 * R) - 0.5 * log(2.0 * 3.14159265358979323846 * R);
}

// W(i0, i1, c) *= exp(-((z - h(i0,i1))^2 - off) / (2R)): Hadamard product of the
// supercore with the (exact, merged-mode) likelihood of a two-mode component.
__global__ void k_lik_apply_2d(int B, float* W, long long W_cap, int N0, int N1, int d, const int* ranks,
                               const float* htab, const float* z, int zstride, int zc, double R,
                               float period, const float* off) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int r2 = ranks[(long long)b * (d + 1) + 2];
  const long long total = (long long)N0 * N1 * r2;
  const float zb = z[(long long)b * zstride + zc];
  const float ob = off[b];
  const float inv2r = (float)(0.5 / R);
  float* Wb = W + (long long)b * W_cap;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / r2;  // i0 * N1 + i1
    const float df = wrap_residual(zb - htab[t], period);
    Wb[e] *= expf(-(df * df - ob) * inv2r);
  }
}

// G_k(a, i, b) *= exp(-((z - h(i))^2 - off) / (2R)): one-mode component.
__global__ void k_lik_apply_1d(int B, float* core, long long cap, int N, int k, int d, const int* ranks,
                               const float* htab, const float* z, int zstride, int zc, double R,
                               float period, const float* off) {
  const int b = blockIdx.y;
  if (b >= B) return;
  const int* rk = ranks + (long long)b * (d + 1);
  const int r0 = rk[k], r1 = rk[k + 1];
  const long long total = (long long)r0 * N * r1;
  const float zb = z[(long long)b * zstride + zc];
  const float ob = off[b];
  const float inv2r = (float)(0.5 / R);
  float* G = core + (long long)b * cap;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)((e / r1) % N);
    const float df = wrap_residual(zb - htab[i], period);
    G[e] *= expf(-(df * df - ob) * inv2r);
  }
}

// -------------------------------------------------------------- moments
// One CTA per filter.  A_kk^(p)(a, b) = sum_i w_p(i) G_kk(a, i, b) with
// w_p(i) = (xi_i - c)^p, p <= 2, accumulated in float64; then vector chains:
//   f_kk = A_kk^(0) f_kk+1 (right sums), mass = f_0 * delta,
//   mean_k  ~ e_k A_k^(1) f_k+1,  E[x_k^2] ~ e_k A_k^(2) f_k+1,
//   E[x_m x_k] ~ u_m A_k^(1) f_k+1 with u_m = e_m A_m^(1) A_m+1^(0) ... A_k-1^(0).
__global__ void k_moments(int B, MomentArgs a, const int* ranks, int rstride, double* Awork,
                          long long awork_stride, double* mass_out, double* mean_out, double* cov_out) {
  extern __shared__ double smd[];
  const int b = blockIdx.x;
  if (b >= B) return;
  const int nc = a.ncores;
  const int P = a.with_moments ? 3 : 1;
  double* f = smd;                              // (nc + 1) x kMaxN
  double* u = f + (kMaxD + 2) * kMaxN;          // nc x kMaxN
  double* e = u + (kMaxD + 1) * kMaxN;          // kMaxN
  double* tmp = e + kMaxN;                      // kMaxN
  double* acc = tmp + kMaxN;                    // 9 x 1024 (group partials)
  double* red = acc + 9 * 1024;                 // 32
  float* xs = reinterpret_cast<float*>(red + 32);  // N: centred coordinates of the current core
  __shared__ double s_mean[kMaxD + 1];
  __shared__ double s_S[(kMaxD + 1) * (kMaxD + 1)];
  const int* rk = ranks + (long long)b * rstride;
  const long long Astride = (long long)kMaxN * kMaxN;
  double* Ab = Awork + (long long)b * awork_stride;

  // ---- per-core weighted sums over the grid index
  for (int kk = 0; kk < nc; ++kk) {
    const int r0 = rk[a.ridx[kk]], r1 = rk[a.ridx[kk + 1]];
    const int N = a.n[kk];
    const float* G = a.core[kk] + (long long)b * a.cap[kk];
    const double* ax = a.axes[kk];
    const double c = a.centre[kk];
    const int npairs = r0 * r1;
    // the centred coordinates in FP32, formed once per core (an FP64
    // subtraction per term and thread would cost more issue time than the
    // whole FP32 sum on this part)
    __syncthreads();
    if (P > 1)
      for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = (float)(ax[i] - c);
    // passes of at most one (alpha, beta) pair per thread (blockDim.x <= 1024
    // pairs, the capacity of each partial-sum slot row of acc)
    const int chunk = (int)blockDim.x;
    for (int pb = 0; pb < npairs; pb += chunk) {
      const int nb = min(chunk, npairs - pb);
      __syncthreads();
      // groups of threads split the grid index of each (alpha, beta); FP32
      // partial sums of at most ceil(N / groups) terms, combined in FP64
      const int groups = max(1, min(3, (int)blockDim.x / nb));
      if ((int)threadIdx.x < nb * groups) {
        const int q = pb + (threadIdx.x % nb);
        const int grp = threadIdx.x / nb;
        const int al = q / r1, be = q - al * r1;
        // four interleaved FP32 partial sums each (a few dozen terms apiece)
        float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
        const float* gp = G + (long long)al * N * r1 + be;
        auto term = [&](int i, float& a0, float& a1, float& a2) {
          const float v = gp[(long long)i * r1];
          a0 += v;
          if (P > 1) {
            const float x = xs[i];
            a1 = fmaf(x, v, a1);
            a2 = fmaf(x * x, v, a2);
          }
        };
        int i = grp;
        for (; i + 3 * groups < N; i += 4 * groups) {
#pragma unroll
          for (int m = 0; m < 4; ++m) term(i + m * groups, s0[m], s1[m], s2[m]);
        }
        for (; i < N; i += groups) term(i, s0[0], s1[0], s2[0]);
        // one slot per (group, pair): no atomics
        acc[grp * 1024 + (q - pb)] = ((double)s0[0] + s0[1]) + ((double)s0[2] + s0[3]);
        if (P > 1) {
          acc[(3 + grp) * 1024 + (q - pb)] = ((double)s1[0] + s1[1]) + ((double)s1[2] + s1[3]);
          acc[(6 + grp) * 1024 + (q - pb)] = ((double)s2[0] + s2[1]) + ((double)s2[2] + s2[3]);
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        for (int p = 0; p < P; ++p) {
          double v = 0.0;
          for (int g = 0; g < groups; ++g) v += acc[(3 * p + g) * 1024 + t];
          acc[p * 1024 + t] = v;  // slot (3 p) * 1024 + t is only read by this thread
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        for (int p = 0; p < P; ++p) Ab[((long long)kk * 3 + p) * Astride + pb + t] = acc[p * 1024 + t];
      }
      __syncthreads();
    }
  }
  __syncthreads();

  // every warp computes the (short, len <= kMaxN) dot product itself: same
  // order everywhere, no barrier, no per-thread loop over warp partials
  auto block_dot = [&](const double* x, const double* y, int len) -> double {
    double s = 0.0;
    for (int t = (int)(threadIdx.x & 31); t < len; t += 32) s += x[t] * y[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  };
  // y (len r1) = x (len r0) * A (r0 x r1)
  auto vecmat = [&](const double* x, const double* A, int r0, int r1, double* y) {
    for (int be = threadIdx.x; be < r1; be += blockDim.x) {
      double s = 0.0;
      for (int al = 0; al < r0; ++al) s += x[al] * A[(long long)al * r1 + be];
      y[be] = s;
    }
    __syncthreads();
  };

  // ---- right sums
  if (threadIdx.x == 0) f[nc * kMaxN] = 1.0;
  __syncthreads();
  for (int kk = nc - 1; kk >= 0; --kk) {
    const int r0 = rk[a.ridx[kk]], r1 = rk[a.ridx[kk + 1]];
    const double* A0 = Ab + ((long long)kk * 3 + 0) * Astride;
    for (int al = threadIdx.x; al < r0; al += blockDim.x) {
      double s = 0.0;
      for (int be = 0; be < r1; ++be) s += A0[(long long)al * r1 + be] * f[(kk + 1) * kMaxN + be];
      f[kk * kMaxN + al] = s;
    }
    __syncthreads();
  }
  const double mraw = f[0];
  if (a.with_moments) {
    if (threadIdx.x == 0) e[0] = 1.0;
    __syncthreads();
    for (int kk = 0; kk < nc; ++kk) {
      const int r0 = rk[a.ridx[kk]], r1 = rk[a.ridx[kk + 1]];
      const double* A0 = Ab + ((long long)kk * 3 + 0) * Astride;
      const double* A1 = Ab + ((long long)kk * 3 + 1) * Astride;
      const double* A2 = Ab + ((long long)kk * 3 + 2) * Astride;
      const double* fr = f + (kk + 1) * kMaxN;
      vecmat(e, A2, r0, r1, tmp);
      const double s2 = block_dot(tmp, fr, r1);
      for (int mm = 0; mm < kk; ++mm) {
        vecmat(u + mm * kMaxN, A1, r0, r1, tmp);
        const double sc = block_dot(tmp, fr, r1);
        if (threadIdx.x == 0) s_S[mm * (kMaxD + 1) + kk] = sc;
        vecmat(u + mm * kMaxN, A0, r0, r1, tmp);
        for (int t = threadIdx.x; t < r1; t += blockDim.x) u[mm * kMaxN + t] = tmp[t];
        __syncthreads();
      }
      vecmat(e, A1, r0, r1, tmp);
      const double s1 = block_dot(tmp, fr, r1);
      for (int t = threadIdx.x; t < r1; t += blockDim.x) u[kk * kMaxN + t] = tmp[t];
      __syncthreads();
      vecmat(e, A0, r0, r1, tmp);
      for (int t = threadIdx.x; t < r1; t += blockDim.x) e[t] = tmp[t];
      if (threadIdx.x == 0) {
        s_mean[kk] = s1;
        s_S[kk * (kMaxD + 1) + kk] = s2;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    mass_out[b] = mraw * a.delta;
    if (a.with_moments && mean_out != nullptr) {
      for (int k = 0; k < nc; ++k) mean_out[(long long)b * nc + k] = a.centre[k] + s_mean[k] / mraw;
      for (int k = 0; k < nc; ++k)
        for (int l = k; l < nc; ++l) {
          const double mk = s_mean[k] / mraw, ml = s_mean[l] / mraw;
          const double v = s_S[k * (kMaxD + 1) + l] / mraw - mk * ml;
          cov_out[((long long)b * nc + k) * nc + l] = v;
          cov_out[((long long)b * nc + l) * nc + k] = v;
        }
    }
  }
  if (a.scale_core != nullptr) {
    const int kk = a.scale_idx;
    const int r0 = rk[a.ridx[kk]], r1 = rk[a.ridx[kk + 1]];
    const long long total = (long long)r0 * a.n[kk] * r1;
    float* G = a.scale_core + (long long)b * a.scale_cap;
    const float inv = (float)(1.0 / (mraw * a.delta));
    for (long long t = threadIdx.x; t < total; t += blockDim.x) G[t] *= inv;
  }
}

constexpr int kMomentMaxN = 4096;  // grid points per mode (the library's limit)
constexpr int kMomentSmemDoubles =
    (kMaxD + 2) * kMaxN + (kMaxD + 1) * kMaxN + 2 * kMaxN + 9 * 1024 + 32 + kMomentMaxN / 2;

}  // namespace

// -------------------------------------------------------------- launchers
static CorePtrs to_ptrs(float* const* p, int d) {
  CorePtrs c{};
  for (int k = 0; k < d; ++k) c.p[k] = p[k];
  return c;
}

void launch_prior(cudaStream_t st, int B, const TTGeom& g, float* const* cores, int* ranks,
                  const double* axes, const double* mean, const double* var) {
  count_launches(1);
  k_prior<<<dim3(B, g.d), 128, 0, st>>>(B, g, to_ptrs(cores, g.d), ranks, axes, mean, var);
}

void launch_shear_expand(cudaStream_t st, int B, const TTGeom& g, int m, int n, int S, int tmin,
                         const float* weights, float* const* cur, float* const* alt,
                         const int* ranks, int virt) {
  count_launches(1);
  const int lo = m < n ? m : n, hi = m < n ? n : m;
  const int ny = virt ? 2 : hi - lo + 1;
  k_shear_expand<<<dim3(32, ny, B), 256, 0, st>>>(B, g, m, n, S, tmin, weights, to_ptrs(cur, g.d),
                                                 to_ptrs(alt, g.d), ranks, virt);
}

void launch_rank_scale(cudaStream_t st, int B, int d, int* ranks, int lo, int hi, int S) {
  count_launches(1);
  k_rank_scale<<<(B + 255) / 256, 256, 0, st>>>(B, d, ranks, lo, hi, S);
}

void launch_block_copy(cudaStream_t st, int B, const TTGeom& g, int lo, int hi,
                       float* const* src, float* const* dst, const int* ranks) {
  count_launches(1);
  k_block_copy<<<dim3(64, hi - lo + 1, B), 256, 0, st>>>(B, g, lo, to_ptrs(src, g.d),
                                                        to_ptrs(dst, g.d), ranks);
}

void launch_acc_piece(cudaStream_t st, int B, const TTGeom& g, int lo, int hi, int p, int maxp,
                      int capr, float* const* cur, float* const* acc, const int* ranks,
                      int* acc_rank, int* piece_off) {
  count_launches(2);
  k_acc_begin<<<(B + 127) / 128, 128, 0, st>>>(B, g.d, lo, hi, p, maxp, capr, ranks, acc_rank,
                                               piece_off);
  k_acc_scatter<<<dim3(64, hi - lo + 1, B), 256, 0, st>>>(B, g, lo, hi, p, maxp, capr,
                                                         to_ptrs(cur, g.d), to_ptrs(acc, g.d),
                                                         ranks, piece_off);
}

void launch_acc_sum(cudaStream_t st, int B, const TTGeom& g, int lo, int hi, int np, int maxp,
                    int capr, float* const* acc, float* const* alt, int* ranks,
                    const int* acc_rank, const int* piece_off) {
  count_launches(2);
  k_acc_gather<<<dim3(64, hi - lo + 1, B), 256, 0, st>>>(B, g, lo, hi, np, maxp, capr,
                                                        to_ptrs(acc, g.d), to_ptrs(alt, g.d),
                                                        ranks, acc_rank, piece_off);
  k_acc_ranks<<<(B + 127) / 128, 128, 0, st>>>(B, g.d, lo, hi, ranks, acc_rank);
}

void launch_plan_mode_apply(cudaStream_t st, int B, int k, const TTGeom& g, const int* ranks,
                            const float* M, const float* cur, float* alt, GemmWork gw, int cap_in) {
  count_launches(1);
  const int total = B * cap_in;
  k_plan_mode_apply<<<(total + 255) / 256, 256, 0, st>>>(B, k, g, ranks, M, cur, alt, gw, cap_in);
  launch_scan_tiles(st, gw);
}

void launch_plan_supercore(cudaStream_t st, int B, const TTGeom& g, const int* ranks,
                           const float* c0, const float* c1, float* W, long long W_cap,
                           GemmWork gw) {
  count_launches(1);
  k_plan_supercore<<<(B + 255) / 256, 256, 0, st>>>(B, g, ranks, c0, c1, W, W_cap, gw);
  launch_scan_tiles(st, gw);
}

void launch_lik_offset(cudaStream_t st, int B, const float* htab, int ntab, const float* z,
                       int zstride, int zc, double R, float period, float* off, double* logoff) {
  if (ntab <= (1 << 16)) {
    count_launches(1);
    k_lik_offset<<<B, 256, 0, st>>>(B, htab, ntab, z, zstride, zc, R, period, off, logoff);
    return;
  }
  // about 16 entries per thread, at most 128 chunks of 256 threads per filter
  const int chunks = (int)std::min<long long>(128, ((long long)ntab + 4095) / 4096);
  count_launches(3);
  k_lik_offset_init<<<(B + 255) / 256, 256, 0, st>>>(B, off);
  k_lik_offset_chunks<<<dim3(chunks, B), 256, 0, st>>>(B, htab, ntab, z, zstride, zc, period, off);
  k_lik_offset_log<<<(B + 255) / 256, 256, 0, st>>>(B, R, off, logoff);
}

void launch_lik_apply_2d(cudaStream_t st, int B, float* W, long long W_cap, int N0, int N1,
                         const int* ranks, int d, const float* htab, const float* z, int zstride,
                         int zc, double R, float period, const float* off) {
  count_launches(1);
  k_lik_apply_2d<<<dim3(64, B), 256, 0, st>>>(B, W, W_cap, N0, N1, d, ranks, htab, z, zstride, zc, R,
                                             period, off);
}

void launch_lik_apply_1d(cudaStream_t st, int B, float* core, long long cap, int N, int k, int d,
                         const int* ranks, const float* htab, const float* z, int zstride, int zc,
                         double R, float period, const float* off) {
  count_launches(1);
  k_lik_apply_1d<<<dim3(16, B), 256, 0, st>>>(B, core, cap, N, k, d, ranks, htab, z, zstride, zc, R,
                                             period, off);
}

void launch_moments(cudaStream_t st, int B, const MomentArgs& a, const int* ranks, int rstride,
                    double* Awork, long long awork_stride, double* mass, double* mean, double* cov) {
  count_launches(1);
  k_moments<<<B, 256, kMomentSmemDoubles * sizeof(double), st>>>(B, a, ranks, rstride, Awork,
                                                                  awork_stride, mass, mean, cov);
}

// log c = log(mass) + logoff, added to the log-likelihood; add != 0: also
// added to this step's log c (a further factor of the same update).
__global__ void k_logc(int B, const double* mass, const double* logoff, double* log_c, double* log_lik,
                       int add) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const double lc = log(mass[b]) + logoff[b];
    log_c[b] = add ? log_c[b] + lc : lc;
    log_lik[b] += lc;
  }
}

void launch_logc(cudaStream_t st, int B, const double* mass, const double* logoff, double* log_c,
                 double* log_lik, int add) {
  count_launches(1);
  k_logc<<<(B + 255) / 256, 256, 0, st>>>(B, mass, logoff, log_c, log_lik, add);
}

// One stage of contracting a TT into its full tensor (a diagnostic for small
// grids): Y[p][i][b] = sum_a X[p][a] G[a][i][b], with X the row vector 1 for
// the first core (ra = 1); float32 cores, float64 accumulation.
__global__ void k_densify_stage(const double* X, long long P, int ra, const float* G, int n, int rb, double* Y) {
  const long long tot = P * n * rb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t % rb);
    const long long pi = t / rb;
    const int i = (int)(pi % n);
    const long long p = pi / n;
    double s = 0.0;
    if (!X) {
      s = (double)G[(long long)i * rb + b];
    } else {
      for (int a = 0; a < ra; ++a) s += X[p * ra + a] * (double)G[((long long)a * n + i) * rb + b];
    }
    Y[t] = s;
  }
}

void launch_densify_stage(cudaStream_t st, const double* X, long long P, int ra, const float* G, int n, int rb,
                          double* Y) {
  count_launches(1);
  const long long tot = P * n * rb;
  const long long blocks = std::min<long long>((tot + 255) / 256, 152LL * 8);
  k_densify_stage<<<(int)std::max<long long>(blocks, 1), 256, 0, st>>>(X, P, ra, G, n, rb, Y);
}

void set_ttops_attributes() {
  cudaFuncSetAttribute(k_moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMomentSmemDoubles * (int)sizeof(double));
}


}  // namespace ttgbf
