// linalg.cu -- stage plans, the SVD of the R factors and the grouped GEMM
// used by TT rounding (Sec. 4.1 "round"; Alg. 2 steps 2 and 4).
//
// One rounding stage (one core of the right-to-left orthogonalisation sweep,
// or one link of the left-to-right truncation sweep) is:
//   plan    -> per filter, the tall matrix whose R factor is needed
//   TSQR    -> R (n x n) by register-resident Householder QR (tsqr.cu)
//   SVD     -> R = U S V^T (pivoted QR, then one-sided Jacobi on the
//              numerically significant rows), rank choice, factors P1, P2
//   plan2   -> GEMM descriptors for "new core = unfolding * P" and
//              "neighbour core = P * neighbour"
//   GEMM    -> grouped SIMT FP32 GEMM over all filters
// Every problem size is read from the device rank array.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace ttgbf {
namespace {

// Smallest magnitude treated as non-zero by the factorisations (above the
// FP32 denormal range, so that 1/x cannot overflow).
constexpr float kTiny = 1e-30f;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place exclusive scan of o[0..n) by one CTA of at most 1024 threads;
// writes the total to o[n].
__device__ void block_scan_inplace(int* o, int n) {
  __shared__ int s_carry;
  __shared__ int s_tmp[1024];
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = (i < n) ? o[i] : 0;
    s_tmp[threadIdx.x] = v;
    __syncthreads();
    for (int s = 1; s < (int)blockDim.x; s <<= 1) {
      const int t = (threadIdx.x >= (unsigned)s) ? s_tmp[threadIdx.x - s] : 0;
      __syncthreads();
      s_tmp[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) o[i] = s_carry + s_tmp[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_tmp[blockDim.x - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) o[n] = s_carry;
  __syncthreads();
}

// ------------------------------------------------------------ Jacobi SVD
// Pair k of round r (k < npad / 2, r < npad - 1) of the circle method on
// npad (even) columns; the sums below stay under 2 m, so one conditional
// subtraction replaces the modulo.
__device__ __forceinline__ void jacobi_pair(int k, int r, int npad, int* p, int* q) {
  const int m = npad - 1;
  if (k == 0) {
    *p = 0;
    *q = 1 + r;
  } else {
    const int a = k + r, b = m - k + r;
    *p = 1 + (a >= m ? a - m : a);
    *q = 1 + (b >= m ? b - m : b);
  }
}

// One sweep's rounds of the one-sided Jacobi method (circle ordering) on the
// kp columns of M (stride ldm floats, zero padded), one pair per group of LPP
// lanes (a warp issues the instructions of 32 / LPP pairs at once): lane gl
// of a group holds the float4s gl + LPP c (c < 32 / LPP) of both columns,
// i.e. the first 128 entries with conflict-free 16-byte accesses, and, with
// EXT (ldm = 160, LPP = 16), lanes gl < 8 also float4 32 + gl.  Returns the
// rotations counted on lanes gl = 0; *cmax gets the largest |cos| of the
// angle between two columns that were rotated (the convergence measure).
template <int LPP, bool EXT>
__device__ __forceinline__ int jacobi_rounds(float* M, float* nrm, int kp, int npad, int ldm,
                                             float floor2, float tol, float* cmax) {
  static_assert(LPP == 8 || LPP == 16, "group width");
  static_assert(!EXT || LPP == 16, "the 160-entry layout uses 16-lane groups");
  constexpr int C4 = 32 / LPP;  // float4 of the first 128 entries per lane
  constexpr int PW = 32 / LPP;  // pairs per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / LPP, gl = lane % LPP;
  const bool gext = EXT && gl < 8;
  float4* const M4 = reinterpret_cast<float4*>(M);
  int myrot = 0;
  float mx = 0.f;
  for (int r = 0; r < npad - 1; ++r) {
    // warp-uniform loop: every group reaches the shuffles of every pass
    for (int q0 = PW * warp; q0 < npad / 2; q0 += PW * nwarps) {
      const int q = q0 + grp;
      int pp = 0, qq = 0;
      bool act = q < npad / 2;
      if (act) {
        jacobi_pair(q, r, npad, &pp, &qq);
        act = pp < kp && qq < kp;
      }
      float4* const xp = M4 + (pp * ldm >> 2);
      float4* const yp = M4 + (qq * ldm >> 2);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 x[C4], y[C4], xe = z4, ye = z4;
#pragma unroll
      for (int c = 0; c < C4; ++c) {
        x[c] = act ? xp[gl + LPP * c] : z4;
        y[c] = act ? yp[gl + LPP * c] : z4;
      }
      if (act && gext) {
        xe = xp[32 + gl];
        ye = yp[32 + gl];
      }
      float g = xe.x * ye.x + xe.y * ye.y + xe.z * ye.z + xe.w * ye.w;
#pragma unroll
      for (int c = 0; c < C4; ++c)
        g += x[c].x * y[c].x + x[c].y * y[c].y + x[c].z * y[c].z + x[c].w * y[c].w;
#pragma unroll
      for (int o = LPP / 2; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
      if (!act) continue;  // no shuffles below
      const float al = nrm[pp], be = nrm[qq];
      if (g == 0.f || fminf(al, be) <= floor2) continue;
      // al, be > 0 here; sqrt(al be) from the approximate reciprocal roots
      const float cosang = fabsf(g) * rsqrtf(al) * rsqrtf(be);
      if (!(cosang > tol)) continue;
      mx = fmaxf(mx, cosang);
      // rotation parameters need not be correctly rounded: (cth, sth)
      // below is orthogonal for any tt
      const float zeta = __fdividef(be - al, 2.f * g);
      const float az = fabsf(zeta);
      const float w = fmaf(zeta, zeta, 1.f);  // >= 1
      const float tt = (az > 1e15f ? __fdividef(0.5f, az) : __fdividef(1.f, az + w * rsqrtf(w))) *
                       (zeta >= 0.f ? 1.f : -1.f);
      const float cth = rsqrtf(fmaf(tt, tt, 1.f));
      const float sth = cth * tt;
      auto rot = [&](const float4& a, const float4& b, float4* pa, float4* pb) {
        *pa = make_float4(cth * a.x - sth * b.x, cth * a.y - sth * b.y, cth * a.z - sth * b.z,
                          cth * a.w - sth * b.w);
        *pb = make_float4(sth * a.x + cth * b.x, sth * a.y + cth * b.y, sth * a.z + cth * b.z,
                          sth * a.w + cth * b.w);
      };
#pragma unroll
      for (int c = 0; c < C4; ++c) rot(x[c], y[c], xp + gl + LPP * c, yp + gl + LPP * c);
      if (gext) rot(xe, ye, xp + 32 + gl, yp + 32 + gl);
      if (gl == 0) {
        nrm[pp] = al - tt * g;
        nrm[qq] = be + tt * g;
        ++myrot;
      }
    }
    __syncthreads();
  }
  *cmax = mx;
  return myrot;
}

// Block sum for the SVD kernel (blockDim a multiple of 32, <= 1024).  Every
// value summed here is non-negative, so FP32 keeps a relative accuracy of
// about n u; FP64 would cost ~60x the issue slots on this part.
__device__ float block_sum_f(float v, float* red) {
  v = warp_sum(v);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (lane == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  // every warp reduces the per-warp partials itself (same order in every
  // warp, so every thread gets the same value)
  return warp_sum(lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f);
}

// Pivoted Householder QR of the n x n matrix A (column-major, ld n, shared
// memory) with its columns in registers: of the nw warps, warp w owns the
// physical columns w + nw t (t < T = ceil(n / nw)) and lane l their rows
// l + 32 e (e < E = ceil(n / 32)), so an update touches no shared memory but
// the reflector.
// Per step: every warp reduces the per-warp pivot candidates; the warp owning
// the pivot forms its reflector (v = 1 at row k, scaled entries below; tau)
// and publishes it; every warp applies it to its remaining columns, writes
// their now final row-k entries R'(k, .) to A, downdates their norms
// (recomputed when more than 99.9 % has cancelled) and leaves its candidate
// for the next step.  Same stopping rule and outputs as the shared-memory
// variant: perm[pos] = physical column at pivot position pos (positions k'..
// n-1 get the columns never pivoted, ascending), R'(r, pos) =
// A[perm[pos] n + r] for r < pos, rdiag = diag(R'), *dropped2 = squared norm
// of the columns left over.  Returns k'.
template <int E, int T>
__device__ __forceinline__ int qrcp_reg(float* A, int n, float* nref, int kcap, float stop2, int* perm,
                        float* rdiag, float* vbuf, int* mark, float* s_red, float* s_redf,
                        int* s_redi, float* s_tau, double* dropped2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float a[T][E];
  float nr2[T];  // current squared norms; nref (shared, n floats, on entry the
                 // initial norms) keeps the norm at the last recomputation
  unsigned alive = 0;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int pc = warp + nw * t;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = lane + 32 * e;
      a[t][e] = (pc < n && i < n) ? A[pc * n + i] : 0.f;
    }
    nr2[t] = pc < n ? nref[pc] : 0.f;
    if (pc < n) alive |= 1u << t;
  }
  auto candidates = [&]() {
    float rl = 0.f, bv = -1.f;
    int bx = n;
#pragma unroll
    for (int t = 0; t < T; ++t)
      if ((alive >> t) & 1u) {
        rl += nr2[t];
        if (nr2[t] > bv) {
          bv = nr2[t];
          bx = warp + nw * t;
        }
      }
    if (lane == 0) {
      s_red[warp] = rl;
      s_redf[warp] = bv;
      s_redi[warp] = bx;
    }
  };
  candidates();
  __syncthreads();
  int k = 0;
  for (;; ++k) {
    // every warp reduces the nw candidates (same result everywhere)
    const float rem = warp_sum(lane < nw ? s_red[lane] : 0.f);
    float best = lane < nw ? s_redf[lane] : -1.f;
    int bi = lane < nw ? s_redi[lane] : n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (k >= kcap || (k > 0 && rem <= stop2) || bi >= n) {
      *dropped2 = (double)rem;
      break;
    }
    const int ek = k >> 5, lk = k & 31;
    if (warp == bi % nw) {
      const int tp = bi / nw;
      float col[E];
#pragma unroll
      for (int e = 0; e < E; ++e) col[e] = 0.f;
#pragma unroll
      for (int t = 0; t < T; ++t)
        if (t == tp) {
#pragma unroll
          for (int e = 0; e < E; ++e) col[e] = a[t][e];
        }
      float ak = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e == ek) ak = col[e];
      const float alpha = __shfl_sync(0xffffffffu, ak, lk);
      float ss = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (lane + 32 * e > k) ss = fmaf(col[e], col[e], ss);
      ss = warp_sum(ss);
      float tot = fmaf(alpha, alpha, ss), tail2 = ss, scale = 1.f;
      // squares are exact enough unless the sum leaves [1e-30, 1e30]; such
      // columns take a second pass scaled by the column maximum
      const bool rescale = tot != 0.f && !(tot >= 1e-30f && tot <= 1e30f);
      if (rescale) {
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (lane + 32 * e > k) mx = fmaxf(mx, fabsf(col[e]));
        mx = fmaxf(warp_max(mx), fabsf(alpha));
        const float inv = mx > 0.f ? 1.f / mx : 0.f;
        float s2 = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (lane + 32 * e > k) {
            const float x = col[e] * inv;
            s2 = fmaf(x, x, s2);
          }
        s2 = warp_sum(s2);
        const float al = alpha * inv;
        tot = fmaf(al, al, s2);
        tail2 = s2;
        scale = mx;
      }
      float tau = 0.f, beta = alpha, scl = 0.f;
      if (tail2 > 0.f && tot > 0.f) {
        const float rs = rsqrtf(tot);
        const float nm = tot * rs * scale;
        const float aa = fabsf(alpha);
        beta = alpha >= 0.f ? -nm : nm;
        tau = fmaf(aa / scale, rs, 1.f);  // (|alpha| + nm) / nm
        const float am = aa + nm;
        scl = alpha >= 0.f ? __frcp_rn(am) : -__frcp_rn(am);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < n) vbuf[i] = i > k ? col[e] * scl : (i == k ? 1.f : 0.f);
      }
      if (lane == 0) {
        *s_tau = tau;
        rdiag[k] = beta;
        perm[k] = bi;
      }
      alive &= ~(1u << tp);
    }
    __syncthreads();
    const float tau = *s_tau;
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = lane + 32 * e;
      v[e] = i < n ? vbuf[i] : 0.f;
    }
    float dot[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      float d0 = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e) d0 = fmaf(v[e], a[t][e], d0);
      dot[t] = d0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int t = 0; t < T; ++t) dot[t] += __shfl_xor_sync(0xffffffffu, dot[t], o);
    float rl = 0.f, bv = -1.f;
    int bx = n;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      if (!((alive >> t) & 1u)) continue;  // warp-uniform
      const float f = tau * dot[t];
#pragma unroll
      for (int e = 0; e < E; ++e) a[t][e] = fmaf(-f, v[e], a[t][e]);
      float xk = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e == ek) xk = a[t][e];
      const float rk = __shfl_sync(0xffffffffu, xk, lk);
      const int pc = warp + nw * t;
      if (lane == lk) A[pc * n + k] = rk;  // R'(k, pc) is final
      float nr = nr2[t] - rk * rk;
      if (!(nr >= 1e-3f * nref[pc])) {  // cancelled (or NaN): recompute
        float sq = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e)
          if (lane + 32 * e > k) sq = fmaf(a[t][e], a[t][e], sq);
        nr = warp_sum(sq);
        __syncwarp();
        if (lane == 0) nref[pc] = nr;
      }
      nr2[t] = nr;
      rl += nr;
      if (nr > bv || (nr == bv && pc < bx)) {
        bv = nr;
        bx = pc;
      }
    }
    if (lane == 0) {
      s_red[warp] = rl;
      s_redf[warp] = bv;
      s_redi[warp] = bx;
    }
    __syncthreads();
  }
  // positions k..n-1: the columns never pivoted, ascending (mark the
  // pivots in `mark` (n ints), then one warp compacts the rest)
  for (int c = threadIdx.x; c < n; c += blockDim.x) mark[c] = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) mark[perm[q]] = 1;
  __syncthreads();
  if (warp == 0) {
    int pos = k;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int c = c0 + lane;
      const bool left = c < n && mark[c] == 0;
      const unsigned bal = __ballot_sync(0xffffffffu, left);
      if (left) perm[pos + __popc(bal & ((1u << lane) - 1u))] = c;
      pos += __popc(bal);
    }
  }
  __syncthreads();
  return k;
}

// SVD of the n x n R factor of problem b, in three steps:
//  1. Householder QR with column pivoting, R P = Q' R', stopped once the
//     columns left over have Frobenius norm below the stage's drop level (or
//     after rank_cap + 16 steps when truncating); their norm is added to the
//     discarded tail.  Pivoting also preconditions step 2.  The columns stay
//     in registers (qrcp_reg) for 32 warps, and for 16 warps up to 96
//     columns; otherwise in shared memory.
//  2. One-sided Jacobi on the k' x n leading rows of R' (their transposes as
//     k' columns of length n): only k' - 1 rounds per sweep, one pair per
//     8- or 16-lane group (jacobi_rounds), stopped once a sweep's rotations
//     are in the quadratic regime.
//  3. The right singular vectors (normalised columns, in the order of
//     decreasing singular value) get one Loewdin correction (classical
//     Gram-Schmidt applied twice when they are further from orthonormal) and
//     are un-permuted, so that the factor pair the stage applies (V S^-1 with
//     S V^T, or S^-1 V^T with V S) multiplies to an exact projector.
// Then the stage's rank choice and factor output.  One CTA per filter; the
// FP64 scalars (norm, threshold, tails, rank choice) are formed by thread 0.
__global__ void __launch_bounds__(1024) k_svd(TsqrWork w, int B, int mode, int rank_cap, double eps,
                                             int d, int first, RoundState rs, float* P1, float* P2,
                                             float* core0_out, long long core0_cap, double* flops) {
  extern __shared__ float sm[];
  const int b = blockIdx.x;
  if (b >= B) return;
  const TsqrProblem p = w.prob[b];
  const int n = p.src.n;
  const float* R = ((p.nlev - 1) & 1) ? p.stack1 : p.stack0;
  float* A = sm;                        // QRCP work, column-major n x n (ld n); later Q of step 3
  float* M = sm + kMaxN * kMaxN;        // Jacobi matrix, column-major n x k' (ld n)
  float* nrm = M + kMaxN * kMaxN;       // [kMaxN] squared column norms
  float* sig = nrm + kMaxN;             // [kMaxN] sorted singular values
  float* rdiag = sig + kMaxN;           // [kMaxN] diagonal of R'
  float* coef = rdiag + kMaxN;          // [kMaxN] Gram-Schmidt coefficients
  int* perm = (int*)(coef + kMaxN);     // [kMaxN] column permutation of the QRCP
  int* pinv = perm + kMaxN;             // [kMaxN] its inverse
  int* ord = pinv + kMaxN;              // [kMaxN] Jacobi columns by decreasing norm
  __shared__ float s_red[32];
  __shared__ float s_redf[32];
  __shared__ int s_redi[32];
  __shared__ float s_tau;
  __shared__ int s_rot, s_rank;
  __shared__ double s_flops;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  for (int t = tid; t < n * n; t += blockDim.x) {
    const int i = t / n, c = t - i * n;
    A[c * n + i] = R[t];
  }
  for (int c = tid; c < n; c += blockDim.x) perm[c] = c;
  if (tid == 0) s_flops = 0.0;
  __syncthreads();
  for (int c = warp; c < n; c += nwarps) {
    float s = 0.f;
    for (int i = lane; i < n; i += 32) s += A[c * n + i] * A[c * n + i];
    s = warp_sum(s);
    if (lane == 0) nrm[c] = s;
  }
  __syncthreads();
  float totf;
  {
    float s = 0.f;
    for (int c = tid; c < n; c += blockDim.x) s += nrm[c];
    totf = block_sum_f(s, s_red);
  }
  // The FP64 scalars (norm, truncation threshold) are formed by thread 0
  // alone: FP64 instructions issue at a small fraction of the FP32 rate on
  // this part, so a few of them per thread would cost more than the FP32
  // work around them.  The per-step tests use the FP32 threshold stop2f.
  __shared__ float s_stop2f;
  double normA = 0.0, delta = 0.0;
  if (tid == 0) {
    const double tot = (double)totf;
    if (mode != kStageRight) normA = first ? sqrt(tot) : rs.normA[b];
    delta = (mode == kStageRight || d <= 1) ? 0.0 : eps * normA / sqrt((double)(d - 1));
    // orthogonalisation drops what is left once it is at the FP32 noise level
    // of R (1e-7 sqrt(n) ||R||_F); truncation stops once the rest is below
    // 0.3 delta
    const double stop2 = (mode == kStageRight) ? 1e-14 * n * tot : 0.09 * delta * delta;
    s_stop2f = (float)stop2;
  }
  __syncthreads();
  const float stop2f = s_stop2f;
  const int kcap = (mode == kStageRight) ? n : min(n, rank_cap + 16);

  // ---- 1. QR with column pivoting.  Columns never move: perm[pos] is the
  // physical column at pivot position pos, and R'(r, pos) = A[perm[pos] n + r].
  // Two barriers per step: warp 0 picks the pivot and forms its reflector;
  // then every warp updates its trailing columns, downdates their norms
  // (recomputed when more than 99.9 % has cancelled) and leaves its part of
  // the next pivot search.
  // With 32 warps, or 16 warps and n <= 96, the columns live in registers
  // (qrcp_reg); otherwise in shared memory.
  int k = 0;
  double dropped2 = 0.0;
  float* vbuf = coef;  // the pivot's reflector; coef is free until step 3
  // (pinv serves as scratch; it is set from perm after the QR)
#define TTGBF_QRCP(E, T)                                                                 \
  k = qrcp_reg<E, T>(A, n, nrm, kcap, stop2f, perm, rdiag, vbuf, pinv, s_red, s_redf, s_redi, \
                     &s_tau, &dropped2)
  const bool reg = nwarps == 32 || (nwarps == 16 && n <= 96);
  if (nwarps == 32) {
    const int E = (n + 31) >> 5;
    if (E <= 1) TTGBF_QRCP(1, 1);
    else if (E == 2) TTGBF_QRCP(2, 2);
    else if (E == 3) TTGBF_QRCP(3, 3);
    else if (E == 4) TTGBF_QRCP(4, 4);
    else TTGBF_QRCP(5, 5);
  } else if (reg) {
    const int T = (n + 15) >> 4;  // 16 warps
    if (T <= 1) TTGBF_QRCP(1, 1);
    else if (T == 2) TTGBF_QRCP(1, 2);
    else if (T == 3) TTGBF_QRCP(2, 3);
    else if (T == 4) TTGBF_QRCP(2, 4);
    else if (T == 5) TTGBF_QRCP(3, 5);
    else TTGBF_QRCP(3, 6);
  }
#undef TTGBF_QRCP
  if (!reg) {
    float* nref = reinterpret_cast<float*>(ord + kMaxN);  // norm at the last recomputation
    for (int c = tid; c < n; c += blockDim.x) nref[c] = nrm[c];
    {
      float rl = 0.f, bv = -1.f;
      int bx = n;
      for (int c = warp; c < n; c += nwarps) {  // same column split as the updates below
        const float v = nrm[c];
        rl += v;
        if (v > bv) {
          bv = v;
          bx = c;
        }
      }
      if (lane == 0) {
        s_red[warp] = rl;
        s_redf[warp] = bv;
        s_redi[warp] = bx;
      }
    }
    __syncthreads();
    for (;; ++k) {
      // every warp reduces the per-warp partials (same result everywhere)
      const float rem = warp_sum(lane < nwarps ? s_red[lane] : 0.f);
      float best = lane < nwarps ? s_redf[lane] : -1.f;
      int bi = lane < nwarps ? s_redi[lane] : n;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (k >= kcap || (k > 0 && rem <= stop2f) || bi >= n) {
        dropped2 = (double)rem;
        break;
      }
      if (warp == 0) {
        const int pv = perm[bi];
        __syncwarp();
        if (lane == 0) {
          perm[bi] = perm[k];
          perm[k] = pv;
        }
        float* colk = A + pv * n;
        float ss = 0.f;
        for (int i = k + 1 + lane; i < n; i += 32) ss = fmaf(colk[i], colk[i], ss);
        ss = warp_sum(ss);
        const float alpha = colk[k];
        float tot = fmaf(alpha, alpha, ss), tail2 = ss, scale = 1.f;
        // squares are exact enough unless the sum leaves [1e-30, 1e30]; such
        // columns take a second pass scaled by the column maximum
        const bool rescale = tot != 0.f && !(tot >= 1e-30f && tot <= 1e30f);
        if (rescale) {
          float mx = 0.f;
          for (int i = k + 1 + lane; i < n; i += 32) mx = fmaxf(mx, fabsf(colk[i]));
          mx = fmaxf(warp_max(mx), fabsf(alpha));
          const float inv = mx > 0.f ? 1.f / mx : 0.f;
          float s2 = 0.f;
          for (int i = k + 1 + lane; i < n; i += 32) {
            const float x = colk[i] * inv;
            s2 = fmaf(x, x, s2);
          }
          s2 = warp_sum(s2);
          const float al = alpha * inv;
          tot = fmaf(al, al, s2);
          tail2 = s2;
          scale = mx;
        }
        float tau = 0.f, beta = alpha, scl = 0.f;
        if (tail2 > 0.f && tot > 0.f) {
          const float rs = rsqrtf(tot);
          const float nm = tot * rs * scale;
          const float aa = fabsf(alpha);
          beta = alpha >= 0.f ? -nm : nm;
          tau = fmaf(aa / scale, rs, 1.f);  // (|alpha| + nm) / nm
          const float am = aa + nm;
          scl = alpha >= 0.f ? __frcp_rn(am) : -__frcp_rn(am);
          for (int i = k + 1 + lane; i < n; i += 32) colk[i] *= scl;
        }
        __syncwarp();
        if (lane == 0) {
          s_tau = tau;
          rdiag[k] = beta;
          colk[k] = 1.f;
        }
      }
      __syncthreads();
      const float tau = s_tau;
      const float* colk = A + perm[k] * n;
      float rl = 0.f, bv = -1.f;
      int bx = n;
      for (int c = k + 1 + warp; c < n; c += nwarps) {
        const int pc = perm[c];
        float* colc = A + pc * n;
        if (tau != 0.f) {
          float dot = 0.f;
          for (int i = k + lane; i < n; i += 32) dot = fmaf(colk[i], colc[i], dot);
          dot = warp_sum(dot) * tau;
          for (int i = k + lane; i < n; i += 32) colc[i] = fmaf(-dot, colk[i], colc[i]);
          __syncwarp();
        }
        const float rk = colc[k];
        float nr = nrm[pc] - rk * rk;
        if (!(nr >= 1e-3f * nref[pc])) {  // cancelled (or NaN): recompute
          float sq = 0.f;
          for (int i = k + 1 + lane; i < n; i += 32) sq = fmaf(colc[i], colc[i], sq);
          nr = warp_sum(sq);
          if (lane == 0) nref[pc] = nr;
        }
        if (lane == 0) nrm[pc] = nr;
        rl += nr;
        if (nr > bv || (nr == bv && c < bx)) {
          bv = nr;
          bx = c;
        }
      }
      if (lane == 0) {
        s_red[warp] = rl;
        s_redf[warp] = bv;
        s_redi[warp] = bx;
      }
      __syncthreads();
    }
  }
  // dropped2: squared norm of the columns left over
  const int kp = k;  // >= 1
  // ---- 2. Jacobi on the k' leading rows of R' as columns of length n,
  // stored with stride ldm (128 or 160, zero padded) so that a lane holds
  // 4 consecutive entries (16-byte shared loads and stores)
  const int ldm = n <= 128 ? 128 : kMaxN;
  const bool ext = ldm > 128;  // lanes 0..7 hold a second group of 4 (entries 128..159)
  for (int t = tid; t < kp * ldm; t += blockDim.x) {
    const int r = t / ldm, c = t - r * ldm;
    M[t] = (c >= n || c < r) ? 0.f : (c == r ? rdiag[r] : A[perm[c] * n + r]);
  }
  for (int c = tid; c < n; c += blockDim.x) pinv[perm[c]] = c;
  __syncthreads();
  auto col4 = [&](int c, int part) -> float4* {
    return reinterpret_cast<float4*>(M + c * ldm) + (part ? 32 + lane : lane);
  };
  auto sq4 = [](const float4& x) { return x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w; };
  auto col_norm2 = [&](int c) {
    float s = sq4(*col4(c, 0));
    if (ext && lane < 8) s += sq4(*col4(c, 1));
    return warp_sum(s);
  };
  const int npad = (kp + 1) & ~1;
  const float tol = 5e-7f * sqrtf((float)n);
  const float quad = sqrtf(tol);
  __shared__ int s_cmax;
  for (int sweep = 0; sweep < 40 && npad >= 2; ++sweep) {
    for (int c = warp; c < kp; c += nwarps) {
      const float s = col_norm2(c);
      if (lane == 0) nrm[c] = s;
    }
    if (tid == 0) {
      s_rot = 0;
      s_cmax = 0;
    }
    __syncthreads();
    float tnorm = 0.f;
    for (int c = lane; c < kp; c += 32) tnorm += nrm[c];
    tnorm = warp_sum(tnorm);
    const float floor2 = 1e-14f * tnorm;
    float cmax = 0.f;
    const int myrot = ext ? jacobi_rounds<16, true>(M, nrm, kp, npad, ldm, floor2, tol, &cmax)
                          : jacobi_rounds<8, false>(M, nrm, kp, npad, ldm, floor2, tol, &cmax);
    if (myrot > 0) {  // counted on one lane per pair group
      atomicAdd(&s_rot, myrot);
      atomicMax(&s_cmax, __float_as_int(cmax));  // non-negative: int order = float order
    }
    const int any = __syncthreads_or(myrot > 0);
    if (tid == 0) {
      const double nn = (double)n;
      s_flops += 0.5 * kp * (kp - 1.0) * 2.0 * nn + (double)s_rot * 6.0 * nn + 2.0 * nn * kp;
    }
    __syncthreads();
    if (!any) break;
    // one-sided Jacobi converges quadratically: once every rotation of a
    // sweep had |cos| below sqrt(tol), the next sweep's are of order
    // cmax^2 < tol, so that sweep (which would rotate little or nothing) is
    // skipped; what it would leave is far below the FP32 level of the
    // factors after the Loewdin correction of step 3
    if (__int_as_float(s_cmax) < quad) break;
  }
  // singular values and their order
  for (int c = warp; c < kp; c += nwarps) {
    const float s = col_norm2(c);
    if (lane == 0) nrm[c] = sqrtf(s);
  }
  __syncthreads();
  for (int c = tid; c < kp; c += blockDim.x)
    if (!(nrm[c] >= 0.f) || isinf(nrm[c])) nrm[c] = -1.f;
  __syncthreads();
  for (int c = tid; c < kp; c += blockDim.x) {
    const float v = nrm[c];
    int pos = 0;
    for (int e = 0; e < kp; ++e) {
      const float u = nrm[e];
      pos += (u > v) || (u == v && e < c);
    }
    sig[pos] = v < 0.f ? 0.f : v;
    ord[pos] = c;
  }
  __syncthreads();
  if (tid == 0) {
    const double nn = (double)n;
    s_flops += 2.0 * nn * nn * kp + (double)kp * kp * 4.0 * nn * 2.0;
  }
  // ---- rank choice
  if (tid == 0) {
    int r;
    if (mode == kStageRight) {
      const float s0 = sig[0];
      r = 0;
      while (r < kp && sig[r] > 1e-7f * s0) ++r;
      if (r < 1) r = 1;
    } else {
      if (first) rs.normA[b] = normA;
      // tail2[r] = sum_{t >= r} sig_t^2 + dropped2; smallest r >= 1 with tail <= delta
      double acc = dropped2;
      int reps = kp + ((sqrt(acc) <= delta) ? 0 : 1);
      for (int j = kp - 1; j >= 1; --j) {
        acc += (double)sig[j] * (double)sig[j];
        if (sqrt(acc) <= delta) reps = j; else break;
      }
      r = min(min(reps, rank_cap), kp);
      if (r < 1) r = 1;
      double tail = dropped2;
      for (int j = r; j < kp; ++j) tail += (double)sig[j] * (double)sig[j];
      const double rel = normA > 0.0 ? sqrt(tail) / normA : 0.0;
      rs.tail_sum[b] += rel;
      if (rel > rs.tail_max[b]) rs.tail_max[b] = rel;
      if (reps > rank_cap) rs.cap_hits[b] += 1;
    }
    s_rank = r;
    rs.newrank[b] = r;
    if (flops != nullptr) {
      double f = s_flops;
      for (int j = 0; j < kp; ++j) f += (double)(n - j) * (2.0 + 6.0 * (n - j - 1));
      atomicAdd(flops, f);
    }
  }
  __syncthreads();
  const int r = s_rank;
  // ---- 3. orthonormal right singular vectors of the kept rank:
  // Q[t] = M[ord[t]] / sig[t] (column t of A, t < r), then one symmetric
  // (Loewdin) correction Q <- Q (3 I - Q^T Q) / 2, which leaves Q^T Q = I to
  // second order in the Jacobi residual; classical Gram-Schmidt applied
  // twice if that residual is not small.  The factor pair the stage applies
  // then multiplies to an exact projector.
  for (int t = warp; t < r; t += nwarps) {
    const float st = sig[t];
    const float inv = st >= kTiny ? 1.f / st : 0.f;
    const float* src = M + ord[t] * ldm;
    for (int i = lane; i < n; i += 32) A[t * n + i] = src[i] * inv;
  }
  __syncthreads();
  float* E = M;  // r x r Gram (ld r); M is free now
  float dev = 0.f;
  for (int q = warp; q < r * r; q += nwarps) {
    const int s0 = q / r, t0 = q - s0 * r;
    if (t0 < s0) continue;
    float dt = 0.f;
    for (int i = lane; i < n; i += 32) dt = fmaf(A[s0 * n + i], A[t0 * n + i], dt);
    dt = warp_sum(dt);
    if (lane == 0) {
      E[s0 * r + t0] = dt;
      E[t0 * r + s0] = dt;
    }
    const float dd = fabsf(dt - (s0 == t0 && sig[s0] >= kTiny ? 1.f : 0.f));
    dev = (dd > dev || dd != dd) ? dd : dev;  // NaN propagates
  }
  // largest deviation from the identity, NaN counted as large
  const int bad = __syncthreads_or(!(dev <= 1e-3f));
  if (!bad) {
    // rows of Q (r values each) times (3 I - E) / 2, one warp per row
    for (int i = warp; i < n; i += nwarps) {
      float acc[(kMaxN + 31) / 32];
#pragma unroll
      for (int m = 0; m < (kMaxN + 31) / 32; ++m) acc[m] = 0.f;
      for (int s1 = 0; s1 < r; ++s1) {
        const float v = A[s1 * n + i];
#pragma unroll
        for (int m = 0; m < (kMaxN + 31) / 32; ++m) {
          const int t = lane + 32 * m;
          if (t < r) acc[m] = fmaf(v, (s1 == t ? 1.5f : 0.f) - 0.5f * E[s1 * r + t], acc[m]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < (kMaxN + 31) / 32; ++m) {
        const int t = lane + 32 * m;
        if (t < r) A[t * n + i] = acc[m];
      }
    }
    __syncthreads();
  } else {
    for (int t = 0; t < r; ++t) {
      float* qt = A + t * n;
      if (sig[t] >= kTiny) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int s1 = warp; s1 < t; s1 += nwarps) {
            const float* qs = A + s1 * n;
            float dot = 0.f;
            for (int i = lane; i < n; i += 32) dot += qs[i] * qt[i];
            dot = warp_sum(dot);
            if (lane == 0) coef[s1] = dot;
          }
          __syncthreads();
          for (int i = tid; i < n; i += blockDim.x) {
            float v = qt[i];
            for (int s1 = 0; s1 < t; ++s1) v -= coef[s1] * A[s1 * n + i];
            qt[i] = v;
          }
          __syncthreads();
        }
        float nq = 0.f;
        for (int i = tid; i < n; i += blockDim.x) nq += qt[i] * qt[i];
        nq = block_sum_f(nq, s_red);
        const float sc = nq > 1e-20f ? rsqrtf(nq) : 0.f;  // a vector that cancelled is dropped
        for (int i = tid; i < n; i += blockDim.x) qt[i] *= sc;
        __syncthreads();
      }
    }
  }
  float* p1 = P1 + (long long)b * kMaxN * kMaxN;
  float* p2 = P2 + (long long)b * kMaxN * kMaxN;
  for (int t = tid; t < n * r; t += blockDim.x) {
    const int i = t / r, j = t - i * r;  // i < n (row of V, original order), j < r
    const float v = A[j * n + pinv[i]];
    const float s = sig[j];
    const float inv = s >= kTiny ? 1.f / s : 0.f;
    if (mode == kStageRight) {
      p1[j * kMaxN + i] = v * inv;  // P1 = S^-1 V^T  (r x n)
      p2[i * kMaxN + j] = v * s;    // P2 = V S       (n x r)
    } else if (mode == kStageLeft) {
      p1[i * kMaxN + j] = v * inv;  // P1 = V S^-1    (n x r)
      p2[j * kMaxN + i] = v * s;    // P2 = S V^T     (r x n)
    } else {
      core0_out[(long long)b * core0_cap + (long long)i * r + j] = v;  // core 0 = V_r (n x r)
      p2[j * kMaxN + i] = v;                                          // P2 = V_r^T   (r x n)
    }
  }
}

// ------------------------------------------------------------------ GEMM
// Tile shapes (rows x columns) of the grouped GEMM.  The rounding's products
// are tall-skinny or short-wide (one side is a rank <= 160, often 16), so a
// descriptor with n <= 32 takes 128 x 32 tiles and one with m <= 32 takes
// 32 x 128 tiles; the rest take 64 x 64.  256 threads, 4 x 4 outputs each.
__host__ __device__ constexpr int gemm_bm(int shape) { return shape == 1 ? 128 : (shape == 2 ? 32 : 64); }
__host__ __device__ constexpr int gemm_bn(int shape) { return shape == 1 ? 32 : (shape == 2 ? 128 : 64); }
__device__ __forceinline__ int gemm_shape(int m, int n) { return n <= 32 ? 1 : (m <= 32 ? 2 : 0); }

constexpr int kGemmK = 16;          // k per shared-memory stage
constexpr int kGemmPitch = 128 + 4;  // floats per k-row of a tile (16-byte aligned rows)

// One BM x BN tile of C = A B, k in chunks of 16 through shared memory with
// the next chunk's global loads issued before the current chunk's FMAs.
template <int BM, int BN>
__device__ __forceinline__ void gemm_tile(const GemmDesc& g, int row0, int col0, float (*As)[kGemmPitch],
                                          float (*Bs)[kGemmPitch]) {
  constexpr int TX = BN / 4;           // threads along n
  constexpr int LA = BM * kGemmK / 256;  // A elements per thread per chunk
  constexpr int LB = BN * kGemmK / 256;  // B elements per thread per chunk
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      const int ar = e / kGemmK, ak = e % kGemmK;
      const int gr = row0 + ar, gk = k0 + ak;
      ra[q] = (gr < g.m && gk < g.k) ? __ldg(g.A + (long long)gr * g.lda + gk) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      const int bk = e / BN, bc = e % BN;
      const int hk = k0 + bk, hc = col0 + bc;
      rb[q] = (hk < g.k && hc < g.n) ? __ldg(g.B + (long long)hk * g.ldb + hc) : 0.f;
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < g.k; k0 += kGemmK) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[e % kGemmK][e / kGemmK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[e / BN][e % BN] = rb[q];
    }
    __syncthreads();
    if (k0 + kGemmK < g.k) fetch(k0 + kGemmK);
#pragma unroll
    for (int kk = 0; kk < kGemmK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 bq = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty * 4 + i;
    if (r >= g.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx * 4 + j;
      if (c < g.n) g.C[(long long)r * g.ldc + c] = acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(256, 4) k_gemm_grouped(GemmWork w, double* flops) {
  __shared__ __align__(16) float As[kGemmK][kGemmPitch];
  __shared__ __align__(16) float Bs[kGemmK][kGemmPitch];
  const int total = w.tiles[w.ndesc];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = w.ndesc;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.tiles[mid] <= t) lo = mid; else hi = mid;
    }
    const GemmDesc g = w.desc[lo];
    const int bm = gemm_bm(g.shape), bn = gemm_bn(g.shape);
    const int tn_count = (g.n + bn - 1) / bn;
    const int local = t - w.tiles[lo];
    const int tm = local / tn_count, tn = local - tm * tn_count;
    const int row0 = tm * bm, col0 = tn * bn;
    if (g.shape == 1) gemm_tile<128, 32>(g, row0, col0, As, Bs);
    else if (g.shape == 2) gemm_tile<32, 128>(g, row0, col0, As, Bs);
    else gemm_tile<64, 64>(g, row0, col0, As, Bs);
    if (threadIdx.x == 0 && flops != nullptr) {
      const int tm_rows = min(bm, g.m - row0), tn_cols = min(bn, g.n - col0);
      atomicAdd(flops, 2.0 * tm_rows * tn_cols * (double)g.k);
    }
  }
}

// Tile shapes and the exclusive prefix of tile counts of descriptors already
// written (one CTA).
__device__ void scan_tiles_block(GemmWork w) {
  for (int i = threadIdx.x; i < w.ndesc; i += blockDim.x) {
    GemmDesc& g = w.desc[i];
    if (w.tc != kContractFp32) {
      const bool tr = g.n > g.m;
      g.shape = tr ? kTcShapeT : kTcShapeN;
      const int lng = tr ? g.n : g.m, sht = tr ? g.m : g.n;
      w.tiles[i] = (g.m > 0 && g.n > 0) ? ((lng + kTcTileM - 1) / kTcTileM) * ((sht + kTcTileN - 1) / kTcTileN) : 0;
      continue;
    }
    const int sh = gemm_shape(g.m, g.n);
    g.shape = sh;
    const int bm = gemm_bm(sh), bn = gemm_bn(sh);
    w.tiles[i] = (g.m > 0 && g.n > 0) ? ((g.m + bm - 1) / bm) * ((g.n + bn - 1) / bn) : 0;
  }
  __syncthreads();
  block_scan_inplace(w.tiles, w.ndesc);
}

__global__ void k_scan_tiles(GemmWork w) { scan_tiles_block(w); }

// ----------------------------------------------------------------- plans
// Per filter: the tall matrix of this stage and its TSQR schedule.
__global__ void k_plan_stage(TsqrWork w, int B, int mode, int k, TTGeom g, const int* ranks,
                             const float* core_k, const float* W, long long W_cap, int N0, int N1,
                             float* stack0, float* stack1, long long stack_cap, int slots,
                             int elem, int slice_blocks) {
  const int d = g.d;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int* rk = ranks + (long long)b * (d + 1);
    TsqrProblem p;
    if (mode == kStageRight) {
      // X = core k as r_k x (n_k r_{k+1}); the R factor of X^T
      const int r0 = rk[k], r1 = rk[k + 1];
      const long long cols = (long long)g.n[k] * r1;
      p.src.p = core_k + (long long)b * g.cap[k];
      p.src.rs = 1;
      p.src.cs = cols;
      p.src.M = (int)cols;
      p.src.n = r0;
    } else if (mode == kStageLeft) {
      // Y = core k as (r_k n_k) x r_{k+1}
      const int r0 = rk[k], r1 = rk[k + 1];
      p.src.p = core_k + (long long)b * g.cap[k];
      p.src.rs = r1;
      p.src.cs = 1;
      p.src.M = r0 * g.n[k];
      p.src.n = r1;
    } else {
      // W = supercore of modes 0,1 as N0 x (N1 r_2); the R factor of W^T
      const long long cols = (long long)N1 * rk[2];
      p.src.p = W + (long long)b * W_cap;
      p.src.rs = 1;
      p.src.cs = cols;
      p.src.M = (int)cols;
      p.src.n = N0;
    }
    const int n = p.src.n;
    const long long M = p.src.M;
    // slices of at least eight blocks, and no more per filter than the
    // resident CTAs can run at once across the batch (fewer slice R
    // factors to combine at the end)
    const long long srows = tsqr_slice_rows(slice_blocks);
    long long nsl = (M + srows - 1) / srows;
    const long long per = slots / B > 1 ? slots / B : 1;
    if (nsl > per) nsl = per;
    const long long fit = stack_cap / ((long long)elem * n * n);
    if (nsl > fit) nsl = fit;
    if (nsl > kTsqrMaxSlices) nsl = kTsqrMaxSlices;
    if (nsl < 1) nsl = 1;
    p.slice = (int)((M + nsl - 1) / nsl);
    p.nslice = (int)((M + p.slice - 1) / p.slice);
    p.nlev = p.nslice > 1 ? 2 : 1;
    p.stack0 = stack0 + (long long)b * stack_cap;
    p.stack1 = stack1 + (long long)b * stack_cap;
    w.offset[b] = p.nslice;  // counts, scanned below
    w.counter[b] = 0;
    w.prob[b] = p;
  }
  __syncthreads();
  block_scan_inplace(w.offset, B);
}

// Per filter: GEMM descriptors that apply the stage's small factors, then
// the rank update.
// vS > 0 (RIGHT only): core k-1 is the middle core of a shear block kept in
// its unexpanded form G (r x n x r'); its expanded form is G (x) I_vS on both
// links (index a vS + u), so core k-1 x P2 splits into one (n x r') x
// (r' x rn) product per (a, u) with the rows b vS + u of P2.  Filter b's
// descriptors then start at b * dstride.
__global__ void k_plan_gemm_stage(int B, int mode, int k, TTGeom g, int* ranks, const int* newrank,
                                  const float* cur_a, float* alt_a, const float* cur_b, float* alt_b,
                                  const float* P1, const float* P2, const float* W, long long W_cap,
                                  int N1, GemmWork gw, int vS, int dstride) {
  const int d = g.d;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int* rk = ranks + (long long)b * (d + 1);
    const int rn = newrank[b];
    const float* p1 = P1 + (long long)b * kMaxN * kMaxN;
    const float* p2 = P2 + (long long)b * kMaxN * kMaxN;
    if (mode == kStageRight) {
      // a = core k (r_k x n_k r_{k+1}), b = core k-1 ((r_{k-1} n_{k-1}) x r_k)
      const int rkk = rk[k], r1 = rk[k + 1], rm = rk[k - 1];
      const int cols = g.n[k] * r1;
      GemmDesc x{p1, cur_a + (long long)b * g.cap[k], alt_a + (long long)b * g.cap[k], rn, cols, rkk,
                 kMaxN, cols, cols};
      if (vS > 0) {
        const int Nm = g.n[k - 1], rkt = rkk / vS;
        GemmDesc* dd = gw.desc + (long long)b * dstride;
        dd[0] = x;
        for (int q = 0; q + 1 < dstride; ++q) {
          GemmDesc y{nullptr, nullptr, nullptr, 0, 0, 0, 1, 1, 1};
          if (q < rm) {
            const int a = q / vS, u = q - a * vS;
            y = GemmDesc{cur_b + (long long)b * g.cap[k - 1] + (long long)a * Nm * rkt, p2 + u * kMaxN,
                         alt_b + (long long)b * g.cap[k - 1] + (long long)q * Nm * rn, Nm, rn, rkt,
                         rkt, vS * kMaxN, rn};
          }
          dd[1 + q] = y;
        }
      } else {
        GemmDesc y{cur_b + (long long)b * g.cap[k - 1], p2, alt_b + (long long)b * g.cap[k - 1],
                   rm * g.n[k - 1], rn, rkk, rkk, kMaxN, rn};
        gw.desc[2 * b] = x;
        gw.desc[2 * b + 1] = y;
      }
      rk[k] = rn;
    } else if (mode == kStageLeft) {
      // a = core k ((r_k n_k) x r_{k+1}), b = core k+1 (r_{k+1} x n_{k+1} r_{k+2})
      const int r0 = rk[k], r1 = rk[k + 1], r2 = rk[k + 2];
      const int cols = g.n[k + 1] * r2;
      GemmDesc x{cur_a + (long long)b * g.cap[k], p1, alt_a + (long long)b * g.cap[k], r0 * g.n[k], rn,
                 r1, r1, kMaxN, rn};
      GemmDesc y{p2, cur_b + (long long)b * g.cap[k + 1], alt_b + (long long)b * g.cap[k + 1], rn, cols,
                 r1, kMaxN, cols, cols};
      gw.desc[2 * b] = x;
      gw.desc[2 * b + 1] = y;
      rk[k + 1] = rn;
    } else {
      // new core 1 = V_r^T W  (r x N1 r_2); core 0 was written by the Jacobi kernel
      const int r2 = rk[2];
      const int cols = N1 * r2;
      const int N0 = g.n[0];
      GemmDesc y{p2, W + (long long)b * W_cap, alt_b + (long long)b * g.cap[1], rn, cols, N0, kMaxN,
                 cols, cols};
      gw.desc[b] = y;
      rk[1] = rn;
    }
  }
  // descriptors of this CTA are in global memory: make them visible to the
  // whole block before the tile scan reads them
  __threadfence_block();
  __syncthreads();
  scan_tiles_block(gw);
}

}  // namespace

// -------------------------------------------------------------- launchers
void launch_plan_stage(cudaStream_t st, int B, int mode, int k, const TTGeom& g, const int* ranks,
                       const float* core_k, const float* W, long long W_cap, int N0, int N1,
                       TsqrWork w, float* stack0, float* stack1, long long stack_cap, int slots,
                       int elem, int slice_blocks) {
  count_launches(1);
  k_plan_stage<<<1, 1024, 0, st>>>(w, B, mode, k, g, ranks, core_k, W, W_cap, N0, N1, stack0, stack1,
                                   stack_cap, slots, elem, slice_blocks);
}

void launch_svd(cudaStream_t st, TsqrWork w, int B, int mode, int rank_cap, double eps, int d,
                   int first, RoundState rs, float* P1, float* P2, float* core0_out,
                   long long core0_cap, double* flops, int left_threads) {
  count_launches(1);
  // truncation stages have at most rank_cap + 16 Jacobi columns: half the warps
  // suffice (two CTAs per SM); the split of the merged 2-site core (n = N_0)
  // takes 32 warps so that its pivoted QR keeps the columns in registers
  const int threads = mode == kStageLeft ? left_threads : 1024;
  k_svd<<<B, threads, kJacobiSmemFloats * sizeof(float), st>>>(w, B, mode, rank_cap, eps, d, first, rs, P1,
                                                             P2, core0_out, core0_cap, flops);
}

void launch_plan_gemm_stage(cudaStream_t st, int B, int mode, int k, const TTGeom& g, int* ranks,
                            const int* newrank, const float* cur_a, float* alt_a,
                            const float* cur_b, float* alt_b, const float* P1, const float* P2,
                            const float* W, long long W_cap, int N1, GemmWork gw, int vS,
                            int dstride) {
  count_launches(1);
  k_plan_gemm_stage<<<1, 1024, 0, st>>>(B, mode, k, g, ranks, newrank, cur_a, alt_a, cur_b, alt_b, P1,
                                        P2, W, W_cap, N1, gw, vS, dstride);
}

void launch_gemm(cudaStream_t st, GemmWork gw, int grid, double* flops) {
  if (gw.tc != kContractFp32) {
    launch_gemm_tc(st, gw, std::max(1, grid / 2), flops);
    return;
  }
  count_launches(1);
  k_gemm_grouped<<<grid, 256, 0, st>>>(gw, flops);
}

void launch_scan_tiles(cudaStream_t st, GemmWork gw) {
  count_launches(1);
  k_scan_tiles<<<1, 1024, 0, st>>>(gw);
}

void set_kernel_attributes() {
  cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kJacobiSmemFloats * (int)sizeof(float));
}

}  // namespace ttgbf
