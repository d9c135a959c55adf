// rsvd64.cu -- float64 R factor and SVD for the truncating stages of TT
// rounding (Sec. 4.1 "round"; Alg. 2 steps 2 and 4), the precision option
// TTGBF_PRECISION_FP64 of ttgbf_opts.
//
// The cores stay float32.  In this mode the stages that decide a truncation
// (the left-to-right sweep and the split of the merged 2-site core) form the
// R factor of their tall matrix and its SVD in float64, so the discarded
// singular values near the threshold eps ||A|| / sqrt(d - 1) are those of the
// float32 data to float64 accuracy rather than to the float32 backward error
// of a float32 Householder QR (about u sqrt(n) ||A||, u = 6e-8).  The
// orthogonalisation sweep, which truncates nothing, stays in float32.
//
//   k_tsqr64: Householder QR of row blocks of 64 rows against a running upper
//             triangular R kept packed in shared memory (one reflector per
//             column touches row j of R and the block only); the same slice
//             and last-CTA combine scheme as the float32 TSQR, with float64
//             slice factors on the stacks.
//   k_svd64:  column-pivoted Householder QR of R stopped at the stage's drop
//             level (remaining norm <= 0.3 delta) or after rank_cap + 16
//             steps, then one-sided Jacobi (Hestenes) on the k' leading rows
//             of R' in float64 until no pair's cosine exceeds 4 n u64; rank
//             choice and the stage's factors as the float32 SVD kernel makes
//             them (written in float32).
// GB300 issues float64 at a small fraction of its float32 rate, so this mode
// costs several times the float32 one; it is an accuracy option.
#include <math.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kQ64Threads = 256;
constexpr int kQ64Rows = 64;  // rows per block; two per lane of the reflector warp

__device__ __forceinline__ int tri_off(int j, int n) { return j * n - (j * (j - 1)) / 2; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// R factor of rows [row0, row0 + M) of (p, rs, cs), n columns, written
// row-major n x n (zeros below the diagonal) to out.  Rp: packed upper
// triangle (row j from tri_off(j, n), entries c >= j); Bk: 64 x ldb block.
template <typename SrcT, bool kCoherent>
__device__ void q64_rows(const SrcT* p, long long rs, long long cs, long long row0, long long M,
                         int n, double* out, double* Rp, double* Bk, int ldb, double* v,
                         double* s_tau) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntri = n * (n + 1) / 2;
  for (int t = tid; t < ntri; t += kQ64Threads) Rp[t] = 0.0;
  for (long long done = 0; done < M; done += kQ64Rows) {
    const long long rows = (M - done < kQ64Rows) ? M - done : kQ64Rows;
    __syncthreads();  // R zeroed / previous block finished
    for (int t = tid; t < kQ64Rows * n; t += kQ64Threads) {
      const int i = t / n, c = t - i * n;
      double x = 0.0;
      if (i < rows) {
        const SrcT* src = p + (row0 + done + i) * rs + (long long)c * cs;
        x = kCoherent ? (double)__ldcg(src) : (double)__ldg(src);
      }
      Bk[i * ldb + c] = x;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const int rj = tri_off(j, n);
      if (warp == 0) {
        const double x0 = Bk[(2 * lane) * ldb + j], x1 = Bk[(2 * lane + 1) * ldb + j];
        const double ss = warp_sum_d(x0 * x0 + x1 * x1);
        const double alpha = Rp[rj];
        double tau = 0.0;
        if (ss > 0.0) {
          const double nm = sqrt(fma(alpha, alpha, ss));
          const double beta = alpha >= 0.0 ? -nm : nm;
          tau = (beta - alpha) / beta;
          const double sc = 1.0 / (alpha - beta);
          v[2 * lane] = x0 * sc;
          v[2 * lane + 1] = x1 * sc;
          if (lane == 0) Rp[rj] = beta;
        }
        if (lane == 0) *s_tau = tau;
      }
      __syncthreads();
      const double tau = *s_tau;
      if (tau != 0.0) {
        for (int c = j + 1 + tid; c < n; c += kQ64Threads) {
          const double rjc = Rp[rj + c - j];
          double dot = rjc;  // v is 1 on row j of R
#pragma unroll 8
          for (int i = 0; i < kQ64Rows; ++i) dot = fma(v[i], Bk[i * ldb + c], dot);
          const double f = tau * dot;
          Rp[rj + c - j] = rjc - f;
#pragma unroll 8
          for (int i = 0; i < kQ64Rows; ++i) Bk[i * ldb + c] = fma(-f, v[i], Bk[i * ldb + c]);
        }
      }
      __syncthreads();
    }
  }
  for (int t = tid; t < n * n; t += kQ64Threads) {
    const int i = t / n, c = t - i * n;
    out[t] = (c >= i) ? Rp[tri_off(i, n) + c - i] : 0.0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kQ64Threads, 1) k_tsqr64(TsqrWork w, int B, int* counter,
                                                            double* flops) {
  extern __shared__ double sm64[];
  __shared__ double s_tau;
  __shared__ int s_last;
  const int total = w.offset[B];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = B;  // offset[lo] <= item < offset[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.offset[mid] <= item) lo = mid; else hi = mid;
    }
    const int b = lo;
    const TsqrProblem pp = w.prob[b];
    const int s = item - w.offset[b];
    const int n = pp.src.n;
    const int ldb = n | 1;  // odd stride: the reflector warp's column reads spread over the banks
    double* Rp = sm64;
    double* Bk = Rp + (n * (n + 1) / 2 + 1);
    double* v = Bk + kQ64Rows * ldb;
    double* st0 = reinterpret_cast<double*>(pp.stack0);
    double* st1 = reinterpret_cast<double*>(pp.stack1);
    if (pp.nslice == 1) {
      q64_rows<float, false>(pp.src.p, pp.src.rs, pp.src.cs, 0, pp.src.M, n, st0, Rp, Bk, ldb, v,
                             &s_tau);
    } else {
      const long long r0 = (long long)s * pp.slice;
      const long long rows = (pp.src.M - r0 < pp.slice) ? pp.src.M - r0 : pp.slice;
      q64_rows<float, false>(pp.src.p, pp.src.rs, pp.src.cs, r0, rows, n,
                             st0 + (long long)s * n * n, Rp, Bk, ldb, v, &s_tau);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(counter + b, 1) == pp.nslice - 1);
      __syncthreads();
      if (!s_last) continue;
      __threadfence();
      q64_rows<double, true>(st0, n, 1, 0, (long long)pp.nslice * n, n, st1, Rp, Bk, ldb, v, &s_tau);
    }
    if (threadIdx.x == 0 && flops != nullptr) {
      const double Md = (double)pp.src.M, k = Md < n ? Md : (double)n;
      atomicAdd(flops, 2.0 * Md * n * k - 2.0 * k * k * k / 3.0);
    }
    __syncthreads();
  }
}

int tsqr64_smem_bytes(int n) {
  return (int)sizeof(double) * (n * (n + 1) / 2 + 1 + kQ64Rows * (n | 1) + kQ64Rows);
}

// ------------------------------------------------------------------ SVD
constexpr int kS64Threads = 512;
constexpr int kS64Warps = kS64Threads / 32;
constexpr int kS64MaxKeep = 80;  // Jacobi rows k' (their float64 copy fits the stage's P1 area)

__device__ double block_sum_d(double v, double* red) {
  v = warp_sum_d(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  return warp_sum_d(lane < kS64Warps ? red[lane] : 0.0);
}

__global__ void __launch_bounds__(kS64Threads) k_svd64(TsqrWork w, int B, int mode, int rank_cap,
                                                       double eps, int d, int first, RoundState rs,
                                                       float* P1, float* P2, float* core0_out,
                                                       long long core0_cap, double* flops) {
  extern __shared__ double sd[];
  __shared__ double s_red[32], s_redf[32], s_tau, s_dropped;
  __shared__ int s_redi[32], s_kp, s_rank, s_rot;
  __shared__ double s_flops;
  const int b = blockIdx.x;
  if (b >= B) return;
  const TsqrProblem p = w.prob[b];
  const int n = p.src.n;
  const double* R = reinterpret_cast<const double*>(((p.nlev - 1) & 1) ? p.stack1 : p.stack0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* A = sd;              // n x n column-major (ld n): QRCP work, later the Jacobi rows
  double* nrm = A + n * n;     // [n] squared column norms (current)
  double* nref = nrm + n;      // [n] norms at the last recomputation
  double* rdiag = nref + n;    // [n] diagonal of R'
  double* sig = rdiag + n;     // [n] sorted singular values
  int* perm = reinterpret_cast<int*>(sig + n);  // [n] physical column at pivot position
  int* pinv = perm + n;                         // [n] its inverse
  int* ord = pinv + n;                          // [n] Jacobi rows by decreasing norm

  for (int t = tid; t < n * n; t += kS64Threads) {
    const int i = t / n, c = t - i * n;
    A[c * n + i] = __ldcg(R + t);
  }
  for (int c = tid; c < n; c += kS64Threads) perm[c] = c;
  if (tid == 0) s_flops = 0.0;
  __syncthreads();
  for (int c = warp; c < n; c += kS64Warps) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s = fma(A[c * n + i], A[c * n + i], s);
    s = warp_sum_d(s);
    if (lane == 0) {
      nrm[c] = s;
      nref[c] = s;
    }
  }
  __syncthreads();
  double tot = 0.0;
  for (int c = tid; c < n; c += kS64Threads) tot += nrm[c];
  tot = block_sum_d(tot, s_red);
  const double normA = first ? sqrt(tot) : rs.normA[b];
  const double delta = d <= 1 ? 0.0 : eps * normA / sqrt((double)(d - 1));
  const double stop2 = 0.09 * delta * delta;
  int kcap = rank_cap + 16;
  if (kcap > kS64MaxKeep) kcap = kS64MaxKeep;
  if (kcap > n) kcap = n;

  // ---- 1. QR with column pivoting (columns stay in place; perm[pos] is the
  // physical column at pivot position pos).
  __syncthreads();  // every warp has read the block sum from s_red
  {
    double rl = 0.0, bv = -1.0;
    int bx = n;
    for (int pos = warp; pos < n; pos += kS64Warps) {
      const double v = nrm[pos];
      rl += v;
      if (v > bv) {
        bv = v;
        bx = pos;
      }
    }
    if (lane == 0) {
      s_red[warp] = rl;
      s_redf[warp] = bv;
      s_redi[warp] = bx;
    }
  }
  __syncthreads();
  int k = 0;
  for (;; ++k) {
    double rem = warp_sum_d(lane < kS64Warps ? s_red[lane] : 0.0);
    double best = lane < kS64Warps ? s_redf[lane] : -1.0;
    int bi = lane < kS64Warps ? s_redi[lane] : n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (k >= kcap || (k > 0 && rem <= stop2) || bi >= n) {
      if (tid == 0) {
        s_dropped = rem;
        s_kp = k;
      }
      break;
    }
    if (warp == 0) {
      const int pv = perm[bi];
      __syncwarp();
      if (lane == 0) {
        perm[bi] = perm[k];
        perm[k] = pv;
      }
      double* colk = A + pv * n;
      double ss = 0.0;
      for (int i = k + 1 + lane; i < n; i += 32) ss = fma(colk[i], colk[i], ss);
      ss = warp_sum_d(ss);
      const double alpha = colk[k];
      double tau = 0.0, beta = alpha;
      if (ss > 0.0) {
        const double nm = sqrt(fma(alpha, alpha, ss));
        beta = alpha >= 0.0 ? -nm : nm;
        tau = (beta - alpha) / beta;
        const double sc = 1.0 / (alpha - beta);
        for (int i = k + 1 + lane; i < n; i += 32) colk[i] *= sc;
      }
      __syncwarp();
      if (lane == 0) {
        s_tau = tau;
        rdiag[k] = beta;
        colk[k] = 1.0;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    const double* colk = A + perm[k] * n;
    double rl = 0.0, bv = -1.0;
    int bx = n;
    for (int pos = k + 1 + warp; pos < n; pos += kS64Warps) {
      const int pc = perm[pos];
      double* colc = A + pc * n;
      if (tau != 0.0) {
        double dot = 0.0;
        for (int i = k + lane; i < n; i += 32) dot = fma(colk[i], colc[i], dot);
        dot = warp_sum_d(dot) * tau;
        for (int i = k + lane; i < n; i += 32) colc[i] = fma(-dot, colk[i], colc[i]);
        __syncwarp();
      }
      const double rk = colc[k];
      double nr = nrm[pc] - rk * rk;
      if (!(nr >= 1e-8 * nref[pc])) {  // cancelled (or NaN): recompute
        double sq = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) sq = fma(colc[i], colc[i], sq);
        nr = warp_sum_d(sq);
        if (lane == 0) nref[pc] = nr;
      }
      if (lane == 0) nrm[pc] = nr;
      rl += nr;
      if (nr > bv || (nr == bv && pos < bx)) {
        bv = nr;
        bx = pos;
      }
    }
    if (lane == 0) {
      s_red[warp] = rl;
      s_redf[warp] = bv;
      s_redi[warp] = bx;
    }
    __syncthreads();
  }
  __syncthreads();
  const int kp = s_kp;  // >= 1
  const double dropped2 = s_dropped;
  for (int c = tid; c < n; c += kS64Threads) pinv[perm[c]] = c;
  // ---- 2. the k' leading rows of R' (pivot order) as vectors of length n,
  // through this filter's P1 area (kp n doubles <= kMaxN^2 floats), into
  // shared memory where A was
  double* Mg = reinterpret_cast<double*>(P1 + (long long)b * kMaxN * kMaxN);
  for (int t = tid; t < kp * n; t += kS64Threads) {
    const int r = t / n, c = t - r * n;
    Mg[t] = c < r ? 0.0 : (c == r ? rdiag[r] : A[perm[c] * n + r]);
  }
  __syncthreads();
  double* M = A;
  for (int t = tid; t < kp * n; t += kS64Threads) M[t] = Mg[t];
  __syncthreads();
  const int npad = (kp + 1) & ~1;
  const double tol = 4.0 * n * 2.220446049250313e-16;
  double tnorm = 0.0;
  for (int t = tid; t < kp * n; t += kS64Threads) tnorm = fma(M[t], M[t], tnorm);
  tnorm = block_sum_d(tnorm, s_red);
  const double floor2 = 1e-300 + 1e-30 * tnorm;
  int sweeps = 0;
  for (; sweeps < 40 && npad >= 2; ++sweeps) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    int myrot = 0;
    for (int r = 0; r < npad - 1; ++r) {
      for (int q = warp; q < npad / 2; q += kS64Warps) {
        // pair q of round r of the circle method on npad slots
        int pp, qq;
        const int m1 = npad - 1;
        if (q == 0) {
          pp = 0;
          qq = 1 + r;
        } else {
          const int a = q + r, c2 = m1 - q + r;
          pp = 1 + (a >= m1 ? a - m1 : a);
          qq = 1 + (c2 >= m1 ? c2 - m1 : c2);
        }
        if (pp >= kp || qq >= kp) continue;  // warp-uniform
        double* x = M + pp * n;
        double* y = M + qq * n;
        double al = 0.0, be = 0.0, g = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double xi = x[i], yi = y[i];
          al = fma(xi, xi, al);
          be = fma(yi, yi, be);
          g = fma(xi, yi, g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (g == 0.0 || fmin(al, be) <= floor2 || !(fabs(g) > tol * sqrt(al * be))) continue;
        const double zeta = (be - al) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        const double cth = 1.0 / sqrt(fma(t, t, 1.0));
        const double sth = cth * t;
        for (int i = lane; i < n; i += 32) {
          const double xi = x[i], yi = y[i];
          x[i] = cth * xi - sth * yi;
          y[i] = sth * xi + cth * yi;
        }
        if (lane == 0) ++myrot;
      }
      __syncthreads();
    }
    if (myrot > 0) atomicAdd(&s_rot, myrot);
    __syncthreads();
    if (tid == 0) s_flops += 0.5 * kp * (kp - 1.0) * 6.0 * n + (double)s_rot * 6.0 * n;
    const int any = s_rot;
    __syncthreads();
    if (any == 0) break;
  }
  // singular values (row norms) and their order
  for (int r = warp; r < kp; r += kS64Warps) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s = fma(M[r * n + i], M[r * n + i], s);
    s = warp_sum_d(s);
    if (lane == 0) nrm[r] = sqrt(s);
  }
  __syncthreads();
  for (int r = tid; r < kp; r += kS64Threads)
    if (!(nrm[r] >= 0.0) || isinf(nrm[r])) nrm[r] = -1.0;
  __syncthreads();
  for (int r = tid; r < kp; r += kS64Threads) {
    const double v = nrm[r];
    int pos = 0;
    for (int e = 0; e < kp; ++e) {
      const double u = nrm[e];
      pos += (u > v) || (u == v && e < r);
    }
    sig[pos] = v < 0.0 ? 0.0 : v;
    ord[pos] = r;
  }
  __syncthreads();
  // ---- rank choice (the truncation rule of the float32 kernel)
  if (tid == 0) {
    if (first) rs.normA[b] = normA;
    double acc = dropped2;
    int reps = kp + ((sqrt(acc) <= delta) ? 0 : 1);
    for (int j = kp - 1; j >= 1; --j) {
      acc += sig[j] * sig[j];
      if (sqrt(acc) <= delta) reps = j; else break;
    }
    int r = min(min(reps, rank_cap), kp);
    if (r < 1) r = 1;
    double tail = dropped2;
    for (int j = r; j < kp; ++j) tail += sig[j] * sig[j];
    const double rel = normA > 0.0 ? sqrt(tail) / normA : 0.0;
    rs.tail_sum[b] += rel;
    if (rel > rs.tail_max[b]) rs.tail_max[b] = rel;
    if (reps > rank_cap) rs.cap_hits[b] += 1;
    s_rank = r;
    rs.newrank[b] = r;
    if (flops != nullptr) {
      double f = s_flops + 2.0 * n * (double)n;
      for (int j = 0; j < kp; ++j) f += 4.0 * (double)(n - j) * (n - j);
      atomicAdd(flops, f);
    }
  }
  __syncthreads();
  const int r = s_rank;
  // ---- factors: V(i, j) = (row ord[j] of the Jacobi matrix at position
  // pinv[i]) / sig[j], in the original column order i
  float* p1 = P1 + (long long)b * kMaxN * kMaxN;
  float* p2 = P2 + (long long)b * kMaxN * kMaxN;
  for (int t = tid; t < n * r; t += kS64Threads) {
    const int i = t / r, j = t - i * r;
    const double s = sig[j];
    const double inv = s > 1e-300 ? 1.0 / s : 0.0;
    const double vv = M[ord[j] * n + pinv[i]] * inv;
    if (mode == kStageLeft) {
      p1[i * kMaxN + j] = (float)(vv * inv);  // P1 = V S^-1 (n x r)
      p2[j * kMaxN + i] = (float)(vv * s);    // P2 = S V^T (r x n)
    } else {
      core0_out[(long long)b * core0_cap + (long long)i * r + j] = (float)vv;  // core 0 = V_r
      p2[j * kMaxN + i] = (float)vv;                                         // P2 = V_r^T
    }
  }
}

int svd64_smem_bytes() {
  return (int)(sizeof(double) * (kMaxN * kMaxN + 4 * kMaxN) + sizeof(int) * 3 * kMaxN);
}

}  // namespace

void launch_tsqr64(cudaStream_t st, TsqrWork w, int B, int grid, double* flops) {
  count_launches(1);
  k_tsqr64<<<grid, kQ64Threads, tsqr64_smem_bytes(kMaxN), st>>>(w, B, w.counter, flops);
}

void launch_svd64(cudaStream_t st, TsqrWork w, int B, int mode, int rank_cap, double eps, int d,
                  int first, RoundState rs, float* P1, float* P2, float* core0_out,
                  long long core0_cap, double* flops) {
  count_launches(1);
  k_svd64<<<B, kS64Threads, svd64_smem_bytes(), st>>>(w, B, mode, rank_cap, eps, d, first, rs, P1,
                                                      P2, core0_out, core0_cap, flops);
}

void set_rsvd64_attributes() {
  cudaFuncSetAttribute(k_tsqr64, cudaFuncAttributeMaxDynamicSharedMemorySize, tsqr64_smem_bytes(kMaxN));
  cudaFuncSetAttribute(k_svd64, cudaFuncAttributeMaxDynamicSharedMemorySize, svd64_smem_bytes());
}

}  // namespace ttgbf
