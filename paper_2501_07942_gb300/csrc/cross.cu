// cross.cu -- deterministic tensor-train cross (Sec. 3: the black-box
// approximation from skeletons, Eq. matrixDecomp, with maximum-volume choices
// of rows and columns) of the product of a likelihood factor with the block of
// cores lo..hi of every filter's density TT: the update of Alg. 2, step 2, for
// a factor that couples several modes.
//
// The block tensor T(a, i_lo, ..., i_hi, b) = L(i_lo..i_hi) [G_lo ... G_hi](a, b)
// has k = hi - lo + 1 "virtual" modes: (a, i_lo) first, (i_hi, b) last, the
// grid index in between.  With the density's cores left of lo left- and right
// of hi right-orthonormal (the caller's canonical form), approximating T
// approximates L (.) P with the same relative error.
//
// One CTA per filter takes one step of a sweep at block mode q:
//   * the step's fiber matrix, float32, column-major in the filter's scratch:
//     left-to-right rows (alpha in I_q, v in mode q), columns beta in J_{q+1};
//     right-to-left rows (v, beta in J_{q+1}), columns alpha in I_q; entries
//     T(alpha, v, beta) = L(...) U_q[alpha] G_q(v) V_{q+1}[beta], U and V the
//     products of the density's cores along each set element (interfaces);
//   * the maximum-volume rows of its column space: Gaussian elimination with
//     partial row pivoting for a start (on the fiber matrix itself: the rows
//     are those of the same elimination on an orthonormal basis Q of its
//     columns, the two differing by an upper triangular factor), B =
//     Q Q[rows]^-1 from the elimination's multipliers (L L1^-1), then
//     single-row exchanges while an entry of B exceeds 1 + delta (the largest
//     entry, the first in row-major order at a tie);
//   * the new index set (table offsets and interfaces) and, in the final
//     sweep, the core B in the density's layout.
// The start steps choose right sets from the density block alone (columns:
// its rank index) and pad them to the link's size with the rows of largest
// norm.  The last kernel writes the last core, the fibers T(I_{k-1}, v), and
// the block's new ranks.
//
// With CrossArgs::trans set the block is instead the 2-site block (lo, lo+1)
// after one factor of the textbook transition (ttgbf_predict_exact): there
// is no likelihood table, and its fibers are sums over the old grid index of
// the shifted Gaussian times the block (trans_fibers_lr / trans_fibers_rl);
// the elimination, exchanges and index sets are the same.
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kCT = 512;  // threads per CTA
constexpr int kCW = kCT / 32;
constexpr int S = kCrossMaxS;
constexpr float kDelta = 0.05f;
constexpr int kMaxvolIters = 100;

__device__ __forceinline__ bool better(float v1, long long i1, float v2, long long i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}

// Largest value (the smallest index at a tie) over the block; every thread
// gets the winner's index (-1 when no thread offered one).
__device__ long long block_argmax(float v, long long i, float* rv, long long* ri, float* best) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(v2, i2, v, i)) {
      v = v2;
      i = i2;
    }
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    rv[threadIdx.x >> 5] = v;
    ri[threadIdx.x >> 5] = i;
  }
  __syncthreads();
  float bv = -1.f;
  long long bi = -1;
  for (int w = 0; w < kCW; ++w)
    if (ri[w] >= 0 && (bi < 0 || better(rv[w], ri[w], bv, bi))) {
      bv = rv[w];
      bi = ri[w];
    }
  *best = bv;
  return bi;
}

// Per-filter geometry of the block.
struct Geo {
  int k;
  int r[kMaxD + 1];      // density ranks at links lo .. lo + k
  long long nv[kMaxD];   // virtual mode sizes
  __device__ int rl(int q) const { return q == 0 ? 1 : r[q]; }
  __device__ int rr(int q) const { return q == k - 1 ? 1 : r[q + 1]; }
  __device__ long long grid(const CrossArgs& a, int q, long long v) const {
    if (q == 0) return v % a.N[0];
    if (q == k - 1) return v / r[k];
    return v;
  }
};

// Reads the block's ranks; false if one exceeds the cross rank (the caller's
// rounding keeps them within the rank cap, which is at most s).
__device__ bool load_geo(const CrossArgs& a, int b, Geo* g) {
  const int* rk = a.ranks + (long long)b * (a.d + 1);
  g->k = a.k;
  for (int t = 0; t <= a.k; ++t) {
    g->r[t] = rk[a.lo + t];
    if (g->r[t] < 1 || g->r[t] > a.s) return false;
  }
  for (int q = 0; q < a.k; ++q) {
    long long n = a.N[q];
    if (q == 0) n *= g->r[0];
    if (q == a.k - 1) n *= g->r[a.k];
    g->nv[q] = n;
  }
  return true;
}

__device__ __forceinline__ float lik_at(const CrossArgs& a, long long idx, float zb, float ob, float inv2r) {
  const float df = wrap_residual(zb - a.htab[idx], a.period);
  return expf(-(df * df - ob) * inv2r);
}

// The textbook transition's mode factor K(j, i, i') of a transition block.
__device__ __forceinline__ float trans_k(const CrossArgs& a, int j, int i, int i1) {
  const float x = (a.tlo0 + ((float)j + 0.5f) * a.tdx0) - a.tF0 * (a.tlo0 + ((float)i + 0.5f) * a.tdx0) -
                  a.tF1 * (a.tlo1 + ((float)i1 + 0.5f) * a.tdx1);
  return a.tkc * expf(-0.5f * x * x * a.tiq);
}

// The old indices i where K(j, i, i') is not below exp(-32) of its peak (8
// standard deviations from x = 0): the window around the i that solves
// F0 xi0_i = xi0_j - F1 xi1_i', clamped to the axis.
__device__ __forceinline__ void trans_window(const CrossArgs& a, int j, int i1, int N0, int* ilo, int* ihi) {
  *ilo = 0;
  *ihi = N0 - 1;
  if (!(a.twin > 0.f)) return;
  const float xj = a.tlo0 + ((float)j + 0.5f) * a.tdx0;
  const float x1 = a.tlo1 + ((float)i1 + 0.5f) * a.tdx1;
  const float ic = ((xj - a.tF1 * x1) / a.tF0 - a.tlo0) / a.tdx0 - 0.5f;
  *ilo = max(0, (int)floorf(ic - a.twin));
  *ihi = min(N0 - 1, (int)ceilf(ic + a.twin));
}

// Transition block, left-to-right fibers at mode 0: column be of F is
// T((a, j), v1_be) = sum_i K(j, i, i'_be) y(a, i), y(a, i) = G_0(a, i, :) . V_1[be]
// (y staged in the scratch Y, r_a N_0 floats).
__device__ void trans_fibers_lr(const CrossArgs& a, const float* G0, int rr0, long long M, int sR,
                                const long long* oJ, const float* V1, int rlast, float* F, float* Y) {
  const int N0 = a.N[0], s = a.s;
  for (int be = 0; be < sR; ++be) {
    const int i1 = (int)(oJ[be] / rlast);
    for (long long t = threadIdx.x; t < M; t += blockDim.x) {
      float acc = 0.f;
      for (int c = 0; c < rr0; ++c) acc = fmaf(G0[t * rr0 + c], V1[be * s + c], acc);
      Y[t] = acc;
    }
    __syncthreads();
    for (long long row = threadIdx.x; row < M; row += blockDim.x) {
      const int aa = (int)row / N0, j = (int)row - aa * N0;
      const float* y = Y + (long long)aa * N0;
      int ilo, ihi;
      trans_window(a, j, i1, N0, &ilo, &ihi);
      float acc = 0.f;
      for (int i = ilo; i <= ihi; ++i) acc = fmaf(trans_k(a, j, i, i1), y[i], acc);
      F[(long long)be * M + row] = acc;
    }
    __syncthreads();
  }
}

// Transition block, fibers along mode 1 for the left elements alpha = (a, j)
// in oI (raw virtual indices): out(v1, al) = sum_c h(i', c) G_1(c, i', b) with
// h(i', c) = sum_i K(j, i, i') G_0(a, i, c) (staged in Y, N_1 r_1 floats),
// written at F + al * M: column al of a fiber matrix (ld M), or row al of the
// last core (M = its row length).
__device__ void trans_fibers_rl(const CrossArgs& a, const float* G0, const float* G1, int r1, int rb, int sL,
                                const long long* oI, float* F, long long M, float* Y) {
  const int N0 = a.N[0], N1 = a.N[1];
  constexpr int kC = 16;  // columns of h per pass: K(j, i, i') is evaluated once per kC columns
  const int npass = (r1 + kC - 1) / kC;
  for (int al = 0; al < sL; ++al) {
    const int aa = (int)(oI[al] / N0), jj = (int)(oI[al] - (long long)aa * N0);
    for (int e = threadIdx.x; e < N1 * npass; e += blockDim.x) {
      const int i1 = e / npass, c0 = (e - i1 * npass) * kC;
      const int nc = min(kC, r1 - c0);
      float acc[kC];
#pragma unroll
      for (int t = 0; t < kC; ++t) acc[t] = 0.f;
      const float* g = G0 + (long long)aa * N0 * r1 + c0;
      int ilo, ihi;
      trans_window(a, jj, i1, N0, &ilo, &ihi);
      for (int i = ilo; i <= ihi; ++i) {
        const float kv = trans_k(a, jj, i, i1);
        const float* gi = g + (long long)i * r1;
#pragma unroll
        for (int t = 0; t < kC; ++t)
          if (t < nc) acc[t] = fmaf(kv, gi[t], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < kC; ++t)
        if (t < nc) Y[i1 * r1 + c0 + t] = acc[t];
    }
    __syncthreads();
    for (long long row = threadIdx.x; row < (long long)N1 * rb; row += blockDim.x) {
      const int i1 = (int)row / rb, bb = (int)row - i1 * rb;
      float acc = 0.f;
      for (int c = 0; c < r1; ++c) acc = fmaf(Y[i1 * r1 + c], G1[((long long)c * N1 + i1) * rb + bb], acc);
      F[(long long)al * M + row] = acc;  // column al of the fiber matrix, or row al of the last core
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool taken(const unsigned* mask, long long i) {
  return (mask[i >> 5] >> (i & 31)) & 1u;
}

__global__ void __launch_bounds__(kCT) k_cross_step(CrossArgs a, int q, int kind) {
  const int b = blockIdx.x;
  if (b >= a.B) return;
  __shared__ float s_brow[S];
  __shared__ float s_Qp[S * S];  // the right interfaces while the fibers are built; then L1
  __shared__ float s_U[S * S];   // the left interfaces while the fibers are built
  __shared__ float s_rv[kCW];
  __shared__ long long s_ri[kCW];
  __shared__ long long s_piv[S];
  const int tid = threadIdx.x;
  const int k = a.k, s = a.s, ld = a.d + 1;
  const bool first = (kind == kCrossStart && q == k - 1);
  if (first) {
    if (tid == 0) a.status[b] = 0;
  } else if (a.status[b] != 0) {
    return;  // an earlier step of this cross was skipped
  }
  Geo g;
  if (!load_geo(a, b, &g)) {
    if (tid == 0) a.status[b] = 1;
    return;
  }
  int* szI = a.sz + (long long)b * 2 * ld;
  int* szJ = szI + ld;
  long long* offI = a.offI + (long long)b * ld * s;
  long long* offJ = a.offJ + (long long)b * ld * s;
  float* U = a.U + (long long)b * ld * s * s;
  float* V = a.V + (long long)b * ld * s * s;
  if (first) {
    // the empty sets at both ends: one element, interface [1]
    if (tid == 0) {
      szI[0] = 1;
      offI[0] = 0;
      U[0] = 1.f;
      szJ[k] = 1;
      offJ[(long long)k * s] = 0;
      V[(long long)k * s * s] = 1.f;
    }
    __syncthreads();
  }
  const long long nq = g.nv[q];
  const int rlq = g.rl(q), rrq = g.rr(q);
  const float* G = a.core[q] + (long long)b * a.cap[q];
  const bool lr = (kind == kCrossLR || kind == kCrossFinal);
  const int sL = (kind == kCrossStart) ? 0 : szI[q];
  const int sR = szJ[q + 1];
  long long M;
  int ncol, target;
  if (lr) {
    M = (long long)sL * nq;
    ncol = sR;
    target = sR;
  } else if (kind == kCrossRL) {
    M = nq * sR;
    ncol = sL;
    target = sL;
  } else {
    M = nq * sR;
    ncol = rlq;
    long long left = 1, right = 1;
    for (int t = 0; t < q; ++t) left = min(left * g.nv[t], 1LL << 30);
    for (int t = q; t < k; ++t) right = min(right * g.nv[t], 1LL << 30);
    target = (int)min((long long)s, min(left, right));
  }
  if (ncol > M) ncol = (int)M;
  if (target > M) target = (int)M;
  if (M * ncol > a.fcap || M > a.mcap || ncol < 1 || target < 1 ||
      (kind == kCrossFinal && M * target > a.cap[q])) {
    if (tid == 0) a.status[b] = 2;
    return;
  }
  const long long* oIq = offI + (long long)q * s;
  const long long* oJn = offJ + (long long)(q + 1) * s;
  const float* Uq = U + (long long)q * s * s;
  const float* Vn = V + (long long)(q + 1) * s * s;
  float* F = a.F + (long long)b * a.fcap;
  float* Qb = a.Qb + (long long)b * a.fcap;
  float* rn = a.rn + (long long)b * a.mcap;
  unsigned* mask = a.mask + (long long)b * (a.mcap / 32 + 1);
  const float zb = a.trans ? 0.f : a.z[(long long)b * a.zstride + a.zc];
  const float ob = a.trans ? 0.f : a.off[b];
  const float inv2r = (float)(0.5 / a.R);
  const long long strq = a.stride[q];

  // ---- fiber matrix F (M x ncol, column-major)
  if (!a.trans) {
    // the step's interfaces in shared memory (read once per fiber entry)
    for (int e = tid; e < sL * rlq; e += kCT) {
      const int al = e / rlq, c = e - al * rlq;
      s_U[al * S + c] = Uq[al * s + c];
    }
    for (int e = tid; e < sR * rrq; e += kCT) {
      const int be = e / rrq, c = e - be * rrq;
      s_Qp[be * S + c] = Vn[be * s + c];
    }
    __syncthreads();
  }
  if (a.trans && lr) {
    trans_fibers_lr(a, G, rrq, M, sR, oJn, Vn, g.r[k], F, Qb);
  } else if (a.trans && kind == kCrossRL) {
    trans_fibers_rl(a, a.core[0] + (long long)b * a.cap[0], G, g.r[1], g.r[k], sL, oIq, F, M, Qb);
  }
  for (long long row = tid; row < M && !(a.trans && kind != kCrossStart); row += kCT) {
    if (lr) {
      const int al = (int)((int)row / (int)nq);  // M < 2^31 (M <= mcap)
      const long long v = row - (long long)al * nq;
      float w[S];
      for (int cp = 0; cp < rrq; ++cp) {
        float acc = 0.f;
        for (int c = 0; c < rlq; ++c) acc = fmaf(s_U[al * S + c], G[((long long)c * nq + v) * rrq + cp], acc);
        w[cp] = acc;
      }
      const long long base = oIq[al] + g.grid(a, q, v) * strq;
      for (int be = 0; be < sR; ++be) {
        float acc = 0.f;
        for (int cp = 0; cp < rrq; ++cp) acc = fmaf(w[cp], s_Qp[be * S + cp], acc);
        F[(long long)be * M + row] = acc * lik_at(a, base + oJn[be], zb, ob, inv2r);
      }
    } else {
      const long long v = (int)row / sR;
      const int be = (int)(row - v * sR);
      float y[S];
      for (int c = 0; c < rlq; ++c) {
        float acc = 0.f;
        for (int cp = 0; cp < rrq; ++cp) acc = fmaf(G[((long long)c * nq + v) * rrq + cp], s_Qp[be * S + cp], acc);
        y[c] = acc;
      }
      if (kind == kCrossStart) {
        float nn = 0.f;
        for (int c = 0; c < ncol; ++c) {
          F[(long long)c * M + row] = y[c];
          nn = fmaf(y[c], y[c], nn);
        }
        rn[row] = nn;
      } else {
        const long long baseJ = g.grid(a, q, v) * strq + oJn[be];
        for (int al = 0; al < sL; ++al) {
          float acc = 0.f;
          for (int c = 0; c < rlq; ++c) acc = fmaf(s_U[al * S + c], y[c], acc);
          F[(long long)al * M + row] = acc * lik_at(a, oIq[al] + baseJ, zb, ob, inv2r);
        }
      }
    }
  }
  __syncthreads();

  // ---- maxvol start rows: Gaussian elimination with partial row pivoting on
  // the fiber matrix itself.  Its rows are those the same elimination picks
  // on an orthonormal basis Q of the columns (F = Q R, R upper triangular,
  // leaves every residual column a multiple of Q's), and it needs no basis.
  // A row not yet pivoted keeps its multipliers L(i, j) in column j.
  const int n = ncol;
  const int nm = min(n, target);
  const long long mwords = M / 32 + 1;
  for (long long e = tid; e < mwords; e += kCT) mask[e] = 0u;
  __syncthreads();
  float best;
  for (int j = 0; j < nm; ++j) {
    float bv = -1.f;
    long long bi = -1;
    for (long long i = tid; i < M; i += kCT) {
      if (taken(mask, i)) continue;
      const float x = fabsf(F[(long long)j * M + i]);
      if (bi < 0 || better(x, i, bv, bi)) {
        bv = x;
        bi = i;
      }
    }
    const long long p = block_argmax(bv, bi, s_rv, s_ri, &best);
    if (p < 0) {  // no free row: cannot happen while nm <= M
      if (tid == 0) a.status[b] = 3;
      return;
    }
    const float pv = F[(long long)j * M + p];
    const int len = nm - j - 1;
    for (int e = tid; e < len; e += kCT) s_brow[e] = F[(long long)(j + 1 + e) * M + p];
    __syncthreads();  // every thread has read pv and the pivot row before they change
    for (long long i = tid; i < M; i += kCT) {
      if (i == p || taken(mask, i)) continue;
      const float l = pv != 0.f ? F[(long long)j * M + i] / pv : 0.f;
      F[(long long)j * M + i] = l;
      for (int e = 0; e < len; ++e) F[(long long)(j + 1 + e) * M + i] -= l * s_brow[e];
    }
    if (tid == 0) {
      s_piv[j] = p;
      mask[p >> 5] |= 1u << (p & 31);
    }
    __syncthreads();
  }
  // B = F F[rows]^-1 = L L1^-1 (L1 = L[rows], unit lower triangular), in place
  // of F: a pivot row is the unit row of its place; another row solves
  // x L1 = L(i, :) from the last column down
  for (int e = tid; e < nm * nm; e += kCT) {
    const int r = e / nm, c = e - r * nm;
    s_Qp[r * S + c] = c < r ? F[(long long)c * M + s_piv[r]] : (c == r ? 1.f : 0.f);
  }
  __syncthreads();
  for (long long i = tid; i < M; i += kCT) {
    if (taken(mask, i)) {
      int r = 0;
      while (r < nm && s_piv[r] != i) ++r;
      for (int c = 0; c < nm; ++c) F[(long long)c * M + i] = (c == r) ? 1.f : 0.f;
      continue;
    }
    float x[S];
    for (int c = nm - 1; c >= 0; --c) {
      float v = F[(long long)c * M + i];
      for (int c2 = c + 1; c2 < nm; ++c2) v = fmaf(-x[c2], s_Qp[c2 * S + c], v);
      x[c] = v;
    }
    for (int c = 0; c < nm; ++c) F[(long long)c * M + i] = x[c];
  }
  __syncthreads();
  // each row's largest |B(i, c)| and the first column holding it, kept in
  // the (now free) scratch Qb by the row's owner and refreshed by each
  // exchange's update, so an exchange scans M row maxima, not M x nm entries
  float* rmax = Qb;
  int* rcol = reinterpret_cast<int*>(Qb + M);
  for (long long i = tid; i < M; i += kCT) {
    float mv = -1.f;
    int mc = 0;
    for (int c = 0; c < nm; ++c) {
      const float x = fabsf(F[(long long)c * M + i]);
      if (x > mv) {
        mv = x;
        mc = c;
      }
    }
    rmax[i] = mv;
    rcol[i] = mc;
  }
  __syncthreads();
  for (int it = 0; it < kMaxvolIters; ++it) {
    float bv = -1.f;
    long long bi = -1;
    for (long long i = tid; i < M; i += kCT) {
      const long long e = i * nm + rcol[i];  // row-major position: the tie order
      if (bi < 0 || better(rmax[i], e, bv, bi)) {
        bv = rmax[i];
        bi = e;
      }
    }
    const long long e = block_argmax(bv, bi, s_rv, s_ri, &best);
    if (e < 0 || !(best > 1.f + kDelta)) break;
    const long long is = e / nm;
    const int js = (int)(e - is * nm);
    const float pvv = F[(long long)js * M + is];
    for (int c = tid; c < nm; c += kCT) s_brow[c] = F[(long long)c * M + is] - (c == js ? 1.f : 0.f);
    if (tid == 0) s_piv[js] = is;
    __syncthreads();
    for (long long i = tid; i < M; i += kCT) {
      const float f = F[(long long)js * M + i] / pvv;
      float mv = -1.f;
      int mc = 0;
      for (int c = 0; c < nm; ++c) {
        const float x = F[(long long)c * M + i] - f * s_brow[c];
        F[(long long)c * M + i] = x;
        if (fabsf(x) > mv) {
          mv = fabsf(x);
          mc = c;
        }
      }
      rmax[i] = mv;
      rcol[i] = mc;
    }
    __syncthreads();
  }
  // start sets: pad with the rows of largest norm
  if (target > nm) {
    for (long long e = tid; e < mwords; e += kCT) mask[e] = 0u;
    __syncthreads();
    if (tid == 0)
      for (int j = 0; j < nm; ++j) mask[s_piv[j] >> 5] |= 1u << (s_piv[j] & 31);
    __syncthreads();
    for (int j = nm; j < target; ++j) {
      float bv = -1.f;
      long long bi = -1;
      for (long long i = tid; i < M; i += kCT) {
        if (taken(mask, i)) continue;
        if (bi < 0 || better(rn[i], i, bv, bi)) {
          bv = rn[i];
          bi = i;
        }
      }
      const long long p = block_argmax(bv, bi, s_rv, s_ri, &best);
      if (p < 0) {  // no free row: cannot happen while target <= M
        if (tid == 0) a.status[b] = 3;
        return;
      }
      if (tid == 0) {
        s_piv[j] = p;
        mask[p >> 5] |= 1u << (p & 31);
      }
      __syncthreads();
    }
  }
  __syncthreads();

  // ---- the new index set and its interfaces
  if (lr) {
    long long* oN = offI + (long long)(q + 1) * s;
    float* Un = U + (long long)(q + 1) * s * s;
    for (int e = tid; e < target * rrq; e += kCT) {
      const int j = e / rrq, cp = e - j * rrq;
      const long long row = s_piv[j];
      const int al = (int)(row / nq);
      const long long v = row - (long long)al * nq;
      float acc = 0.f;
      for (int c = 0; c < rlq; ++c) acc = fmaf(Uq[al * s + c], G[((long long)c * nq + v) * rrq + cp], acc);
      Un[j * s + cp] = acc;
      if (cp == 0) oN[j] = a.trans ? row : oIq[al] + g.grid(a, q, v) * strq;
    }
    if (tid == 0) szI[q + 1] = target;
  } else {
    long long* oN = offJ + (long long)q * s;
    float* Vq = V + (long long)q * s * s;
    for (int e = tid; e < target * rlq; e += kCT) {
      const int j = e / rlq, c = e - j * rlq;
      const long long row = s_piv[j];
      const long long v = row / sR;
      const int be = (int)(row - v * sR);
      float acc = 0.f;
      for (int cp = 0; cp < rrq; ++cp) acc = fmaf(G[((long long)c * nq + v) * rrq + cp], Vn[be * s + cp], acc);
      Vq[j * s + c] = acc;
      if (c == 0) oN[j] = a.trans ? row : g.grid(a, q, v) * strq + oJn[be];
    }
    if (tid == 0) szJ[q] = target;
  }
  if (kind == kCrossFinal) {
    // core q = B in the density's layout [alpha][v][j]
    float* O = a.out[q] + (long long)b * a.cap[q];
    for (long long row = tid; row < M; row += kCT)
      for (int j = 0; j < target; ++j) O[row * target + j] = F[(long long)j * M + row];
  }
}

// The last core (fibers T(I_{k-1}, v) over the last virtual mode) and the
// block's new ranks.
__global__ void __launch_bounds__(kCT) k_cross_last(CrossArgs a) {
  const int b = blockIdx.x;
  if (b >= a.B) return;
  const int tid = threadIdx.x, k = a.k, s = a.s, ld = a.d + 1;
  Geo g;
  if (!load_geo(a, b, &g)) return;
  if (a.status[b] != 0) return;
  const int* szI = a.sz + (long long)b * 2 * ld;
  const int q = k - 1;
  const int sL = szI[q];
  const long long nq = g.nv[q];
  const int rlq = g.rl(q);
  if ((long long)sL * nq > a.cap[q]) return;
  const long long* oI = a.offI + ((long long)b * ld + q) * s;
  const float* Uq = a.U + ((long long)b * ld + q) * s * s;
  const float* G = a.core[q] + (long long)b * a.cap[q];
  float* O = a.out[q] + (long long)b * a.cap[q];
  if (a.trans) {
    trans_fibers_rl(a, a.core[0] + (long long)b * a.cap[0], G, g.r[1], g.r[k], sL, oI, O, nq,
                    a.Qb + (long long)b * a.fcap);
  }
  const float zb = a.trans ? 0.f : a.z[(long long)b * a.zstride + a.zc];
  const float ob = a.trans ? 0.f : a.off[b];
  const float inv2r = (float)(0.5 / a.R);
  for (long long e = tid; e < (long long)sL * nq && !a.trans; e += kCT) {
    const int al = (int)(e / nq);
    const long long v = e - (long long)al * nq;
    float acc = 0.f;
    for (int c = 0; c < rlq; ++c) acc = fmaf(Uq[al * s + c], G[(long long)c * nq + v], acc);
    O[e] = acc * lik_at(a, oI[al] + g.grid(a, q, v) * a.stride[q], zb, ob, inv2r);
  }
  __syncthreads();
  if (tid == 0) {
    int* rk = a.ranks + (long long)b * ld;
    for (int l = 1; l < k; ++l) rk[a.lo + l] = szI[l];
  }
}

}  // namespace

void launch_cross_step(cudaStream_t st, const CrossArgs& a, int q, int kind) {
  count_launches(1);
  k_cross_step<<<a.B, kCT, 0, st>>>(a, q, kind);
}

void launch_cross_last(cudaStream_t st, const CrossArgs& a) {
  count_launches(1);
  k_cross_last<<<a.B, kCT, 0, st>>>(a);
}

}  // namespace ttgbf
