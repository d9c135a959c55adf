// tsqr.cu -- R factor of the tall matrices of TT rounding (Sec. 4.1 "round";
// Alg. 2 step 2), batched over filters: Householder QR with the matrix held in
// registers.
//
// One CTA (16 warps) holds a 256 x n tile, n <= 160, in registers: lane
// (warp w, half h, row lane l) owns rows l + 16 a (a < 16) of the columns
// 32 q + 2 w + h.  Column j's reflector is formed by the 16 lanes that hold
// it and broadcast through shared memory; every other column's dot product
// with it is a 16-lane shuffle reduction.  One __syncthreads per column: the
// owner of column j + 1 forms the next reflector right after its own update
// (double-buffered reflectors), so the sync also publishes it.
//
// A filter's rows are cut into slices, one CTA each.  A slice is consumed in
// passes: the first pass factors 256 rows; each later pass keeps the n x n R
// on top of the tile and factors it together with the next 256 - n rows (the
// rows of R below the current column are known zeros and are skipped).  The
// slice R factors go to a per-filter stack; the CTA that finishes last
// (atomic counter after a memory fence; no CTA ever waits on another) stacks
// them and factors the stack the same way.  The result is the n x n R
// (row-major, zeros below the diagonal) in stack0 (one slice) or stack1.
#include <math.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kQrThreads = 512;
constexpr int kQrRL = 16;                // row lanes per half-warp
constexpr int kQrRPL = 16;               // rows per lane
constexpr int kQrRows = kQrRL * kQrRPL;  // tile rows
static_assert(kQrRows == kTsqrTileRows, "tile geometry");
constexpr int kQrSlots = 32;             // column slots per register column (16 warps x 2)
constexpr int kQrMaxCPL = (kMaxN + kQrSlots - 1) / kQrSlots;
constexpr float kQrTiny = 1e-30f;  // column entries below this count as zero

static_assert(kQrRows > kMaxN, "each pass must take new rows below R");
static_assert(kQrMaxCPL <= 5, "register budget");

struct QrShared {
  float v[2][kQrRows];
  float tau[2];
  int last;
};

// Rows [first, kQrRows) of the tile from source rows row0 + (i - first),
// zero past nrows.  `coherent` loads bypass L1 (data written by other CTAs
// during this kernel).
template <int CPL>
__device__ __forceinline__ void qr_load(float (&A)[kQrRPL][CPL], const float* p, long long rs,
                                        long long cs, long long row0, long long nrows, int first,
                                        int n, int rl, int slot, bool coherent) {
  const float* base = p + row0 * rs + (long long)slot * cs;
  const long long qstep = (long long)kQrSlots * cs;
#pragma unroll
  for (int a = 0; a < kQrRPL; ++a) {
    const int i = rl + kQrRL * a;
    if (i < first) continue;
    const long long r = i - first;
    const float* rowp = base + r * rs;
    const bool rok = r < nrows;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      float x = 0.f;
      if (rok && kQrSlots * q + slot < n) x = coherent ? __ldcg(rowp + q * qstep) : __ldg(rowp + q * qstep);
      A[a][q] = x;
    }
  }
}

// Reflector H = I - tau v v^T (v_j = 1) that zeroes column j (register
// column Q, so j >= 32 Q) below row j.  Executed by the whole owner warp;
// half `own` holds the column.  Writes v (rows >= 32 Q; the rows above are
// never read for this column group) and tau, and leaves beta on the
// diagonal and zeros below it.
template <int CPL, int Q>
__device__ __forceinline__ void qr_reflector(float (&A)[kQrRPL][CPL], int j, int rl, bool own,
                                             float* v, float* tau_out) {
  constexpr int A0 = 2 * Q;
  float s0 = 0.f, s1 = 0.f, alpha = 0.f;
#pragma unroll
  for (int a = A0; a < kQrRPL; ++a) {
    const int i = rl + kQrRL * a;
    const float x = A[a][Q];
    const float x2 = (i > j) ? x * x : 0.f;
    if (a & 1) s1 += x2; else s0 += x2;
    if (i == j) alpha = x;
  }
  float ss = s0 + s1;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  alpha = __shfl_sync(0xffffffffu, alpha, (threadIdx.x & 16) | (j & 15));
  // |x|^2 sums are exact enough unless they leave [1e-30, 1e30]; such columns
  // take a second pass scaled by the column maximum
  const float tot = fmaf(alpha, alpha, ss);
  const bool rescale = tot != 0.f && !(tot >= 1e-30f && tot <= 1e30f);
  float nm = sqrtf(tot), tail2 = ss;
  if (__any_sync(0xffffffffu, rescale)) {
    float mx = 0.f;
#pragma unroll
    for (int a = A0; a < kQrRPL; ++a) {
      const int i = rl + kQrRL * a;
      if (i >= j) mx = fmaxf(mx, fabsf(A[a][Q]));
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float inv = (rescale && mx >= kQrTiny) ? 1.f / mx : 0.f;
    float s2 = 0.f;
#pragma unroll
    for (int a = A0; a < kQrRPL; ++a) {
      const int i = rl + kQrRL * a;
      const float x = A[a][Q] * inv;
      if (i > j) s2 = fmaf(x, x, s2);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (rescale) {
      const float al = alpha * inv;
      nm = mx * sqrtf(fmaf(al, al, s2));
      tail2 = s2;  // only its sign (zero or not) is used below
    }
  }
  float tau = 0.f, beta = alpha, scl = 0.f;
  if (tail2 > 0.f) {
    beta = alpha >= 0.f ? -nm : nm;
    const float am = alpha - beta;  // sign(alpha) (|alpha| + nm): no cancellation
    tau = -am / beta;                // (beta - alpha) / beta, in [1, 2]
    scl = 1.f / am;
  }
  if (own) {
#pragma unroll
    for (int a = A0; a < kQrRPL; ++a) {
      const int i = rl + kQrRL * a;
      const float x = A[a][Q];
      v[i] = (i > j) ? x * scl : (i == j ? 1.f : 0.f);
      A[a][Q] = (i > j) ? 0.f : (i == j ? beta : x);
    }
    if (rl == 0) *tau_out = tau;
  }
}

// Row block a of the tile is skipped by every reflector of column group
// Q0: rows above 32 Q0 are zero in v; with R on top of the tile (HASR), so
// are the blocks strictly between the group and row 32 (CPL - 1) < n, where
// R is known zero; blocks at or past NA hold no rows of this pass.
template <int CPL, bool HASR, int NA, int Q0>
__device__ __forceinline__ constexpr bool qr_skip(int a) {
  return a < 2 * Q0 || a >= NA || (HASR && a >= 2 * Q0 + 2 && a < 2 * (CPL - 1));
}

// Reflector entries of this lane's rows for column group Q0.
template <int CPL, bool HASR, int NA, int Q0>
__device__ __forceinline__ void qr_vload(float (&vr)[kQrRPL], int rl, const float* v) {
#pragma unroll
  for (int a = 0; a < kQrRPL; ++a)
    if (!qr_skip<CPL, HASR, NA, Q0>(a)) vr[a] = v[rl + kQrRL * a];
}

// Apply the reflector of column j (j in [32 Q0, 32 Q0 + 32)) to the
// columns after j among register columns [QA, QB).
template <int CPL, bool HASR, int NA, int Q0, int QA, int QB>
__device__ __forceinline__ void qr_apply(float (&A)[kQrRPL][CPL], const float* v, int j, int rl,
                                         int slot, float tau) {
  if constexpr (QA < QB) {
    float vr[kQrRPL];
    qr_vload<CPL, HASR, NA, Q0>(vr, rl, v);
    float dot[CPL];
#pragma unroll
    for (int q = QA; q < QB; ++q) dot[q] = 0.f;
#pragma unroll
    for (int a = 0; a < kQrRPL; ++a) {
      if (qr_skip<CPL, HASR, NA, Q0>(a)) continue;
#pragma unroll
      for (int q = QA; q < QB; ++q) dot[q] = fmaf(vr[a], A[a][q], dot[q]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int q = QA; q < QB; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
    for (int q = QA; q < QB; ++q) {
      const int c = kQrSlots * q + slot;
      dot[q] = (c > j) ? tau * dot[q] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < kQrRPL; ++a) {
      if (qr_skip<CPL, HASR, NA, Q0>(a)) continue;
#pragma unroll
      for (int q = QA; q < QB; ++q) A[a][q] = fmaf(-dot[q], vr[a], A[a][q]);
    }
  }
}

// Steps j in [32 Q0, 32 Q0 + 32) of a pass (register column group Q0 is
// static, so every register index below is static).  The owner warp of
// column j + 1 updates that register column first, forms the next
// reflector, then updates its other columns, so the reflector's latency
// overlaps the other warps' updates.
template <int CPL, bool HASR, int NA, int Q0>
__device__ __forceinline__ void qr_group(float (&A)[kQrRPL][CPL], int n, QrShared& sh, int rl,
                                         int half, int warp, int slot) {
  for (int s = 0; s < kQrSlots; ++s) {
    const int j = kQrSlots * Q0 + s;
    if (j >= n) break;
    const int buf = j & 1;
    const float tau = sh.tau[buf];
    const int jn = j + 1;
    const bool owner = jn < n && warp == ((jn & 31) >> 1);
    const bool own = half == (jn & 1);
    const float* v = sh.v[buf];
    if (owner) {
      if (s + 1 < kQrSlots) {
        if (tau != 0.f) qr_apply<CPL, HASR, NA, Q0, Q0, Q0 + 1>(A, v, j, rl, slot, tau);
        qr_reflector<CPL, Q0>(A, jn, rl, own, sh.v[buf ^ 1], &sh.tau[buf ^ 1]);
        if (tau != 0.f) qr_apply<CPL, HASR, NA, Q0, Q0 + 1, CPL>(A, v, j, rl, slot, tau);
      } else if constexpr (Q0 + 1 < CPL) {
        if (tau != 0.f) qr_apply<CPL, HASR, NA, Q0, Q0 + 1, Q0 + 2>(A, v, j, rl, slot, tau);
        qr_reflector<CPL, Q0 + 1>(A, jn, rl, own, sh.v[buf ^ 1], &sh.tau[buf ^ 1]);
        if (tau != 0.f) {
          qr_apply<CPL, HASR, NA, Q0, Q0, Q0 + 1>(A, v, j, rl, slot, tau);
          qr_apply<CPL, HASR, NA, Q0, Q0 + 2, CPL>(A, v, j, rl, slot, tau);
        }
      }
    } else if (tau != 0.f) {
      qr_apply<CPL, HASR, NA, Q0, Q0, CPL>(A, v, j, rl, slot, tau);
    }
    __syncthreads();
  }
  if constexpr (Q0 + 1 < CPL) {
    if (kQrSlots * (Q0 + 1) < n) qr_group<CPL, HASR, NA, Q0 + 1>(A, n, sh, rl, half, warp, slot);
  }
}

// Householder QR of the tile's n columns; R ends in rows < n.  HASR: rows
// < n already hold an upper triangular R.
// NA: row blocks that hold rows of this pass (the rest are zero).
template <int CPL, bool HASR, int NA>
__device__ __forceinline__ void qr_pass(float (&A)[kQrRPL][CPL], int n, QrShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane & 15, half = lane >> 4, slot = 2 * warp + half;
  if (warp == 0) qr_reflector<CPL, 0>(A, 0, rl, half == 0, sh.v[0], &sh.tau[0]);
  __syncthreads();
  qr_group<CPL, HASR, NA, 0>(A, n, sh, rl, half, warp, slot);
}

// R factor of rows [row0, row0 + M) of (p, rs, cs), n columns, by passes;
// written row-major n x n to out.
template <int CPL>
__device__ __noinline__ void qr_rows(const float* p, long long rs, long long cs, long long row0,
                                     long long M, int n, bool coherent, float* out, QrShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane & 15, slot = 2 * warp + (lane >> 4);
  float A[kQrRPL][CPL];
  qr_load<CPL>(A, p, rs, cs, row0, M, 0, n, rl, slot, coherent);
  long long done = M < kQrRows ? M : kQrRows;
  if (M <= kQrRows / 2) {
    qr_pass<CPL, false, kQrRPL / 2>(A, n, sh);  // rows 128.. are zero
  } else {
    qr_pass<CPL, false, kQrRPL>(A, n, sh);
  }
  while (done < M) {
    qr_load<CPL>(A, p, rs, cs, row0 + done, M - done, n, n, rl, slot, coherent);
    done += kQrRows - n;
    qr_pass<CPL, true, kQrRPL>(A, n, sh);
  }
#pragma unroll
  for (int a = 0; a < kQrRPL; ++a) {
    const int i = rl + kQrRL * a;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = kQrSlots * q + slot;
      if (i < n && c < n) out[(long long)i * n + c] = A[a][q];
    }
  }
}

// Fields are read from global memory where they are used, so that none of
// them stays live in registers across the passes.
template <int CPL>
__device__ void qr_item(const TsqrProblem* pp, int b, int s, int* counter, double* flops,
                        QrShared& sh) {
  const int n = pp->src.n;
  const int nslice = pp->nslice;
  if (nslice == 1) {
    qr_rows<CPL>(pp->src.p, pp->src.rs, pp->src.cs, 0, pp->src.M, n, false, pp->stack0, sh);
  } else {
    const long long r0 = (long long)s * pp->slice;
    const long long M = pp->src.M;
    const long long rows = (M - r0 < pp->slice) ? M - r0 : pp->slice;
    qr_rows<CPL>(pp->src.p, pp->src.rs, pp->src.cs, r0, rows, n, false,
                 pp->stack0 + (long long)s * n * n, sh);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh.last = (atomicAdd(counter + b, 1) == nslice - 1);
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    qr_rows<CPL>(pp->stack0, n, 1, 0, (long long)nslice * n, n, true, pp->stack1, sh);
  }
  if (threadIdx.x == 0 && flops != nullptr) {
    // Householder R factor of an M x n matrix: 2 M n^2 - 2 n^3 / 3
    const double M = (double)pp->src.M;
    const double k = M < n ? M : (double)n;
    atomicAdd(flops, 2.0 * M * n * k - 2.0 * k * k * k / 3.0);
  }
}

__global__ void __launch_bounds__(kQrThreads, 1) k_tsqr(TsqrWork w, int B, int* counter,
                                                         double* flops) {
  __shared__ QrShared sh;
  const int total = w.offset[B];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int lo = 0, hi = B;  // offset[lo] <= item < offset[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.offset[mid] <= item) lo = mid; else hi = mid;
    }
    const int b = lo;
    const TsqrProblem* pp = w.prob + b;
    const int s = item - w.offset[b];
    const int cpl = (pp->src.n + kQrSlots - 1) / kQrSlots;
    switch (cpl) {
      case 1: qr_item<1>(pp, b, s, counter, flops, sh); break;
      case 2: qr_item<2>(pp, b, s, counter, flops, sh); break;
      case 3: qr_item<3>(pp, b, s, counter, flops, sh); break;
      case 4: qr_item<4>(pp, b, s, counter, flops, sh); break;
      default: qr_item<5>(pp, b, s, counter, flops, sh); break;
    }
    __syncthreads();
  }
}

}  // namespace

void launch_tsqr(cudaStream_t st, TsqrWork w, int B, int grid, double* flops) {
  count_launches(1);
  k_tsqr<<<grid, kQrThreads, 0, st>>>(w, B, w.counter, flops);
}

}  // namespace ttgbf
