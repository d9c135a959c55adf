// tsqr.cu -- R factor of the tall matrices of TT rounding (Sec. 4.1 "round";
// Alg. 2 step 2), batched over filters: structured Householder QR with the
// running R in shared memory and the incoming rows in registers.
//
// A CTA of 8 warps keeps the n x n upper-triangular R of the rows it has
// consumed in shared memory (zero at the start) and takes the rows in blocks
// of 128: lane (warp w, half h, row lane l) holds rows 8 l + a (a < 8) of
// the block for the columns 16 q + w + 8 h (q < ceil(n / 16)).  Column j of
// [R; block] is reduced by one reflector that touches only row j of R and
// the block (R is triangular), so a block costs n steps of
//   reflector: norm of the block's column j (16-lane shuffle sum) with
//              R(j, j); v = the block's column scaled, v = 1 on R's row j;
//   update:    every column c > j: d = R(j, c) + v . block(:, c) (16-lane
//              shuffle sum), R(j, c) -= tau d, block(:, c) -= tau d v.
// One barrier per column.  The owner of column j + 1 updates that column
// first and forms the next reflector (double-buffered in shared memory)
// before its other columns, so the barrier also publishes it.  Two CTAs run
// per SM (R of up to 160 x 160 floats each), so one CTA's reflector latency
// overlaps the other's updates.
//
// A filter's rows are cut into slices, one CTA each.  The slice R factors
// go to a per-filter stack; the CTA that finishes last (atomic counter after
// a memory fence; no CTA ever waits on another) factors the stacked R's the
// same way.  The result is the n x n R (row-major, zeros below the diagonal)
// in stack0 (one slice) or stack1 (several).
#include <math.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kQrThreads = 256;
constexpr int kQrRL = 16;                // row lanes per half-warp
constexpr int kQrRPL = 8;                // rows per lane
constexpr int kQrRows = kQrRL * kQrRPL;  // rows per block
static_assert(kQrRows == kTsqrTileRows, "block geometry");
constexpr int kQrSlots = 16;  // column slots per register column (8 warps x 2 halves)
constexpr int kQrMaxCPL = (kMaxN + kQrSlots - 1) / kQrSlots;
static_assert(kQrMaxCPL <= 10, "register budget");
constexpr int kQrLd = kMaxN;  // row stride of R in shared memory

// Reflectors rotate through four buffers: the owner of a column publishes
// the next reflector and finishes its own other columns after the barrier,
// so a reflector can still be read two steps later.
struct __align__(16) QrShared {
  float v[4][kQrRows];
  float tau[4];
  int last;
};

// Named barriers 1..3 (step j uses 1 + j % 3).  A warp that only arrives at
// one step's barrier (the owner, which does not wait) is never the owner of
// two consecutive steps (consecutive columns belong to different warps), so
// it waits at the next barrier and no warp reaches the same barrier id again
// before that barrier's previous use completed.
__device__ __forceinline__ void qr_bar_sync(int id) {
  static_assert(kQrThreads == 256, "barrier thread count");
  if (id == 1) asm volatile("bar.sync 1, 256;" ::: "memory");
  else if (id == 2) asm volatile("bar.sync 2, 256;" ::: "memory");
  else asm volatile("bar.sync 3, 256;" ::: "memory");
}
__device__ __forceinline__ void qr_bar_arrive(int id) {
  if (id == 1) asm volatile("bar.arrive 1, 256;" ::: "memory");
  else if (id == 2) asm volatile("bar.arrive 2, 256;" ::: "memory");
  else asm volatile("bar.arrive 3, 256;" ::: "memory");
}

// Rows [row0, row0 + 128) of (p, rs, cs) into the block, zero past nrows.
// `coherent` loads bypass L1 (data written by other CTAs of this kernel).
template <int CPL>
__device__ __forceinline__ void qr_load(float (&A)[kQrRPL][CPL], const float* p, long long rs,
                                        long long cs, long long row0, long long nrows, int n,
                                        int rl, int slot, bool coherent) {
  const float* base = p + row0 * rs + (long long)slot * cs;
  const long long qstep = (long long)kQrSlots * cs;
#pragma unroll
  for (int a = 0; a < kQrRPL; ++a) {
    const int i = rl * kQrRPL + a;
    const float* rowp = base + (long long)i * rs;
    const bool rok = i < nrows;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      float x = 0.f;
      if (rok && kQrSlots * q + slot < n)
        x = coherent ? __ldcg(rowp + q * qstep) : __ldg(rowp + q * qstep);
      A[a][q] = x;
    }
  }
}

// Reflector of column j (register column Q) of [R; block], executed by the
// whole owner warp; half `own` holds the column.  Writes v (block rows) and
// tau, puts beta in R(j, j) and zeroes the block's column.  With
// nm = ||(R(j, j), block(:, j))||, beta = -sign(alpha) nm, tau = (|alpha| +
// nm) / nm and v = x / (alpha - beta): one reciprocal square root and one
// reciprocal on the dependency chain.
template <int CPL, int Q>
__device__ __forceinline__ void qr_reflector(float (&A)[kQrRPL][CPL], int j, int rl, bool own,
                                             float* Rs, float* v, float* tau_out) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int a = 0; a < kQrRPL; a += 2) {
    s0 = fmaf(A[a][Q], A[a][Q], s0);
    s1 = fmaf(A[a + 1][Q], A[a + 1][Q], s1);
  }
  float ss = s0 + s1;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float alpha = Rs[j * kQrLd + j];
  // squares are exact enough unless the sum leaves [1e-30, 1e30]; such
  // columns take a second pass scaled by the column maximum
  float tot = fmaf(alpha, alpha, ss), tail2 = ss, scale = 1.f;
  const bool rescale = tot != 0.f && !(tot >= 1e-30f && tot <= 1e30f);
  if (__any_sync(0xffffffffu, rescale)) {
    float mx = 0.f;
#pragma unroll
    for (int a = 0; a < kQrRPL; ++a) mx = fmaxf(mx, fabsf(A[a][Q]));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mx = fmaxf(mx, fabsf(alpha));
    const float inv = (rescale && mx > 0.f) ? 1.f / mx : 0.f;
    float s2 = 0.f;
#pragma unroll
    for (int a = 0; a < kQrRPL; ++a) {
      const float x = A[a][Q] * inv;
      s2 = fmaf(x, x, s2);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (rescale) {
      const float al = alpha * inv;
      tot = fmaf(al, al, s2);  // of the scaled column; nm = mx sqrt(tot)
      tail2 = s2;
      scale = mx;
    }
  }
  float tau = 0.f, beta = alpha, scl = 0.f;
  if (tail2 > 0.f) {
    const float rs = rsqrtf(tot);
    const float nm = tot * rs * scale;
    const float aa = fabsf(alpha);
    beta = alpha >= 0.f ? -nm : nm;
    tau = fmaf(aa / scale, rs, 1.f);  // (|alpha| + nm) / nm
    const float am = aa + nm;         // |alpha - beta|
    scl = alpha >= 0.f ? __frcp_rn(am) : -__frcp_rn(am);
  }
  if (own) {
    // v of rows 8 rl + (0..3) at float4 rl, rows 8 rl + (4..7) at float4
    // 16 + rl: a half's 16-byte accesses cover contiguous 256 bytes
    float4* v4 = reinterpret_cast<float4*>(v);
    v4[rl] = make_float4(A[0][Q] * scl, A[1][Q] * scl, A[2][Q] * scl, A[3][Q] * scl);
    v4[kQrRL + rl] = make_float4(A[4][Q] * scl, A[5][Q] * scl, A[6][Q] * scl, A[7][Q] * scl);
#pragma unroll
    for (int a = 0; a < kQrRPL; ++a) A[a][Q] = 0.f;
    if (rl == 0) {
      *tau_out = tau;
      Rs[j * kQrLd + j] = beta;
    }
  }
}

// Apply the reflector of column j (j in [16 Q0, 16 Q0 + 16)) to the columns
// after j among register columns [QA, QB).  Row lane 0 carries R(j, c).
template <int CPL, int Q0, int QA, int QB>
__device__ __forceinline__ void qr_apply(float (&A)[kQrRPL][CPL], float* Rs, const float* v, int j,
                                         int rl, int slot, float tau) {
  if constexpr (QA < QB) {
    float vr[kQrRPL];
    {
      const float4* v4 = reinterpret_cast<const float4*>(v);
      const float4 v0 = v4[rl], v1 = v4[kQrRL + rl];
      vr[0] = v0.x; vr[1] = v0.y; vr[2] = v0.z; vr[3] = v0.w;
      vr[4] = v1.x; vr[5] = v1.y; vr[6] = v1.z; vr[7] = v1.w;
    }
    // R(j, c) enters through row lane 0; columns of groups after Q0 all lie
    // after j
    float rj[CPL], dot[CPL];
#pragma unroll
    for (int q = QA; q < QB; ++q) {
      const int c = kQrSlots * q + slot;
      const bool live = q > Q0 || c > j;
      rj[q] = (rl == 0 && live) ? Rs[j * kQrLd + c] : 0.f;
    }
#pragma unroll
    for (int q = QA; q < QB; ++q) {
      float d0 = rj[q], d1 = 0.f;
#pragma unroll
      for (int a = 0; a < kQrRPL; a += 2) {
        d0 = fmaf(vr[a], A[a][q], d0);
        d1 = fmaf(vr[a + 1], A[a + 1][q], d1);
      }
      dot[q] = d0 + d1;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int q = QA; q < QB; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
    for (int q = QA; q < QB; ++q) {
      const int c = kQrSlots * q + slot;
      const bool live = q > Q0 || c > j;
      const float f = live ? tau * dot[q] : 0.f;
      if (live && rl == 0) Rs[j * kQrLd + c] = rj[q] - f;
#pragma unroll
      for (int a = 0; a < kQrRPL; ++a) A[a][q] = fmaf(-f, vr[a], A[a][q]);
    }
  }
}

// Steps j in [16 Q0, 16 Q0 + 16) of a block (register column group Q0 is
// static, so every register index below is static).
template <int CPL, int Q0>
__device__ __forceinline__ void qr_group(float (&A)[kQrRPL][CPL], int n, float* Rs, QrShared& sh,
                                         int rl, int half, int warp, int slot) {
  for (int s = 0; s < kQrSlots; ++s) {
    const int j = kQrSlots * Q0 + s;
    if (j >= n) break;
    const int buf = j & 3, nbuf = (j + 1) & 3, bar = 1 + j % 3;
    const float tau = sh.tau[buf];
    const int jn = j + 1;
    const bool owner = jn < n && warp == (jn & 7);
    const bool own = half == ((jn >> 3) & 1);
    const float* v = sh.v[buf];
    if (owner) {
      // the owner's chain: update of column jn, its reflector, publish;
      // its other columns are updated after it has arrived
      if (s + 1 < kQrSlots) {
        if (tau != 0.f) qr_apply<CPL, Q0, Q0, Q0 + 1>(A, Rs, v, j, rl, slot, tau);
        qr_reflector<CPL, Q0>(A, jn, rl, own, Rs, sh.v[nbuf], &sh.tau[nbuf]);
        qr_bar_arrive(bar);
        if (tau != 0.f) qr_apply<CPL, Q0, Q0 + 1, CPL>(A, Rs, v, j, rl, slot, tau);
      } else if constexpr (Q0 + 1 < CPL) {
        if (tau != 0.f) qr_apply<CPL, Q0, Q0 + 1, Q0 + 2>(A, Rs, v, j, rl, slot, tau);
        qr_reflector<CPL, Q0 + 1>(A, jn, rl, own, Rs, sh.v[nbuf], &sh.tau[nbuf]);
        qr_bar_arrive(bar);
        if (tau != 0.f) {
          qr_apply<CPL, Q0, Q0, Q0 + 1>(A, Rs, v, j, rl, slot, tau);
          qr_apply<CPL, Q0, Q0 + 2, CPL>(A, Rs, v, j, rl, slot, tau);
        }
      } else {
        qr_bar_sync(bar);  // not reached: jn < n <= 16 CPL
      }
    } else {
      if (tau != 0.f) qr_apply<CPL, Q0, Q0, CPL>(A, Rs, v, j, rl, slot, tau);
      qr_bar_sync(bar);
    }
  }
  if constexpr (Q0 + 1 < CPL) {
    if (kQrSlots * (Q0 + 1) < n) qr_group<CPL, Q0 + 1>(A, n, Rs, sh, rl, half, warp, slot);
  }
}

// R factor of rows [row0, row0 + M) of (p, rs, cs), n columns: blocks of
// 128 rows folded into R (shared memory), then R written row-major n x n to
// out.
template <int CPL>
__device__ __noinline__ void qr_rows(const float* p, long long rs, long long cs, long long row0,
                                     long long M, int n, bool coherent, float* out, float* Rs,
                                     QrShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // consecutive columns belong to different warps, so the owner of the next
  // column has finished the previous step's updates when its reflector is due
  const int rl = lane & 15, half = lane >> 4, slot = warp + 8 * half;
  for (int t = threadIdx.x; t < n * kQrLd; t += kQrThreads) Rs[t] = 0.f;
  float A[kQrRPL][CPL];
  for (long long done = 0; done < M; done += kQrRows) {
    qr_load<CPL>(A, p, rs, cs, row0 + done, M - done, n, rl, slot, coherent);
    __syncthreads();  // R zeroed / previous block's last step complete
    if (warp == 0) qr_reflector<CPL, 0>(A, 0, rl, half == 0, Rs, sh.v[0], &sh.tau[0]);
    __syncthreads();
    qr_group<CPL, 0>(A, n, Rs, sh, rl, half, warp, slot);
  }
  for (int t = threadIdx.x; t < n * n; t += kQrThreads) {
    const int i = t / n, c = t - i * n;
    out[t] = (c >= i) ? Rs[i * kQrLd + c] : 0.f;
  }
  __syncthreads();
}

// Fields are read from global memory where they are used, so that none of
// them stays live in registers across the blocks.
template <int CPL>
__device__ void qr_item(const TsqrProblem* pp, int b, int s, int* counter, double* flops,
                        float* Rs, QrShared& sh) {
  const int n = pp->src.n;
  const int nslice = pp->nslice;
  if (nslice == 1) {
    qr_rows<CPL>(pp->src.p, pp->src.rs, pp->src.cs, 0, pp->src.M, n, false, pp->stack0, Rs, sh);
  } else {
    const long long r0 = (long long)s * pp->slice;
    const long long M = pp->src.M;
    const long long rows = (M - r0 < pp->slice) ? M - r0 : pp->slice;
    qr_rows<CPL>(pp->src.p, pp->src.rs, pp->src.cs, r0, rows, n, false,
                 pp->stack0 + (long long)s * n * n, Rs, sh);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh.last = (atomicAdd(counter + b, 1) == nslice - 1);
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    qr_rows<CPL>(pp->stack0, n, 1, 0, (long long)nslice * n, n, true, pp->stack1, Rs, sh);
  }
  if (threadIdx.x == 0 && flops != nullptr) {
    // Householder R factor of an M x n matrix: 2 M n^2 - 2 n^3 / 3
    const double M = (double)pp->src.M;
    const double k = M < n ? M : (double)n;
    atomicAdd(flops, 2.0 * M * n * k - 2.0 * k * k * k / 3.0);
  }
}

__global__ void __launch_bounds__(kQrThreads, 2) k_tsqr(TsqrWork w, int B, int* counter,
                                                         double* flops) {
  extern __shared__ float Rs[];  // kMaxN x kQrLd
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
      case 1: qr_item<1>(pp, b, s, counter, flops, Rs, sh); break;
      case 2: qr_item<2>(pp, b, s, counter, flops, Rs, sh); break;
      case 3: qr_item<3>(pp, b, s, counter, flops, Rs, sh); break;
      case 4: qr_item<4>(pp, b, s, counter, flops, Rs, sh); break;
      case 5: qr_item<5>(pp, b, s, counter, flops, Rs, sh); break;
      case 6: qr_item<6>(pp, b, s, counter, flops, Rs, sh); break;
      case 7: qr_item<7>(pp, b, s, counter, flops, Rs, sh); break;
      case 8: qr_item<8>(pp, b, s, counter, flops, Rs, sh); break;
      case 9: qr_item<9>(pp, b, s, counter, flops, Rs, sh); break;
      default: qr_item<10>(pp, b, s, counter, flops, Rs, sh); break;
    }
    __syncthreads();
  }
}

constexpr int kQrSmemBytes = kMaxN * kQrLd * (int)sizeof(float);

}  // namespace

void launch_tsqr(cudaStream_t st, TsqrWork w, int B, int grid, double* flops) {
  count_launches(1);
  k_tsqr<<<2 * grid, kQrThreads, kQrSmemBytes, st>>>(w, B, w.counter, flops);
}

void set_tsqr_attributes() {
  cudaFuncSetAttribute(k_tsqr, cudaFuncAttributeMaxDynamicSharedMemorySize, kQrSmemBytes);
}

}  // namespace ttgbf
