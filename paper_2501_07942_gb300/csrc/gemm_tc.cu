// gemm_tc.cu -- the grouped GEMM of the TT contractions (the rank-r core
// products of Sec. 4.1 "round", the per-mode operators and the 2-site merge of
// the update) on the fifth-generation tensor cores: tcgen05.mma of kind::tf32
// with float32 accumulators in tensor memory (TMEM).
//
// A tile is 128 entries along the longer side of C by 32 along the shorter
// one (C^T = B^T A^T when n > m), so the MMA's M = 128 rows always run along
// the tall dimension of the rounding's tall-skinny products.  Per tile:
//   * 128 threads (4 warps) stage k in chunks of 16: both operands K-major in
//     shared memory, in the no-swizzle canonical layout of 8-row x 16-byte
//     core matrices (core matrices adjacent along k 128 bytes apart, along
//     the rows 512 bytes apart).  The loads are plain global loads: the
//     operands' leading dimensions are ranks and need not be multiples of 16
//     bytes, so the staging converts as it copies.  Each float is rounded to
//     TF32 (round to nearest); in the split mode (3xTF32) the remainder
//     x - hi is rounded as well and staged beside it.
//   * thread 0 issues two MMAs of K = 8 per chunk (six in the split mode:
//     lo*hi, hi*lo, hi*hi, the lo*lo term is below float32 rounding) and
//     commits them to the chunk's mbarrier; two staging buffers alternate,
//     so the next chunk is staged while the tensor core works on this one.
//   * after the last commit the four warps read their 32 TMEM lanes (rows of
//     the tile) with tcgen05.ld and write C.
// The TMEM allocation is 32 columns per CTA; with 40 KB of shared memory per
// CTA at most five CTAs share an SM, so an allocation never waits.  Every
// mbarrier wait gives up after one second of the global timer: the tile is
// then written as NaN, *status is set, and the CTA frees its TMEM and returns.
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace ttgbf {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcKC = 16;                         // k per staged chunk
constexpr int kTcABytes = kTcTileM * kTcKC * 4;   // one operand chunk, 128 rows: 8 KB
constexpr int kTcBBytes = kTcTileN * kTcKC * 4;   // 32 rows: 2 KB
constexpr int kTcBufBytes = 2 * (kTcABytes + kTcBBytes);  // hi and lo parts
constexpr int kTcTmemCols = 32;
constexpr unsigned long long kTcWaitNs = 1000000000ull;  // one second

// Instruction descriptor of tcgen05.mma kind::tf32: D float32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcTileN >> 3) << 17) |
                              ((uint32_t)(kTcTileM >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29: core matrices adjacent along k), stride byte
// offset >> 4 (bits 32-45: adjacent 8-row groups), the fixed 0b001 at bits
// 46-48, no base offset, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Byte offset of element (i, k) of a staged operand chunk (k < 16).
__device__ __forceinline__ int tc_off(int i, int k) {
  return ((i >> 3) << 9) + ((k >> 2) << 7) + ((i & 7) << 4) + ((k & 3) << 2);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of the given parity of an mbarrier; false after the
// time limit.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kTcWaitNs) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One operand of a tile: element (i, k) at p[i * si + k * sk], i < ilim, k < K.
struct TcSrc {
  const float* p;
  long long si, sk;
  int ilim;
};

// Element q of this thread's share of an operand chunk with R rows (R a
// multiple or a divisor of the 128 threads): (i, k) = (i0 + q di, k0 + q dk),
// consecutive threads along whichever index is contiguous in memory.
struct TcMap {
  int i0, k0, di, dk;
};
template <int R>
__device__ __forceinline__ TcMap tc_map(bool kcontig) {
  const int tid = threadIdx.x;
  if (kcontig) return TcMap{tid / kTcKC, tid % kTcKC, kTcThreads / kTcKC, 0};
  if (R >= kTcThreads) return TcMap{tid, 0, 0, 1};  // R == 128: one k per element
  return TcMap{tid % R, tid / R, 0, kTcThreads / R};
}

// Global loads of k in [k0, k0 + 16) of an operand with R rows (zero past
// the operand's edges).
template <int R>
__device__ __forceinline__ void tc_load(const TcSrc& s, int k0, int K, float (&v)[R * kTcKC / kTcThreads]) {
  static_assert(R == kTcThreads || kTcThreads % R == 0, "operand rows");
  const TcMap m = tc_map<R>(s.sk == 1);
  const float* p = s.p + (long long)m.i0 * s.si + (long long)(k0 + m.k0) * s.sk;
  const long long step = (long long)m.di * s.si + (long long)m.dk * s.sk;
#pragma unroll
  for (int q = 0; q < R * kTcKC / kTcThreads; ++q) {
    const bool in = m.i0 + q * m.di < s.ilim && k0 + m.k0 + q * m.dk < K;
    v[q] = in ? __ldg(p + q * step) : 0.f;
  }
}

// The loaded values, rounded to TF32, into the staging layout (and their
// rounded remainders into lo).
template <int R, bool kSplit>
__device__ __forceinline__ void tc_store(const TcSrc& s, const float (&v)[R * kTcKC / kTcThreads], uint8_t* hi,
                                         uint8_t* lo) {
  const TcMap m = tc_map<R>(s.sk == 1);
#pragma unroll
  for (int q = 0; q < R * kTcKC / kTcThreads; ++q) {
    const int off = tc_off(m.i0 + q * m.di, m.k0 + q * m.dk);
    const uint32_t h = to_tf32(v[q]);
    *reinterpret_cast<uint32_t*>(hi + off) = h;
    if (kSplit) *reinterpret_cast<uint32_t*>(lo + off) = to_tf32(v[q] - __uint_as_float(h));
  }
}

template <bool kSplit>
__global__ void __launch_bounds__(kTcThreads, 4) k_gemm_tc(GemmWork w, double* flops) {
  __shared__ __align__(1024) uint8_t s_buf[2][kTcBufBytes];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  const int total = w.tiles[w.ndesc];
  if ((int)blockIdx.x >= total) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  uint32_t phase[2] = {0u, 0u};
  bool failed = false;
  for (int t = blockIdx.x; t < total && !failed; t += gridDim.x) {
    int lo = 0, hi = w.ndesc;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (w.tiles[mid] <= t) lo = mid; else hi = mid;
    }
    const GemmDesc g = w.desc[lo];
    const bool tr = g.shape == kTcShapeT;  // tile rows along C's columns
    const int lng = tr ? g.n : g.m, sht = tr ? g.m : g.n;
    const int nshort = (sht + kTcTileN - 1) / kTcTileN;
    const int local = t - w.tiles[lo];
    const int l0 = (local / nshort) * kTcTileM, s0 = (local % nshort) * kTcTileN;
    // operand A of the MMA: 128 rows along the long side; B: 32 along the short side
    TcSrc sa, sb;
    if (!tr) {
      sa = TcSrc{g.A + (long long)l0 * g.lda, g.lda, 1, lng - l0};
      sb = TcSrc{g.B + s0, 1, g.ldb, sht - s0};
    } else {
      sa = TcSrc{g.B + l0, 1, g.ldb, lng - l0};
      sb = TcSrc{g.A + (long long)s0 * g.lda, g.lda, 1, sht - s0};
    }
    const int nch = (g.k + kTcKC - 1) / kTcKC;
    // chunk c + 1's global loads are issued before chunk c's MMAs, so their
    // latency overlaps the tensor core's work and the next buffer wait
    float va[kTcTileM * kTcKC / kTcThreads], vb[kTcTileN * kTcKC / kTcThreads];
    if (nch > 0) {
      tc_load<kTcTileM>(sa, 0, g.k, va);
      tc_load<kTcTileN>(sb, 0, g.k, vb);
    }
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      if (c >= 2) {  // the MMAs of chunk c - 2 have read this buffer
        const bool ok = mbar_wait(smem_u32(&s_bar[b]), phase[b]);
        phase[b] ^= 1u;
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
      }
      uint8_t* base = s_buf[b];
      tc_store<kTcTileM, kSplit>(sa, va, base, base + kTcABytes + kTcBBytes);
      tc_store<kTcTileN, kSplit>(sb, vb, base + kTcABytes, base + 2 * kTcABytes + kTcBBytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (c + 1 < nch) {
        tc_load<kTcTileM>(sa, (c + 1) * kTcKC, g.k, va);
        tc_load<kTcTileN>(sb, (c + 1) * kTcKC, g.k, vb);
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ah = smem_u32(base), bh = ah + kTcABytes;
        const uint32_t al = bh + kTcBBytes, bl = al + kTcABytes;
#pragma unroll
        for (int s = 0; s < kTcKC / 8; ++s) {
          const uint32_t so = s * 256;  // two 16-byte core-matrix columns per K = 8
          const uint32_t acc0 = (c > 0 || s > 0) ? 1u : 0u;
          if (kSplit) {
            tc_mma(tmem, tc_desc(al + so), tc_desc(bh + so), acc0);
            tc_mma(tmem, tc_desc(ah + so), tc_desc(bl + so), 1u);
            tc_mma(tmem, tc_desc(ah + so), tc_desc(bh + so), 1u);
          } else {
            tc_mma(tmem, tc_desc(ah + so), tc_desc(bh + so), acc0);
          }
        }
        tc_commit(smem_u32(&s_bar[b]));
      }
    }
    if (!failed && nch > 0) {  // the last one or two chunks' commits
      bool ok = true;
      if (nch >= 2) {
        const int b = nch & 1;  // chunk nch - 2
        ok = mbar_wait(smem_u32(&s_bar[b]), phase[b]);
        phase[b] ^= 1u;
      }
      {
        const int b = (nch - 1) & 1;
        ok = mbar_wait(smem_u32(&s_bar[b]), phase[b]) && ok;
        phase[b] ^= 1u;
      }
      if (__syncthreads_or(!ok)) failed = true;
    }
    tc_fence_after();
    // epilogue: thread (warp, lane) holds tile row 32 warp + lane; its 32
    // columns are read in two halves of 16
    const int i = warp * 32 + lane;
#pragma unroll
    for (int h = 0; h < kTcTileN / 16; ++h) {
      uint32_t v[16];
      if (nch > 0 && !failed) {
        tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * h, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = failed ? 0x7fc00000u : 0u;  // NaN marks a tile given up
      }
      if (l0 + i < lng) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cj = s0 + 16 * h + j;
          if (cj >= sht) break;
          const float x = __uint_as_float(v[j]);
          if (!tr) g.C[(long long)(l0 + i) * g.ldc + cj] = x;
          else g.C[(long long)cj * g.ldc + l0 + i] = x;
        }
      }
    }
    if (tid == 0 && flops != nullptr && !failed) {
      const int rows = min(kTcTileM, lng - l0), cols = min(kTcTileN, sht - s0);
      atomicAdd(flops, 2.0 * rows * cols * (double)g.k);
    }
    // every warp's TMEM reads are done before the next tile's first MMA
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (failed) {  // a last bounded wait for tensor-core work still in flight
    mbar_wait(smem_u32(&s_bar[0]), phase[0]);
    mbar_wait(smem_u32(&s_bar[1]), phase[1]);
    if (tid == 0 && w.status != nullptr) atomicExch(w.status, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

}  // namespace

void launch_gemm_tc(cudaStream_t st, GemmWork gw, int grid, double* flops) {
  count_launches(1);
  if (gw.tc == kContractTf32x3) k_gemm_tc<true><<<grid, kTcThreads, 0, st>>>(gw, flops);
  else k_gemm_tc<false><<<grid, kTcThreads, 0, st>>>(gw, flops);
}

}  // namespace ttgbf
