// Tensor-core correlation of a batch with an approximate dictionary (BF16 or per-atom scaled
// E4M3): G[b][j] = scale_j sigma_b sum_n q_jn r^_bn, on the 5th-generation tensor cores.
//
// One CTA computes a 128-atom x 256-signal tile: warp 0 streams 128-byte K-slices of both
// operands into a 4-stage shared-memory ring with TMA (128B swizzle), warp 1 issues
// tcgen05.mma (M = 128, N = 256, FP32 accumulators in TMEM) and commits each stage back to the
// producer, warps 2-5 read the accumulators with tcgen05.ld and scale/store them.  Tiles whose
// 256 signals are all on other ladder levels (or finished) exit before allocating anything.
// Every mbarrier wait is bounded: on expiry the CTA records an error and still frees its TMEM.
//
// Paper: the correlation A~^T rho of the proximal update (eq:ISTA_update) with the approximate
// dictionaries of Section III; here batched over signals, which makes it a dense contraction.
#include <algorithm>
#include <cstring>

#include <cudaTypedefs.h>

#include "tc_gemm.cuh"

namespace lasso {

constexpr uint32_t TC_WAIT_POLLS = 1u << 22;   // bounded mbarrier waits (seconds, never forever)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t i = 0; i < TC_WAIT_POLLS; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA instruction descriptor: FP32 accumulation, A and B K-major, M x N tile.
// ab_format: 1 = BF16 (kind::f16), 0 = E4M3 (kind::f8f6f4).
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t ab_format, uint32_t M, uint32_t N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout: rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused by swizzled K-major layouts)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

template <int FP8>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  if constexpr (FP8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The signal of slot n0 + c0 + lane (lane's column of a 32-column chunk), its scale, and whether
// the slot is live; the epilogue warps broadcast them by shuffle (no barrier among them).
struct TcCol {
  int on, sig;
  float sigma;
};
__device__ __forceinline__ TcCol tc_col(int64_t slot, int64_t nslots, const int* __restrict__ list,
                                        const float* __restrict__ sigma) {
  TcCol c;
  c.on = slot < nslots;
  c.sig = c.on ? (list ? list[slot] : (int)slot) : 0;
  c.sigma = c.on ? (sigma ? sigma[c.sig] : 1.f) : 0.f;
  return c;
}

// Persistent over the tiles: CTA c takes tiles c, c + gridDim.x, ... of the (atom tile, signal
// tile) grid of the live slots, atom tile fastest (consecutive CTAs share the signal tile's
// residual rows in L2).  Two TMEM accumulators (512 columns): tile i accumulates in buffer i % 2
// while the epilogue drains tile i - 1 from the other, and the TMA ring runs on across tiles.  A
// launch with no live slot exits at once.
template <int FP8>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_corr(const __grid_constant__ CUtensorMap tma, const __grid_constant__ CUtensorMap tmb,
          const __grid_constant__ CUtensorMap tma2, const __grid_constant__ CUtensorMap tmb2, int64_t K, int64_t B,
          int nkb, int nphase, const float* __restrict__ scale, const float* __restrict__ sigma,
          const int* __restrict__ list, const int* __restrict__ count, float* __restrict__ Gfull,
          int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  __shared__ int s_fail;
  __shared__ uint32_t s_tmem;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                                    // TC_STAGES x 16 KB
  uint8_t* sB = base + TC_STAGES * TC_BM * 128;          // TC_STAGES x 32 KB
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * TC_BN * 128);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accf = empty + TC_STAGES;                    // [2]: tile in buffer b accumulated
  uint64_t* acce = accf + 2;                             // [2]: buffer b drained by the epilogue

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nslots = count ? (int64_t)*count : B;
  const int tm = (int)((K + TC_BM - 1) / TC_BM);
  const int total = tm * (int)((nslots + TC_BN - 1) / TC_BN);
  if ((int)blockIdx.x >= total) return;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accf[0], 1);
    mbar_init(&accf[1], 1);
    mbar_init(&acce[0], 4);
    mbar_init(&acce[1], 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(2 * TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr int KB_ELEMS = FP8 ? 128 : 64;   // elements per 128-byte K-slice
  const int nk = nkb * nphase;               // phases: a^T r (1); a1^T r1, a1^T r2, a2^T r1 (3)

  if (warp == 0) {
    // ---- TMA producer: the k-slices of every tile of this CTA, one ring
    if (lane == 0) {
      int g = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x) {
        const int64_t m0 = (int64_t)(t % tm) * TC_BM, n0 = (int64_t)(t / tm) * TC_BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % TC_STAGES;
          const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
          const int phase = kb / nkb, kk = kb - phase * nkb;
          if (g >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
            s_fail = 1;
            stop = true;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)(TC_BM + TC_BN) * 128u);
          tma_load_2d(phase == 2 ? &tma2 : &tma, &full[s], sA + s * TC_BM * 128, kk * KB_ELEMS, (int)m0);
          tma_load_2d(phase == 1 ? &tmb2 : &tmb, &full[s], sB + s * TC_BN * 128, kk * KB_ELEMS, (int)n0);
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc(FP8 ? 0u : 1u, TC_BM, TC_BN);
      int g = 0, it = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x, ++it) {
        const int buf = it & 1;
        if (it >= 2) {
          // the epilogue has drained this buffer's previous tile
          if (!mbar_wait(&acce[buf], (uint32_t)((it >> 1) - 1) & 1u)) {
            s_fail = 1;
            break;
          }
          tc_fence_after();
        }
        const uint32_t dst = tmem + (uint32_t)(buf * TC_BN);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % TC_STAGES;
          const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
          if (!mbar_wait(&full[s], ph)) {
            s_fail = 1;
            stop = true;
            break;
          }
          tc_fence_after();
          const uint64_t ad = umma_sdesc(smem_u32(sA + s * TC_BM * 128));
          const uint64_t bd = umma_sdesc(smem_u32(sB + s * TC_BN * 128));
#pragma unroll
          for (int k = 0; k < 4; ++k)   // four 32-byte K-steps per 128-byte slice
            umma<FP8>(dst, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (!stop) umma_commit(&accf[buf]);   // arrives once the tile's MMAs have completed
      }
    }
  } else {
    // ---- epilogue: TMEM lane quarter (warp % 4) holds atoms m0 + 32 q .. + 31
    const int q = warp & 3;
    int it = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      const int buf = it & 1;
      const int64_t m0 = (int64_t)(t % tm) * TC_BM, n0 = (int64_t)(t / tm) * TC_BN;
      if (!mbar_wait(&accf[buf], (uint32_t)(it >> 1) & 1u)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const int64_t row = m0 + q * 32 + lane;
      const float sc = row < K ? (scale ? scale[row] : 1.f) : 0.f;
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        const TcCol mine = tc_col(n0 + c0 + lane, nslots, list, sigma);
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_BN + c0), r);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int on = __shfl_sync(0xffffffffu, mine.on, i);
          const int sig = __shfl_sync(0xffffffffu, mine.sig, i);
          const float sg = __shfl_sync(0xffffffffu, mine.sigma, i);
          if (on && row < K) Gfull[(int64_t)sig * K + row] = __uint_as_float(r[i]) * sc * sg;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// The same product with promoted accumulation.  The MMAs of k-block g (TC_GROUP consecutive
// 128-byte K-slices, over the phases in order) accumulate from zero into TMEM buffer g % 2
// (columns [256 (g % 2), 256 (g % 2) + 256)); when a k-block's MMAs complete, the eight epilogue
// warps load it with tcgen05.ld and add it to FP32 registers (round to nearest), then release the
// buffer.  Warp 2 + e reads TMEM lane quarter (warp % 4) and the column half e / 4, so each
// epilogue thread holds 128 running sums (one atom, 128 signals).  The tensor-core accumulation
// chain is one k-block long; the k-block sums are added in FP32.  Persistent over the tiles like
// k_tc_corr; the k-block counter runs on across a CTA's tiles.
template <int FP8>
__global__ void __launch_bounds__(TCP_THREADS, 1)
k_tc_corr_kb(const __grid_constant__ CUtensorMap tma, const __grid_constant__ CUtensorMap tmb,
             const __grid_constant__ CUtensorMap tma2, const __grid_constant__ CUtensorMap tmb2, int64_t K, int64_t B,
             int nkb, int nphase, const float* __restrict__ scale, const float* __restrict__ sigma,
             const int* __restrict__ list, const int* __restrict__ count, float* __restrict__ Gfull,
             int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  __shared__ int s_fail;
  __shared__ uint32_t s_tmem;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + TC_STAGES * TC_BM * 128;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * TC_BN * 128);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accf = empty + TC_STAGES;     // [2]: k-block in buffer b complete (tcgen05.commit)
  uint64_t* acce = accf + 2;              // [2]: buffer b read by the 8 epilogue warps

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nslots = count ? (int64_t)*count : B;
  const int tm = (int)((K + TC_BM - 1) / TC_BM);
  const int total = tm * (int)((nslots + TC_BN - 1) / TC_BN);
  if ((int)blockIdx.x >= total) return;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accf[0], 1);
    mbar_init(&accf[1], 1);
    mbar_init(&acce[0], 8);
    mbar_init(&acce[1], 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(2 * TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr int KB_ELEMS = FP8 ? 128 : 64;
  const int nk = nkb * nphase;
  const int ng = (nk + TC_GROUP - 1) / TC_GROUP;   // k-blocks per tile

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x) {
        const int64_t m0 = (int64_t)(t % tm) * TC_BM, n0 = (int64_t)(t / tm) * TC_BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % TC_STAGES;
          const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
          const int phase = kb / nkb, kk = kb - phase * nkb;
          if (g >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
            s_fail = 1;
            stop = true;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)(TC_BM + TC_BN) * 128u);
          tma_load_2d(phase == 2 ? &tma2 : &tma, &full[s], sA + s * TC_BM * 128, kk * KB_ELEMS, (int)m0);
          tma_load_2d(phase == 1 ? &tmb2 : &tmb, &full[s], sB + s * TC_BN * 128, kk * KB_ELEMS, (int)n0);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc(FP8 ? 0u : 1u, TC_BM, TC_BN);
      int g = 0, gb = 0;   // k-slice and k-block counters of this CTA
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x, gb += ng) {
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int gg = gb + kb / TC_GROUP;
          const bool first = (kb % TC_GROUP) == 0;
          const int buf = gg & 1;
          if (first && gg >= 2) {
            // the epilogue has read this buffer's previous k-block
            if (!mbar_wait(&acce[buf], (uint32_t)((gg >> 1) - 1) & 1u)) {
              s_fail = 1;
              stop = true;
              break;
            }
            tc_fence_after();
          }
          const int s = g % TC_STAGES;
          const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
          if (!mbar_wait(&full[s], ph)) {
            s_fail = 1;
            stop = true;
            break;
          }
          tc_fence_after();
          const uint64_t ad = umma_sdesc(smem_u32(sA + s * TC_BM * 128));
          const uint64_t bd = umma_sdesc(smem_u32(sB + s * TC_BN * 128));
          const uint32_t dst = tmem + (uint32_t)(buf * TC_BN);
#pragma unroll
          for (int k = 0; k < 4; ++k) umma<FP8>(dst, ad + 2 * k, bd + 2 * k, idesc, (first && k == 0) ? 0u : 1u);
          umma_commit(&empty[s]);
          if ((kb % TC_GROUP) == TC_GROUP - 1 || kb == nk - 1) umma_commit(&accf[buf]);
        }
      }
    }
  } else {
    const int e = warp - 2;
    const int q = warp & 3;                  // TMEM lane quarter this warp may read
    const int h = e >> 2;                    // column half
    int gb = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, gb += ng) {
      const int64_t m0 = (int64_t)(t % tm) * TC_BM, n0 = (int64_t)(t / tm) * TC_BN;
      const int64_t row = m0 + q * 32 + lane;
      float acc[TC_BN / 2];
#pragma unroll
      for (int i = 0; i < TC_BN / 2; ++i) acc[i] = 0.f;
      bool ok = true;
      for (int g = 0; g < ng; ++g) {
        const int gg = gb + g;
        const int buf = gg & 1;
        if (!mbar_wait(&accf[buf], (uint32_t)(gg >> 1) & 1u)) {
          ok = false;
          s_fail = 1;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < TC_BN / 64; ++c) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_BN + h * (TC_BN / 2) + c * 32), r);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[c * 32 + i] = __fadd_rn(acc[c * 32 + i], __uint_as_float(r[i]));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[buf]);
      }
      if (!ok) break;
      const float sc = row < K ? (scale ? scale[row] : 1.f) : 0.f;
#pragma unroll
      for (int c = 0; c < TC_BN / 64; ++c) {
        const TcCol mine = tc_col(n0 + h * (TC_BN / 2) + c * 32 + lane, nslots, list, sigma);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int on = __shfl_sync(0xffffffffu, mine.on, i);
          const int sig = __shfl_sync(0xffffffffu, mine.sig, i);
          const float sg = __shfl_sync(0xffffffffu, mine.sigma, i);
          if (on && row < K) Gfull[(int64_t)sig * K + row] = acc[c * 32 + i] * sc * sg;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ------------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static int encode_2d(CUtensorMap* map, const void* ptr, int64_t rows, int64_t ld, int fp8, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_last_error("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  const int es = fp8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  return LASSO_OK;
}

int tc_make_operands(const void* level_data, const void* level_data2, int64_t K, const void* rq, const void* rq2,
                     int64_t B, int64_t ldN, int fp8, TcOperands* out) {
  const bool split = level_data2 != nullptr || rq2 != nullptr;
  if ((ldN * (fp8 ? 1 : 2)) % 16 != 0 || (reinterpret_cast<uintptr_t>(level_data) & 15) ||
      (reinterpret_cast<uintptr_t>(rq) & 15) || (split && (fp8 || !level_data2 || !rq2)) ||
      (reinterpret_cast<uintptr_t>(level_data2) & 15) || (reinterpret_cast<uintptr_t>(rq2) & 15))
    return LASSO_ERR_INVALID_ARG;
  out->fp8 = fp8;
  out->nphase = split ? 3 : 1;
  out->promote = split ? 1 : 0;
  int rc = encode_2d(&out->a, level_data, K, ldN, fp8, TC_BM);
  if (rc) return rc;
  rc = encode_2d(&out->b, rq, B, ldN, fp8, TC_BN);
  if (rc) return rc;
  if (!split) {
    out->a2 = out->a;
    out->b2 = out->b;
    return LASSO_OK;
  }
  rc = encode_2d(&out->a2, level_data2, K, ldN, 0, TC_BM);
  if (rc) return rc;
  return encode_2d(&out->b2, rq2, B, ldN, 0, TC_BN);
}

void tc_launch_corr(const TcOperands& ops, int64_t K, int64_t B, int64_t ldN, const float* scale,
                    const float* sigma, const int* list, const int* count, float* Gfull, int* err,
                    cudaStream_t stream) {
  static bool attr[2] = {false, false};
  static bool attr_kb = false;
  const int es = ops.fp8 ? 1 : 2;
  const int nkb = (int)((ldN * es + 127) / 128);   // 128-byte K-slices (TMA zero-fills the tail)
  // persistent CTAs: at most one per SM (each holds about 200 KB of shared memory and all of TMEM)
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int64_t tiles = ((K + TC_BM - 1) / TC_BM) * ((B + TC_BN - 1) / TC_BN);
  const dim3 grid((unsigned)std::min<int64_t>(tiles, sms));
  if (ops.promote && !ops.fp8) {
    if (!attr_kb) {
      cudaFuncSetAttribute(k_tc_corr_kb<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM);
      attr_kb = true;
    }
    k_tc_corr_kb<0><<<grid, TCP_THREADS, TCP_SMEM, stream>>>(ops.a, ops.b, ops.a2, ops.b2, K, B, nkb, ops.nphase,
                                                             scale, sigma, list, count, Gfull, err);
    return;
  }
  if (ops.fp8) {
    if (!attr[1]) {
      cudaFuncSetAttribute(k_tc_corr<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      attr[1] = true;
    }
    k_tc_corr<1><<<grid, TC_THREADS, TC_SMEM, stream>>>(ops.a, ops.b, ops.a2, ops.b2, K, B, nkb, ops.nphase, scale,
                                                        sigma, list, count, Gfull, err);
  } else {
    if (!attr[0]) {
      cudaFuncSetAttribute(k_tc_corr<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      attr[0] = true;
    }
    k_tc_corr<0><<<grid, TC_THREADS, TC_SMEM, stream>>>(ops.a, ops.b, ops.a2, ops.b2, K, B, nkb, ops.nphase, scale,
                                                        sigma, list, count, Gfull, err);
  }
}

// ------------------------------------------------------------------ self-test

__device__ __forceinline__ uint32_t tc_hash(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return (uint32_t)x;
}

// Operands with a wide dynamic range: |v| = 2^e (1 + m / 8), e in [-6, 5] (E4M3 exact) or BF16
// values of a uniform grid; `positive` makes every product the same sign (worst accumulation).
__global__ void k_tc_fill(uint8_t* __restrict__ dst, int64_t rows, int64_t ld, int64_t N, int fp8, int positive,
                          uint64_t seed) {
  const int64_t total = rows * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t % ld;
    const uint32_t h = tc_hash(seed * 0x9E3779B97F4A7C15ull + (uint64_t)t);
    float v = 0.f;
    if (n < N) {
      const int e = (int)(h % 12) - 6;
      const int m = (int)((h >> 8) % 8);
      v = ldexpf(1.f + m / 8.f, e);
      if (!positive && ((h >> 16) & 1)) v = -v;
    }
    if (fp8) dst[t] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    else reinterpret_cast<__nv_bfloat16*>(dst)[t] = __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ double tc_val(const uint8_t* p, int64_t idx, int fp8) {
  if (fp8) {
    __half_raw hr = __nv_cvt_fp8_to_halfraw(p[idx], __NV_E4M3);
    return (double)__half2float(__half(hr));
  }
  return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
}

// FP64 reference and error statistics: err / sum|a r| and err / (gamma_n(u_tc) sum|a r|).
// Split mode (A2, R2 non-null): the reference is a1^T r1 + a1^T r2 + a2^T r1.
__global__ void k_tc_check(const uint8_t* __restrict__ A, const uint8_t* __restrict__ R, const uint8_t* __restrict__ A2,
                           const uint8_t* __restrict__ R2, const float* __restrict__ G, int64_t K, int64_t B, int64_t ld,
                           int fp8, double gam, unsigned long long* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= K * B) return;
  const int64_t j = t % K, b = t / K;
  double s = 0.0, sa = 0.0;
  for (int64_t n = 0; n < ld; ++n) {
    const double a = tc_val(A, j * ld + n, fp8), r = tc_val(R, b * ld + n, fp8);
    const double p = a * r;
    s += p;
    sa += fabs(p);
    if (A2) {
      const double p2 = a * tc_val(R2, b * ld + n, 0), p3 = tc_val(A2, j * ld + n, 0) * r;
      s += p2 + p3;
      sa += fabs(p2) + fabs(p3);
    }
  }
  const double err = fabs((double)G[b * K + j] - s);
  const double rel = sa > 0.0 ? err / sa : 0.0;
  const double ratio = sa > 0.0 ? err / (gam * sa) : 0.0;
  atomicMax(&out[0], __double_as_longlong(rel));
  atomicMax(&out[1], __double_as_longlong(ratio));
}

int tc_selftest(int mode, int64_t K, int64_t N, int64_t B, double* max_rel, double* max_ratio) {
  const int fp8 = mode == 1 ? 1 : 0;
  const bool split = mode == 2;
  const int64_t ld = round_up(N, 16);
  const int es = fp8 ? 1 : 2;
  uint8_t *A = nullptr, *R = nullptr, *A2 = nullptr, *R2 = nullptr;
  float* G = nullptr;
  int* err = nullptr;
  unsigned long long* out = nullptr;
  int rc = LASSO_OK;
  if (cudaMalloc(&A, K * ld * es) != cudaSuccess || cudaMalloc(&R, B * ld * es) != cudaSuccess ||
      cudaMalloc(&G, K * B * 4) != cudaSuccess || cudaMalloc(&err, 4) != cudaSuccess ||
      cudaMalloc(&out, 16) != cudaSuccess ||
      (split && (cudaMalloc(&A2, K * ld * 2) != cudaSuccess || cudaMalloc(&R2, B * ld * 2) != cudaSuccess)))
    rc = LASSO_ERR_NOMEM;
  double rel = 0.0, ratio = 0.0;
  for (int positive = 0; positive < 2 && rc == LASSO_OK; ++positive) {
    cudaMemset(err, 0, 4);
    cudaMemset(out, 0, 16);
    cudaMemset(G, 0, K * B * 4);
    k_tc_fill<<<1024, 256>>>(A, K, ld, N, fp8, positive, 11 + positive);
    k_tc_fill<<<1024, 256>>>(R, B, ld, N, fp8, positive, 29 + positive);
    if (split) {
      k_tc_fill<<<1024, 256>>>(A2, K, ld, N, 0, positive, 47 + positive);
      k_tc_fill<<<1024, 256>>>(R2, B, ld, N, 0, positive, 53 + positive);
    }
    TcOperands ops;
    rc = tc_make_operands(A, A2, K, R, R2, B, ld, fp8, &ops);
    if (rc) break;
    tc_launch_corr(ops, K, B, ld, nullptr, nullptr, nullptr, nullptr, G, err, 0);
    const int nk = (int)(ld / (fp8 ? 32 : 16));
    // split (promoted): one k-block's chain of TC_GROUP * 64 products and 4 TC_GROUP k-steps with
    // u_tc, then the FP32 sum of the k-blocks; plain: one chain over all products
    const double gam = split ? tc_promoted_gamma(ld, 3)
                             : gamma_n(((double)ld + nk), fp8 ? TC_U_FP8 : TC_U_BF16);
    k_tc_check<<<(unsigned)((K * B + 255) / 256), 256>>>(A, R, A2, R2, G, K, B, ld, fp8, gam, out);
    int herr = 0;
    unsigned long long h[2] = {0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(h, out, 16, cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_last_error(cudaGetErrorString(cudaGetLastError()), __FILE__, __LINE__);
      rc = LASSO_ERR_CUDA;
      break;
    }
    if (herr) {
      rc = LASSO_ERR_TIMEOUT;
      break;
    }
    double r0, r1;
    memcpy(&r0, &h[0], 8);
    memcpy(&r1, &h[1], 8);
    rel = fmax(rel, r0);
    ratio = fmax(ratio, r1);
  }
  cudaFree(A);
  cudaFree(R);
  cudaFree(A2);
  cudaFree(R2);
  cudaFree(G);
  cudaFree(err);
  cudaFree(out);
  if (max_rel) *max_rel = rel;
  if (max_ratio) *max_ratio = ratio;
  return rc;
}

}  // namespace lasso

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_tc_selftest(int mode, int64_t K, int64_t N, int64_t B, double* max_rel_err,
                                 double* max_err_over_bound) {
  lasso::clear_last_error();
  if (K <= 0 || N <= 0 || B <= 0 || K * B > (int64_t)1 << 28 || mode < 0 || mode > 2) return LASSO_ERR_INVALID_ARG;
  return lasso::tc_selftest(mode, K, N, B, max_rel_err, max_err_over_bound);
}
