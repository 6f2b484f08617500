// Device building blocks of one FISTA pass over the preserved atoms: atom-row dot products
// with compensated accumulation, and the sparse residual accumulation.
//
// Rounding model (folded into the stable test by the callers, see LevelDev):
//  * the exact FP32 level uses Dot2 (error-free products, TwoSum accumulation): the error of
//    the unrounded result is second order, <= 2 gamma_{2n}^2 sum_i |a_i rho^_i|;
//  * BF16 / FP8 levels: 2 products (the first rounded, the second fused) are summed in FP32
//    and the pair is added exactly (TwoSum) into a double-float accumulator, so
//    |g^ - a~^T rho^| <= gamma_3 sum_i |a~_i rho^_i|;
//  * FP64-arithmetic levels: plain FP64 FMA chains.
#pragma once

#include "common.cuh"

namespace lasso {

__device__ __forceinline__ float2 bf16x2_to_f2(uint32_t v) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
  return __bfloat1622float2(h);
}

__device__ __forceinline__ float2 fp8x2_to_f2(uint16_t v) {
  __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)v, __NV_E4M3);
  return __half22float2(*reinterpret_cast<__half2*>(&hr));
}

// Add the pair a0 r0 + a1 r1 (first product rounded, second fused) to the accumulator.
__device__ __forceinline__ void df_pair(DF& acc, float a0, float r0, float a1, float r1) {
  float p = __fmul_rn(a0, r0);
  p = __fmaf_rn(a1, r1, p);
  acc.add(p);
}

__device__ __forceinline__ DF df_warp_reduce(DF acc) {
#pragma unroll
  for (int m = 16; m; m >>= 1) acc.merge(df_shfl_xor(acc, m));
  return acc;
}

// Warp dot product of atom row j of level L with the staged vector rho (shared memory).
// rho_f: FP32 staging (float levels); rho_d: FP64 staging (FP64-arithmetic levels).
// Returns the same value in every lane.
__device__ __forceinline__ double warp_atom_dot(const LevelDev& L, int64_t j, int ldN, const float* __restrict__ rho_f,
                                                const double* __restrict__ rho_d, int lane) {
  switch (L.kind) {
    case LK_F32: {
      const float4* row = reinterpret_cast<const float4*>((const float*)L.data + j * L.ld);
      const float4* rs = reinterpret_cast<const float4*>(rho_f);
      DF acc;
      acc.init();
      const int nv = ldN >> 2;
#pragma unroll 4
      for (int k = lane; k < nv; k += 32) {
        float4 a = __ldg(row + k);
        float4 r = rs[k];
        dot2_add(acc, a.x, r.x);
        dot2_add(acc, a.y, r.y);
        dot2_add(acc, a.z, r.z);
        dot2_add(acc, a.w, r.w);
      }
      return df_warp_reduce(acc).value();
    }
    case LK_BF16: {
      const uint4* row = reinterpret_cast<const uint4*>((const __nv_bfloat16*)L.data + j * L.ld);
      const float4* rs = reinterpret_cast<const float4*>(rho_f);
      DF acc;
      acc.init();
      const int nv = ldN >> 3;
#pragma unroll 2
      for (int k = lane; k < nv; k += 32) {
        uint4 a = __ldg(row + k);
        float4 r0 = rs[2 * k], r1 = rs[2 * k + 1];
        float2 a0 = bf16x2_to_f2(a.x), a1 = bf16x2_to_f2(a.y), a2 = bf16x2_to_f2(a.z), a3 = bf16x2_to_f2(a.w);
        df_pair(acc, a0.x, r0.x, a0.y, r0.y);
        df_pair(acc, a1.x, r0.z, a1.y, r0.w);
        df_pair(acc, a2.x, r1.x, a2.y, r1.y);
        df_pair(acc, a3.x, r1.z, a3.y, r1.w);
      }
      return df_warp_reduce(acc).value();
    }
    case LK_FP8: {
      const uint4* row = reinterpret_cast<const uint4*>((const uint8_t*)L.data + j * L.ld);
      const float4* rs = reinterpret_cast<const float4*>(rho_f);
      DF acc;
      acc.init();
      const int nv = ldN >> 4;
      for (int k = lane; k < nv; k += 32) {
        uint4 a = __ldg(row + k);
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 r = rs[4 * k + q];
          float2 lo = fp8x2_to_f2((uint16_t)(w[q] & 0xffffu));
          float2 hi = fp8x2_to_f2((uint16_t)(w[q] >> 16));
          df_pair(acc, lo.x, r.x, lo.y, r.y);
          df_pair(acc, hi.x, r.z, hi.y, r.w);
        }
      }
      return df_warp_reduce(acc).value() * (double)L.scale[j];
    }
    case LK_F64: {
      const double2* row = reinterpret_cast<const double2*>((const double*)L.data + j * L.ld);
      const double2* rs = reinterpret_cast<const double2*>(rho_d);
      double s = 0.0;
      const int nv = ldN >> 1;
      for (int k = lane; k < nv; k += 32) {
        double2 a = __ldg(row + k);
        double2 r = rs[k];
        s = fma(a.x, r.x, s);
        s = fma(a.y, r.y, s);
      }
      return warp_sum(s);
    }
    case LK_F32D: {
      const float4* row = reinterpret_cast<const float4*>((const float*)L.data + j * L.ld);
      const double2* rs = reinterpret_cast<const double2*>(rho_d);
      double s = 0.0;
      const int nv = ldN >> 2;
      for (int k = lane; k < nv; k += 32) {
        float4 a = __ldg(row + k);
        double2 r0 = rs[2 * k], r1 = rs[2 * k + 1];
        s = fma((double)a.x, r0.x, s);
        s = fma((double)a.y, r0.y, s);
        s = fma((double)a.z, r1.x, s);
        s = fma((double)a.w, r1.y, s);
      }
      return warp_sum(s);
    }
  }
  return 0.0;
}

// Dot2 (error-free products, TwoSum accumulation) of atom row j of an FP32 level with rho, all in
// FP32: the double-float result s + c is rounded once to FP32 (within 3 u |g|, which the bound
// of the caller covers); the same value in every lane.
__device__ __forceinline__ float warp_atom_dot_tight_f(const LevelDev& L, int64_t j, int ldN,
                                                      const float* __restrict__ rho_f, int lane) {
  const float4* row = reinterpret_cast<const float4*>((const float*)L.data + j * L.ld);
  const float4* rs = reinterpret_cast<const float4*>(rho_f);
  DF acc;
  acc.init();
  const int nv = ldN >> 2;
#pragma unroll 4
  for (int k = lane; k < nv; k += 32) {
    const float4 a = __ldg(row + k);
    const float4 r = __ldg(rs + k);
    dot2_add(acc, a.x, r.x);
    dot2_add(acc, a.y, r.y);
    dot2_add(acc, a.z, r.z);
    dot2_add(acc, a.w, r.w);
  }
  acc = df_warp_reduce(acc);
  return __fadd_rn(acc.s, acc.c);
}

// Fast warp dot product for the bulk of a pass: plain FMA chains (two independent FP32 or FP64
// accumulators per lane), rho read through L1 straight from global memory.  The rounding error
// is bounded by gamma_{ld/32 + 8} sum_i |a_i rho_i| (the LevelDev's gam_corr), which the stable
// test absorbs; the certificate of the exact FP32 level is tightened separately (Dot2).
template <typename VT>
__device__ __forceinline__ float4 rho4_f(const VT* __restrict__ rho, int q) {
  if constexpr (sizeof(VT) == 4) {
    return __ldg(reinterpret_cast<const float4*>(rho) + q);
  } else {
    const double2* p = reinterpret_cast<const double2*>(rho) + 2 * q;
    double2 a = __ldg(p), b = __ldg(p + 1);
    return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

template <typename VT>
__device__ __forceinline__ double warp_atom_dot_fast(const LevelDev& L, int64_t j, int ldN, const VT* __restrict__ rho,
                                                     int lane) {
  switch (L.kind) {
    case LK_F32: {
      const float4* row = reinterpret_cast<const float4*>((const float*)L.data + j * L.ld);
      float s0 = 0.f, s1 = 0.f;
      const int nv = ldN >> 2;
      int k = lane;
      for (; k + 32 < nv; k += 64) {
        const float4 a = __ldg(row + k), b = __ldg(row + k + 32);
        const float4 r = rho4_f(rho, k), t = rho4_f(rho, k + 32);
        s0 = __fmaf_rn(a.x, r.x, s0); s0 = __fmaf_rn(a.y, r.y, s0); s0 = __fmaf_rn(a.z, r.z, s0); s0 = __fmaf_rn(a.w, r.w, s0);
        s1 = __fmaf_rn(b.x, t.x, s1); s1 = __fmaf_rn(b.y, t.y, s1); s1 = __fmaf_rn(b.z, t.z, s1); s1 = __fmaf_rn(b.w, t.w, s1);
      }
      if (k < nv) {
        const float4 a = __ldg(row + k);
        const float4 r = rho4_f(rho, k);
        s0 = __fmaf_rn(a.x, r.x, s0); s0 = __fmaf_rn(a.y, r.y, s0); s0 = __fmaf_rn(a.z, r.z, s0); s0 = __fmaf_rn(a.w, r.w, s0);
      }
      return warp_sum_f(__fadd_rn(s0, s1));
    }
    case LK_BF16: {
      const uint4* row = reinterpret_cast<const uint4*>((const __nv_bfloat16*)L.data + j * L.ld);
      float s0 = 0.f, s1 = 0.f;
      const int nv = ldN >> 3;
#pragma unroll 2
      for (int k = lane; k < nv; k += 32) {
        const uint4 a = __ldg(row + k);
        const float4 r0 = rho4_f(rho, 2 * k), r1 = rho4_f(rho, 2 * k + 1);
        const float2 a0 = bf16x2_to_f2(a.x), a1 = bf16x2_to_f2(a.y), a2 = bf16x2_to_f2(a.z), a3 = bf16x2_to_f2(a.w);
        s0 = __fmaf_rn(a0.x, r0.x, s0); s1 = __fmaf_rn(a0.y, r0.y, s1);
        s0 = __fmaf_rn(a1.x, r0.z, s0); s1 = __fmaf_rn(a1.y, r0.w, s1);
        s0 = __fmaf_rn(a2.x, r1.x, s0); s1 = __fmaf_rn(a2.y, r1.y, s1);
        s0 = __fmaf_rn(a3.x, r1.z, s0); s1 = __fmaf_rn(a3.y, r1.w, s1);
      }
      return warp_sum_f(__fadd_rn(s0, s1));
    }
    case LK_FP8: {
      const uint4* row = reinterpret_cast<const uint4*>((const uint8_t*)L.data + j * L.ld);
      float s0 = 0.f, s1 = 0.f;
      const int nv = ldN >> 4;
      for (int k = lane; k < nv; k += 32) {
        const uint4 a = __ldg(row + k);
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 r = rho4_f(rho, 4 * k + q);
          const float2 lo = fp8x2_to_f2((uint16_t)(w[q] & 0xffffu));
          const float2 hi = fp8x2_to_f2((uint16_t)(w[q] >> 16));
          s0 = __fmaf_rn(lo.x, r.x, s0); s1 = __fmaf_rn(lo.y, r.y, s1);
          s0 = __fmaf_rn(hi.x, r.z, s0); s1 = __fmaf_rn(hi.y, r.w, s1);
        }
      }
      return __fmul_rn(warp_sum_f(__fadd_rn(s0, s1)), L.scale[j]);
    }
    case LK_F64: {
      const double2* row = reinterpret_cast<const double2*>((const double*)L.data + j * L.ld);
      const double2* rs = reinterpret_cast<const double2*>(rho);
      double s = 0.0;
      const int nv = ldN >> 1;
      for (int k = lane; k < nv; k += 32) {
        const double2 a = __ldg(row + k);
        const double2 r = __ldg(rs + k);
        s = fma(a.x, r.x, s);
        s = fma(a.y, r.y, s);
      }
      return warp_sum(s);
    }
    case LK_F32D: {
      const float4* row = reinterpret_cast<const float4*>((const float*)L.data + j * L.ld);
      const double2* rs = reinterpret_cast<const double2*>(rho);
      double s = 0.0;
      const int nv = ldN >> 2;
      for (int k = lane; k < nv; k += 32) {
        const float4 a = __ldg(row + k);
        const double2 r0 = __ldg(rs + 2 * k), r1 = __ldg(rs + 2 * k + 1);
        s = fma((double)a.x, r0.x, s);
        s = fma((double)a.y, r0.y, s);
        s = fma((double)a.z, r1.x, s);
        s = fma((double)a.w, r1.y, s);
      }
      return warp_sum(s);
    }
  }
  return 0.0;
}

// Two atoms at once with four 16-byte loads of each row in flight per lane (float levels only):
// the correlation pass is bound by the bytes in flight from L2, not by arithmetic.  Same
// rounding model as warp_atom_dot_fast (FP32 FMA chains, two accumulators per atom).
template <typename VT>
__device__ __forceinline__ void warp_atom_dot2_fast(const LevelDev& L, int64_t j0, int64_t j1, int ldN,
                                                    const VT* __restrict__ rho, int lane, float& g0, float& g1) {
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
  if (L.kind == LK_F32) {
    const float4* r0 = reinterpret_cast<const float4*>((const float*)L.data + j0 * L.ld);
    const float4* r1 = reinterpret_cast<const float4*>((const float*)L.data + j1 * L.ld);
    const int nv = ldN >> 2;
    int k = lane;
    for (; k + 32 < nv; k += 64) {
      const float4 x0 = __ldg(r0 + k), x1 = __ldg(r0 + k + 32), y0 = __ldg(r1 + k), y1 = __ldg(r1 + k + 32);
      const float4 p = rho4_f(rho, k), q = rho4_f(rho, k + 32);
      a0 = __fmaf_rn(x0.x, p.x, a0); a0 = __fmaf_rn(x0.y, p.y, a0); a0 = __fmaf_rn(x0.z, p.z, a0); a0 = __fmaf_rn(x0.w, p.w, a0);
      a1 = __fmaf_rn(x1.x, q.x, a1); a1 = __fmaf_rn(x1.y, q.y, a1); a1 = __fmaf_rn(x1.z, q.z, a1); a1 = __fmaf_rn(x1.w, q.w, a1);
      b0 = __fmaf_rn(y0.x, p.x, b0); b0 = __fmaf_rn(y0.y, p.y, b0); b0 = __fmaf_rn(y0.z, p.z, b0); b0 = __fmaf_rn(y0.w, p.w, b0);
      b1 = __fmaf_rn(y1.x, q.x, b1); b1 = __fmaf_rn(y1.y, q.y, b1); b1 = __fmaf_rn(y1.z, q.z, b1); b1 = __fmaf_rn(y1.w, q.w, b1);
    }
    if (k < nv) {
      const float4 x0 = __ldg(r0 + k), y0 = __ldg(r1 + k);
      const float4 p = rho4_f(rho, k);
      a0 = __fmaf_rn(x0.x, p.x, a0); a0 = __fmaf_rn(x0.y, p.y, a0); a0 = __fmaf_rn(x0.z, p.z, a0); a0 = __fmaf_rn(x0.w, p.w, a0);
      b0 = __fmaf_rn(y0.x, p.x, b0); b0 = __fmaf_rn(y0.y, p.y, b0); b0 = __fmaf_rn(y0.z, p.z, b0); b0 = __fmaf_rn(y0.w, p.w, b0);
    }
  } else if (L.kind == LK_BF16) {
    const uint4* r0 = reinterpret_cast<const uint4*>((const __nv_bfloat16*)L.data + j0 * L.ld);
    const uint4* r1 = reinterpret_cast<const uint4*>((const __nv_bfloat16*)L.data + j1 * L.ld);
    const int nv = ldN >> 3;
    int k = lane;
    auto acc = [&](float& s0, float& s1, const uint4 a, const float4 p, const float4 q) {
      const float2 e0 = bf16x2_to_f2(a.x), e1 = bf16x2_to_f2(a.y), e2 = bf16x2_to_f2(a.z), e3 = bf16x2_to_f2(a.w);
      s0 = __fmaf_rn(e0.x, p.x, s0); s1 = __fmaf_rn(e0.y, p.y, s1);
      s0 = __fmaf_rn(e1.x, p.z, s0); s1 = __fmaf_rn(e1.y, p.w, s1);
      s0 = __fmaf_rn(e2.x, q.x, s0); s1 = __fmaf_rn(e2.y, q.y, s1);
      s0 = __fmaf_rn(e3.x, q.z, s0); s1 = __fmaf_rn(e3.y, q.w, s1);
    };
    for (; k + 32 < nv; k += 64) {
      const uint4 x0 = __ldg(r0 + k), x1 = __ldg(r0 + k + 32), y0 = __ldg(r1 + k), y1 = __ldg(r1 + k + 32);
      const float4 p0 = rho4_f(rho, 2 * k), q0 = rho4_f(rho, 2 * k + 1);
      const float4 p1 = rho4_f(rho, 2 * (k + 32)), q1 = rho4_f(rho, 2 * (k + 32) + 1);
      acc(a0, a1, x0, p0, q0);
      acc(a0, a1, x1, p1, q1);
      acc(b0, b1, y0, p0, q0);
      acc(b0, b1, y1, p1, q1);
    }
    if (k < nv) {
      const uint4 x0 = __ldg(r0 + k), y0 = __ldg(r1 + k);
      const float4 p0 = rho4_f(rho, 2 * k), q0 = rho4_f(rho, 2 * k + 1);
      acc(a0, a1, x0, p0, q0);
      acc(b0, b1, y0, p0, q0);
    }
  } else {   // LK_FP8
    const uint4* r0 = reinterpret_cast<const uint4*>((const uint8_t*)L.data + j0 * L.ld);
    const uint4* r1 = reinterpret_cast<const uint4*>((const uint8_t*)L.data + j1 * L.ld);
    const int nv = ldN >> 4;
    auto acc = [&](float& s0, float& s1, const uint4 a, int k) {
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 r = rho4_f(rho, 4 * k + q);
        const float2 lo = fp8x2_to_f2((uint16_t)(w[q] & 0xffffu));
        const float2 hi = fp8x2_to_f2((uint16_t)(w[q] >> 16));
        s0 = __fmaf_rn(lo.x, r.x, s0); s1 = __fmaf_rn(lo.y, r.y, s1);
        s0 = __fmaf_rn(hi.x, r.z, s0); s1 = __fmaf_rn(hi.y, r.w, s1);
      }
    };
    int k = lane;
    for (; k + 32 < nv; k += 64) {
      const uint4 x0 = __ldg(r0 + k), x1 = __ldg(r0 + k + 32), y0 = __ldg(r1 + k), y1 = __ldg(r1 + k + 32);
      acc(a0, a1, x0, k);
      acc(a0, a1, x1, k + 32);
      acc(b0, b1, y0, k);
      acc(b0, b1, y1, k + 32);
    }
    if (k < nv) {
      const uint4 x0 = __ldg(r0 + k), y0 = __ldg(r1 + k);
      acc(a0, a1, x0, k);
      acc(b0, b1, y0, k);
    }
  }
  float u = __fadd_rn(a0, a1), v = __fadd_rn(b0, b1);
#pragma unroll
  for (int m = 16; m; m >>= 1) {
    u = __fadd_rn(u, __shfl_xor_sync(0xffffffffu, u, m));
    v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  }
  if (L.kind == LK_FP8) {
    u = __fmul_rn(u, L.scale[j0]);
    v = __fmul_rn(v, L.scale[j1]);
  }
  g0 = u;
  g1 = v;
}

// Four consecutive rows [r0, r0 + 4) of atom j (r0 a multiple of 4), as FP32 / FP64.
__device__ __forceinline__ float4 load4_f(const LevelDev& L, int64_t j, int r0) {
  switch (L.kind) {
    case LK_F32:
      return __ldg(reinterpret_cast<const float4*>((const float*)L.data + j * L.ld + r0));
    case LK_BF16: {
      uint2 v = __ldg(reinterpret_cast<const uint2*>((const __nv_bfloat16*)L.data + j * L.ld + r0));
      float2 a = bf16x2_to_f2(v.x), b = bf16x2_to_f2(v.y);
      return make_float4(a.x, a.y, b.x, b.y);
    }
    case LK_FP8: {
      uint32_t v = __ldg(reinterpret_cast<const unsigned int*>((const uint8_t*)L.data + j * L.ld + r0));
      float2 a = fp8x2_to_f2((uint16_t)(v & 0xffffu)), b = fp8x2_to_f2((uint16_t)(v >> 16));
      return make_float4(a.x, a.y, b.x, b.y);
    }
  }
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// The same for a storage kind known at compile time (lets a loop keep several loads in flight).
template <int KIND>
__device__ __forceinline__ float4 load4_t(const LevelDev& L, int64_t j, int r0) {
  if constexpr (KIND == LK_F32) {
    return __ldg(reinterpret_cast<const float4*>((const float*)L.data + j * L.ld + r0));
  } else if constexpr (KIND == LK_BF16) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>((const __nv_bfloat16*)L.data + j * L.ld + r0));
    float2 a = bf16x2_to_f2(v.x), b = bf16x2_to_f2(v.y);
    return make_float4(a.x, a.y, b.x, b.y);
  } else {
    uint32_t v = __ldg(reinterpret_cast<const unsigned int*>((const uint8_t*)L.data + j * L.ld + r0));
    float2 a = fp8x2_to_f2((uint16_t)(v & 0xffffu)), b = fp8x2_to_f2((uint16_t)(v >> 16));
    return make_float4(a.x, a.y, b.x, b.y);
  }
}

// Residual accumulation acc[v] += sum_q w_q a~_{j_q}[r0 + v] over cnt staged nonzeros, eight
// atom segments in flight per thread: error-free products (Dot2) when d2, plain FMA chains
// otherwise (acc[v].s only).
template <int KIND>
__device__ __forceinline__ void res_accumulate(const LevelDev& L, const int32_t* s_idx, const float* s_wf, int cnt,
                                               int r0, bool d2, DF* acc) {
  int q = 0;
  for (; q + 8 <= cnt; q += 8) {
    float4 av[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) av[u] = load4_t<KIND>(L, s_idx[q + u], r0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float w = s_wf[q + u];
      if (d2) {
        dot2_add(acc[0], w, av[u].x);
        dot2_add(acc[1], w, av[u].y);
        dot2_add(acc[2], w, av[u].z);
        dot2_add(acc[3], w, av[u].w);
      } else {
        acc[0].s = __fmaf_rn(w, av[u].x, acc[0].s);
        acc[1].s = __fmaf_rn(w, av[u].y, acc[1].s);
        acc[2].s = __fmaf_rn(w, av[u].z, acc[2].s);
        acc[3].s = __fmaf_rn(w, av[u].w, acc[3].s);
      }
    }
  }
  for (; q < cnt; ++q) {
    const float4 av = load4_t<KIND>(L, s_idx[q], r0);
    const float w = s_wf[q];
    if (d2) {
      dot2_add(acc[0], w, av.x);
      dot2_add(acc[1], w, av.y);
      dot2_add(acc[2], w, av.z);
      dot2_add(acc[3], w, av.w);
    } else {
      acc[0].s = __fmaf_rn(w, av.x, acc[0].s);
      acc[1].s = __fmaf_rn(w, av.y, acc[1].s);
      acc[2].s = __fmaf_rn(w, av.z, acc[2].s);
      acc[3].s = __fmaf_rn(w, av.w, acc[3].s);
    }
  }
}

struct D4 {
  double x, y, z, w;
};

__device__ __forceinline__ D4 load4_d(const LevelDev& L, int64_t j, int r0) {
  if (L.kind == LK_F64) {
    const double2* p = reinterpret_cast<const double2*>((const double*)L.data + j * L.ld + r0);
    double2 a = __ldg(p), b = __ldg(p + 1);
    return D4{a.x, a.y, b.x, b.y};
  }
  float4 f = __ldg(reinterpret_cast<const float4*>((const float*)L.data + j * L.ld + r0));
  return D4{f.x, f.y, f.z, f.w};
}

}  // namespace lasso
