// Dictionary preparation (a one-time step per dictionary): packing, atom norms, BF16 / FP8
// copies, Kronecker scales and truncations, exact per-atom error bounds eps_j and the step
// size L by power iteration.  All error bounds are evaluated in FP64 on the device.
//
// Paper: approximate dictionaries A = A~ + E with per-atom bounds eps_j >= ||a~_j - a_j||_2
// (eq:approx_dict, Section III-B); ladder {A~^i} with A~^I = A (Section IV); SuKro sums of
// Kronecker products (Section V-A).
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dict.cuh"
#include "tc_gemm.cuh"

namespace lasso {

// ------------------------------------------------------------------------------ kernels

// dst[j * ldN + n] = src(n, j) as FP64 (zero padding up to ldN).
template <typename Tin>
__global__ void k_pack_f64(const Tin* __restrict__ src, int64_t N, int64_t K, int64_t ld, int atom_major,
                           double* __restrict__ dst, int64_t ldN) {
  int64_t total = K * ldN;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = t / ldN, n = t % ldN;
    double v = 0.0;
    if (n < N) v = (double)(atom_major ? src[j * ld + n] : src[n * ld + j]);
    dst[t] = v;
  }
}

// FP64 norm of every atom row (warp per atom).
__global__ void k_row_norms_f64(const double* __restrict__ a, int64_t ldN, int64_t N, int64_t K,
                                double* __restrict__ out) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double s = 0.0;
    for (int64_t n = lane; n < N; n += 32) {
      double v = a[j * ldN + n];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) out[j] = sqrt(s);
  }
}

// Optional normalisation in FP64, then rounding to the exact level's type.
template <typename T>
__global__ void k_store_exact(const double* __restrict__ a64, const double* __restrict__ norms, int normalize,
                              int64_t ldN, int64_t K, T* __restrict__ dst) {
  int64_t total = K * ldN;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    double v = a64[t];
    if (normalize) {
      double nr = norms[t / ldN];
      v = nr > 0.0 ? v / nr : 0.0;
    }
    dst[t] = (T)v;
  }
}

// Exact atom norms of the stored exact level, rounded up (so that R' ||a_j|| never shrinks).
// The fixed relative margins of this file's FP64 norms (1e-13) and error norms (1e-12) are sized
// for the longest signals the solver accepts (ldN <= 24576): a lane's chain then holds at most 768
// squares and the 32-lane tree adds 5 levels, so a sum of squares is off by at most
// gamma_773(2^-53) ~ 8.6e-14 relative and its square root by half that.
template <typename T>
__global__ void k_exact_norms(const T* __restrict__ a, int64_t ldN, int64_t N, int64_t K, double* __restrict__ out,
                              float* __restrict__ atn, double* __restrict__ kappa) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double s = 0.0;
    for (int64_t n = lane; n < N; n += 32) {
      double v = (double)a[j * ldN + n];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      double nr = sqrt(s) * (1.0 + 1e-13);
      out[j] = nr;
      atn[j] = __double2float_ru(nr);
      kappa[j] = nr;
    }
  }
}

__device__ __forceinline__ double load_exact(const void* p, int kind, int64_t idx) {
  return kind == LK_F64 ? ((const double*)p)[idx] : (double)((const float*)p)[idx];
}

// BF16 copy (round to nearest even) of the exact level.
__global__ void k_quant_bf16(const void* __restrict__ ex, int ex_kind, int64_t total, __nv_bfloat16* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    float v = (float)load_exact(ex, ex_kind, t);
    dst[t] = __float2bfloat16_rn(v);
  }
}

// FP32 copy of an FP64 exact level.
__global__ void k_quant_f32(const double* __restrict__ ex, int64_t total, float* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (float)ex[t];
}

// Per-atom scaled E4M3 copy: s_j = fl32(max_i |a_ij| / 448), q_ij = E4M3_satfinite(fl32(a_ij / s_j)).
__global__ void k_quant_fp8(const void* __restrict__ ex, int ex_kind, int64_t ldN, int64_t N, int64_t K,
                            __nv_fp8_storage_t* __restrict__ dst, float* __restrict__ scale) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double m = 0.0;
    for (int64_t n = lane; n < N; n += 32) m = fmax(m, fabs((double)(float)load_exact(ex, ex_kind, j * ldN + n)));
    m = warp_max(m);
    float s = (float)(m / 448.0);
    if (!(s > 0.f)) s = 1.f;
    if (lane == 0) scale[j] = s;
    for (int64_t n = lane; n < ldN; n += 32) {
      float a = n < N ? (float)load_exact(ex, ex_kind, j * ldN + n) : 0.f;
      float v = __fdiv_rn(a, s);
      dst[j * ldN + n] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

__device__ __forceinline__ double load_level(const void* p, int kind, const float* scale, int64_t j, int64_t idx) {
  switch (kind) {
    case LK_F64: return ((const double*)p)[idx];
    case LK_F32:
    case LK_F32D: return (double)((const float*)p)[idx];
    case LK_BF16: return (double)__bfloat162float(((const __nv_bfloat16*)p)[idx]);
    case LK_FP8: {
      __half_raw hr = __nv_cvt_fp8_to_halfraw(((const __nv_fp8_storage_t*)p)[idx], __NV_E4M3);
      return (double)__half2float(__half(hr)) * (double)scale[j];
    }
  }
  return 0.0;
}

// eps_j = ||a~_j - a_j|| and ||a~_j|| in FP64 (warp per atom), eps inflated to stay an upper bound.
__global__ void k_level_eps(const void* __restrict__ ap, int akind, const float* __restrict__ scale,
                            const void* __restrict__ ex, int ex_kind, int64_t ldN, int64_t N, int64_t K,
                            double* __restrict__ eps, float* __restrict__ atn, double* __restrict__ kappa) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double se = 0.0, sa = 0.0;
    for (int64_t n = lane; n < N; n += 32) {
      double a = load_level(ap, akind, scale, j, j * ldN + n);
      double e = a - load_exact(ex, ex_kind, j * ldN + n);
      se = fma(e, e, se);
      sa = fma(a, a, sa);
    }
    se = warp_sum(se);
    sa = warp_sum(sa);
    if (lane == 0) {
      eps[j] = sqrt(se) * (1.0 + 1e-12);
      double an = sqrt(sa) * (1.0 + 1e-13);
      atn[j] = __double2float_ru(an);
      kappa[j] = an;
    }
  }
}

// Gram tensors of Kronecker factors: G[r][s][k] = sum_n M_r[n, k] M_s[n, k] (FP64).
__global__ void k_kron_gram(const float* __restrict__ M, int R, int Nn, int Kk, double* __restrict__ G) {
  int total = R * R * Kk;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int k = t % Kk, rs = t / Kk, s = rs % R, r = rs / R;
    double acc = 0.0;
    for (int n = 0; n < Nn; ++n)
      acc = fma((double)M[((int64_t)r * Nn + n) * Kk + k], (double)M[((int64_t)s * Nn + n) * Kk + k], acc);
    G[t] = acc;
  }
}

// Sum over r, s in [r0, r1) of GB[r][s][k1] GC[r][s][k2].
__device__ __forceinline__ double kron_gram_sum(const double* GB, const double* GC, int R, int K1, int K2, int k1,
                                                int k2, int r0, int r1) {
  double acc = 0.0;
  for (int r = r0; r < r1; ++r)
    for (int s = r0; s < r1; ++s)
      acc = fma(GB[((int64_t)r * R + s) * K1 + k1], GC[((int64_t)r * R + s) * K2 + k2], acc);
  return acc;
}

// d_j = 1 / ||(sum_r B_r (x) C_r) e_j|| (FP64, Gram identity).
// Column scale d_j of A = (sum_r B_r (x) C_r) diag(d): 1 / ||column j|| (unit atoms) when
// normalize != 0, else 1 (the Kronecker sum as given); anorm_j >= ||a_j|| in both cases.
__global__ void k_kron_scale(const double* __restrict__ GB, const double* __restrict__ GC, int R, int K1, int K2,
                             int normalize, double* __restrict__ d, float* __restrict__ df, double* __restrict__ anorm) {
  int K = K1 * K2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
    double sq = kron_gram_sum(GB, GC, R, K1, K2, j / K2, j % K2, 0, R);
    if (normalize) {
      double dj = sq > 0.0 ? 1.0 / sqrt(sq) : 0.0;
      d[j] = dj;
      df[j] = (float)dj;
      anorm[j] = 1.0 + 1e-12;   // unit atoms (FP64 rounding of d_j covered by the slack)
    } else {
      d[j] = 1.0;
      df[j] = 1.0f;
      // the Gram sum of 2 R^2 terms, then a square root: relative error far below 1e-12
      anorm[j] = sqrt(fmax(sq, 0.0)) * (1.0 + 1e-12);
    }
  }
}

// Truncation to the first Rk terms: eps_j (tail terms), ||a~_j|| (head terms) and
// kappa_j = d_j sum_{r<Rk} ||B_r[:, k1]|| ||C_r[:, k2]|| (rounding-bound weight of the small GEMMs).
__global__ void k_kron_level(const double* __restrict__ GB, const double* __restrict__ GC, const double* __restrict__ d,
                             int R, int K1, int K2, int Rk, double* __restrict__ eps, float* __restrict__ atn,
                             double* __restrict__ kappa) {
  int K = K1 * K2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
    int k1 = j / K2, k2 = j % K2;
    // ||sum_{r>=Rk} ...||^2 from the tail block of the Gram tensors
    double t2 = 0.0;
    for (int r = Rk; r < R; ++r)
      for (int s = Rk; s < R; ++s) t2 = fma(GB[((int64_t)r * R + s) * K1 + k1], GC[((int64_t)r * R + s) * K2 + k2], t2);
    double head = kron_gram_sum(GB, GC, R, K1, K2, k1, k2, 0, Rk);
    double kap = 0.0;
    for (int r = 0; r < Rk; ++r)
      kap += sqrt(fmax(GB[((int64_t)r * R + r) * K1 + k1], 0.0)) * sqrt(fmax(GC[((int64_t)r * R + r) * K2 + k2], 0.0));
    eps[j] = d[j] * sqrt(fmax(t2, 0.0)) * (1.0 + 1e-12) + 1e-15;
    atn[j] = __double2float_ru(d[j] * sqrt(fmax(head, 0.0)) * (1.0 + 1e-12));
    kappa[j] = d[j] * kap * (1.0 + 1e-12);
  }
}

// Dense FP32 rounding of the exact Kronecker dictionary and its rounding error eps_j (warp per atom).
__global__ void k_kron_dense_f32(const float* __restrict__ Bf, const float* __restrict__ Cf, const double* __restrict__ d,
                                 int R, int N1, int K1, int N2, int K2, int64_t ldN, float* __restrict__ dst,
                                 double* __restrict__ eps, float* __restrict__ atn, double* __restrict__ kappa) {
  int lane = threadIdx.x & 31;
  int64_t K = (int64_t)K1 * K2, N = (int64_t)N1 * N2;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    int k1 = (int)(j / K2), k2 = (int)(j % K2);
    double se = 0.0, sa = 0.0;
    for (int64_t n = lane; n < ldN; n += 32) {
      float f = 0.f;
      if (n < N) {
        int n1 = (int)(n / N2), n2 = (int)(n % N2);
        double v = 0.0;
        for (int r = 0; r < R; ++r)
          v += (double)Bf[((int64_t)r * N1 + n1) * K1 + k1] * (double)Cf[((int64_t)r * N2 + n2) * K2 + k2];
        v *= d[j];
        f = (float)v;
        double e = (double)f - v;
        se = fma(e, e, se);
        sa = fma((double)f, (double)f, sa);
      }
      dst[j * ldN + n] = f;
    }
    se = warp_sum(se);
    sa = warp_sum(sa);
    if (lane == 0) {
      // FP64 evaluation of the exact entries carries ~R ulps of relative error per entry.
      eps[j] = sqrt(se) * (1.0 + 1e-12) + 4.0 * (R + 2) * U64;
      double an = sqrt(sa) * (1.0 + 1e-13);
      atn[j] = __double2float_ru(an);
      kappa[j] = an;
    }
  }
}

// The FP64 rung of a Kronecker dictionary: the atoms a_j = d_j sum_r B_r[:, k1] (x) C_r[:, k2]
// evaluated in FP64 (one warp per atom).  Each entry is R products summed and scaled by d_j, so
// its error is at most gamma_{R+1}(u64) d_j sum_r |B| |C|; eps_j bounds the norm of those errors,
// kappa_j = ||a~_j|| (the rung's own rounding weight) and atn_j = ||a~_j|| rounded up.
__global__ void k_kron_dense_f64(const float* __restrict__ Bf, const float* __restrict__ Cf, const double* __restrict__ d,
                                 int R, int N1, int K1, int N2, int K2, int64_t ldN, double* __restrict__ dst,
                                 double* __restrict__ eps, float* __restrict__ atn, double* __restrict__ kappa) {
  int lane = threadIdx.x & 31;
  int64_t K = (int64_t)K1 * K2, N = (int64_t)N1 * N2;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    int k1 = (int)(j / K2), k2 = (int)(j % K2);
    double sabs = 0.0, sa = 0.0;
    for (int64_t n = lane; n < ldN; n += 32) {
      double v = 0.0;
      if (n < N) {
        int n1 = (int)(n / N2), n2 = (int)(n % N2);
        double va = 0.0;
        for (int r = 0; r < R; ++r) {
          const double p = (double)Bf[((int64_t)r * N1 + n1) * K1 + k1] * (double)Cf[((int64_t)r * N2 + n2) * K2 + k2];
          v += p;
          va += fabs(p);
        }
        v *= d[j];
        va *= fabs(d[j]);
        sabs = fma(va, va, sabs);
        sa = fma(v, v, sa);
      }
      dst[j * ldN + n] = v;
    }
    sabs = warp_sum(sabs);
    sa = warp_sum(sa);
    if (lane == 0) {
      eps[j] = gamma_n((double)R + 3.0, U64) * sqrt(sabs) * (1.0 + 1e-12);
      const double an = sqrt(sa) * (1.0 + 1e-13);
      atn[j] = __double2float_ru(an);
      kappa[j] = an;
    }
  }
}

// eps_j + gam kappa_j and ||a_j||, rounded up to FP32 (bounds used by FP32 device code).
__global__ void k_round_up_f32(const double* __restrict__ eps, const double* __restrict__ kappa, double gam,
                               int64_t K, float* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = __double2float_ru(kappa ? eps[j] + gam * kappa[j] : eps[j]);
}

static int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 1 << 20);
}

__global__ void k_round_up3_f32(const double* __restrict__ eps, const double* __restrict__ kappa, double gam,
                                const double* __restrict__ extra, int64_t K, float* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = __double2float_ru((eps[j] + gam * kappa[j] + extra[j]) * (1.0 + 4.0 * U64));
}

// BF16 split of the FP32 exact atoms, one warp per atom: a1 = bf16(a), a2 = bf16(a - a1) (both
// differences are exact in FP32), the remainder norm ||a - a1 - a2|| and ||a2|| / kappa_j.
__global__ void k_split_bf16(const float* __restrict__ A, int64_t K, int64_t ld, const double* __restrict__ kappa,
                             __nv_bfloat16* __restrict__ s1, __nv_bfloat16* __restrict__ s2, double* __restrict__ e3,
                             double* __restrict__ ratio2) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (j >= K) return;
  double se = 0.0, s2n = 0.0;
  for (int64_t n = lane; n < ld; n += 32) {
    const float a = A[j * ld + n];
    const __nv_bfloat16 h1 = __float2bfloat16_rn(a);
    const float r1 = __fsub_rn(a, __bfloat162float(h1));
    const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(h2));
    s1[j * ld + n] = h1;
    s2[j * ld + n] = h2;
    se = fma((double)r2, (double)r2, se);
    const double v2 = (double)__bfloat162float(h2);
    s2n = fma(v2, v2, s2n);
  }
  se = warp_sum(se);
  s2n = warp_sum(s2n);
  if (lane == 0) {
    e3[j] = sqrt(se) * (1.0 + 1e-12);
    ratio2[j] = kappa[j] > 0.0 ? sqrt(s2n) * (1.0 + 1e-12) / kappa[j] : 0.0;
  }
}

int ensure_split(lasso_dict* d) {
  HostLevel& h = d->exact;
  if (h.split1) return LASSO_OK;
  if (h.kind != LK_F32 || !h.data || !h.kappa) return LASSO_ERR_INVALID_ARG;
  const size_t elems = (size_t)d->K * d->ldN;
  double* ratio = nullptr;
  if (cudaMalloc(&h.split1, elems * 2) != cudaSuccess || cudaMalloc(&h.split2, elems * 2) != cudaSuccess ||
      cudaMalloc(&h.e3, d->K * sizeof(double)) != cudaSuccess || cudaMalloc(&ratio, d->K * sizeof(double)) != cudaSuccess) {
    cudaFree(h.split1);
    cudaFree(h.split2);
    cudaFree(h.e3);
    cudaFree(ratio);
    h.split1 = h.split2 = nullptr;
    h.e3 = nullptr;
    set_last_error("no device memory for the BF16 split of the dictionary", __FILE__, __LINE__);
    return LASSO_ERR_NOMEM;
  }
  k_split_bf16<<<grid_for(d->K * 32), 256>>>((const float*)h.data, d->K, d->ldN, h.kappa,
                                                (__nv_bfloat16*)h.split1, (__nv_bfloat16*)h.split2, h.e3, ratio);
  LASSO_CUDA_TRY(cudaGetLastError());
  std::vector<double> r(d->K);
  LASSO_CUDA_TRY(cudaMemcpy(r.data(), ratio, d->K * sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(ratio);
  double c2 = 0.0;
  for (double v : r) c2 = std::max(c2, v);
  h.c2 = c2 * (1.0 + 1e-9);
  return LASSO_OK;
}

// ------------------------------------------------------------------ power iteration kernels (FP64)

__device__ __forceinline__ double level_elem(const LevelDev& L, int64_t j, int64_t n) {
  return load_level(L.data, L.kind, L.scale, j, j * L.ld + n);
}

// w = A~^T v (dense level; warp per atom)
__global__ void k_pi_rmatvec_dense(LevelDev L, int64_t N, int64_t K, const double* __restrict__ v, double* __restrict__ w) {
  int lane = threadIdx.x & 31;
  int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = wi; j < K; j += nw) {
    double s = 0.0;
    for (int64_t n = lane; n < N; n += 32) s = fma(level_elem(L, j, n), v[n], s);
    s = warp_sum(s);
    if (lane == 0) w[j] = s;
  }
}

// w = A~ x (dense level; block of rows x slice of atoms, FP64 atomics)
__global__ void k_pi_matvec_dense(LevelDev L, int64_t N, int64_t K, int64_t kslice, const double* __restrict__ x,
                                  double* __restrict__ w) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  int64_t j0 = blockIdx.y * kslice, j1 = min(K, j0 + kslice);
  double s = 0.0;
  for (int64_t j = j0; j < j1; ++j) {
    double xj = x[j];
    if (xj != 0.0) s = fma(level_elem(L, j, n), xj, s);
  }
  atomicAdd(&w[n], s);
}

// Kronecker: T[r][k1][n2] = sum_n1 B_r[n1, k1] P[n1, n2]
__global__ void k_pi_kron_t1(LevelDev L, const double* __restrict__ v, double* __restrict__ T) {
  int64_t total = (int64_t)L.R * L.K1 * L.N2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int n2 = (int)(t % L.N2), k1 = (int)((t / L.N2) % L.K1), r = (int)(t / ((int64_t)L.N2 * L.K1));
    double s = 0.0;
    for (int n1 = 0; n1 < L.N1; ++n1)
      s = fma((double)L.B[((int64_t)r * L.N1 + n1) * L.K1 + k1], v[(int64_t)n1 * L.N2 + n2], s);
    T[t] = s;
  }
}
// g[k1 K2 + k2] = d sum_r sum_n2 T[r][k1][n2] C_r[n2, k2]
__global__ void k_pi_kron_t2(LevelDev L, const double* __restrict__ T, const double* __restrict__ d, double* __restrict__ w) {
  int64_t K = (int64_t)L.K1 * L.K2;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x) {
    int k1 = (int)(j / L.K2), k2 = (int)(j % L.K2);
    double s = 0.0;
    for (int r = 0; r < L.R; ++r)
      for (int n2 = 0; n2 < L.N2; ++n2)
        s = fma(T[((int64_t)r * L.K1 + k1) * L.N2 + n2], (double)L.C[((int64_t)r * L.N2 + n2) * L.K2 + k2], s);
    w[j] = d[j] * s;
  }
}
// U[r][n1][k2] = sum_k1 B_r[n1, k1] (d x)[k1, k2]
__global__ void k_pi_kron_m1(LevelDev L, const double* __restrict__ x, const double* __restrict__ d, double* __restrict__ U) {
  int64_t total = (int64_t)L.R * L.N1 * L.K2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int k2 = (int)(t % L.K2), n1 = (int)((t / L.K2) % L.N1), r = (int)(t / ((int64_t)L.K2 * L.N1));
    double s = 0.0;
    for (int k1 = 0; k1 < L.K1; ++k1) {
      int64_t j = (int64_t)k1 * L.K2 + k2;
      s = fma((double)L.B[((int64_t)r * L.N1 + n1) * L.K1 + k1], d[j] * x[j], s);
    }
    U[t] = s;
  }
}
// w[n1 N2 + n2] = sum_r sum_k2 U[r][n1][k2] C_r[n2, k2]
__global__ void k_pi_kron_m2(LevelDev L, const double* __restrict__ U, double* __restrict__ w) {
  int64_t N = (int64_t)L.N1 * L.N2;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    int n1 = (int)(n / L.N2), n2 = (int)(n % L.N2);
    double s = 0.0;
    for (int r = 0; r < L.R; ++r)
      for (int k2 = 0; k2 < L.K2; ++k2)
        s = fma(U[((int64_t)r * L.N1 + n1) * L.K2 + k2], (double)L.C[((int64_t)r * L.N2 + n2) * L.K2 + k2], s);
    w[n] = s;
  }
}

// Products of sparse factors (FP64).  out = S v, or S^T v through the stored CSR of S^T.
__global__ void k_faust_mv64(FaustFactor F, int transpose, const double* __restrict__ in, double* __restrict__ out) {
  const int rows = transpose ? F.cols : F.rows;
  const int32_t* rp = transpose ? F.rpT : F.rp;
  const int32_t* ci = transpose ? F.ciT : F.ci;
  const float* v = transpose ? F.vT : F.v;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < rows; n += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = rp[n]; p < rp[n + 1]; ++p) s = fma((double)v[p], in[ci[p]], s);
    out[n] = s;
  }
}

// Explicit product, atom-major: T[j, n] = S_{J-1}[n, j] for the last factor (|S| when absval;
// the caller zeroes T; each (n, j) occurs once in a canonical CSR) ...
__global__ void k_faust_last64(FaustFactor F, int absval, int64_t ld, double* __restrict__ T) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < F.rows; n += (int64_t)gridDim.x * blockDim.x)
    for (int p = F.rp[n]; p < F.rp[n + 1]; ++p) {
      const double v = F.v[p];
      T[(int64_t)F.ci[p] * ld + n] = absval ? fabs(v) : v;
    }
}

// ... then Tout[j, n] = sum over row n of S_f of S_f[n, c] Tin[j, c] for f = J-2, ..., 0.
__global__ void k_faust_stage64(FaustFactor F, int absval, int64_t K, int64_t ld, const double* __restrict__ Tin,
                                double* __restrict__ Tout) {
  const int64_t total = K * F.rows;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / F.rows;
    const int n = (int)(t % F.rows);
    const double* row = Tin + j * ld;
    double s = 0.0;
    for (int p = F.rp[n]; p < F.rp[n + 1]; ++p) {
      const double v = F.v[p];
      s = fma(absval ? fabs(v) : v, row[F.ci[p]], s);
    }
    Tout[j * ld + n] = s;
  }
}

// kappa_j = ||(|S_0| ... |S_{J-1}|) e_j|| from the explicit absolute product (warp per atom).
__global__ void k_faust_kappa(const double* __restrict__ P, int64_t ld, int64_t N, int64_t K, double* __restrict__ kappa) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double s = 0.0;
    for (int64_t n = lane; n < N; n += 32) s = fma(P[j * ld + n], P[j * ld + n], s);
    s = warp_sum(s);
    if (lane == 0) kappa[j] = sqrt(s) * (1.0 + 1e-12);
  }
}

// eps_j = ||a~_j - a_j|| from the explicit product, plus gam64 kappa_j for its own FP64
// evaluation (|P^ - P| <= gamma |S_0| ... |S_{J-1}| entrywise); ||a~_j|| rounded up.
__global__ void k_faust_eps(const double* __restrict__ P, int64_t ld, const void* __restrict__ ex, int ex_kind,
                            int64_t ldN, int64_t N, int64_t K, double gam64, const double* __restrict__ kappa,
                            double* __restrict__ eps, float* __restrict__ atn) {
  int lane = threadIdx.x & 31;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < K; j += nw) {
    double se = 0.0, sa = 0.0;
    for (int64_t n = lane; n < N; n += 32) {
      const double a = P[j * ld + n];
      const double e = a - load_exact(ex, ex_kind, j * ldN + n);
      se = fma(e, e, se);
      sa = fma(a, a, sa);
    }
    se = warp_sum(se);
    sa = warp_sum(sa);
    if (lane == 0) {
      eps[j] = sqrt(se) * (1.0 + 1e-12) + gam64 * kappa[j];
      atn[j] = __double2float_ru((sqrt(sa) + gam64 * kappa[j]) * (1.0 + 1e-12));
    }
  }
}

__global__ void k_norm_scale(double* __restrict__ v, int64_t n, double* __restrict__ out_norm) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], v[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = sqrt(t);
  }
  __syncthreads();
  double nr = sh[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = nr > 0.0 ? v[i] / nr : 0.0;
  if (threadIdx.x == 0) *out_norm = nr;
}

__global__ void k_fill(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// ------------------------------------------------------------------------------ host side


static int alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return LASSO_ERR_NOMEM;
  }
  return LASSO_OK;
}

static double host_mean_max(const double* dptr, int64_t K, double* mx) {
  std::vector<double> h(K);
  cudaMemcpy(h.data(), dptr, K * sizeof(double), cudaMemcpyDeviceToHost);
  double s = 0.0, m = 0.0;
  for (double v : h) {
    s += v;
    m = std::max(m, v);
  }
  *mx = m;
  return K ? s / K : 0.0;
}

// Rounding constants of a level for a solve iterating in FP32 (vt_double = false) or FP64.
// Dense float levels: BF16 / FP8 fold 2 products into a double-float accumulator; the exact
// FP32 level uses error-free products (TwoProduct + TwoSum), so its error is second order.
static void level_rounding(const lasso_dict* d, const HostLevel& h, bool vt_double, bool tc, LevelDev& L) {
  const double N = (double)d->ldN;
  const double stage = vt_double ? U32 : 0.0;   // rho rounded to FP32 for float arithmetic
  const double nl = std::ceil(N / 32.0) + 8.0;   // per-lane chain + cross-lane levels
  if (tc && (h.kind == LK_BF16 || h.kind == LK_FP8)) {
    // tensor-core accumulation of N products (k-steps of 16 BF16 / 32 E4M3), then the atom and
    // signal scales and the FP32 store
    const bool f8 = h.kind == LK_FP8;
    L.gam_corr = gamma_n(N + N / (f8 ? 32.0 : 16.0) + 3.0, f8 ? TC_U_FP8 : TC_U_BF16) + stage;
    L.gam_tight = L.gam_corr;
    L.res_model = RES_FOLD;
    L.gam_res = gamma_n(f8 ? 7.0 : 6.0, U32);
    return;
  }
  if (tc && h.kind == LK_F32) {
    // split form on the tensor cores: the three BF16 products a1 r1, a1 r2, a2 r1 with promoted
    // accumulation (each k-block a tensor-core chain, the k-block sums added in FP32), then the
    // FP32 store; the sum of |a1 r1| + |a1 r2| + |a2 r1| is <= (1 + 2^-7)^2 kappa_j ||rho||.  The
    // certificate atoms are recomputed from the FP32 data with error-free products (gam_tight),
    // the residual as for the FP32 level.
    L.gam_corr = 1.02 * tc_promoted_gamma(d->ldN, 3) + 2.0 * U32 + stage;
    L.gam_tight = 2.0 * gamma_n(2.0 * nl, U32) * gamma_n(2.0 * nl, U32) + stage;
    L.res_model = RES_DOT2;
    L.gam_res = vt_double ? U32 : 0.0;
    return;
  }
  switch (h.kind) {
    case LK_F64:
    case LK_F32D:
      L.gam_corr = gamma_n(nl, U64);
      L.gam_tight = L.gam_corr;
      L.res_model = RES_CHAIN;
      L.gam_res = 0.0;
      break;
    case LK_F32:
      // bulk passes: plain FMA chains of nl terms; certificate: Dot2, whose error is
      // <= 2 gamma_{2n}^2 sum |a_i rho_i| for a chain of n terms
      L.gam_corr = gamma_n(nl + 2.0, U32) + stage;
      L.gam_tight = 2.0 * gamma_n(2.0 * nl, U32) * gamma_n(2.0 * nl, U32) + stage;
      L.res_model = RES_DOT2;
      L.gam_res = vt_double ? U32 : 0.0;          // z rounded to FP32 in the products
      break;
    case LK_BF16:
      L.gam_corr = gamma_n(nl + 2.0, U32) + stage;
      L.res_model = RES_FOLD;
      L.gam_res = gamma_n(6.0, U32);
      break;
    case LK_FP8:
      L.gam_corr = gamma_n(nl + 3.0, U32) + stage;
      L.res_model = RES_FOLD;
      L.gam_res = gamma_n(7.0, U32);
      break;
    case LK_KRON:
      L.gam_corr = gamma_n((double)d->N1 + (double)h.param * d->N2 + 3.0, U32) + stage;
      L.res_model = RES_FOLD;
      L.gam_res = gamma_n((double)d->K1 + (double)h.param * d->K2 + 5.0, U32);
      break;
    case LK_FAUST:
      // FP32 FMA chains along the CSR rows, one factor after the other: the stages' relative
      // errors compose to gamma of the summed longest rows, weighted entrywise by
      // |S_0| ... |S_{J-1}|, whose column norms are kappa_j
      L.gam_corr = gamma_n((double)h.n_adj + 3.0, U32) + stage;
      L.gam_tight = L.gam_corr;
      L.res_model = RES_FOLD;
      L.gam_res = gamma_n((double)h.n_fwd + 5.0, U32);
      break;
  }
}

static int finish_level(lasso_dict* d, HostLevel& h) {
  LASSO_CUDA_TRY(cudaGetLastError());
  LASSO_CUDA_TRY(cudaDeviceSynchronize());
  h.eps_mean = host_mean_max(h.eps, d->K, &h.eps_max);
  return LASSO_OK;
}

static int alloc_level_vectors(lasso_dict* d, HostLevel& h) {
  int rc;
  if ((rc = alloc((void**)&h.eps, d->K * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&h.kappa, d->K * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&h.atnorm, d->K * sizeof(float)))) return rc;
  return LASSO_OK;
}

static void free_level(HostLevel& h) {
  if (h.owns_data && h.data) cudaFree(h.data);
  cudaFree(h.scale);
  cudaFree(h.eps);
  cudaFree(h.kappa);
  cudaFree(h.atnorm);
  for (auto* e : h.epsr32) cudaFree(e);
  if (h.owns_data || h.kind == LK_KRON || h.kind == LK_FAUST) {
    cudaFree(h.kappa32);
    cudaFree(h.eps32);
  }
  if (h.kind == LK_FAUST) {
    cudaFree(h.fbuf);
    cudaFree(h.fac);
  }
  cudaFree(h.split1);
  cudaFree(h.split2);
  cudaFree(h.e3);
  cudaFree(h.epsr32_split);
  h = HostLevel();
}

// FP32 copies of the per-atom bounds for the iterate precision of a solve (computed once).
static int ensure_level_f32(const lasso_dict* d, const HostLevel& hc, bool vt_double, bool tc, const LevelDev& L) {
  HostLevel& h = const_cast<HostLevel&>(hc);
  if (!h.kappa32) {
    LASSO_CUDA_TRY(cudaMalloc(&h.kappa32, d->K * sizeof(float)));
    k_round_up_f32<<<grid_for(d->K), 256>>>(h.kappa, nullptr, 0.0, d->K, h.kappa32);
    LASSO_CUDA_TRY(cudaGetLastError());
    LASSO_CUDA_TRY(cudaDeviceSynchronize());
  }
  if (!h.eps32) {
    LASSO_CUDA_TRY(cudaMalloc(&h.eps32, d->K * sizeof(float)));
    k_round_up_f32<<<grid_for(d->K), 256>>>(h.eps, nullptr, 0.0, d->K, h.eps32);
    LASSO_CUDA_TRY(cudaGetLastError());
    LASSO_CUDA_TRY(cudaDeviceSynchronize());
  }
  if (tc && h.kind == LK_F32) {
    // split tensor-core exact level: eps_j + gam_corr kappa_j + ||a_j - a1_j - a2_j||
    if (!h.split1 || !h.e3) return LASSO_ERR_INVALID_ARG;
    if (!h.epsr32_split) {
      LASSO_CUDA_TRY(cudaMalloc(&h.epsr32_split, d->K * sizeof(float)));
      k_round_up3_f32<<<grid_for(d->K), 256>>>(h.eps, h.kappa, L.gam_corr, h.e3, d->K, h.epsr32_split);
      LASSO_CUDA_TRY(cudaGetLastError());
      LASSO_CUDA_TRY(cudaDeviceSynchronize());
    }
    return LASSO_OK;
  }
  float*& dst = h.epsr32[(vt_double ? 1 : 0) + (tc ? 2 : 0)];
  if (dst) return LASSO_OK;
  if (getenv("LASSO_TRACE_STEPS")) fprintf(stderr, "[lasso trace] level bounds: kind %d\n", h.kind);
  LASSO_CUDA_TRY(cudaMalloc(&dst, d->K * sizeof(float)));
  k_round_up_f32<<<grid_for(d->K), 256>>>(h.eps, h.kappa, L.gam_corr, d->K, dst);
  LASSO_CUDA_TRY(cudaGetLastError());
  // one-time set-up on the legacy stream: finish it before any solve stream reads the bounds
  LASSO_CUDA_TRY(cudaDeviceSynchronize());
  return LASSO_OK;
}

LevelDev make_level_dev(const lasso_dict* d, const HostLevel& h, bool vt_double, bool tc) {
  LevelDev L;
  memset(&L, 0, sizeof(L));
  L.kind = h.kind;
  L.ld = d->ldN;
  L.data = h.data;
  L.scale = h.scale;
  L.eps = h.eps;
  L.kappa = h.kappa;
  L.atnorm = h.atnorm;
  L.rc = h.rc;
  const bool split = tc && h.kind == LK_F32 && !vt_double && h.split1 != nullptr;
  tc = (tc && (h.kind == LK_BF16 || h.kind == LK_FP8)) || split;
  L.tc = tc ? 1 : 0;
  L.split = split ? 1 : 0;
  L.c2 = split ? h.c2 : 0.0;
  if (split) {
    // the plain FP32 bounds serve the fast checks outside the bulk pass (full-dictionary check)
    LevelDev Ls = L;
    Ls.tc = 0;
    Ls.split = 0;
    level_rounding(d, h, vt_double, false, Ls);
    if (h.eps && ensure_level_f32(d, h, vt_double, false, Ls) == LASSO_OK)
      L.epsr32_simt = h.epsr32[vt_double ? 1 : 0];
  }
  level_rounding(d, h, vt_double, tc, L);
  if (h.eps && ensure_level_f32(d, h, vt_double, tc, L) == LASSO_OK) {
    L.epsr32 = split ? h.epsr32_split : h.epsr32[(vt_double ? 1 : 0) + (tc ? 2 : 0)];
    L.kappa32 = h.kappa32;
    L.eps32 = h.eps32;
    if (!split) L.epsr32_simt = L.epsr32;
    if (split && !L.epsr32_simt) L.epsr32 = nullptr;
  } else if (h.eps) {
    L.epsr32 = nullptr;   // build_dict_dev rejects a level without its FP32 bounds
  }
  if (h.kind == LK_KRON) {
    L.B = d->Bf;
    L.C = d->Cf;
    L.dscale = h.dscale;
    L.R = h.param;
    L.N1 = d->N1;
    L.K1 = d->K1;
    L.N2 = d->N2;
    L.K2 = d->K2;
  }
  if (h.kind == LK_FAUST) {
    L.fac = h.fac;
    L.J = h.J;
    L.fdim = h.fdim;
  }
  return L;
}

int ensure_rung64(lasso_dict* d) {
  if (d->rung64.kind >= 0) return LASSO_OK;
  if (d->exact_kind != LK_F32) return LASSO_OK;
  HostLevel& h = d->rung64;
  if (d->is_kron) {
    // the exact A is the FP64 Kronecker sum, whose FP32 rounding (the exact level's data) carries
    // eps_j of a few 1e-8: enough to floor certificates near 1e-6 at small lambda.  The rung
    // holds its own FP64 evaluation, with eps_j of FP64 rounding only.
    HostLevel r;
    r.kind = LK_F64;
    r.api_kind = -1;
    r.u = U64;
    r.rc = 1.0;
    int rc;
    if ((rc = alloc(&r.data, (size_t)d->K * d->ldN * sizeof(double)))) return rc;
    if ((rc = alloc_level_vectors(d, r))) {
      free_level(r);
      return rc;
    }
    k_kron_dense_f64<<<grid_for(d->K * 32), 256>>>(d->Bf, d->Cf, d->d, d->R, d->N1, d->K1, d->N2, d->K2, d->ldN,
                                                   (double*)r.data, r.eps, r.atnorm, r.kappa);
    if ((rc = finish_level(d, r))) {
      free_level(r);
      return rc;
    }
    h = r;
    return LASSO_OK;
  }
  h = d->exact;               // shares the FP32 data and vectors of the exact level
  h.owns_data = false;
  h.kind = LK_F32D;
  for (auto& e : h.epsr32) e = nullptr;
  h.kappa32 = nullptr;
  h.eps32 = nullptr;
  h.split1 = h.split2 = nullptr;
  h.e3 = nullptr;
  h.epsr32_split = nullptr;
  return LASSO_OK;
}

static bool dict_trace() { return getenv("LASSO_TRACE_STEPS") != nullptr; }

int build_dict_dev(lasso_dict* d, bool final_fp64, DictDev* out, std::vector<const HostLevel*>* order,
                   bool tc_levels, bool tc_exact, bool split_level) {
  if (dict_trace()) fprintf(stderr, "[lasso trace] build_dict_dev: enter\n");
  memset(out, 0, sizeof(*out));
  out->N = (int)d->N;
  out->K = (int)d->K;
  out->ldN = d->ldN;
  out->anorm = d->anorm;
  if (!d->anorm32) {
    LASSO_CUDA_TRY(cudaMalloc(&d->anorm32, d->K * sizeof(float)));
    k_round_up_f32<<<grid_for(d->K), 256>>>(d->anorm, nullptr, 0.0, d->K, d->anorm32);
    LASSO_CUDA_TRY(cudaGetLastError());
    LASSO_CUDA_TRY(cudaDeviceSynchronize());
  }
  out->anorm32 = d->anorm32;
  if (d->anorm_max <= 0.0) {
    std::vector<double> h(d->K);
    LASSO_CUDA_TRY(cudaMemcpy(h.data(), d->anorm, d->K * sizeof(double), cudaMemcpyDeviceToHost));
    double m = 0.0;
    for (double v : h) m = std::max(m, v);
    d->anorm_max = m;
  }
  out->amax = d->anorm_max;
  if (dict_trace()) fprintf(stderr, "[lasso trace] build_dict_dev: atom norms ready\n");
  std::vector<const HostLevel*> lv;
  for (auto& h : d->approx) lv.push_back(&h);
  const bool vt64 = final_fp64 || d->exact_kind == LK_F64;
  split_level = split_level && !tc_exact && !vt64 && d->exact_kind == LK_F32 && d->exact.data;
  if (split_level) {
    int rc = ensure_split(d);
    if (rc) return rc;
    lv.push_back(&d->exact);   // the split form of the exact atoms (tensor cores)
  }
  lv.push_back(&d->exact);
  if (final_fp64 && d->exact_kind == LK_F32) {
    int rc = ensure_rung64(d);
    if (rc) return rc;
    lv.push_back(&d->rung64);
  }
  if ((int)lv.size() > MAX_LEVELS) return LASSO_ERR_INVALID_ARG;
  out->n_levels = (int)lv.size();
  const bool vt_double = final_fp64 || d->exact_kind == LK_F64;
  if (tc_exact && !vt_double && d->exact_kind == LK_F32) {
    int rc = ensure_split(d);
    if (rc) return rc;
  }
  const size_t split_idx = split_level ? d->approx.size() : lv.size();   // first entry of the exact atoms
  for (size_t i = 0; i < lv.size(); ++i) {
    const bool is_exact = lv[i] == &d->exact;
    const bool is_split = i == split_idx;
    out->lv[i] = make_level_dev(d, *lv[i], vt_double,
                                is_split ? true : (is_exact ? (tc_exact && !vt_double) : tc_levels));
    if (is_split) out->lv[i].rc = SPLIT_RC;
    if (!out->lv[i].epsr32) return LASSO_ERR_CUDA;
  }
  if (order) *order = lv;
  return LASSO_OK;
}

// ------------------------------------------------------------------ power iteration

static int level_sq_norm(lasso_dict* d, const HostLevel& h, int iters, double* out) {
  LevelDev L = make_level_dev(d, h);
  const int64_t N = d->N, K = d->K;
  double *v = nullptr, *w = nullptr, *tmp = nullptr, *nrm = nullptr;
  int rc;
  if ((rc = alloc((void**)&v, K * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&w, std::max(N, K) * sizeof(double)))) return rc;
  int64_t tsz = 16;
  if (h.kind == LK_KRON)
    tsz = std::max<int64_t>((int64_t)h.param * d->K1 * d->N2, (int64_t)h.param * d->N1 * d->K2);
  if (h.kind == LK_FAUST) tsz = 2 * (int64_t)h.fdim;
  if ((rc = alloc((void**)&tmp, tsz * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&nrm, sizeof(double)))) return rc;
  k_fill<<<grid_for(K), 256>>>(v, K, 1.0 / std::sqrt((double)K));
  double s = 0.0;
  const int64_t kslice = 512;
  for (int it = 0; it < iters; ++it) {
    // w = A~ v
    if (h.kind == LK_FAUST) {
      const double* src = v;
      for (int f = h.J - 1; f >= 0; --f) {
        double* dst = f == 0 ? w : tmp + ((h.J - 1 - f) & 1) * (int64_t)h.fdim;
        k_faust_mv64<<<grid_for(h.fac_h[f].rows), 256>>>(h.fac_h[f], 0, src, dst);
        src = dst;
      }
    } else if (h.kind == LK_KRON) {
      k_pi_kron_m1<<<grid_for(tsz), 256>>>(L, v, d->d, tmp);
      k_pi_kron_m2<<<grid_for(N), 256>>>(L, tmp, w);
    } else {
      cudaMemsetAsync(w, 0, N * sizeof(double));
      dim3 g((unsigned)((N + 127) / 128), (unsigned)((K + kslice - 1) / kslice));
      k_pi_matvec_dense<<<g, 128>>>(L, N, K, kslice, v, w);
    }
    // v = A~^T w
    if (h.kind == LK_FAUST) {
      const double* src = w;
      for (int f = 0; f < h.J; ++f) {
        double* dst = f == h.J - 1 ? v : tmp + (f & 1) * (int64_t)h.fdim;
        k_faust_mv64<<<grid_for(h.fac_h[f].cols), 256>>>(h.fac_h[f], 1, src, dst);
        src = dst;
      }
    } else if (h.kind == LK_KRON) {
      k_pi_kron_t1<<<grid_for(tsz), 256>>>(L, w, tmp);
      k_pi_kron_t2<<<grid_for(K), 256>>>(L, tmp, d->d, v);
    } else {
      k_pi_rmatvec_dense<<<grid_for(K * 32), 256>>>(L, N, K, w, v);
    }
    k_norm_scale<<<1, 1024>>>(v, K, nrm);
  }
  LASSO_CUDA_TRY(cudaGetLastError());
  LASSO_CUDA_TRY(cudaMemcpy(&s, nrm, sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(v);
  cudaFree(w);
  cudaFree(tmp);
  cudaFree(nrm);
  *out = s;
  return LASSO_OK;
}

int dict_prepare(lasso_dict* d, double L_override) {
  if (L_override > 0.0) {
    d->L = L_override;
    d->prepared = true;
    return LASSO_OK;
  }
  double m = 0.0, s = 0.0;
  int rc = level_sq_norm(d, d->exact, 200, &s);
  if (rc) return rc;
  m = s;
  for (auto& h : d->approx) {
    rc = level_sq_norm(d, h, 200, &s);
    if (rc) return rc;
    m = std::max(m, s);
  }
  d->L = 1.001 * m;
  d->prepared = true;
  return LASSO_OK;
}

}  // namespace lasso

using namespace lasso;

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_dict_create_dense(const void* A, lasso_dtype dt, int64_t N, int64_t K, int64_t ld,
                                       int atom_major, int normalize, int host_ptr, lasso_dict** out) {
  lasso::clear_last_error();
  if (!out) return LASSO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || N <= 0 || K <= 0 || (dt != LASSO_F64 && dt != LASSO_F32)) return LASSO_ERR_INVALID_ARG;
  if (atom_major ? ld < N : ld < K) return LASSO_ERR_INVALID_ARG;
  if (N > (1 << 24) || K > (1 << 30)) {
    set_last_error("lasso_dict_create_dense: N above 2^24 or K above 2^30", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  lasso_dict* d = new lasso_dict();
  cudaGetDevice(&d->device);
  d->N = N;
  d->K = K;
  d->ldN = round_up(N, 16);
  d->exact_kind = dt == LASSO_F64 ? LK_F64 : LK_F32;
  const size_t esz = dt == LASSO_F64 ? 8 : 4;
  const size_t in_elems = atom_major ? (size_t)(K - 1) * ld + N : (size_t)(N - 1) * ld + K;
  void* src = const_cast<void*>(A);
  void* tmp_in = nullptr;
  double *a64 = nullptr, *norms = nullptr;
  int rc = LASSO_OK;
  if (host_ptr) {
    if ((rc = alloc(&tmp_in, in_elems * esz))) goto fail;
    if (cudaMemcpy(tmp_in, A, in_elems * esz, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = LASSO_ERR_CUDA;
      goto fail;
    }
    src = tmp_in;
  }
  if ((rc = alloc((void**)&a64, (size_t)K * d->ldN * sizeof(double)))) goto fail;
  if ((rc = alloc((void**)&norms, K * sizeof(double)))) goto fail;
  if (dt == LASSO_F64)
    k_pack_f64<double><<<grid_for(K * d->ldN), 256>>>((const double*)src, N, K, ld, atom_major, a64, d->ldN);
  else
    k_pack_f64<float><<<grid_for(K * d->ldN), 256>>>((const float*)src, N, K, ld, atom_major, a64, d->ldN);
  k_row_norms_f64<<<grid_for(K * 32), 256>>>(a64, d->ldN, N, K, norms);
  {
    HostLevel& h = d->exact;
    h.kind = d->exact_kind;
    h.api_kind = dt == LASSO_F64 ? -1 : -2;
    if ((rc = alloc(&h.data, (size_t)K * d->ldN * esz))) goto fail;
    if (dt == LASSO_F64)
      k_store_exact<double><<<grid_for(K * d->ldN), 256>>>(a64, norms, normalize, d->ldN, K, (double*)h.data);
    else
      k_store_exact<float><<<grid_for(K * d->ldN), 256>>>(a64, norms, normalize, d->ldN, K, (float*)h.data);
    if ((rc = alloc_level_vectors(d, h))) goto fail;
    if ((rc = alloc((void**)&d->anorm, K * sizeof(double)))) goto fail;
    cudaMemset(h.eps, 0, K * sizeof(double));
    if (dt == LASSO_F64)
      k_exact_norms<double><<<grid_for(K * 32), 256>>>((const double*)h.data, d->ldN, N, K, d->anorm, h.atnorm, h.kappa);
    else
      k_exact_norms<float><<<grid_for(K * 32), 256>>>((const float*)h.data, d->ldN, N, K, d->anorm, h.atnorm, h.kappa);
    if (cudaGetLastError() != cudaSuccess) {
      rc = LASSO_ERR_CUDA;
      goto fail;
    }
    h.rc = 1.0;
    if ((rc = finish_level(d, h))) goto fail;
  }
  cudaFree(tmp_in);
  cudaFree(a64);
  cudaFree(norms);
  *out = d;
  return LASSO_OK;
fail:
  cudaFree(tmp_in);
  cudaFree(a64);
  cudaFree(norms);
  lasso_dict_destroy(d);
  return rc;
}

extern "C" int lasso_dict_create_kron(const float* B, const float* C, int R, int N1, int K1, int N2, int K2,
                                      int normalize, int host_ptr, lasso_dict** out) {
  lasso::clear_last_error();
  if (!out) return LASSO_ERR_INVALID_ARG;
  *out = nullptr;
  if (!B || !C || R <= 0 || N1 <= 0 || K1 <= 0 || N2 <= 0 || K2 <= 0 || R > 64) return LASSO_ERR_INVALID_ARG;
  lasso_dict* d = new lasso_dict();
  cudaGetDevice(&d->device);
  d->is_kron = true;
  d->R = R;
  d->N1 = N1;
  d->K1 = K1;
  d->N2 = N2;
  d->K2 = K2;
  d->N = (int64_t)N1 * N2;
  d->K = (int64_t)K1 * K2;
  d->ldN = round_up(d->N, 16);
  d->exact_kind = LK_F32;
  const size_t nb = (size_t)R * N1 * K1, nc = (size_t)R * N2 * K2;
  int rc = LASSO_OK;
  float* dfl = nullptr;
  if ((rc = alloc((void**)&d->Bf, nb * 4))) goto fail;
  if ((rc = alloc((void**)&d->Cf, nc * 4))) goto fail;
  if (cudaMemcpy(d->Bf, B, nb * 4, host_ptr ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemcpy(d->Cf, C, nc * 4, host_ptr ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice) != cudaSuccess) {
    rc = LASSO_ERR_CUDA;
    goto fail;
  }
  if ((rc = alloc((void**)&d->gramB, (size_t)R * R * K1 * 8))) goto fail;
  if ((rc = alloc((void**)&d->gramC, (size_t)R * R * K2 * 8))) goto fail;
  if ((rc = alloc((void**)&d->d, d->K * 8))) goto fail;
  if ((rc = alloc((void**)&dfl, d->K * 4))) goto fail;
  if ((rc = alloc((void**)&d->anorm, d->K * 8))) goto fail;
  k_kron_gram<<<grid_for((int64_t)R * R * K1), 256>>>(d->Bf, R, N1, K1, d->gramB);
  k_kron_gram<<<grid_for((int64_t)R * R * K2), 256>>>(d->Cf, R, N2, K2, d->gramC);
  k_kron_scale<<<grid_for(d->K), 256>>>(d->gramB, d->gramC, R, K1, K2, normalize, d->d, dfl, d->anorm);
  {
    HostLevel& h = d->exact;
    h.kind = LK_F32;
    h.api_kind = -2;
    h.dscale = nullptr;
    if ((rc = alloc(&h.data, (size_t)d->K * d->ldN * 4))) goto fail;
    if ((rc = alloc_level_vectors(d, h))) goto fail;
    k_kron_dense_f32<<<grid_for(d->K * 32), 256>>>(d->Bf, d->Cf, d->d, R, N1, K1, N2, K2, d->ldN, (float*)h.data, h.eps,
                                                   h.atnorm, h.kappa);
    if (cudaGetLastError() != cudaSuccess) {
      rc = LASSO_ERR_CUDA;
      goto fail;
    }
    h.rc = 1.0;
    if ((rc = finish_level(d, h))) goto fail;
  }
  // the FP32 copy of d shared by every Kronecker level
  d->exact.dscale = dfl;
  *out = d;
  return LASSO_OK;
fail:
  cudaFree(dfl);
  lasso_dict_destroy(d);
  return rc;
}

extern "C" int lasso_dict_add_level(lasso_dict* d, lasso_level_kind kind, int param) {
  lasso::clear_last_error();
  if (!d || (int)d->approx.size() + 1 >= MAX_LEVELS - 1) return LASSO_ERR_INVALID_ARG;
  HostLevel h;
  h.api_kind = kind;
  h.param = param;
  const int64_t K = d->K, N = d->N, ldN = d->ldN, total = K * ldN;
  int rc;
  switch (kind) {
    case LASSO_LEVEL_BF16: {
      h.kind = LK_BF16;
      if ((rc = alloc(&h.data, total * 2))) return rc;
      k_quant_bf16<<<grid_for(total), 256>>>(d->exact.data, d->exact.kind, total, (__nv_bfloat16*)h.data);
      if ((rc = alloc_level_vectors(d, h))) return rc;
      k_level_eps<<<grid_for(K * 32), 256>>>(h.data, LK_BF16, nullptr, d->exact.data, d->exact.kind, ldN, N, K, h.eps,
                                             h.atnorm, h.kappa);
      h.rc = 0.5 * (d->exact.kind == LK_F64 ? 0.5 : 1.0);
      break;
    }
    case LASSO_LEVEL_FP8: {
      h.kind = LK_FP8;
      if ((rc = alloc(&h.data, total))) return rc;
      if ((rc = alloc((void**)&h.scale, K * 4))) return rc;
      k_quant_fp8<<<grid_for(K * 32), 256>>>(d->exact.data, d->exact.kind, ldN, N, K, (__nv_fp8_storage_t*)h.data,
                                             h.scale);
      if ((rc = alloc_level_vectors(d, h))) return rc;
      k_level_eps<<<grid_for(K * 32), 256>>>(h.data, LK_FP8, h.scale, d->exact.data, d->exact.kind, ldN, N, K, h.eps,
                                             h.atnorm, h.kappa);
      h.rc = 0.25 * (d->exact.kind == LK_F64 ? 0.5 : 1.0);
      break;
    }
    case LASSO_LEVEL_F32: {
      if (d->exact.kind != LK_F64) return LASSO_ERR_INVALID_ARG;
      h.kind = LK_F32;
      if ((rc = alloc(&h.data, total * 4))) return rc;
      k_quant_f32<<<grid_for(total), 256>>>((const double*)d->exact.data, total, (float*)h.data);
      if ((rc = alloc_level_vectors(d, h))) return rc;
      k_level_eps<<<grid_for(K * 32), 256>>>(h.data, LK_F32, nullptr, d->exact.data, d->exact.kind, ldN, N, K, h.eps,
                                             h.atnorm, h.kappa);
      h.rc = 0.5;
      break;
    }
    case LASSO_LEVEL_KRON: {
      if (!d->is_kron || param <= 0 || param > d->R) return LASSO_ERR_INVALID_ARG;
      h.kind = LK_KRON;
      h.owns_data = false;
      h.data = nullptr;
      h.dscale = d->exact.dscale;
      if ((rc = alloc_level_vectors(d, h))) return rc;
      k_kron_level<<<grid_for(K), 256>>>(d->gramB, d->gramC, d->d, d->R, d->K1, d->K2, param, h.eps, h.atnorm, h.kappa);
      // theoretical relative complexity R' (2 N1 K1 K2 + 2 N1 K2 N2) / (2 N K)
      h.rc = (double)param * ((double)d->N1 * d->K1 * d->K2 + (double)d->N1 * d->K2 * d->N2) / ((double)N * K);
      break;
    }
    default:
      return LASSO_ERR_INVALID_ARG;
  }
  LASSO_CUDA_TRY(cudaGetLastError());
  if ((rc = finish_level(d, h))) return rc;
  d->approx.push_back(h);
  d->prepared = false;
  return LASSO_OK;
}

void lasso_workspace_free(lasso::Workspace* ws);

namespace {

// Explicit FP64 product of the factors (|S_f| when absval), atom-major K x ld, into `out`
// (`tmp` is the other buffer of the ping-pong).  Returns the buffer holding the result.
double* faust_explicit(const HostLevel& h, int64_t K, int64_t ld, int absval, double* out, double* tmp) {
  double* bufs[2] = {out, tmp};
  // the last factor lands in the buffer that, after J - 1 stages, is `out`
  int cur = (h.J - 1) & 1;
  cudaMemsetAsync(bufs[cur], 0, (size_t)K * ld * sizeof(double));
  k_faust_last64<<<grid_for(h.fac_h[h.J - 1].rows), 256>>>(h.fac_h[h.J - 1], absval, ld, bufs[cur]);
  for (int f = h.J - 2; f >= 0; --f) {
    k_faust_stage64<<<grid_for(K * h.fac_h[f].rows), 256>>>(h.fac_h[f], absval, K, ld, bufs[cur], bufs[cur ^ 1]);
    cur ^= 1;
  }
  return bufs[cur];
}

}  // namespace

extern "C" int lasso_dict_add_level_faust(lasso_dict* d, int J, const int64_t* dims, const int64_t* indptr,
                                          const int32_t* indices, const float* values) {
  lasso::clear_last_error();
  if (!d || (int)d->approx.size() + 1 >= MAX_LEVELS - 1) return LASSO_ERR_INVALID_ARG;
  if (J < 1 || J > 16 || !dims || !indptr || !indices || !values) return LASSO_ERR_INVALID_ARG;
  for (int f = 0; f <= J; ++f)
    if (dims[f] < 1 || dims[f] > (1 << 30)) return LASSO_ERR_INVALID_ARG;
  if (dims[0] != d->N || dims[J] != d->K) return LASSO_ERR_INVALID_ARG;
  // validate every factor on the host (so that every device index stays in range) and lay the
  // CSR arrays of S_f and S_f^T out in one buffer, each array 16-byte aligned
  struct Lay { int64_t rows, cols, nnz, rp, ci, v, rpT, ciT, vT; };
  std::vector<Lay> lay(J);
  int64_t po = 0, no = 0, bytes = 0, nnz_total = 0;
  int n_fwd = 0, n_adj = 0, fdim = 0;
  auto take = [&](int64_t b) { const int64_t at = bytes; bytes += round_up(std::max<int64_t>(b, 16), 16); return at; };
  for (int f = 0; f < J; ++f) {
    Lay& l = lay[f];
    l.rows = dims[f];
    l.cols = dims[f + 1];
    const int64_t* rp = indptr + po;
    if (rp[0] != 0) return LASSO_ERR_INVALID_ARG;
    int64_t longest = 0;
    for (int64_t n = 0; n < l.rows; ++n) {
      if (rp[n + 1] < rp[n]) return LASSO_ERR_INVALID_ARG;
      longest = std::max(longest, rp[n + 1] - rp[n]);
    }
    l.nnz = rp[l.rows];
    if (l.nnz >= ((int64_t)1 << 31)) return LASSO_ERR_INVALID_ARG;
    std::vector<int64_t> colcount(l.cols, 0);
    for (int64_t n = 0; n < l.rows; ++n)
      for (int64_t p = rp[n]; p < rp[n + 1]; ++p) {
        const int32_t c = indices[no + p];
        if (c < 0 || c >= l.cols) return LASSO_ERR_INVALID_ARG;
        if (p > rp[n] && c <= indices[no + p - 1]) return LASSO_ERR_INVALID_ARG;
        if (!std::isfinite(values[no + p])) return LASSO_ERR_INVALID_ARG;
        ++colcount[c];
      }
    int64_t longest_t = 0;
    for (int64_t c : colcount) longest_t = std::max(longest_t, c);
    n_fwd += (int)longest;
    n_adj += (int)longest_t;
    fdim = std::max<int>(fdim, (int)std::max(l.rows, l.cols));
    l.rp = take((l.rows + 1) * 4);
    l.ci = take(l.nnz * 4);
    l.v = take(l.nnz * 4);
    l.rpT = take((l.cols + 1) * 4);
    l.ciT = take(l.nnz * 4);
    l.vT = take(l.nnz * 4);
    nnz_total += l.nnz;
    po += l.rows + 1;
    no += l.nnz;
  }
  // host staging: CSR of S_f as given, CSR of S_f^T by a counting sort over the columns (rows of
  // S_f^T keep the increasing order of the original rows)
  std::vector<unsigned char> stage((size_t)bytes, 0);
  po = 0;
  no = 0;
  for (int f = 0; f < J; ++f) {
    const Lay& l = lay[f];
    const int64_t* rp = indptr + po;
    int32_t* rp32 = reinterpret_cast<int32_t*>(&stage[l.rp]);
    int32_t* ci32 = reinterpret_cast<int32_t*>(&stage[l.ci]);
    float* v32 = reinterpret_cast<float*>(&stage[l.v]);
    int32_t* rpT = reinterpret_cast<int32_t*>(&stage[l.rpT]);
    int32_t* ciT = reinterpret_cast<int32_t*>(&stage[l.ciT]);
    float* vT = reinterpret_cast<float*>(&stage[l.vT]);
    for (int64_t n = 0; n <= l.rows; ++n) rp32[n] = (int32_t)rp[n];
    memcpy(ci32, indices + no, l.nnz * 4);
    memcpy(v32, values + no, l.nnz * 4);
    for (int64_t c = 0; c <= l.cols; ++c) rpT[c] = 0;
    for (int64_t p = 0; p < l.nnz; ++p) ++rpT[ci32[p] + 1];
    for (int64_t c = 0; c < l.cols; ++c) rpT[c + 1] += rpT[c];
    std::vector<int32_t> next(rpT, rpT + l.cols);
    for (int64_t n = 0; n < l.rows; ++n)
      for (int64_t p = rp[n]; p < rp[n + 1]; ++p) {
        const int32_t q = next[ci32[p]]++;
        ciT[q] = (int32_t)n;
        vT[q] = v32[p];
      }
    po += l.rows + 1;
    no += l.nnz;
  }
  HostLevel h;
  h.kind = LK_FAUST;
  h.api_kind = LASSO_LEVEL_FAUST;
  h.param = J;
  h.owns_data = false;
  h.J = J;
  h.fdim = fdim;
  h.n_fwd = n_fwd;
  h.n_adj = n_adj;
  const int64_t K = d->K, N = d->N, ldN = d->ldN;
  const int64_t ld = std::max<int64_t>(fdim, ldN);
  double *P = nullptr, *Q = nullptr;
  int rc = LASSO_OK;
  auto fail = [&](int code) {
    cudaFree(P);
    cudaFree(Q);
    free_level(h);
    return code;
  };
  if ((rc = alloc(&h.fbuf, (size_t)bytes))) return fail(rc);
  if (cudaMemcpy(h.fbuf, stage.data(), (size_t)bytes, cudaMemcpyHostToDevice) != cudaSuccess) return fail(LASSO_ERR_CUDA);
  unsigned char* base = static_cast<unsigned char*>(h.fbuf);
  for (int f = 0; f < J; ++f) {
    const Lay& l = lay[f];
    FaustFactor F;
    F.rows = (int)l.rows;
    F.cols = (int)l.cols;
    F.rp = reinterpret_cast<const int32_t*>(base + l.rp);
    F.ci = reinterpret_cast<const int32_t*>(base + l.ci);
    F.v = reinterpret_cast<const float*>(base + l.v);
    F.rpT = reinterpret_cast<const int32_t*>(base + l.rpT);
    F.ciT = reinterpret_cast<const int32_t*>(base + l.ciT);
    F.vT = reinterpret_cast<const float*>(base + l.vT);
    h.fac_h.push_back(F);
  }
  if ((rc = alloc((void**)&h.fac, J * sizeof(FaustFactor)))) return fail(rc);
  if (cudaMemcpy(h.fac, h.fac_h.data(), J * sizeof(FaustFactor), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LASSO_ERR_CUDA);
  if ((rc = alloc_level_vectors(d, h))) return fail(rc);
  if ((rc = alloc((void**)&P, (size_t)K * ld * sizeof(double)))) return fail(rc);
  if ((rc = alloc((void**)&Q, (size_t)K * ld * sizeof(double)))) return fail(rc);
  // kappa_j from |S_0| ... |S_{J-1}|, then eps_j and ||a~_j|| from the signed product
  const double* Pa = faust_explicit(h, K, ld, 1, P, Q);
  k_faust_kappa<<<grid_for(K * 32), 256>>>(Pa, ld, N, K, h.kappa);
  const double* Pv = faust_explicit(h, K, ld, 0, P, Q);
  k_faust_eps<<<grid_for(K * 32), 256>>>(Pv, ld, d->exact.data, d->exact.kind, ldN, N, K,
                                         gamma_n((double)n_fwd + 2.0, U64), h.kappa, h.eps, h.atnorm);
  if (cudaGetLastError() != cudaSuccess) return fail(LASSO_ERR_CUDA);
  if ((rc = finish_level(d, h))) return fail(rc);
  cudaFree(P);
  cudaFree(Q);
  P = Q = nullptr;
  h.rc = (double)nnz_total / ((double)N * (double)K);
  d->approx.push_back(h);
  d->faust_dim = std::max(d->faust_dim, fdim);
  d->prepared = false;
  // the solve workspaces are sized for the levels they saw: rebuild them with this level's scratch
  if (d->ws) lasso_workspace_free(d->ws);
  if (d->ws64) lasso_workspace_free(d->ws64);
  d->ws = d->ws64 = nullptr;
  return LASSO_OK;
}

extern "C" int lasso_dict_set_rc(lasso_dict* d, int level, double rc) {
  lasso::clear_last_error();
  if (!d || level < 0 || level > (int)d->approx.size() || !(rc > 0.0)) return LASSO_ERR_INVALID_ARG;
  HostLevel& h = level == (int)d->approx.size() ? d->exact : d->approx[level];
  h.rc = rc;
  h.rc_set = true;
  return LASSO_OK;
}

extern "C" int lasso_dict_prepare(lasso_dict* d, double L_override) {
  lasso::clear_last_error();
  if (!d) return LASSO_ERR_INVALID_ARG;
  return dict_prepare(d, L_override);
}

extern "C" int lasso_dict_info(const lasso_dict* d, lasso_dict_info_t* info) {
  lasso::clear_last_error();
  if (!d || !info) return LASSO_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->N = d->N;
  info->K = d->K;
  info->n_levels = (int)d->approx.size() + 1;
  info->L = d->L;
  for (size_t i = 0; i <= d->approx.size() && i < 8; ++i) {
    const HostLevel& h = i < d->approx.size() ? d->approx[i] : d->exact;
    info->kind[i] = h.api_kind;
    info->rc[i] = h.rc;
    info->eps_mean[i] = h.eps_mean;
    info->eps_max[i] = h.eps_max;
  }
  return LASSO_OK;
}

__global__ void k_level_to_f64(LevelDev L, int64_t N, int64_t K, double* __restrict__ out) {
  int64_t total = K * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = t / N, n = t % N;
    out[t] = load_level(L.data, L.kind, L.scale, j, j * L.ld + n);
  }
}

extern "C" int lasso_dict_level_host(const lasso_dict* d, int level, double* eps_host, double* atoms_host) {
  lasso::clear_last_error();
  if (!d || level < 0 || level > (int)d->approx.size()) return LASSO_ERR_INVALID_ARG;
  const HostLevel& h = level == (int)d->approx.size() ? d->exact : d->approx[level];
  if (eps_host) LASSO_CUDA_TRY(cudaMemcpy(eps_host, h.eps, d->K * 8, cudaMemcpyDeviceToHost));
  if (atoms_host) {
    if (level_structured(h.kind)) {
      set_last_error("lasso_dict_level_host: a structured level has no dense atoms to copy", __FILE__, __LINE__);
      return LASSO_ERR_UNSUPPORTED;
    }
    double* tmp = nullptr;
    int rc = alloc((void**)&tmp, (size_t)d->K * d->N * 8);
    if (rc) return rc;
    k_level_to_f64<<<grid_for(d->K * d->N), 256>>>(make_level_dev(d, h), d->N, d->K, tmp);
    LASSO_CUDA_TRY(cudaGetLastError());
    LASSO_CUDA_TRY(cudaMemcpy(atoms_host, tmp, (size_t)d->K * d->N * 8, cudaMemcpyDeviceToHost));
    cudaFree(tmp);
  }
  return LASSO_OK;
}

extern "C" void lasso_dict_destroy(lasso_dict* d) {
  if (!d) return;
  if (d->ws) lasso_workspace_free(d->ws);
  if (d->ws64) lasso_workspace_free(d->ws64);
  for (auto& h : d->approx) free_level(h);
  cudaFree(d->exact.dscale);
  d->exact.dscale = nullptr;
  free_level(d->exact);
  cudaFree(d->Bf);
  cudaFree(d->Cf);
  cudaFree(d->d);
  cudaFree(d->gramB);
  cudaFree(d->gramC);
  cudaFree(d->anorm);
  cudaFree(d->anorm32);
  if (d->rung64.kind >= 0) {
    if (d->rung64.owns_data) {
      free_level(d->rung64);   // the Kronecker dictionary's own FP64 rung
    } else {
      for (auto* e : d->rung64.epsr32) cudaFree(e);
      cudaFree(d->rung64.kappa32);
      cudaFree(d->rung64.eps32);
    }
  }
  delete d;
}
