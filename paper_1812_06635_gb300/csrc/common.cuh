// Shared device types and helpers of the GB300 screened Lasso library.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "../../include/lasso.h"

namespace lasso {

constexpr int MAX_LEVELS = 8;
constexpr int VEC_BYTES = 16;        // every dense row is padded to a multiple of 16 elements
constexpr int CORR_CHUNK = 32;       // smallest work item (atoms of the preserved list); batches use 4x
constexpr int RES_THREADS = 512;

// Arithmetic kind of a level.
enum LevelKind : int {
  LK_F64 = 0,     // FP64 data, FP64 accumulation
  LK_F32 = 1,     // FP32 data, error-free FP32 products and compensated accumulation (Dot2)
  LK_BF16 = 2,    // BF16 data, FP32 products, compensated accumulation
  LK_FP8 = 3,     // E4M3 data with per-atom FP32 scale, FP32 products
  LK_KRON = 4,    // sum of Kronecker products, FP32 small GEMMs
  LK_F32D = 5,    // FP32 data, FP64 accumulation (final FP64 rung of an FP32 dictionary)
  LK_FAUST = 6    // product of sparse factors (CSR), FP32 sparse products
};

// Structured levels form their products over every atom in batched kernels (A~ z into AZ,
// A~^T rho into Gfull); the correlation pass only reads them.
__host__ __device__ inline bool level_structured(int k) { return k == LK_KRON || k == LK_FAUST; }
__host__ __device__ inline bool level_is_dense(int k) { return !level_structured(k); }
enum ResModel : int { RES_FOLD = 0, RES_CHAIN = 1, RES_DOT2 = 2 };
__host__ __device__ inline bool level_fp64_arith(int k) { return k == LK_F64 || k == LK_F32D; }

// One sparse factor S_f (rows x cols) of a product level, in CSR and as the CSR of S_f^T.
struct FaustFactor {
  int rows, cols;
  const int32_t* rp;        // rows + 1 row pointers
  const int32_t* ci;        // column indices, increasing within a row
  const float* v;
  const int32_t* rpT;       // S_f^T: cols + 1 row pointers
  const int32_t* ciT;
  const float* vT;
};

// One rung of the ladder, as the kernels see it.
struct LevelDev {
  int kind;
  int64_t ld;               // dense: elements per atom row (multiple of 16)
  const void* data;         // dense: K x ld atom-major
  const float* scale;       // FP8: per-atom scale
  const double* eps;        // eps_j >= ||a~_j - a_j|| (dictionary error only)
  const double* kappa;      // kappa_j: bound of sum_i |a~_ij| |v_i| / ||v|| (||a~_j|| or Kronecker form)
  const float* atnorm;      // ||a~_j||
  const float* epsr32;      // eps_j + gam_corr kappa_j rounded up to FP32 (bulk bound in FP32 code)
  const float* kappa32;     // kappa_j rounded up to FP32
  const float* eps32;       // eps_j rounded up to FP32
  const float* epsr32_simt; // eps_j + (FP32 SIMT product bound) kappa_j: fast checks outside the bulk pass
  // Split tensor-core form of the exact FP32 level: a = a1 + a2 + e3 (a1, a2 BF16), correlated as
  // a1^T r1 + a1^T r2 + a2^T r1 with rho = r1 + r2 + r3; c2 >= max_j ||a2_j|| / kappa_j bounds the
  // dropped a2^T r2 through the per-signal term (k_quant_rho folds c2 ||r2|| into dq).
  int split;
  double c2;
  void* rq2;                // split: second BF16 operand of the residuals
  int tc;                   // 1: batched correlation on the tensor cores (BF16 / FP8 levels)
  void* rq;                 // tensor-core levels: quantised residuals (B x ld, BF16 or E4M3)
  float* rsig;              // tensor-core levels: per-signal scale of the quantised residual
  // Rounding of the correlation: |g^_j - a~_j^T rho^| <= gam_corr kappa_j ||rho^|| + 3 u_g |g^_j|,
  // so the stable test and the dual scaling use eps_j + gam_corr kappa_j in place of eps_j.
  double gam_corr;
  double gam_tight;         // exact FP32 level: bound of the Dot2 recomputation (certificate)
  // Rounding of the residual, e_r >= ||rho^ - (y - A~ z)||:
  //   RES_FOLD:  gam_res sum_j |z_j| kappa_j + 2 u ||rho^||
  //   RES_CHAIN: gamma_{nnz+4}(u64) sum_j |z_j| kappa_j + 2 u ||rho^||
  //   RES_DOT2:  (3 gamma_{2 nnz + 2}(u32)^2 + gam_res) sum_j |z_j| kappa_j + 2 u ||rho^||
  int res_model;
  double gam_res;
  double rc;                // relative complexity (Algorithm 2)
  // Kronecker factors (LK_KRON): A~ = (sum_{r<R} B_r (x) C_r) diag(d)
  const float* B;
  const float* C;
  const float* dscale;      // d_j as FP32 (the FP64 value enters through kappa / eps)
  int R, N1, K1, N2, K2;
  // Product of sparse factors (LK_FAUST): A~ = S_0 S_1 ... S_{J-1} (device array of J factors);
  // fdim = the largest dimension of any factor (length of the scratch vectors)
  const FaustFactor* fac;
  int J, fdim;
};

struct DictDev {
  int N, K, n_levels;
  int64_t ldN;              // padded signal length (multiple of 16)
  const double* anorm;      // exact ||a_j||_2, rounded up
  const float* anorm32;     // the same rounded up to FP32
  double amax;              // max_j ||a_j||_2
  LevelDev lv[MAX_LEVELS];
};

// Per-signal solver state (device memory, one per signal).
struct SigState {
  double lam, yy, ynorm, t, beta;
  double l1, sum_epsz, sum_kapz;     // of the current point z_t (its nonzero list)
  double gap, Gp, Gt, gamma, Rp, delta, sp;
  double lam_max_lb, lam_max_ub;
  // snapshot of the pass whose reduced certificate met tol, awaiting the full-dictionary check
  double c_rr, c_yr, c_l1, c_epsz, c_kapz, c_m1;
  double dq;                         // ||rho - rho^||: quantisation of the tensor-core operand
  double rr, yr;                     // ||rho^||^2 and y^T rho^ of the current pass (k_residual)
  float nrho_ru;                     // ||rho^|| rounded up to FP32
  float thr_f, beta_f;               // lam / L and the FISTA momentum, as FP32 (update of the pass)
  float c_nrho_ru;                   // ||rho^|| of the snapshot, rounded up
  unsigned pm1, pm2;                 // per-pass maxima of the correlation (FP32 bit patterns, >= 0)
  // screening scalars of the pass: |s'|, |s'| ||rho||, test radius, |s~|, R~, 1 / lam
  double t_abs_sp, t_c_eps, t_Rs, t_abs_st, t_Rt, t_inv_lam;
  int act, scr, snap;                // outcome of the pass, screen flag, snapshot
  int res_tight, c_res_tight;        // residual with error-free products (next passes, sticky / the snapshot)
  int corr_tight;                    // exact level: correlations with error-free products (sticky)
  int res_used;                      // the products the current pass's residual was formed with
                                     // (k_residual): the rounding model of its bound follows it
  double best_cert;                  // exact level: best certificate so far
  int stall, pad2;                   // exact level: passes without a 2 % improvement of it
  int c_nnz, pending, next_check, pad1;
  int level, n_kept, parity, n_nz, status, done, iters, Kt, n_chunks, pad0;
  int level_passes[MAX_LEVELS];
};

// e_r >= ||rho^ - (y - A~ z)|| for the residual of the current pass (see LevelDev).
__device__ __forceinline__ double residual_bound(const LevelDev& L, double sum_kapz, int n_nz, double nrho,
                                                 bool vt64, bool fast = false);

// Knobs of a solve, as kernels see them.
struct SolveParams {
  double tol, Gamma, tau, L;
  double inv_L;             // 1 / L
  int algo, rule, screen_every, max_iter;
  int B;
  int chunk;                // atoms per correlation work item (multiple of CORR_CHUNK)
  int full_gap;             // 1: stop on the full-dictionary gap (checked explicitly)
  int stall_passes;         // exact FP32 level: passes without progress that mark a signal saturated (0: off)
  int corr_grid;            // blocks of the correlation pass (the per-pass chunk keeps it busy)
  int z_f32;                // FP64 iterates whose point is returned in FP32: the extrapolated point z
                            // (the certified and returned point) is kept FP32-representable
};

// Internal status of a signal whose FP32 iterates stopped improving on the exact level: the
// host solves it again with FP64 iterates (never returned to callers; reported as
// LASSO_ERR_MAXITER when that second solve is disabled).
constexpr int LASSO_ST_SATURATED = 2;

// ------------------------------------------------------------------ error-free transforms
// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-float accumulator (s, c): value s + c.
struct DF {
  float s, c;
  __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float p) {
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void merge(const DF& o) {
    float t, e;
    two_sum(s, o.s, t, e);
    s = t;
    c = __fadd_rn(__fadd_rn(c, o.c), e);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Dot2 step (Ogita, Rump & Oishi, "Accurate sum and dot product", 2005): the product is split
// exactly as p + q (FMA), p enters the running sum through TwoSum and the errors gather in c.
__device__ __forceinline__ void dot2_add(DF& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float q = __fmaf_rn(a, b, -p);
  float t, e;
  two_sum(acc.s, p, t, e);
  acc.s = t;
  acc.c = __fadd_rn(acc.c, __fadd_rn(e, q));
}

__device__ __forceinline__ DF df_shfl_xor(const DF& v, int m) {
  DF o;
  o.s = __shfl_xor_sync(0xffffffffu, v.s, m);
  o.c = __shfl_xor_sync(0xffffffffu, v.c, m);
  return o;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
// Sum of non-negative FP32 terms rounded upward at every step: an upper bound of the exact sum.
__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

constexpr double U32 = 5.9604644775390625e-08;    // 2^-24
constexpr double U64 = 1.1102230246251565e-16;    // 2^-53

// gamma_n = n u / (1 - n u) (Higham): bound of the relative error of an n-term recursive sum.
__host__ __device__ inline double gamma_n(double n, double u) { return n * u / (1.0 - n * u); }


// ------------------------------------------------------------------ host error helpers
#define LASSO_CUDA_TRY(expr)                                                          \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      lasso::set_last_error(cudaGetErrorString(_e), __FILE__, __LINE__);              \
      return _e == cudaErrorMemoryAllocation ? LASSO_ERR_NOMEM : LASSO_ERR_CUDA;      \
    }                                                                                 \
  } while (0)

void set_last_error(const char* msg, const char* file, int line);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace lasso

namespace lasso {
__device__ __forceinline__ double residual_bound(const LevelDev& L, double sum_kapz, int n_nz, double nrho,
                                                 bool vt64, bool fast) {
  const double urho = vt64 ? U64 : U32;
  // fast: FP32 residual as plain FMA chains over the nonzeros (one chain per row), then y - acc
  if (fast && !vt64 && !level_structured(L.kind) && !level_fp64_arith(L.kind))
    return gamma_n((double)n_nz + 4.0, U32) * sum_kapz + 2.0 * urho * nrho;
  switch (L.res_model) {
    case RES_CHAIN:
      return gamma_n((double)n_nz + 4.0, U64) * sum_kapz + 2.0 * urho * nrho;
    case RES_DOT2: {
      const double g = gamma_n(2.0 * n_nz + 2.0, U32);
      // 2 g^2: Dot2 sum; g^2 more for the final FP32 rounding of y - (s + c), u |c| <= u g (...)
      return (3.0 * g * g + L.gam_res) * sum_kapz + 2.0 * urho * nrho;
    }
    default:
      return L.gam_res * sum_kapz + 2.0 * urho * nrho;
  }
}
}  // namespace lasso
