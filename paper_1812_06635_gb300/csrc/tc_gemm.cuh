// Tensor-core correlation G = A~ R^^T for the batched BF16 / FP8 levels (tcgen05 + TMA + TMEM).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace lasso {

constexpr int TC_BM = 128;        // atoms per tile (TMEM lanes)
constexpr int TC_BN = 256;        // signals per tile (TMEM columns, FP32 accumulators)
constexpr int TC_STAGES = 4;      // TMA ring depth (48 KB per stage)
constexpr int TC_THREADS = 192;   // warp 0: TMA producer, warp 1: MMA issuer, warps 2-5: epilogue
constexpr int TC_SMEM = TC_STAGES * (TC_BM + TC_BN) * 128 + 1024 + 256;

// Rounding model of the tensor-core accumulation (products of BF16 / E4M3 operands are exact in
// FP32; the sum of n products is taken as an FP32 chain with unit roundoff u_tc, no better than
// 2^-22 for BF16 and 2^-19 for E4M3 inputs).  tests/test_gpu_tc.py checks the observed error
// against this bound on adversarial and random inputs.
constexpr double TC_U_BF16 = 2.384185791015625e-07;   // 2^-22
constexpr double TC_U_FP8 = 1.9073486328125e-06;      // 2^-19

// Promoted accumulation (the split form): the MMAs of each k-block of TC_GROUP 128-byte
// K-slices accumulate in one of two TMEM buffers; eight epilogue warps add every finished
// k-block into FP32 registers (round to nearest) while the next k-block accumulates in the other
// buffer.  The tensor-core chain then spans one k-block instead of the whole signal length.
constexpr int TC_GROUP = 2;                 // 128-byte K-slices per promoted k-block
constexpr int TCP_THREADS = 320;            // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int TCP_SMEM = TC_SMEM;

struct TcOperands {
  CUtensorMap a;          // dictionary level: K rows (atoms) x ldN, K-major
  CUtensorMap b;          // quantised residuals: B rows (signal slots) x ldN, K-major
  CUtensorMap a2, b2;     // split form (nphase 3): second BF16 parts of the atoms / residuals
  int fp8;                // 1: kind::f8f6f4 E4M3, 0: kind::f16 BF16
  int nphase;             // 1: a^T r; 3: a1^T r1 + a1^T r2 + a2^T r1 in one accumulator
  int promote;            // 1: promoted accumulation (k-blocks of TC_GROUP slices summed in FP32)
};

// Number of promoted k-blocks of a product of ldN elements in `nphase` phases.
inline int tc_groups(int64_t ldN, int fp8, int nphase) {
  const int nkb = (int)((ldN * (fp8 ? 1 : 2) + 127) / 128);
  return (nkb * nphase + TC_GROUP - 1) / TC_GROUP;
}

// Rounding bound of the promoted BF16 product relative to sum |a_i r_i| (all phases): each
// k-block is a tensor-core chain of TC_GROUP (64 products + 4 k-steps) with unit roundoff
// u_tc = 2^-22, and the k-block sums are added in FP32 with round to nearest.
inline double tc_promoted_gamma(int64_t ldN, int nphase) {
  const double gk = gamma_n(TC_GROUP * (64.0 + 4.0), TC_U_BF16);
  const double gr = gamma_n((double)tc_groups(ldN, 0, nphase), U32);
  return gk + gr * (1.0 + gk);
}

// Encode the tensor maps (host); level_data2 / rq2 non-null selects the split form.  Returns
// LASSO_OK or an error status.
int tc_make_operands(const void* level_data, const void* level_data2, int64_t K, const void* rq, const void* rq2,
                     int64_t B, int64_t ldN, int fp8, TcOperands* out);

// Gfull[b][j] = scale_j * sigma_b * sum_n q_jn r^_bn for the signals listed in slots
// [0, *count) of `list` (row s of the residual operand belongs to signal list[s]); tiles past the
// count exit at once.  list == nullptr: slot s is signal s (count B).  err: set to 1 if a
// pipeline wait gave up.
void tc_launch_corr(const TcOperands& ops, int64_t K, int64_t B, int64_t ldN, const float* scale,
                    const float* sigma, const int* list, const int* count, float* Gfull, int* err,
                    cudaStream_t stream);

// Self-test: random K x N operands and B signals through the tensor-core GEMM, compared with an
// FP64 evaluation of the same products; reports the largest error relative to sum |a_i r_i|.
// mode 0: BF16, 1: E4M3, 2: split BF16 (three products, promoted accumulation).
int tc_selftest(int mode, int64_t K, int64_t N, int64_t B, double* max_rel, double* max_abs_bound_ratio);

}  // namespace lasso
