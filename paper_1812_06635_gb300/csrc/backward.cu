// Derivative of the Lasso solution through its support system (the differentiation pattern;
// not in the paper).  From the KKT conditions of Section II, on the support S with signs s,
// A_S^T (A_S x_S - y) + lambda s = 0; for a loss gradient g = dL/dx:
//   u = (A_S^T A_S)^{-1} g_S,  dL/dy = A_S u,  dL/dA[:, S] += r u^T - (A_S u) x_S^T,  r = y - A_S x_S.
// One block per signal: support compaction, FP64 Gram (exact FP32 products), Cholesky, two
// triangular solves, then dy and the rank-2 update of dA (FP32 atomics across the batch).
#include <algorithm>
#include <vector>

#include "dict.cuh"

namespace lasso {

constexpr int BW_THREADS = 256;

__global__ void k_support_count(const float* __restrict__ X, int64_t K, int32_t* __restrict__ counts) {
  const int b = blockIdx.x;
  int c = 0;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) c += X[(int64_t)b * K + j] != 0.f;
  c = warp_sum_i(c);
  __shared__ int sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    counts[b] = t;
  }
}

__device__ __forceinline__ double exact_elem(const LevelDev& L, int64_t j, int64_t n) {
  return L.kind == LK_F64 ? ((const double*)L.data)[j * L.ld + n] : (double)((const float*)L.data)[j * L.ld + n];
}

__global__ void __launch_bounds__(BW_THREADS)
k_backward(LevelDev L, int N, int64_t K, int mmax, const float* __restrict__ Y, const float* __restrict__ X,
           const float* __restrict__ Gl, float* __restrict__ dY, float* __restrict__ dA, int32_t* __restrict__ Sbuf,
           double* __restrict__ Mbuf, double* __restrict__ vbuf) {
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = BW_THREADS / 32;
  int32_t* S = Sbuf + (int64_t)b * mmax;
  double* M = Mbuf + (int64_t)b * mmax * mmax;
  double* u = vbuf + (int64_t)b * (2 * mmax + 2 * (int64_t)N);
  double* xs = u + mmax;
  double* Au = xs + mmax;
  double* r = Au + N;
  __shared__ int s_cnt[BW_THREADS / 32];
  __shared__ int s_base;
  __shared__ double s_d;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  // ---- ordered support list
  for (int64_t t0 = 0; t0 < K; t0 += BW_THREADS) {
    const int64_t j = t0 + threadIdx.x;
    const bool nz = j < K && X[(int64_t)b * K + j] != 0.f;
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) s_cnt[wid] = __popc(bal);
    __syncthreads();
    int off = s_base;
    for (int w = 0; w < wid; ++w) off += s_cnt[w];
    if (nz) {
      const int q = off + __popc(bal & ((1u << lane) - 1u));
      S[q] = (int32_t)j;
      xs[q] = (double)X[(int64_t)b * K + j];
      u[q] = (double)Gl[(int64_t)b * K + j];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < nw; ++w) s_base += s_cnt[w];
    __syncthreads();
  }
  const int m = s_base;
  if (m == 0) {
    for (int n = threadIdx.x; n < N; n += BW_THREADS) dY[(int64_t)b * N + n] = 0.f;
    return;
  }
  // ---- Gram M = A_S^T A_S (lower triangle), warp per entry
  const int npairs = m * (m + 1) / 2;
  for (int pq = wid; pq < npairs; pq += nw) {
    int p = (int)((sqrt(8.0 * pq + 1.0) - 1.0) * 0.5);
    while ((p + 1) * (p + 2) / 2 <= pq) ++p;
    while (p * (p + 1) / 2 > pq) --p;
    const int q = pq - p * (p + 1) / 2;
    double acc = 0.0;
    for (int n = lane; n < N; n += 32) acc = fma(exact_elem(L, S[p], n), exact_elem(L, S[q], n), acc);
    acc = warp_sum(acc);
    if (lane == 0) M[(int64_t)p * mmax + q] = acc;
  }
  __syncthreads();
  // ---- Cholesky M = C C^T (lower, in place)
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double dkk = M[(int64_t)k * mmax + k];
      s_d = dkk > 0.0 ? sqrt(dkk) : 0.0;
      M[(int64_t)k * mmax + k] = s_d;
    }
    __syncthreads();
    const double dk = s_d;
    for (int i = k + 1 + threadIdx.x; i < m; i += BW_THREADS)
      M[(int64_t)i * mmax + k] = dk > 0.0 ? M[(int64_t)i * mmax + k] / dk : 0.0;
    __syncthreads();
    const int rem = m - k - 1;
    const int ntri = rem * (rem + 1) / 2;
    for (int t = threadIdx.x; t < ntri; t += BW_THREADS) {
      int i = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int jj = t - i * (i + 1) / 2;
      const int ii = k + 1 + i, j2 = k + 1 + jj;
      M[(int64_t)ii * mmax + j2] -= M[(int64_t)ii * mmax + k] * M[(int64_t)j2 * mmax + k];
    }
    __syncthreads();
  }
  // ---- solve C w = g_S, then C^T u = w (u holds g_S on entry)
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      const double dkk = M[(int64_t)k * mmax + k];
      u[k] = dkk > 0.0 ? u[k] / dkk : 0.0;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += BW_THREADS) u[i] -= M[(int64_t)i * mmax + k] * u[k];
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {
    if (threadIdx.x == 0) {
      const double dkk = M[(int64_t)k * mmax + k];
      u[k] = dkk > 0.0 ? u[k] / dkk : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += BW_THREADS) u[i] -= M[(int64_t)k * mmax + i] * u[k];
    __syncthreads();
  }
  // ---- A_S u, r = y - A_S x_S, dL/dy = A_S u
  for (int n = threadIdx.x; n < N; n += BW_THREADS) {
    double au = 0.0, ax = 0.0;
    for (int p = 0; p < m; ++p) {
      const double a = exact_elem(L, S[p], n);
      au = fma(a, u[p], au);
      ax = fma(a, xs[p], ax);
    }
    Au[n] = au;
    r[n] = (double)Y[(int64_t)b * N + n] - ax;
    dY[(int64_t)b * N + n] = (float)au;
  }
  __syncthreads();
  // ---- dL/dA[:, S] += r u^T - (A_S u) x_S^T   (row j of the atom-major gradient)
  if (dA) {
    for (int p = wid; p < m; p += nw) {
      const int64_t j = S[p];
      const double up = u[p], xp = xs[p];
      for (int n = lane; n < N; n += 32) atomicAdd(&dA[j * N + n], (float)(r[n] * up - Au[n] * xp));
    }
  }
}

}  // namespace lasso

using namespace lasso;

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_backward(lasso_dict* d, const float* d_Y, const float* d_X, const float* d_G, int64_t B,
                              float* d_dY, float* d_dA, void* stream) {
  lasso::clear_last_error();
  if (!d || !d_Y || !d_X || !d_G || !d_dY || B <= 0) return LASSO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* counts = nullptr;
  LASSO_CUDA_TRY(cudaMalloc(&counts, B * 4));
  k_support_count<<<(unsigned)B, 256, 0, st>>>(d_X, d->K, counts);
  std::vector<int32_t> hc(B);
  cudaError_t e = cudaMemcpyAsync(hc.data(), counts, B * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(counts);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  int mmax = 1;
  for (int32_t c : hc) mmax = std::max(mmax, (int)c);
  if (mmax > 1024) {
    set_last_error("lasso_backward: a signal's support exceeds 1024 atoms", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  int32_t* Sbuf = nullptr;
  double *Mbuf = nullptr, *vbuf = nullptr;
  if (cudaMalloc(&Sbuf, (size_t)B * mmax * 4) != cudaSuccess ||
      cudaMalloc(&Mbuf, (size_t)B * mmax * mmax * 8) != cudaSuccess ||
      cudaMalloc(&vbuf, (size_t)B * (2 * mmax + 2 * d->N) * 8) != cudaSuccess) {
    cudaFree(Sbuf);
    cudaFree(Mbuf);
    cudaFree(vbuf);
    return LASSO_ERR_NOMEM;
  }
  LevelDev L = make_level_dev(d, d->exact);
  k_backward<<<(unsigned)B, BW_THREADS, 0, st>>>(L, (int)d->N, d->K, mmax, d_Y, d_X, d_G, d_dY, d_dA, Sbuf, Mbuf, vbuf);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(Sbuf);
  cudaFree(Mbuf);
  cudaFree(vbuf);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  return LASSO_OK;
}
