// Read bandwidth of data resident in L2, for the roofline of kernels whose operands stay in L2
// across a batch (the correlation pass re-reads a dictionary that fits in L2 once per signal).
//
// One launch reads an L2-resident buffer `rounds` times with 16-byte loads that bypass L1
// (ld.global.cg); each round starts at a rotated offset, so no SM re-reads its own lines.  The
// grid fills every SM; the time comes from CUDA events around the timed launch.
#include "common.cuh"

namespace lasso {

__global__ void __launch_bounds__(256) k_l2_read(const float4* __restrict__ buf, int64_t n4, int rounds,
                                                  float* __restrict__ sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  for (int r = 0; r < rounds; ++r) {
    const int64_t off = ((int64_t)r * 7919 * 256) % n4;
    int64_t i = tid;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      int64_t k0 = i + off, k1 = i + stride + off, k2 = i + 2 * stride + off, k3 = i + 3 * stride + off;
      if (k0 >= n4) k0 -= n4;
      if (k1 >= n4) k1 -= n4;
      if (k2 >= n4) k2 -= n4;
      if (k3 >= n4) k3 -= n4;
      const float4 v0 = __ldcg(buf + k0), v1 = __ldcg(buf + k1), v2 = __ldcg(buf + k2), v3 = __ldcg(buf + k3);
      a0 += v0.x + v0.y + v0.z + v0.w;
      a1 += v1.x + v1.y + v1.z + v1.w;
      a2 += v2.x + v2.y + v2.z + v2.w;
      a3 += v3.x + v3.y + v3.z + v3.w;
    }
    for (; i < n4; i += stride) {
      int64_t k = i + off;
      if (k >= n4) k -= n4;
      const float4 v = __ldcg(buf + k);
      a0 += v.x + v.y + v.z + v.w;
    }
  }
  // the buffer holds zeros: the store never happens, but the loads cannot be dropped
  if (a0 + a1 + a2 + a3 != 0.f) sink[0] = a0 + a1 + a2 + a3;
}

}  // namespace lasso

using namespace lasso;

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_probe_l2_read(int64_t bytes, int rounds, double* gbs) {
  lasso::clear_last_error();
  if (!gbs || bytes < (1 << 20) || bytes > ((int64_t)96 << 20) || rounds < 1 || rounds > 1000)
    return LASSO_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  LASSO_CUDA_TRY(cudaGetDevice(&dev));
  LASSO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float4* buf = nullptr;
  float* sink = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess || cudaMalloc(&sink, 16) != cudaSuccess) {
    cudaFree(buf);
    set_last_error("no device memory for the L2 probe", __FILE__, __LINE__);
    return LASSO_ERR_NOMEM;
  }
  const int64_t n4 = bytes / 16;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LASSO_OK;
  if (cudaMemset(buf, 0, bytes) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = LASSO_ERR_CUDA;
  } else {
    const int grid = sms * 8;
    k_l2_read<<<grid, 256>>>(buf, n4, 2, sink);   // brings the buffer into L2
    cudaEventRecord(e0);
    k_l2_read<<<grid, 256>>>(buf, n4, rounds, sink);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
      set_last_error(cudaGetErrorString(cudaGetLastError()), __FILE__, __LINE__);
      rc = LASSO_ERR_CUDA;
    } else {
      *gbs = (double)bytes * rounds / (ms * 1e-3) / 1e9;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(sink);
  return rc;
}
