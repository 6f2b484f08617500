// lambda_max = ||A^T y||_inf for a batch of signals without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- for instance a process whose device
// memory is entirely handed to another allocator (a framework's caching pool), where a raw
// cudaMalloc can fail although the pool has room, or a latency-critical loop that must not
// pay cudaMalloc's implicit device synchronisation.  The regular entry point
// lasso_lambda_max() sizes its buffers per call and may allocate; this one uses a fixed
// scratch array compiled into the library instead.
//
// The scratch is one file-scope __device__ array (every GPU that loads the library keeps it
// until the process exits).  Host code cannot use the array's name as a device address, so
// the address is looked up once per device with cudaGetSymbolAddress and cached.
#include <cstring>
#include <mutex>

#include "dict.cuh"
#include "kernels.cuh"

namespace lasso {

// Per-block maxima of |a_j^T y_b|: (number of signals) x (atom blocks) doubles at most.
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = 1 << 20;   // 8 MiB
constexpr int NA_ATOMS_PER_BLOCK = 256;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_MAX_SMEM = 200 * 1024;    // y_b staged in shared memory

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Block (chunk, b): max over atoms [chunk * 256, chunk * 256 + 256) of |a_j^T y_b| with the
// exact level's arithmetic (FP64, or FP32 with error-free products); y_b staged in shared memory.
__global__ void __launch_bounds__(NA_THREADS)
k_noalloc_partial_max(LevelDev L, int N, int64_t ldN, int64_t K, const float* __restrict__ Y, int nchunk,
                      double* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  __shared__ double s_max[NA_THREADS / 32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool fp64a = level_fp64_arith(L.kind);
  float* yf = reinterpret_cast<float*>(na_smem);
  double* yd = reinterpret_cast<double*>(na_smem);
  for (int64_t n = threadIdx.x; n < ldN; n += NA_THREADS) {
    const float v = n < N ? Y[(int64_t)b * N + n] : 0.f;
    if (fp64a) yd[n] = (double)v;
    else yf[n] = v;
  }
  __syncthreads();
  double m = 0.0;
  const int64_t j0 = (int64_t)chunk * NA_ATOMS_PER_BLOCK;
  const int64_t j1 = j0 + NA_ATOMS_PER_BLOCK < K ? j0 + NA_ATOMS_PER_BLOCK : K;
  for (int64_t j = j0 + wid; j < j1; j += NA_THREADS / 32) {
    const double g = warp_atom_dot(L, j, (int)ldN, yf, yd, lane);
    m = fmax(m, fabs(g));
  }
  if (lane == 0) s_max[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t = fmax(t, s_max[w]);
    scratch[(int64_t)b * nchunk + chunk] = t;
  }
}

__global__ void k_noalloc_reduce(const double* __restrict__ scratch, int64_t B, int nchunk, double* __restrict__ out) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  double m = 0.0;
  for (int c = 0; c < nchunk; ++c) m = fmax(m, scratch[b * nchunk + c]);
  out[b] = m;
}

// Device address of the scratch array, looked up once per device (with that device current).
static std::mutex g_na_mutex;
static double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

static int noalloc_scratch(double** out) {
  int dev = 0;
  LASSO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) {
    set_last_error("lasso_lambda_max_noalloc: device ordinal above 63", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "null scratch address", __FILE__, __LINE__);
      return LASSO_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return LASSO_OK;
}

}  // namespace lasso

using namespace lasso;

// The exact level as k_noalloc_partial_max reads it.  warp_atom_dot on the exact FP32 / FP64
// level reads only the kind, the row stride and the atom rows, so the descriptor is filled
// from the dictionary's own fields: the regular make_level_dev() may create the level's FP32
// bound arrays on first use, which would allocate and synchronise the device.
static LevelDev exact_level_rows(const lasso_dict* d) {
  LevelDev L;
  memset(&L, 0, sizeof(L));
  L.kind = d->exact.kind;
  L.ld = d->ldN;
  L.data = d->exact.data;
  return L;
}

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_lambda_max_noalloc(const lasso_dict* d, const float* d_Y, int64_t B, double* d_out,
                                        void* stream) {
  lasso::clear_last_error();
  if (!d || !d_Y || !d_out || B <= 0) {
    set_last_error("lasso_lambda_max_noalloc: null dictionary or buffer, or B <= 0", __FILE__, __LINE__);
    return LASSO_ERR_INVALID_ARG;
  }
  if (!d->exact.data || (d->exact.kind != LK_F32 && d->exact.kind != LK_F64)) {
    set_last_error("lasso_lambda_max_noalloc: the dictionary has no dense exact level", __FILE__, __LINE__);
    return LASSO_ERR_INVALID_ARG;
  }
  int dev = -1;
  LASSO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != d->device) {
    set_last_error("lasso_lambda_max_noalloc: the current CUDA device is not the dictionary's device",
                   __FILE__, __LINE__);
    return LASSO_ERR_INVALID_ARG;
  }
  const int64_t nchunk = (d->K + NA_ATOMS_PER_BLOCK - 1) / NA_ATOMS_PER_BLOCK;
  if (B > 65535 || B * nchunk > NOALLOC_SCRATCH_DOUBLES) {
    set_last_error("lasso_lambda_max_noalloc: B * ceil(K / 256) exceeds the 1048576-entry scratch "
                   "(or B > 65535); split the batch", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  const size_t smem = (size_t)d->ldN * (d->exact.kind == LK_F64 ? 8 : 4);
  if (smem > NA_MAX_SMEM) {
    set_last_error("lasso_lambda_max_noalloc: the signal (padded length x element size) exceeds the "
                   "200 KiB of shared memory this kernel stages it in (N <= 51200 for FP32 "
                   "dictionaries, N <= 25600 for FP64)", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  const LevelDev L = exact_level_rows(d);
  cudaStream_t st = (cudaStream_t)stream;
  LASSO_CUDA_TRY(cudaFuncSetAttribute(k_noalloc_partial_max, cudaFuncAttributeMaxDynamicSharedMemorySize, NA_MAX_SMEM));
  k_noalloc_partial_max<<<dim3((unsigned)nchunk, (unsigned)B), NA_THREADS, smem, st>>>(
      L, (int)d->N, d->ldN, d->K, d_Y, (int)nchunk, scratch);
  k_noalloc_reduce<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(scratch, B, (int)nchunk, d_out);
  LASSO_CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}
