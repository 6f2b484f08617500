// The screened FISTA solve on the device: one pass = residual -> correlation fused with the
// proximal update and partial reductions -> gap / dual scaling / stable safe test / switch /
// ordered compaction of the preserved set -> work-item schedule.  Passes are captured in a
// CUDA graph and replayed until every signal has stopped.
//
// Paper: Algorithm 1 (FastL1) and Algorithm 2 (SwitchDictionary); dual points
// eq:theta_dynamic_approx; stable GAP Safe sphere Theorem 1 / Table I; gap ratio
// eq:DefRatioSwitch; look-ahead estimate eq:DefCardinalEstimated; ISTA update
// eq:ISTA_update (FISTA momentum of Beck & Teboulle); stopping rule of Section IV.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <vector>

#include "dict.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace lasso {

constexpr int SCREEN_THREADS = 256;
constexpr int FULL_SET = MAX_LEVELS - 1;    // slot list of the signals under the full-dictionary check
constexpr int CORR_THREADS = 256;
constexpr int RES_ROWS = RES_THREADS * 4;   // rows per residual block
constexpr int GEMM_T = 64;                  // tile of the Kronecker small GEMMs
constexpr int FULL_ITEM_MULT = 8;           // correlation items of levels gathered from a batched product
constexpr double FP32_TOL_FLOOR = 5e-7;     // smallest tolerance solved with FP32 iterates

struct Workspace {
  int64_t B = 0, K = 0, ldN = 0;
  bool vt_double = false;
  bool kron = false;
  int R = 0, N1 = 0, K1 = 0, N2 = 0, K2 = 0;
  void* Yw = nullptr;
  void* Rho = nullptr;
  void* X = nullptr;
  void* Z = nullptr;
  void* G = nullptr;
  void* Xout = nullptr;
  void* nz_val = nullptr;
  int32_t* nz_idx = nullptr;
  int32_t* kept = nullptr;           // 2 x B x K
  uint8_t* mask = nullptr;           // B x K, 1 while the atom is preserved
  int32_t* cand_idx = nullptr;       // B x K, nonzeros of the point awaiting the full check
  void* cand_val = nullptr;          // B x K
  int32_t* offsets2 = nullptr;       // B + 1, work items of the full-dictionary checks
  double* part_full = nullptr;       // B x nch
  float* c0ub = nullptr;             // B x K, |a_j^T y| upper bounds (Dynamic Safe rule)
  double* part_res = nullptr;        // B x nrb x 2
  double* part_corr = nullptr;       // B x nch x 2
  int32_t* offsets = nullptr;        // B + 1
  int32_t* live_list = nullptr;      // B: the signals still running, in order (k_schedule)
  int32_t* counters = nullptr;       // [0] done count, [1] stop flag, [2] chunk, [4] live count,
                                     // [5] preserved atoms of the live signals, [8 + l] signals
                                     // on tensor-core level l
  double* alg_bytes = nullptr;       // [6] algorithmic bytes per kernel kind
  SigState* st = nullptr;
  // Kronecker scratch
  float* Gfull = nullptr;            // B x K
  float* AZ = nullptr;               // B x ldN
  float* Xd = nullptr;               // B x K
  float* Tk = nullptr;               // B x R x max(K1 N2, N1 K2)
  float* Fs = nullptr;               // sparse-factor levels: B x 2 x fdim scratch vectors
  int64_t fs_ld = 0;                 // floats of scratch per signal
  void* rq[MAX_LEVELS] = {nullptr};  // tensor-core levels: quantised residuals (B slots x ldN)
  void* rq2[MAX_LEVELS] = {nullptr}; // split exact level: second BF16 part of the residuals
  float* rsig[MAX_LEVELS] = {nullptr};
  int32_t* tc_slot = nullptr;        // MAX_LEVELS x B: slot of signal b on level l (or -1)
  int32_t* tc_list = nullptr;        // MAX_LEVELS x B: signal in slot s of level l
  int* tc_err = nullptr;
  int32_t* h_counters = nullptr;     // pinned
  cudaStream_t stream = nullptr;     // used when the caller passes the legacy default stream
  int nrb = 0, nch = 0;
};

void free_ws(Workspace* w) {
  if (!w) return;
  void* ptrs[] = {w->Yw, w->Rho, w->X, w->Z, w->G, w->Xout, w->nz_val, w->nz_idx, w->kept, w->c0ub,
                  w->mask, w->cand_idx, w->cand_val, w->offsets2, w->part_full,
                  w->part_res, w->part_corr, w->offsets, w->live_list, w->counters, w->alg_bytes, w->st, w->Gfull,
                  w->AZ, w->Xd, w->Tk,
                  w->Fs};
  for (void* p : ptrs) cudaFree(p);
  for (int l = 0; l < MAX_LEVELS; ++l) {
    cudaFree(w->rq[l]);
    cudaFree(w->rq2[l]);
    cudaFree(w->rsig[l]);
  }
  cudaFree(w->tc_slot);
  cudaFree(w->tc_list);
  cudaFree(w->tc_err);
  cudaFreeHost(w->h_counters);
  if (w->stream) cudaStreamDestroy(w->stream);
  delete w;
}

static int ws_alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return LASSO_ERR_NOMEM;
  }
  return LASSO_OK;
}

static int get_ws(lasso_dict* d, int64_t B, bool vt_double, Workspace** out) {
  Workspace*& slot = vt_double ? d->ws64 : d->ws;
  Workspace* w = slot;
  if (w && w->B >= B) {
    *out = w;
    return LASSO_OK;
  }
  if (w) free_ws(w);
  slot = nullptr;
  w = new Workspace();
  w->B = B;
  w->K = d->K;
  w->ldN = d->ldN;
  w->vt_double = vt_double;
  w->kron = d->is_kron;
  w->R = d->R;
  w->N1 = d->N1;
  w->K1 = d->K1;
  w->N2 = d->N2;
  w->K2 = d->K2;
  w->nrb = (int)((d->N + RES_ROWS - 1) / RES_ROWS);
  w->nch = (int)((d->K + CORR_CHUNK - 1) / CORR_CHUNK);
  const size_t vs = vt_double ? 8 : 4;
  const size_t BK = (size_t)B * d->K, BN = (size_t)B * d->ldN;
  int rc = 0;
  rc |= ws_alloc(&w->Yw, BN * vs);
  rc |= ws_alloc(&w->Rho, BN * vs);
  rc |= ws_alloc(&w->X, BK * vs);
  rc |= ws_alloc(&w->Z, BK * vs);
  rc |= ws_alloc(&w->G, BK * vs);
  rc |= ws_alloc(&w->Xout, BK * vs);
  rc |= ws_alloc(&w->nz_val, BK * vs);
  rc |= ws_alloc((void**)&w->nz_idx, BK * 4);
  rc |= ws_alloc((void**)&w->kept, 2 * BK * 4);
  rc |= ws_alloc((void**)&w->mask, BK);
  rc |= ws_alloc((void**)&w->cand_idx, BK * 4);
  rc |= ws_alloc(&w->cand_val, BK * vs);
  rc |= ws_alloc((void**)&w->offsets2, (size_t)(B + 1) * 4);
  rc |= ws_alloc((void**)&w->part_full, (size_t)B * w->nch * 8);
  rc |= ws_alloc((void**)&w->c0ub, BK * 4);
  rc |= ws_alloc((void**)&w->part_res, (size_t)B * w->nrb * 2 * 8);
  rc |= ws_alloc((void**)&w->part_corr, (size_t)B * w->nch * 2 * 8);
  rc |= ws_alloc((void**)&w->offsets, (size_t)(B + 1) * 4);
  rc |= ws_alloc((void**)&w->live_list, (size_t)B * 4);
  rc |= ws_alloc((void**)&w->counters, 64);
  rc |= ws_alloc((void**)&w->alg_bytes, 16 * sizeof(double));   // [0,6) bytes, [8,16) atom-passes per level
  rc |= ws_alloc((void**)&w->st, (size_t)B * sizeof(SigState));
  rc |= ws_alloc((void**)&w->tc_slot, (size_t)MAX_LEVELS * B * 4);
  rc |= ws_alloc((void**)&w->tc_list, (size_t)MAX_LEVELS * B * 4);
  if (d->is_kron) {
    const size_t tk = (size_t)B * d->R * std::max<int64_t>((int64_t)d->K1 * d->N2, (int64_t)d->N1 * d->K2);
    rc |= ws_alloc((void**)&w->Gfull, BK * 4);
    rc |= ws_alloc((void**)&w->AZ, BN * 4);
    rc |= ws_alloc((void**)&w->Xd, BK * 4);
    rc |= ws_alloc((void**)&w->Tk, tk * 4);
  }
  if (d->faust_dim > 0) {
    w->fs_ld = 2 * (int64_t)d->faust_dim;
    if (!w->Gfull) rc |= ws_alloc((void**)&w->Gfull, BK * 4);
    if (!w->AZ) rc |= ws_alloc((void**)&w->AZ, BN * 4);
    rc |= ws_alloc((void**)&w->Fs, (size_t)B * w->fs_ld * 4);
  }
  rc |= ws_alloc((void**)&w->tc_err, 16);
  if (cudaHostAlloc((void**)&w->h_counters, 64, cudaHostAllocDefault) != cudaSuccess) rc |= 1;
  if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) rc |= 1;
  if (rc) {
    free_ws(w);
    return LASSO_ERR_NOMEM;
  }
  slot = w;
  *out = w;
  return LASSO_OK;
}

// Pointers of the current pass (kernel parameter block).
template <typename VT>
struct PassArgs {
  DictDev dd;
  SolveParams sp;
  const VT* Yw;
  VT* Rho;
  VT* X;
  VT* Z;
  VT* G;
  VT* Xout;
  VT* nz_val;
  int32_t* nz_idx;
  int32_t* kept;
  uint8_t* mask;
  int32_t* cand_idx;
  VT* cand_val;
  int32_t* offsets2;
  double* part_full;
  float* c0ub;
  double* part_res;
  double* part_corr;
  int32_t* offsets;
  int32_t* live_list;
  int32_t* counters;
  double* alg_bytes;
  SigState* st;
  float* Gfull;
  float* AZ;
  float* Xd;
  float* Tk;
  float* Fs;
  int64_t fs_ld;
  int32_t* tc_slot;
  int32_t* tc_list;
  int64_t K, ldN;
  int nrb, nch;
};

__device__ __forceinline__ double level_elem_bytes(int kind) {
  switch (kind) {
    case LK_F64: return 8.0;
    case LK_F32:
    case LK_F32D: return 4.0;
    case LK_BF16: return 2.0;
    case LK_FP8: return 1.0;
  }
  return 0.0;
}

template <typename VT>
__device__ __forceinline__ int32_t* kept_of(const PassArgs<VT>& a, int b, int parity) {
  return a.kept + ((int64_t)parity * a.sp.B + b) * a.K;
}

// Every workspace pointer of a pass (one place, so no entry point can leave one unset).
template <typename VT>
static void fill_pass_args(PassArgs<VT>& pa, Workspace* w, const lasso_dict* d) {
  pa.Yw = (const VT*)w->Yw;
  pa.Rho = (VT*)w->Rho;
  pa.X = (VT*)w->X;
  pa.Z = (VT*)w->Z;
  pa.G = (VT*)w->G;
  pa.Xout = (VT*)w->Xout;
  pa.nz_val = (VT*)w->nz_val;
  pa.nz_idx = w->nz_idx;
  pa.kept = w->kept;
  pa.mask = w->mask;
  pa.cand_idx = w->cand_idx;
  pa.cand_val = (VT*)w->cand_val;
  pa.offsets2 = w->offsets2;
  pa.part_full = w->part_full;
  pa.c0ub = w->c0ub;
  pa.part_res = w->part_res;
  pa.part_corr = w->part_corr;
  pa.offsets = w->offsets;
  pa.live_list = w->live_list;
  pa.counters = w->counters;
  pa.alg_bytes = w->alg_bytes;
  pa.st = w->st;
  pa.Gfull = w->Gfull;
  pa.AZ = w->AZ;
  pa.Xd = w->Xd;
  pa.Tk = w->Tk;
  pa.Fs = w->Fs;
  pa.fs_ld = w->fs_ld;
  pa.tc_slot = w->tc_slot;
  pa.tc_list = w->tc_list;
  pa.K = d->K;
  pa.ldN = d->ldN;
  pa.nrb = w->nrb;
  pa.nch = w->nch;
}

// ------------------------------------------------------------------ init

// ||y||^2, ||y||, FISTA scalars; the preserved set starts as every atom.
template <typename VT>
__global__ void k_init_state(PassArgs<VT> a, const double* __restrict__ lambdas) {
  const int b = blockIdx.x;
  const VT* y = a.Yw + (int64_t)b * a.ldN;
  double s = 0.0;
  for (int n = threadIdx.x; n < a.dd.N; n += blockDim.x) s = fma((double)y[n], (double)y[n], s);
  __shared__ double sh[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  int32_t* kp = kept_of(a, b, 0);
  uint8_t* mk = a.mask + (int64_t)b * a.K;
  for (int64_t j = threadIdx.x; j < a.K; j += blockDim.x) {
    kp[j] = (int32_t)j;
    mk[j] = 1;
  }
  if (threadIdx.x == 0) {
    double yy = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) yy += sh[w];
    SigState st;
    memset(&st, 0, sizeof(st));
    st.lam = lambdas ? lambdas[b] : 1.0;   // null: relative lambda 1 (lambda_max only)
    st.yy = yy;
    st.ynorm = sqrt(yy);
    st.t = 1.0;
    st.beta = 0.0;
    st.level = 0;
    st.n_kept = (int)a.K;
    st.n_chunks = (int)((a.K + a.sp.chunk - 1) / a.sp.chunk);
    st.gap = INFINITY;
    st.best_cert = INFINITY;
    st.status = LASSO_OK;
    if (!(yy < INFINITY) || !(st.lam == st.lam)) {
      st.status = LASSO_ERR_NONFINITE;
      st.done = 1;
    } else if (yy == 0.0) {
      st.done = 1;         // y = 0: x* = 0 with gap 0
      st.gap = 0.0;
      st.n_kept = 0;
    }
    a.st[b] = st;
  }
}

// The schedule of the next pass, in one sweep over the batch (each signal's state read once):
// the correlation work items of the live signals (prefix sums in offsets), the compacted list of
// live signals, the slots of the live signals on each tensor-core level (the rows of that level's
// quantised residual operand, so its GEMM covers only ceil(count / 256) signal tiles), the done
// count, and the pass's chunk: the tuned one, halved (down to 32) while the preserved atoms of the
// live signals would give fewer than two items per block (dyn; from the previous schedule's total).
template <typename VT>
__global__ void __launch_bounds__(1024) k_schedule(PassArgs<VT> a, int dyn) {
  constexpr int NW = 32;
  __shared__ int w_items[NW], w_live[NW], w_lvl[MAX_LEVELS][NW];
  __shared__ long long w_kept[NW];
  __shared__ int t_items, t_live, t_lvl[MAX_LEVELS];
  __shared__ long long t_kept;
  __shared__ int c_items, c_live, c_lvl[MAX_LEVELS];
  __shared__ long long c_kept;
  const int B = a.sp.B;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nl = a.dd.n_levels;
  int chunk = a.sp.chunk;
  if (dyn && sizeof(VT) == 4) {
    const long long t = a.counters[5];
    while (chunk > CORR_CHUNK && t / chunk < 2LL * a.sp.corr_grid) chunk >>= 1;
  }
  if (threadIdx.x == 0) {
    c_items = c_live = 0;
    c_kept = 0;
    for (int l = 0; l < MAX_LEVELS; ++l) c_lvl[l] = 0;
    a.counters[2] = chunk;
  }
  __syncthreads();
  for (int base = 0; base < B; base += blockDim.x) {
    const int b = base + threadIdx.x;
    bool live = false;
    int items = 0, lvl = -1;
    long long nk = 0;
    if (b < B) {
      const SigState& s = a.st[b];
      live = !s.done;
      if (live) {
        lvl = s.level;
        nk = s.n_kept;
        // the FP32 pass gathers the levels formed by a batched product with FULL_ITEM_MULT times
        // larger items; the initial pass and FP64 iterates use the chunk
        const LevelDev& L = a.dd.lv[lvl];
        const int ch = dyn && sizeof(VT) == 4 && (level_structured(L.kind) || L.tc) ? chunk * FULL_ITEM_MULT : chunk;
        items = (int)((nk + ch - 1) / ch);
      }
    }
    int v = items;   // inclusive warp scan of the items
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    long long kw = nk;
#pragma unroll
    for (int m = 16; m; m >>= 1) kw += __shfl_xor_sync(0xffffffffu, kw, m);
    const unsigned lt = (1u << lane) - 1u;
    const unsigned bl = __ballot_sync(0xffffffffu, live);
    unsigned bll[MAX_LEVELS];
#pragma unroll
    for (int l = 0; l < MAX_LEVELS; ++l) bll[l] = __ballot_sync(0xffffffffu, live && lvl == l);
    if (lane == 31) w_items[wid] = v;
    if (lane == 0) {
      w_live[wid] = __popc(bl);
      w_kept[wid] = kw;
#pragma unroll
      for (int l = 0; l < MAX_LEVELS; ++l) w_lvl[l][wid] = __popc(bll[l]);
    }
    __syncthreads();
    if (wid == 0) {
      // exclusive scans over the warps (one lane per warp) and the sweep's totals
      const int nw = (int)(blockDim.x >> 5);
      int xi = lane < nw ? w_items[lane] : 0, xl = lane < nw ? w_live[lane] : 0;
      long long xk = lane < nw ? w_kept[lane] : 0;
      int xv[MAX_LEVELS];
#pragma unroll
      for (int l = 0; l < MAX_LEVELS; ++l) xv[l] = lane < nw ? w_lvl[l][lane] : 0;
      int si = xi, sl = xl, sv[MAX_LEVELS];
#pragma unroll
      for (int l = 0; l < MAX_LEVELS; ++l) sv[l] = xv[l];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int ti = __shfl_up_sync(0xffffffffu, si, o), tl = __shfl_up_sync(0xffffffffu, sl, o);
        if (lane >= o) {
          si += ti;
          sl += tl;
        }
#pragma unroll
        for (int l = 0; l < MAX_LEVELS; ++l) {
          const int tv = __shfl_up_sync(0xffffffffu, sv[l], o);
          if (lane >= o) sv[l] += tv;
        }
      }
#pragma unroll
      for (int m = 16; m; m >>= 1) xk += __shfl_xor_sync(0xffffffffu, xk, m);
      if (lane < nw) {
        w_items[lane] = si - xi;
        w_live[lane] = sl - xl;
#pragma unroll
        for (int l = 0; l < MAX_LEVELS; ++l) w_lvl[l][lane] = sv[l] - xv[l];
      }
      if (lane == 31) {
        t_items = si;
        t_live = sl;
#pragma unroll
        for (int l = 0; l < MAX_LEVELS; ++l) t_lvl[l] = sv[l];
      }
      if (lane == 0) t_kept = xk;
    }
    __syncthreads();
    if (b < B) {
      a.offsets[b] = c_items + w_items[wid] + v - items;
      if (live) a.live_list[c_live + w_live[wid] + __popc(bl & lt)] = b;
      for (int l = 0; l < nl; ++l) {
        if (!a.dd.lv[l].tc) continue;
        const bool on = live && lvl == l;
        const int slot = c_lvl[l] + w_lvl[l][wid] + __popc(bll[l] & lt);
        a.tc_slot[(int64_t)l * B + b] = on ? slot : -1;
        if (on) a.tc_list[(int64_t)l * B + slot] = b;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      c_items += t_items;
      c_live += t_live;
      c_kept += t_kept;
      for (int l = 0; l < MAX_LEVELS; ++l) c_lvl[l] += t_lvl[l];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.offsets[B] = c_items;
    a.counters[0] = B - c_live;   // signals done
    a.counters[4] = c_live;
    a.counters[5] = (int)min(c_kept, (long long)INT_MAX);   // preserved atoms of the live signals
    for (int l = 0; l < nl; ++l)
      if (a.dd.lv[l].tc) a.counters[8 + l] = c_lvl[l];
  }
}

// ------------------------------------------------------------------ residual (dense levels)

// rho^_b = y_b - sum_{j in nz(z_b)} z_bj a~_j, one block per signal (4 rows per thread per row
// group), plus ||rho^||^2 and y^T rho^, which the block finishes itself: the pass scalars land in
// the signal's state (FP64 rr, yr; FP32 ||rho^|| rounded up, lam / L and the FISTA momentum).
// Float iterates keep every per-row operation in FP32 (FP64 runs at 1/64 of the FP32 rate):
// compensated (double-float) sums stand in for FP64 accumulators.
template <typename VT>
__device__ __forceinline__ void residual_signal(const PassArgs<VT>& a, int b) {
  SigState* sp = a.st + b;
  __shared__ int s_live;
  __shared__ int32_t s_idx[RES_THREADS];
  __shared__ float s_wf[RES_THREADS];
  __shared__ double s_wd[RES_THREADS];
  __shared__ double s_red[4][RES_THREADS / 32];
  if (threadIdx.x == 0) s_live = !sp->done;
  __syncthreads();
  if (!s_live) return;
  const int lvl = sp->level, nnz = sp->n_nz;
  const bool tight = sp->res_tight != 0;
  const LevelDev& L = a.dd.lv[lvl];
  const VT* y = a.Yw + (int64_t)b * a.ldN;
  VT* rho = a.Rho + (int64_t)b * a.ldN;
  const int32_t* nzi = a.nz_idx + (int64_t)b * a.K;
  const VT* nzv = a.nz_val + (int64_t)b * a.K;
  const int N = (int)a.dd.N, ldN = (int)a.ldN;
  const int ngroups = (ldN + RES_THREADS * 4 - 1) / (RES_THREADS * 4);
  // FP64 data arithmetic (FP64 level, or FP32 data with FP64 accumulation) or FP64 iterates on
  // a float level: FP64 sums of the residual
  const bool fp64a = level_fp64_arith(L.kind);
  const bool dsum = fp64a || sizeof(VT) == 8;
  DF rrf, yrf;
  rrf.init();
  yrf.init();
  double rrd = 0.0, yrd = 0.0;
  for (int grp = 0; grp < ngroups; ++grp) {
    const int r0 = grp * RES_THREADS * 4 + threadIdx.x * 4;
    const bool active = r0 < N;
    if (fp64a) {
      double out[4] = {0.0, 0.0, 0.0, 0.0};
      if (level_structured(L.kind)) {
        if (active) {
          const float* az = a.AZ + (int64_t)b * a.ldN;
#pragma unroll
          for (int v = 0; v < 4; ++v) out[v] = (double)y[r0 + v] - (double)az[r0 + v];
        }
      } else {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int base = 0; base < nnz; base += RES_THREADS) {
          __syncthreads();
          if (base + threadIdx.x < nnz) {
            s_idx[threadIdx.x] = nzi[base + threadIdx.x];
            s_wd[threadIdx.x] = (double)nzv[base + threadIdx.x];
          }
          __syncthreads();
          const int cnt = min(RES_THREADS, nnz - base);
          if (active)
            for (int q = 0; q < cnt; ++q) {
              const D4 av = load4_d(L, s_idx[q], r0);
              const double w = s_wd[q];
              acc[0] = fma(w, av.x, acc[0]);
              acc[1] = fma(w, av.y, acc[1]);
              acc[2] = fma(w, av.z, acc[2]);
              acc[3] = fma(w, av.w, acc[3]);
            }
        }
        if (active)
#pragma unroll
          for (int v = 0; v < 4; ++v) out[v] = (double)y[r0 + v] - acc[v];
      }
      if (r0 < ldN) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (r0 + v < N) {
            const VT r = (VT)out[v];
            rho[r0 + v] = r;
            rrd = fma((double)r, (double)r, rrd);
            yrd = fma((double)y[r0 + v], (double)r, yrd);
          } else {
            rho[r0 + v] = (VT)0;
          }
        }
      }
      continue;
    }
    // FP32 iterates on a float level: double-float accumulation of the products (Dot2 on the
    // exact FP32 level, exact pairs on BF16 / FP8), FP32 result y - (s + c)
    DF acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v].init();
    if (level_structured(L.kind)) {
      if (active) {
        const float* az = a.AZ + (int64_t)b * a.ldN;
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v].s = az[r0 + v];
      }
    } else {
      float p[4] = {0.f, 0.f, 0.f, 0.f};
      int parity = 0;
      for (int base = 0; base < nnz; base += RES_THREADS) {
        __syncthreads();
        if (base + threadIdx.x < nnz) {
          const int32_t j = nzi[base + threadIdx.x];
          float w = (float)nzv[base + threadIdx.x];
          if (L.kind == LK_FP8) w = __fmul_rn(w, L.scale[j]);
          s_idx[threadIdx.x] = j;
          s_wf[threadIdx.x] = w;
        }
        __syncthreads();
        const int cnt = min(RES_THREADS, nnz - base);
        if (active && (L.kind == LK_F32 || sizeof(VT) == 4)) {
          // Dot2 once the certificate needs it, plain FMA chains before
          const bool d2 = L.kind == LK_F32 && tight;
          if (L.kind == LK_F32) res_accumulate<LK_F32>(L, s_idx, s_wf, cnt, r0, d2, acc);
          else if (L.kind == LK_BF16) res_accumulate<LK_BF16>(L, s_idx, s_wf, cnt, r0, false, acc);
          else res_accumulate<LK_FP8>(L, s_idx, s_wf, cnt, r0, false, acc);
        } else if (active) {
          for (int q = 0; q < cnt; ++q) {
            const float4 av = load4_f(L, s_idx[q], r0);
            const float w = s_wf[q];
            if (parity == 0) {
              p[0] = __fmul_rn(w, av.x);
              p[1] = __fmul_rn(w, av.y);
              p[2] = __fmul_rn(w, av.z);
              p[3] = __fmul_rn(w, av.w);
            } else {
              acc[0].add(__fmaf_rn(w, av.x, p[0]));
              acc[1].add(__fmaf_rn(w, av.y, p[1]));
              acc[2].add(__fmaf_rn(w, av.z, p[2]));
              acc[3].add(__fmaf_rn(w, av.w, p[3]));
            }
            parity ^= 1;
          }
        }
      }
      if (active && parity) {
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v].add(p[v]);
      }
    }
    if (sizeof(VT) == 8 && r0 < ldN) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (r0 + v < N) {
          const double out = (double)y[r0 + v] - acc[v].value();
          const VT r = (VT)out;
          rho[r0 + v] = r;
          rrd = fma((double)r, (double)r, rrd);
          yrd = fma((double)y[r0 + v], (double)r, yrd);
        } else {
          rho[r0 + v] = (VT)0;
        }
      }
    } else if (r0 < ldN) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (r0 + v < N) {
          const float yv = (float)y[r0 + v];
          // y - (s + c): TwoSum of y - s, then the small terms
          float t, e;
          two_sum(yv, -acc[v].s, t, e);
          const float r = __fadd_rn(t, __fsub_rn(e, acc[v].c));
          rho[r0 + v] = (VT)r;
          dot2_add(rrf, r, r);
          dot2_add(yrf, yv, r);
        } else {
          rho[r0 + v] = (VT)0;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (dsum) {
    rrd = warp_sum(rrd);
    yrd = warp_sum(yrd);
    if (lane == 0) {
      s_red[0][wid] = rrd;
      s_red[1][wid] = 0.0;
      s_red[2][wid] = yrd;
      s_red[3][wid] = 0.0;
    }
  } else {
    rrf = df_warp_reduce(rrf);
    yrf = df_warp_reduce(yrf);
    if (lane == 0) {
      s_red[0][wid] = rrf.s;
      s_red[1][wid] = rrf.c;
      s_red[2][wid] = yrf.s;
      s_red[3][wid] = yrf.c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rr = 0.0, yr = 0.0;
    for (int w = 0; w < RES_THREADS / 32; ++w) {
      rr += s_red[0][w] + s_red[1][w];
      yr += s_red[2][w] + s_red[3][w];
    }
    sp->rr = rr;
    sp->yr = yr;
    sp->res_used = tight ? 1 : 0;
    sp->nrho_ru = __double2float_ru(sqrt(rr));
    sp->thr_f = (float)(sp->lam * a.sp.inv_L);
    sp->beta_f = (float)sp->beta;
    if (a.alg_bytes && !level_structured(L.kind)) {
      // nonzero atoms of z (rows of A~), their values and indices, y read and rho written
      const double vs = (double)sizeof(VT);
      atomicAdd(&a.alg_bytes[0], (double)nnz * ((double)N * level_elem_bytes(L.kind) + 4.0 + vs) + 2.0 * N * vs);
    }
  }
}

// Over the live signals (k_schedule's list), one signal per block: launched with one block per
// signal of the batch, the live signals take the first blocks and the hardware balances them.
template <typename VT>
__global__ void __launch_bounds__(RES_THREADS) k_residual(PassArgs<VT> a) {
  const int n = a.counters[4];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    residual_signal<VT>(a, a.live_list[i]);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ correlation + update

enum CorrMode { CORR_PASS = 0, CORR_INIT = 1, CORR_CERT = 2 };

// Correlations g_j = a~_j^T rho^ over one chunk of the preserved list, fused with the FISTA
// update of the chunk's coefficients and with the chunk's maxima max(|g_j| + eps_j ||rho||)
// and max |g_j| (the two dual scalings).  Persistent grid over (signal, chunk) items.
// CORR_INIT: rho := y over every atom with the most precise level (lambda_max, a^T y bounds).
// CORR_CERT: every atom with the most precise level, no update (full-dictionary certificate).
template <typename VT, int MODE>
__global__ void __launch_bounds__(CORR_THREADS) k_corr(PassArgs<VT> a) {
  __shared__ double s_m1[CORR_THREADS / 32], s_m2[CORR_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int B = a.sp.B;
  const int total = a.offsets[B];
  const int ldN = (int)a.ldN;
  const int CH = a.sp.chunk;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    // signal of this item: last b with offsets[b] <= item
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (a.offsets[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    const int b = lo;
    const int chunk = item - a.offsets[b];
    const SigState& s = a.st[b];
    const int lvl = MODE == CORR_PASS ? s.level : a.dd.n_levels - 1;
    const LevelDev& L = a.dd.lv[lvl];
    const bool fp64a = level_fp64_arith(L.kind);
    const int npos = MODE == CORR_PASS ? s.n_kept : (int)a.K;
    const int p0 = chunk * CH, p1 = min(npos, p0 + CH);
    const VT* src = (MODE == CORR_INIT ? a.Yw : a.Rho) + (int64_t)b * a.ldN;
    double rr = 0.0;
    if (MODE == CORR_INIT) {
      rr = s.yy;
    } else {
      rr = s.rr;
    }
    const double nrho = sqrt(rr);
    const double ug = fp64a && sizeof(VT) == 8 ? U64 : U32;
    // the bulk pass bounds its rounding with gam_corr; INIT / CERT use the tight products
    const double gam = MODE == CORR_PASS ? L.gam_corr : L.gam_tight;
    const double inv_L = 1.0 / a.sp.L;
    const double thr = s.lam * inv_L;
    const int32_t* kp = kept_of(a, b, s.parity);
    VT* X = a.X + (int64_t)b * a.K;
    VT* Z = a.Z + (int64_t)b * a.K;
    VT* G = a.G + (int64_t)b * a.K;
    // per-atom epilogue: FP32 arithmetic for FP32 iterates (directed rounding keeps m1 an upper
    // bound); FP64 only when the iterates are FP64
    const float nrho_f = __double2float_ru(nrho);
    const float ga_fac = 1.0000004f;   // >= 1 + 3 u32, rounded up
    const float inv_Lf = (float)inv_L, thr_f = (float)thr, beta_f = (float)s.beta;
    double m1 = 0.0, m2 = 0.0;
    float m1f = 0.f, m2f = 0.f;
    const bool pair = MODE == CORR_PASS && !L.tc && (L.kind == LK_F32 || L.kind == LK_BF16 || L.kind == LK_FP8);
    const bool from_full = level_structured(L.kind) || (MODE == CORR_PASS && L.tc);
    const float dq_f = from_full && L.tc ? __double2float_ru(s.dq * 1.001) : 0.f;
    constexpr int NW = CORR_THREADS / 32;
    for (int base = p0 + wid; base < p1; base += (pair ? 2 : 1) * NW) {
      double gg[2] = {0.0, 0.0};
      int64_t jj[2] = {0, 0};
      int npair = 1;
      jj[0] = MODE == CORR_PASS ? kp[base] : base;
      if (pair && base + NW < p1) {
        npair = 2;
        jj[1] = kp[base + NW];
        float f0, f1;
        warp_atom_dot2_fast<VT>(L, jj[0], jj[1], ldN, src, lane, f0, f1);
        gg[0] = f0;
        gg[1] = f1;
      } else if (from_full) {
        gg[0] = (double)a.Gfull[(int64_t)b * a.K + jj[0]];
      } else if (MODE == CORR_PASS) {
        gg[0] = warp_atom_dot_fast<VT>(L, jj[0], ldN, src, lane);
      } else {
        gg[0] = warp_atom_dot(L, jj[0], ldN, reinterpret_cast<const float*>(src), reinterpret_cast<const double*>(src),
                              lane);
      }
      if (lane != 0) continue;
      for (int q = 0; q < npair; ++q) {
        const int64_t j = jj[q];
        const int pos = base + q * NW;
        if constexpr (sizeof(VT) == 4) {
          const float g = (float)gg[q];
          const float ag = fabsf(g);
          // eps_j + gam kappa_j (FP32, rounded up); the INIT / CERT passes use the tight bound
          const float er = MODE == CORR_PASS ? L.epsr32[j]
                                             : __double2float_ru(L.eps[j] + gam * L.kappa[j]);
          float ub = __fmaf_ru(er, nrho_f, __fmul_ru(ag, ga_fac));
          if (dq_f > 0.f) ub = __fmaf_ru(L.kappa32[j], dq_f, ub);
          if (MODE == CORR_PASS) {
            m1f = fmaxf(m1f, ub);
            m2f = fmaxf(m2f, ag);
          } else {
            // INIT / CERT keep the unrounded error-free value (lambda_max, audit)
            m1 = fmax(m1, fabs(gg[q]) * (1.0 + 4.0 * U64) + (L.eps[j] + gam * L.kappa[j]) * nrho);
            m2 = fmax(m2, fabs(gg[q]));
          }
          if (MODE == CORR_INIT) {
            if (a.c0ub) a.c0ub[(int64_t)b * a.K + j] = ub;
          } else if (MODE == CORR_PASS) {
            const float xj = (float)X[j];
            const float zj = (float)Z[j];
            const float v = __fmaf_rn(g, inv_Lf, zj);
            const float xn = v > thr_f ? v - thr_f : (v < -thr_f ? v + thr_f : 0.f);
            const float zn = a.sp.algo == LASSO_FISTA ? __fmaf_rn(beta_f, xn - xj, xn) : xn;
            X[j] = (VT)xn;
            Z[j] = (VT)zn;
            G[pos] = (VT)g;
          }
        } else {
          const double g = gg[q];
          const double ga = fabs(g) * (1.0 + 3.0 * ug);
          const double epsr = L.eps[j] + gam * L.kappa[j];
          m1 = fmax(m1, ga + epsr * nrho + (dq_f > 0.f ? L.kappa[j] * s.dq * 1.001 : 0.0));
          m2 = fmax(m2, fabs(g));
          if (MODE == CORR_INIT) {
            if (a.c0ub) a.c0ub[(int64_t)b * a.K + j] = __double2float_ru(ga + epsr * nrho);
          } else if (MODE == CORR_PASS) {
            const double xj = (double)X[j];
            const double zj = (double)Z[j];
            const double v = zj + g * inv_L;
            const double xn = v > thr ? v - thr : (v < -thr ? v + thr : 0.0);
            const double zn = a.sp.algo == LASSO_FISTA ? xn + s.beta * (xn - xj) : xn;
            X[j] = (VT)xn;
            Z[j] = a.sp.z_f32 ? (VT)(float)zn : (VT)zn;
            G[pos] = (VT)g;
          }
        }
      }
    }
    if constexpr (sizeof(VT) == 4) {
      if (MODE == CORR_PASS) {
        m1 = m1f;
        m2 = m2f;
      }
    }
    if (lane == 0) {
      s_m1[wid] = m1;
      s_m2[wid] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < CORR_THREADS / 32; ++w) {
        t1 = fmax(t1, s_m1[w]);
        t2 = fmax(t2, s_m2[w]);
      }
      double* pc = a.part_corr + ((int64_t)b * a.nch + chunk) * 2;
      pc[0] = t1;
      pc[1] = t2;
      if (MODE == CORR_PASS && a.alg_bytes && !level_structured(L.kind) && !L.tc) {
        // preserved atoms of the chunk (rows of A~, index, x and z read and written, g written),
        // plus rho once per signal
        const double vs = (double)sizeof(VT);
        atomicAdd(&a.alg_bytes[1], (double)(p1 - p0) * ((double)a.dd.N * level_elem_bytes(L.kind) + 4.0 + 5.0 * vs) +
                                       (chunk == 0 ? a.dd.N * vs : 0.0));
      }
    }
    __syncthreads();
  }
}

// lambda_max bounds, lambda, early exit when lambda >= lambda_max (x* = 0, gap 0).
// Signal of work item `item`: the last b in [lo, hi] with offsets[b] <= item.
__device__ __forceinline__ int item_signal(const int* __restrict__ offsets, int lo, int hi, int item) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The correlation pass for FP32 iterates: g_j = a~_j^T rho^ over the preserved list, fused with
// the FISTA update of those coefficients and with the two maxima of the pass,
// max_j (|g_j| + eps_j ||rho^||) (upper bound, stable scaling) and max_j |g_j|.
// Persistent grid over (signal, chunk) items; the eight warps of a block share an item, each
// warp forming two dot products at a time (lanes 0 and 1 then update the two coefficients).
// Levels whose correlations come from a batched product (tensor cores, Kronecker) only run the
// update, one coefficient per thread.  The signal's pass scalars are FP32 copies prepared by
// k_residual; the maxima go to the signal's state with atomicMax on FP32 bit patterns
// (non-negative values).  Every per-atom operation is FP32; the bounds use directed rounding.
template <typename VT>
__global__ void __launch_bounds__(CORR_THREADS, 4) k_corr_pass(PassArgs<VT> a) {
  static_assert(sizeof(VT) == 4, "FP32 iterates only");
  constexpr int NW = CORR_THREADS / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int B = a.sp.B;
  const int total = a.offsets[B];
  const int ldN = (int)a.ldN;
  const int CH = a.counters[2];      // this pass's chunk (k_schedule)
  const float ga_fac = 1.0000004f;   // >= 1 + 3 u32, rounded up
  const float inv_Lf = (float)a.sp.inv_L;
  const bool fista = a.sp.algo == LASSO_FISTA;
  float bytes = 0.f;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = item_signal(a.offsets, 0, B - 1, item);
    const int chunk = item - a.offsets[b];
    const SigState& s = a.st[b];
    const LevelDev& L = a.dd.lv[s.level];
    const bool from_full = level_structured(L.kind) || L.tc;
    const int CHs = from_full ? CH * FULL_ITEM_MULT : CH;   // gathers take larger items
    const int p0 = chunk * CHs, p1 = min(s.n_kept, p0 + CHs);
    const VT* rho = a.Rho + (int64_t)b * a.ldN;
    const float nrho_f = s.nrho_ru, thr_f = s.thr_f, beta_f = s.beta_f;
    const bool tight = !from_full && L.kind == LK_F32 && s.corr_tight;
    const float dq_f = L.tc ? __double2float_ru(s.dq * 1.001) : 0.f;
    const float gt_f = tight ? __double2float_ru(L.gam_tight) : 0.f;
    const int32_t* kp = kept_of(a, b, s.parity);
    VT* X = a.X + (int64_t)b * a.K;
    VT* Z = a.Z + (int64_t)b * a.K;
    VT* G = a.G + (int64_t)b * a.K;
    float m1 = 0.f, m2 = 0.f;
    auto update = [&](int pos, int32_t j, float g) {
      const float ag = fabsf(g);
      const float er = tight ? __fmaf_ru(gt_f, L.kappa32[j], L.eps32[j]) : L.epsr32[j];
      float ub = __fmaf_ru(er, nrho_f, __fmul_ru(ag, ga_fac));
      if (dq_f > 0.f) ub = __fmaf_ru(L.kappa32[j], dq_f, ub);
      m1 = fmaxf(m1, ub);
      m2 = fmaxf(m2, ag);
      const float xj = (float)X[j], zj = (float)Z[j];
      const float v = __fmaf_rn(g, inv_Lf, zj);
      const float xn = v > thr_f ? v - thr_f : (v < -thr_f ? v + thr_f : 0.f);
      const float zn = fista ? __fmaf_rn(beta_f, xn - xj, xn) : xn;
      X[j] = (VT)xn;
      Z[j] = (VT)zn;
      G[pos] = (VT)g;
    };
    if (from_full) {
      // four positions per thread at a time: their loads are issued before any update stores
      const float* gf = a.Gfull + (int64_t)b * a.K;
      for (int pos0 = p0 + (int)threadIdx.x; pos0 < p1; pos0 += 4 * CORR_THREADS) {
        int32_t jv[4];
        float gv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int pos = pos0 + u * CORR_THREADS;
          jv[u] = pos < p1 ? kp[pos] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = jv[u] >= 0 ? gf[jv[u]] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (jv[u] >= 0) update(pos0 + u * CORR_THREADS, jv[u], gv[u]);
      }
    } else if (tight) {
      // error-free products (Dot2) with their tight bound, near the end of the signal's solve
      for (int base = p0 + wid; base < p1; base += NW) {
        const int32_t j = kp[base];
        const float g = warp_atom_dot_tight_f(L, j, ldN, reinterpret_cast<const float*>(rho), lane);
        if (lane == 0) update(base, j, g);
        if (a.alg_bytes && lane == 0)
          bytes += (float)a.dd.N * level_elem_bytes(L.kind) + 4.f + 5.f * sizeof(VT);
      }
      if (a.alg_bytes && chunk == 0 && wid == 0 && lane == 0) bytes += (float)a.dd.N * sizeof(VT);
    } else {
      for (int base = p0 + wid; base < p1; base += 2 * NW) {
        const bool two = base + NW < p1;
        const int32_t j0 = kp[base], j1 = two ? kp[base + NW] : j0;
        float g0, g1;
        warp_atom_dot2_fast<VT>(L, j0, j1, ldN, rho, lane, g0, g1);
        if (lane == 0) update(base, j0, g0);
        else if (lane == 1 && two) update(base + NW, j1, g1);
        if (a.alg_bytes && lane == 0)
          bytes += (two ? 2.f : 1.f) * ((float)a.dd.N * level_elem_bytes(L.kind) + 4.f + 5.f * sizeof(VT));
      }
      if (a.alg_bytes && chunk == 0 && wid == 0 && lane == 0) bytes += (float)a.dd.N * sizeof(VT);
    }
    m1 = warp_max_f(m1);
    m2 = warp_max_f(m2);
    if (lane == 0 && m1 > 0.f) atomicMax(&a.st[b].pm1, __float_as_uint(m1));
    if (lane == 0 && m2 > 0.f) atomicMax(&a.st[b].pm2, __float_as_uint(m2));
  }
  if (a.alg_bytes && lane == 0 && bytes > 0.f) atomicAdd(&a.alg_bytes[1], (double)bytes);
}

// The initial pass on the tensor cores: g^_j ~ a~_j^T y for every atom from a batched product
// with a tensor-core level (Gfull), bounded by the level's error (eps_j, the accumulation and
// the quantisation of y).  Every atom whose upper bound reaches the largest lower bound could
// attain lambda_max = max_j |a_j^T y| (eq:DefLMax); those are recomputed from the exact data with
// error-free products, so lambda_max keeps the bounds of the exact initial pass.  The other
// atoms keep their tensor-core upper bounds of |a_j^T y| (Dynamic / Static Safe rules).
template <typename VT>
__global__ void __launch_bounds__(256) k_init_tc(PassArgs<VT> a, int lvl) {
  const int b = blockIdx.x;
  SigState* sp = a.st + b;
  __shared__ int s_go;
  __shared__ float s_lb[8];
  __shared__ double s_m1[8], s_m2[8];
  if (threadIdx.x == 0) s_go = !sp->done;
  __syncthreads();
  if (!s_go) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const LevelDev& Lq = a.dd.lv[lvl];
  const LevelDev& Lx = a.dd.lv[a.dd.n_levels - 1];
  const int64_t K = a.K;
  const float* g = a.Gfull + (int64_t)b * K;
  float* c0 = a.c0ub + (int64_t)b * K;
  const double ynorm = sp->ynorm;
  const float yn_f = __double2float_ru(ynorm);
  const float dq_f = __double2float_ru(sp->dq * 1.001);
  // upper bounds of |a_j^T y| for every atom, and the largest lower bound
  float lbm = 0.f;
  for (int64_t j = threadIdx.x; j < K; j += 256) {
    const float ag = fabsf(g[j]);
    const float err = __fmaf_ru(Lq.kappa32[j], dq_f, __fmul_ru(Lq.epsr32[j], yn_f));
    c0[j] = __fadd_ru(__fmul_ru(ag, 1.0000005f), err);
    lbm = fmaxf(lbm, __fsub_rd(__fmul_rd(ag, 0.9999995f), err));
  }
  lbm = warp_max_f(lbm);
  if (lane == 0) s_lb[wid] = lbm;
  __syncthreads();
  float T = 0.f;
  for (int w = 0; w < 8; ++w) T = fmaxf(T, s_lb[w]);
  // candidates: recomputed with error-free products on the exact atoms
  const float* yv = reinterpret_cast<const float*>(a.Yw + (int64_t)b * a.ldN);
  double m1 = 0.0, m2 = 0.0;
  for (int64_t base = (int64_t)wid * 32; base < K; base += 256) {
    const int64_t j = base + lane;
    const bool cand = j < K && c0[j] >= T;
    unsigned m = __ballot_sync(0xffffffffu, cand);
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const int64_t jj = base + l;
      const double gx = warp_atom_dot(Lx, jj, (int)a.ldN, yv, nullptr, lane);
      const double ub = fabs(gx) * (1.0 + 4.0 * U64) + (Lx.eps[jj] + Lx.gam_tight * Lx.kappa[jj]) * ynorm;
      m1 = fmax(m1, ub);
      m2 = fmax(m2, fabs(gx));
      if (lane == 0) c0[jj] = __double2float_ru(ub);
    }
  }
  if (lane == 0) {
    s_m1[wid] = m1;
    s_m2[wid] = m2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < 8; ++w) {
      m1 = fmax(m1, s_m1[w]);
      m2 = fmax(m2, s_m2[w]);
    }
  }
  // the initial-pass maxima as k_init_finish reads them (first chunk; the others empty)
  const int nch = (int)((K + a.sp.chunk - 1) / a.sp.chunk);
  for (int c = threadIdx.x; c < nch; c += 256) {
    double* pc = a.part_corr + ((int64_t)b * a.nch + c) * 2;
    pc[0] = c == 0 ? m1 : 0.0;
    pc[1] = c == 0 ? m2 : 0.0;
  }
}

template <typename VT>
__global__ void k_init_finish(PassArgs<VT> a, int lambda_relative) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.sp.B) return;
  SigState& s = a.st[b];
  if (s.done) return;
  double ub = 0.0, lb = 0.0;
  const int nch = (int)((a.K + a.sp.chunk - 1) / a.sp.chunk);
  for (int c = 0; c < nch; ++c) {
    ub = fmax(ub, a.part_corr[((int64_t)b * a.nch + c) * 2]);
    lb = fmax(lb, a.part_corr[((int64_t)b * a.nch + c) * 2 + 1]);
  }
  s.lam_max_lb = lb;
  s.lam_max_ub = ub;
  if (lambda_relative) s.lam = s.lam * lb;
  if (!(s.lam > 0.0) || !(s.lam < INFINITY)) {
    s.status = LASSO_ERR_INVALID_ARG;
    s.done = 1;
    return;
  }
  if (s.lam >= ub) {
    s.done = 1;
    s.gap = 0.0;
    s.n_kept = 0;
    s.status = LASSO_OK;
  }
  s.n_chunks = (int)((s.n_kept + a.sp.chunk - 1) / a.sp.chunk);
}

// ------------------------------------------------------------------ gap, screening, switch

// FP64 scalars of one pass of one signal, for an upper bound m1 of max_j (|a_j^T rho| +
// eps_j ||rho||) and m2 = max_j |g^_j|:
//   P = 1/2||rho||^2 + lam ||z||_1, theta' = s' rho (stable scaling), theta~ = s~ rho,
//   G' = P - D(theta'), G~ = P - D(theta~), delta = ||rho|| e + e^2/2 with
//   e = sum eps_j |z_j| + (residual rounding), R' = sqrt(2 G' + 2 delta) / lam, gamma = G~ / G',
//   and the certificate (G' + delta) / ||y||^2 of the reduced problem.
struct PassScalars {
  double Gp, Gt, delta, Rp, gamma, sp, abs_st, Rt, cert;
};

template <typename VT>
__device__ PassScalars pass_scalars(const SigState& s, const LevelDev& L, double rr, double yr, double m1, double m2) {
  PassScalars o;
  const double lam = s.lam;
  const double nrho = sqrt(rr);
  const double e_r = residual_bound(L, s.sum_kapz, s.n_nz, nrho, sizeof(VT) == 8, !s.res_used);
  const double e = s.sum_epsz + e_r;
  double sp_ = 0.0, st_ = 0.0;
  if (rr > 0.0) {
    const double beta = yr / (lam * rr);
    sp_ = m1 > 0.0 ? fmin(fmax(beta, -1.0 / m1), 1.0 / m1) : beta;
    st_ = m2 > 0.0 ? fmin(fmax(beta, -1.0 / m2), 1.0 / m2) : beta;
  }
  const double P = 0.5 * rr + lam * s.l1;
  const double Dp = lam * sp_ * yr - 0.5 * lam * lam * sp_ * sp_ * rr;
  const double Dt = lam * st_ * yr - 0.5 * lam * lam * st_ * st_ * rr;
  o.Gp = P - Dp;
  o.Gt = P - Dt;
  o.delta = nrho * e + 0.5 * e * e;
  o.Rp = sqrt(fmax(2.0 * o.Gp + 2.0 * o.delta, 0.0)) / lam;
  o.gamma = o.Gp > 0.0 ? o.Gt / o.Gp : 0.0;
  o.sp = sp_;
  o.abs_st = fabs(st_);
  o.Rt = sqrt(fmax(2.0 * o.Gt, 0.0)) / lam;
  o.cert = fmax(o.Gp + o.delta, 0.0) / s.yy;
  return o;
}

__device__ __forceinline__ void apply_scalars(SigState& s, const PassScalars& ps) {
  s.Gp = ps.Gp;
  s.Gt = ps.Gt;
  s.delta = ps.delta;
  s.Rp = ps.Rp;
  s.gamma = ps.gamma;
  s.sp = ps.sp;
}

// Outcome of the pass for one signal once its certificate is known: stop (converged, or an
// error), snapshot the point for the full-dictionary check, or continue; and the scalars of the
// screening test.  m1_bulk: the pass's own maximum (finiteness check); m1_used: the one the
// certificate used.
template <typename VT>
__device__ void pass_decide(SigState& s, const PassArgs<VT>& a, double m1_bulk, double m1_used,
                            const PassScalars& ps) {
  const int I = a.dd.n_levels - 1;
  const double rr = s.rr, yr = s.yr, gcert = ps.cert;
  const double lam = s.lam;
  const double nrho = sqrt(rr);
  int action = 0;   // 0 continue, 1 stop (converged), 2 stop (error)
  s.snap = 0;       // 1: snapshot the point for the full-dictionary check
  if (!(rr < INFINITY) || !(yr == yr) || !(m1_bulk < INFINITY) || !(s.Gp == s.Gp) || !(s.delta < INFINITY)) {
    s.status = LASSO_ERR_NONFINITE;
    action = 2;
  } else if (s.level == I && gcert <= a.sp.tol && !a.sp.full_gap) {
    s.status = LASSO_OK;
    action = 1;
  } else if (s.level == I && gcert <= a.sp.tol && !s.pending && s.iters >= s.next_check) {
    // the reduced problem is solved to tol: keep iterating while this point's correlations
    // with the rejected atoms are checked (full-dictionary gap, stopping rule of Section IV)
    s.pending = 1;
    s.snap = 1;
  } else if (s.iters >= a.sp.max_iter || a.counters[1]) {
    // pass limit, or the host's wall-clock limit (counters[1]): stop with the current point
    // and its certificate (partial x, last certified gap)
    s.status = a.counters[1] ? LASSO_ERR_TIMEOUT : LASSO_ERR_MAXITER;
    action = 2;
  }
  if (s.level == I || action) s.gap = gcert;
  if (action || s.snap) {
    // the scalars of the point that is returned or checked (full-dictionary gap, audit)
    s.c_rr = rr;
    s.c_yr = yr;
    s.c_l1 = s.l1;
    s.c_epsz = s.sum_epsz;
    s.c_kapz = s.sum_kapz;
    s.c_nnz = s.n_nz;
    s.c_m1 = m1_used;
    s.c_nrho_ru = __double2float_ru(nrho);
    s.c_res_tight = s.res_used;
  }
  // Dynamic Safe radius ||theta' - y/lam|| (Table I)
  const double sp_ = s.sp;
  const double inv_lam = 1.0 / lam;
  const double d2 = sp_ * sp_ * rr - 2.0 * sp_ * yr * inv_lam + s.yy * inv_lam * inv_lam;
  s.scr = rr > 0.0 && (s.iters % a.sp.screen_every) == 0 ? 1 : 0;
  s.act = action;
  s.t_abs_sp = fabs(sp_);
  s.t_c_eps = fabs(sp_) * nrho;
  if (a.sp.rule == LASSO_RULE_GAP) {
    s.t_Rs = s.Rp;
  } else if (a.sp.rule == LASSO_RULE_DST) {
    s.t_Rs = sqrt(fmax(d2, 0.0)) * (1.0 + 4.0 * U64);
  } else {
    // Static Safe sphere around y / lam (eq:static_sphere); lam_max_ub >= lambda_max
    s.t_Rs = s.ynorm * fmax(inv_lam - 1.0 / s.lam_max_ub, 0.0) * (1.0 + 8.0 * U64);
  }
  s.t_abs_st = ps.abs_st;
  s.t_Rt = ps.Rt;
  s.t_inv_lam = inv_lam * (1.0 + 2.0 * U64);
}

// Saturation of the iterates on the exact level: the certificate has not improved by 2 % for
// max(stall_passes, passes / 16) passes (FP32 iterates) or max(stall_passes, passes / 2) passes
// (the FP64 second solve) while still above tol; an FP32 signal stops and is solved again with
// FP64 iterates by the host, an FP64 second solve stops with its best certificate.
template <typename VT>
__device__ __forceinline__ void check_stall(SigState& s, const PassArgs<VT>& a, double cert) {
  if (a.sp.stall_passes <= 0 || s.level != a.dd.n_levels - 1 || s.act != 0 || s.pending) return;
  if (cert < 0.98 * s.best_cert) {
    s.best_cert = cert;
    s.stall = 0;
  } else if (++s.stall >= max(a.sp.stall_passes, s.iters / (int)(sizeof(VT) == 8 ? 2 : 16)) && cert > a.sp.tol) {
    // (the window grows with the pass count: ISTA's gap falls like 1 / k, so a fixed window
    // would eventually show less than 2 % progress on a converging signal; the second solve
    // ends a signal for good, so it waits until the plateau is as long as the progress before
    // it: a certificate stuck at the floor of its FP32 point since pass k stops near pass 2 k,
    // while FISTA on a coherent dictionary can stall for hundreds of passes and then converge)
    s.status = LASSO_ST_SATURATED;
    s.act = 2;
  }
}

// FP64 scalars of the pass, one thread per signal (FP64 issue is shared by the 32 signals of a
// warp instead of one): the certificate, the pass count and the outcome of the pass; on the
// exact FP32 level near convergence, the switch of the signal's correlations to error-free
// products (k_corr_pass, from the next pass on).
template <typename VT>
__global__ void __launch_bounds__(128) k_eval(PassArgs<VT> a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.sp.B) return;
  SigState* sp = a.st + b;
  if (sp->done) return;
  SigState s = *sp;
  const LevelDev& L = a.dd.lv[s.level];
  const int I = a.dd.n_levels - 1;
  const double rr = s.rr, yr = s.yr;
  double m1 = 0.0, m2 = 0.0;
  if constexpr (sizeof(VT) == 4) {
    m1 = (double)__uint_as_float(s.pm1);
    m2 = (double)__uint_as_float(s.pm2);
    s.pm1 = 0u;
    s.pm2 = 0u;
  } else {
    for (int c = 0; c < s.n_chunks; ++c) {
      m1 = fmax(m1, a.part_corr[((int64_t)b * a.nch + c) * 2]);
      m2 = fmax(m2, a.part_corr[((int64_t)b * a.nch + c) * 2 + 1]);
    }
  }
  const PassScalars ps = pass_scalars<VT>(s, L, rr, yr, m1, m2);
  apply_scalars(s, ps);
  s.iters += 1;
  s.level_passes[s.level] += 1;
  if (a.alg_bytes) atomicAdd(&a.alg_bytes[8 + s.level], (double)s.n_kept);
  if (sizeof(VT) == 4 && L.kind == LK_F32 && !L.tc && s.level == I && ps.cert > a.sp.tol && rr > 0.0 &&
      m2 > 0.0 && !s.corr_tight) {
    // would the certificate meet tol with the tight products?  then the next passes compute the
    // correlations with error-free products (sticky)
    const PassScalars pe = pass_scalars<VT>(s, L, rr, yr, m2 * (1.0 + 3.0 * U32), m2);
    if (pe.cert <= a.sp.tol) s.corr_tight = 1;
  }
  pass_decide<VT>(s, a, m1, m1, ps);
  check_stall<VT>(s, a, ps.cert);
  // the next residuals with error-free products once the certificate nears tol, or once the
  // fast residual's rounding bound is a visible part of it (sticky)
  if (!s.res_tight && s.level == I && (ps.cert <= 30.0 * a.sp.tol || ps.delta >= 0.1 * (ps.Gp + ps.delta)))
    s.res_tight = 1;
  *sp = s;
}

// One block per signal, after the pass has been evaluated (k_eval).  In one sweep of the preserved list, every atom is tested (stable GAP or Dynamic Safe
// sphere), K_t is counted, and the preserved list and the nonzero list of z+ are compacted in
// order; Algorithm 2 picks the next level and the sums of the nonzero list close the pass.
// FP32 iterates keep the per-atom work in FP32: tests rounded upward (over-estimating only
// keeps atoms), sum |z_j| compensated, sum eps_j |z_j| and sum kappa_j |z_j| rounded upward.
template <typename VT>
__device__ __forceinline__ void screen_signal(const PassArgs<VT>& a, int b) {
  constexpr bool F32 = sizeof(VT) == 4;
  constexpr int NWS = SCREEN_THREADS / 32;
  SigState* sp = a.st + b;
  __shared__ double sc[16];
  __shared__ int si[12];
  constexpr int SU = 4;
  __shared__ int s_cnt[2][SU][NWS];
  __shared__ int s_warp3[NWS];
  __shared__ double s_red[3][NWS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const SigState& s = *sp;
    si[11] = s.done;
    si[4] = s.n_kept;
    si[5] = s.parity;
    si[6] = s.level;
    si[7] = s.n_nz;
    sc[0] = s.t_abs_sp;
    sc[1] = s.t_c_eps;
    sc[2] = s.t_Rs;
    sc[3] = s.t_abs_st;
    sc[4] = s.t_Rt;
    sc[5] = 1.0 - a.sp.tau;
    sc[6] = 1.0 + 3.0 * (level_fp64_arith(a.dd.lv[s.level].kind) && sizeof(VT) == 8 ? U64 : U32);
    sc[7] = s.t_inv_lam;
    sc[14] = s.dq;
    si[0] = s.act;
    si[1] = s.scr;
    si[2] = s.snap;
  }
  __syncthreads();
  if (si[11]) return;
  const int n_kept = si[4], parity = si[5], level = si[6], n_nz = si[7];
  const LevelDev& L = a.dd.lv[level];
  const int32_t* kp = kept_of(a, b, parity);
  const VT* G = a.G + (int64_t)b * a.K;
  const int action = si[0];
  VT* X = a.X + (int64_t)b * a.K;
  VT* Z = a.Z + (int64_t)b * a.K;
  if (action) {
    // return the certified point z_t (its nonzero list) and stop
    VT* xo = a.Xout + (int64_t)b * a.K;
    for (int q = threadIdx.x; q < n_nz; q += SCREEN_THREADS)
      xo[a.nz_idx[(int64_t)b * a.K + q]] = a.nz_val[(int64_t)b * a.K + q];
    if (threadIdx.x == 0) sp->done = 1;
    return;
  }
  if (si[2]) {
    for (int q = threadIdx.x; q < n_nz; q += SCREEN_THREADS) {
      a.cand_idx[(int64_t)b * a.K + q] = a.nz_idx[(int64_t)b * a.K + q];
      a.cand_val[(int64_t)b * a.K + q] = a.nz_val[(int64_t)b * a.K + q];
    }
  }
  const bool screen = si[1];
  const double abs_sp = sc[0], c_eps = sc[1], Rs = sc[2], abs_st = sc[3], Rt = sc[4], thr = sc[5], gfac = sc[6],
               inv_lam = sc[7], dq = sc[14];
  const bool gap_rule = a.sp.rule == LASSO_RULE_GAP;
  const double* anorm = a.dd.anorm;
  const float* anorm32 = a.dd.anorm32;
  const float* c0 = a.c0ub + (int64_t)b * a.K;
  // FP32 copies of the scalars, rounded so that the FP32 test value stays an upper bound of
  // the exact one (rejection needs test < 1 - tau, so over-estimating only keeps more atoms)
  const float abs_sp_f = __double2float_ru(abs_sp), gfac_f = __double2float_ru(gfac);
  const float c_eps_f = __double2float_ru(c_eps), Rs_f = __double2float_ru(Rs);
  const float inv_lam_f = __double2float_ru(inv_lam), thr_f = __double2float_rd(thr);
  const float abs_st_f = (float)abs_st, Rt_f = (float)Rt;
  const float c_dq_f = L.tc ? __double2float_ru(abs_sp * dq * 1.001) : 0.f;
  auto keep_of = [&](int64_t j, VT g) -> bool {
    if (!screen) return true;
    if constexpr (F32) {
      float mu;
      if (gap_rule) {
        mu = __fadd_ru(__fmaf_ru(L.epsr32[j], c_eps_f, __fmul_ru(__fmul_ru(abs_sp_f, fabsf((float)g)), gfac_f)),
                       __fmul_ru(Rs_f, anorm32[j]));
        if (c_dq_f > 0.f) mu = __fmaf_ru(L.kappa32[j], c_dq_f, mu);
      } else {
        mu = __fadd_ru(__fmul_ru(c0[j], inv_lam_f), __fmul_ru(Rs_f, anorm32[j]));
      }
      return mu >= thr_f;
    } else {
      double mu;
      if (gap_rule)
        mu = abs_sp * fabs((double)g) * gfac + (L.eps[j] + L.gam_corr * L.kappa[j]) * c_eps + Rs * anorm[j] +
             (L.tc ? L.kappa[j] * abs_sp * dq * 1.001 : 0.0);
      else mu = (double)c0[j] * inv_lam + Rs * anorm[j];
      return mu * (1.0 + 4.0 * U64) >= thr;
    }
  };
  // ---- one sweep: K_t (conventional test on A~, eq:DefCardinalEstimated), the stable test,
  // and ordered compaction of the preserved list and of the nonzeros of z+
  int32_t* kn = kept_of(a, b, parity ^ 1);
  int32_t* nzi = a.nz_idx + (int64_t)b * a.K;
  VT* nzv = a.nz_val + (int64_t)b * a.K;
  int base_k = 0, base_z = 0, kt = 0;
  DF l1f;
  l1f.init();
  float sef = 0.f, skf = 0.f;
  double l1 = 0.0, se = 0.0, sk = 0.0;
  // SU positions per thread per step (loads of all of them in flight together)
  for (int t0 = 0; t0 < n_kept; t0 += SU * SCREEN_THREADS) {
    int32_t jv[SU];
    VT gv[SU], zv[SU];
    bool keep[SU], nz[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      const int pos = t0 + u * SCREEN_THREADS + threadIdx.x;
      jv[u] = pos < n_kept ? kp[pos] : -1;
    }
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      const int pos = t0 + u * SCREEN_THREADS + threadIdx.x;
      gv[u] = jv[u] >= 0 ? G[pos] : (VT)0;
      zv[u] = jv[u] >= 0 ? Z[jv[u]] : (VT)0;
    }
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      keep[u] = false;
      nz[u] = false;
      if (jv[u] >= 0) {
        const int64_t j = jv[u];
        if (__fmaf_rn(abs_st_f, fabsf((float)gv[u]), Rt_f * L.atnorm[j]) >= 1.f) ++kt;
        keep[u] = keep_of(j, gv[u]);
        if (!keep[u]) {
          X[j] = (VT)0;
          Z[j] = (VT)0;
          a.mask[(int64_t)b * a.K + j] = 0;
        } else {
          nz[u] = zv[u] != (VT)0;
        }
      }
    }
    unsigned bk[SU], bz[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      bk[u] = __ballot_sync(0xffffffffu, keep[u]);
      bz[u] = __ballot_sync(0xffffffffu, nz[u]);
      if (lane == 0) {
        s_cnt[0][u][wid] = __popc(bk[u]);
        s_cnt[1][u][wid] = __popc(bz[u]);
      }
    }
    __syncthreads();
    // ordered offsets: position order is (u, warp, lane)
    int off_k[SU], off_z[SU];
    int run_k = base_k, run_z = base_z;
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      for (int w = 0; w < NWS; ++w) {
        if (w == wid) {
          off_k[u] = run_k;
          off_z[u] = run_z;
        }
        run_k += s_cnt[0][u][w];
        run_z += s_cnt[1][u][w];
      }
    }
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      if (keep[u]) kn[off_k[u] + __popc(bk[u] & below)] = jv[u];
      if (nz[u]) {
        const int64_t j = jv[u];
        const int q = off_z[u] + __popc(bz[u] & below);
        nzi[q] = jv[u];
        nzv[q] = zv[u];
        if constexpr (F32) {
          const float az = fabsf((float)zv[u]);
          l1f.add(az);
          sef = __fmaf_ru(L.eps32[j], az, sef);
          skf = __fmaf_ru(L.kappa32[j], az, skf);
        } else {
          const double az = fabs((double)zv[u]);
          l1 += az;
          se = fma(L.eps[j], az, se);
          sk = fma(L.kappa[j], az, sk);
        }
      }
    }
    base_k = run_k;
    base_z = run_z;
    __syncthreads();
  }
  kt = warp_sum_i(kt);
  if (lane == 0) s_warp3[wid] = kt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < NWS; ++w) t += s_warp3[w];
    // Algorithm 2
    const int I = a.dd.n_levels - 1;
    int nl = level;
    if (level < I) {
      if (t <= L.rc * (double)a.K) nl = I;
      else if (sp->gamma <= a.sp.Gamma) nl = level + 1;
    }
    si[8] = nl;
    si[9] = t;
  }
  __syncthreads();
  const int new_level = si[8];
  if (new_level != level) {
    // the error sums of the nonzero list belong to the level of the next pass
    const LevelDev& Ln = a.dd.lv[new_level];
    sef = skf = 0.f;
    se = sk = 0.0;
    for (int q = threadIdx.x; q < base_z; q += SCREEN_THREADS) {
      const int64_t j = nzi[q];
      if constexpr (F32) {
        const float az = fabsf((float)nzv[q]);
        sef = __fmaf_ru(Ln.eps32[j], az, sef);
        skf = __fmaf_ru(Ln.kappa32[j], az, skf);
      } else {
        const double az = fabs((double)nzv[q]);
        se = fma(Ln.eps[j], az, se);
        sk = fma(Ln.kappa[j], az, sk);
      }
    }
  }
  if constexpr (F32) {
    l1f = df_warp_reduce(l1f);
    sef = warp_sum_ru(sef);
    skf = warp_sum_ru(skf);
    if (lane == 0) {
      s_red[0][wid] = (double)l1f.s + (double)l1f.c;
      s_red[1][wid] = (double)sef;
      s_red[2][wid] = (double)skf;
    }
  } else {
    l1 = warp_sum(l1);
    se = warp_sum(se);
    sk = warp_sum(sk);
    if (lane == 0) {
      s_red[0][wid] = l1;
      s_red[1][wid] = se;
      s_red[2][wid] = sk;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int w = 0; w < NWS; ++w) {
      t1 += s_red[0][w];
      t2 += s_red[1][w];
      t3 += s_red[2][w];
    }
    SigState& o = *sp;
    o.l1 = t1;
    o.sum_epsz = t2;
    o.sum_kapz = t3;
    o.n_kept = base_k;
    o.n_nz = base_z;
    o.Kt = si[9];
    o.level = new_level;
    o.parity = parity ^ 1;
    o.n_chunks = (base_k + a.sp.chunk - 1) / a.sp.chunk;
    // FISTA: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, momentum (t_k - 1) / t_{k+1} for the next update
    const double tk = o.t;
    const double t1n = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
    const double t2n = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t1n * t1n));
    o.t = t1n;
    o.beta = (t1n - 1.0) / t2n;
  }
}

template <typename VT>
__global__ void __launch_bounds__(SCREEN_THREADS, 4) k_screen(PassArgs<VT> a) {
  const int n = a.counters[4];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    screen_signal<VT>(a, a.live_list[i]);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ full-dictionary check

// Work items of the pending checks: ceil(K / chunk) per pending signal.
template <typename VT>
__global__ void k_schedule_full(PassArgs<VT> a) {
  __shared__ int sh_sum[32];
  __shared__ int sh_cnt[32];
  __shared__ int carry, carry2;
  if (threadIdx.x == 0) {
    carry = 0;
    carry2 = 0;
  }
  __syncthreads();
  const int B = a.sp.B;
  const int nchk = (int)((a.K + a.sp.chunk - 1) / a.sp.chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < B; base += blockDim.x) {
    const int b = base + threadIdx.x;
    const int items = (b < B && a.st[b].pending && !a.st[b].done) ? nchk : 0;
    int v = items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) sh_sum[wid] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      const int nw = blockDim.x >> 5;
      int x = threadIdx.x < nw ? sh_sum[threadIdx.x] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)threadIdx.x >= o) x += t;
      }
      sh_sum[threadIdx.x] = x;
    }
    __syncthreads();
    if (b < B) a.offsets2[b] = carry + (wid ? sh_sum[wid - 1] : 0) + v - items;
    // slot of the signal among those under check (operand rows of the tensor-core check)
    const unsigned bal = __ballot_sync(0xffffffffu, items > 0);
    if (lane == 0) sh_cnt[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = carry2;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
        const int c = sh_cnt[w2];
        sh_cnt[w2] = acc;
        acc += c;
      }
      carry2 = acc;
    }
    __syncthreads();
    if (b < B) {
      const int slot = sh_cnt[wid] + __popc(bal & ((1u << lane) - 1u));
      a.tc_slot[(int64_t)FULL_SET * B + b] = items > 0 ? slot : -1;
      if (items > 0) a.tc_list[(int64_t)FULL_SET * B + slot] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += sh_sum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.offsets2[B] = carry;
    a.counters[8 + FULL_SET] = carry2;
  }
}

// Correlations of the rejected atoms with the snapshot residual (fast products, rigorous
// upper bounds with the exact level's margins); the preserved atoms are covered by c_m1.
template <typename VT>
__global__ void __launch_bounds__(CORR_THREADS) k_full_check(PassArgs<VT> a) {
  __shared__ double s_m[CORR_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int B = a.sp.B;
  const int total = a.offsets2[B];
  const int CH = a.sp.chunk;
  const LevelDev& L = a.dd.lv[a.dd.n_levels - 1];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = item_signal(a.offsets2, 0, B - 1, item);
    const int chunk = item - a.offsets2[b];
    const SigState& s = a.st[b];
    const VT* rho = a.Rho + (int64_t)b * a.ldN;
    const uint8_t* mk = a.mask + (int64_t)b * a.K;
    const float nrho_f = s.c_nrho_ru;
    // an atom whose loose bound reaches the preserved atoms' maximum could decide the scaling:
    // recompute it from the FP32 data with error-free products (tight bound)
    const bool tighten = sizeof(VT) == 4 && L.kind == LK_F32;
    const float T_f = __double2float_rd(s.c_m1);
    const int64_t j0 = (int64_t)chunk * CH, j1 = min((int64_t)a.K, j0 + CH);
    double m = 0.0;
    for (int64_t j = j0 + wid; j < j1; j += CORR_THREADS / 32) {
      if (mk[j]) continue;   // warp-uniform: every lane reads the same flag
      const float g = (float)warp_atom_dot_fast<VT>(L, j, (int)a.ldN, rho, lane);
      const float ub = __fmaf_ru(L.epsr32_simt[j], nrho_f, __fmul_ru(fabsf(g), 1.0000004f));
      if (tighten && ub > T_f) {   // warp-uniform: g is the same in every lane
        const double gd = warp_atom_dot(L, j, (int)a.ldN, reinterpret_cast<const float*>(rho), nullptr, lane);
        m = fmax(m, fabs(gd) * (1.0 + 3.0 * U32) + L.gam_tight * L.kappa[j] * (double)nrho_f);
      } else {
        m = fmax(m, (double)ub);
      }
    }
    if (lane == 0) s_m[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < CORR_THREADS / 32; ++w) t = fmax(t, s_m[w]);
      a.part_full[(int64_t)b * a.nch + chunk] = t;
    }
    __syncthreads();
  }
}

// The full-dictionary check with the tensor cores: the rejected atoms' correlations with the
// snapshot residual come from the batched product of a tensor-core level (Gfull), bounded by
// that level's error; a rejected atom whose bound reaches the preserved atoms' maximum is
// recomputed from the exact data with error-free products.  One block per signal under check.
template <typename VT>
__device__ __forceinline__ void full_check_tc_signal(const PassArgs<VT>& a, int lvl, int b) {
  const SigState& s = a.st[b];
  if (s.done || !s.pending) return;
  __shared__ double s_m[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const LevelDev& Lq = a.dd.lv[lvl];
  const LevelDev& Lx = a.dd.lv[a.dd.n_levels - 1];
  const int64_t K = a.K;
  const float* g = a.Gfull + (int64_t)b * K;
  const uint8_t* mk = a.mask + (int64_t)b * K;
  const float nrho_f = s.c_nrho_ru;
  const float dq_f = __double2float_ru(s.dq * 1.001);
  const float T_f = __double2float_rd(s.c_m1);
  const float* rho = reinterpret_cast<const float*>(a.Rho + (int64_t)b * a.ldN);
  double m = 0.0;
  for (int64_t base = (int64_t)wid * 32; base < K; base += 256) {
    const int64_t j = base + lane;
    bool cand = false;
    if (j < K && !mk[j]) {
      const float err = __fmaf_ru(Lq.kappa32[j], dq_f, __fmul_ru(Lq.epsr32[j], nrho_f));
      const float ub = __fadd_ru(__fmul_ru(fabsf(g[j]), 1.0000005f), err);
      if (ub > T_f) cand = true;
      else m = fmax(m, (double)ub);
    }
    unsigned msk = __ballot_sync(0xffffffffu, cand);
    while (msk) {
      const int l = __ffs(msk) - 1;
      msk &= msk - 1;
      const int64_t jj = base + l;
      const double gx = warp_atom_dot(Lx, jj, (int)a.ldN, rho, nullptr, lane);
      m = fmax(m, fabs(gx) * (1.0 + 3.0 * U32) + Lx.gam_tight * Lx.kappa[jj] * (double)nrho_f);
    }
  }
  m = warp_max(m);
  if (lane == 0) s_m[wid] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = fmax(t, s_m[w]);
    s_m[0] = t;
  }
  __syncthreads();
  const int nchk = (int)((K + a.sp.chunk - 1) / a.sp.chunk);
  for (int c = threadIdx.x; c < nchk; c += 256) a.part_full[(int64_t)b * a.nch + c] = c == 0 ? s_m[0] : 0.0;
}

// Over the signals under the check (k_schedule_full's slot list).
template <typename VT>
__global__ void __launch_bounds__(256) k_full_check_tc(PassArgs<VT> a, int lvl) {
  const int n = a.counters[8 + FULL_SET];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    full_check_tc_signal<VT>(a, lvl, a.tc_list[(int64_t)FULL_SET * a.sp.B + i]);
    __syncthreads();
  }
}

// Full-dictionary gap of the snapshot point; stop (and return it) when it meets tol.
template <typename VT>
__device__ __forceinline__ void full_finish_signal(const PassArgs<VT>& a, int b) {
  SigState* sp = a.st + b;
  __shared__ int s_stop, s_run;
  // one thread reads the flags (thread 0 rewrites the state below), so the whole block agrees
  if (threadIdx.x == 0) s_run = sp->pending && !sp->done;
  __syncthreads();
  if (!s_run) return;
  if (threadIdx.x == 0) {
    SigState s = *sp;
    const LevelDev& L = a.dd.lv[a.dd.n_levels - 1];
    const int nchk = (int)((a.K + a.sp.chunk - 1) / a.sp.chunk);
    double m1 = s.c_m1;
    for (int c = 0; c < nchk; ++c) m1 = fmax(m1, a.part_full[(int64_t)b * a.nch + c]);
    const double lam = s.lam, rr = s.c_rr, yr = s.c_yr, nrho = sqrt(rr);
    double sf = 0.0;
    if (rr > 0.0) {
      const double beta = yr / (lam * rr);
      sf = m1 > 0.0 ? fmin(fmax(beta, -1.0 / m1), 1.0 / m1) : beta;
    }
    const double e = s.c_epsz + residual_bound(L, s.c_kapz, s.c_nnz, nrho, sizeof(VT) == 8, !s.c_res_tight);
    const double P = 0.5 * rr + lam * s.c_l1;
    const double D = lam * sf * yr - 0.5 * lam * lam * sf * sf * rr;
    const double g = fmax(P - D + nrho * e + 0.5 * e * e, 0.0) / s.yy;
    s.pending = 0;
    s_stop = g <= a.sp.tol;
    if (s_stop) {
      s.gap = g;
      s.status = LASSO_OK;
    } else {
      s.next_check = s.iters + 4;
    }
    *sp = s;
  }
  __syncthreads();
  if (s_stop) {
    VT* xo = a.Xout + (int64_t)b * a.K;
    const int n = sp->c_nnz;
    for (int q = threadIdx.x; q < n; q += blockDim.x) xo[a.cand_idx[(int64_t)b * a.K + q]] = a.cand_val[(int64_t)b * a.K + q];
    __syncthreads();
    if (threadIdx.x == 0) sp->done = 1;
  }
}

template <typename VT>
__global__ void k_full_finish(PassArgs<VT> a) {
  const int n = a.counters[8 + FULL_SET];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    full_finish_signal<VT>(a, a.tc_list[(int64_t)FULL_SET * a.sp.B + i]);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ tensor-core operand

// Quantise rho^ of the signals on a tensor-core level into their slot rows of the GEMM operand
// (BF16; E4M3 with the per-signal scale sigma = max |rho| / 448; or the split r1 + r2 of two
// BF16 parts for the split exact level) and bound dq >= ||rho^ - (quantised rho^)||: the
// correlation of the quantised operand differs from a~_j^T rho^ by at most kappa_j dq, which the
// bounds add.  The split level adds c2 ||r2|| for the product a2^T r2 it leaves out.  FP32
// iterates: exact differences (BF16, split) or one rounding (E4M3), squares summed upward.
template <typename VT>
__device__ __forceinline__ void quant_rho_signal(const PassArgs<VT>& a, int lvl, int fp8, int slot_set, int b) {
  const int B = a.sp.B;
  // rows: the level's own slots (slot_set -2), every live signal in its own row (-1: the initial
  // pass, rho = y), or the slots of another list (the signals under the full-dictionary check)
  const int slot = slot_set == -1 ? (a.st[b].done ? -1 : b)
                                  : a.tc_slot[(int64_t)(slot_set == -2 ? lvl : slot_set) * B + b];
  if (slot < 0) return;
  __shared__ float s_max[8];
  __shared__ double s_sum[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const LevelDev& L = a.dd.lv[lvl];
  const VT* rho = a.Rho + (int64_t)b * a.ldN;
  const int N = a.dd.N;
  const int64_t row = (int64_t)slot * a.ldN;
  float sg = 1.f;
  if (fp8) {
    float m = 0.f;
    for (int n = threadIdx.x; n < N; n += 256) m = fmaxf(m, fabsf((float)rho[n]));
    m = warp_max_f(m);
    if (lane == 0) s_max[wid] = m;
    __syncthreads();
    float mx = 0.f;
    for (int w = 0; w < 8; ++w) mx = fmaxf(mx, s_max[w]);
    sg = mx > 0.f ? mx / 448.f : 1.f;
  }
  double dq2 = 0.0, r22 = 0.0;
  if constexpr (sizeof(VT) == 8) {
    // FP64 iterates: differences in FP64
    if (fp8) {
      uint8_t* out = reinterpret_cast<uint8_t*>(L.rq) + row;
      for (int n = threadIdx.x; n < a.ldN; n += 256) {
        const double r = n < N ? (double)rho[n] : 0.0;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fdiv_rn((float)r, sg), __NV_SATFINITE, __NV_E4M3);
        out[n] = q;
        __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        const double e = r - (double)__half2float(__half(hr)) * (double)sg;
        dq2 = fma(e, e, dq2);
      }
    } else {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(L.rq) + row;
      for (int n = threadIdx.x; n < a.ldN; n += 256) {
        const double r = n < N ? (double)rho[n] : 0.0;
        const __nv_bfloat16 q = __float2bfloat16_rn((float)r);
        out[n] = q;
        const double e = r - (double)__bfloat162float(q);
        dq2 = fma(e, e, dq2);
      }
    }
    dq2 = warp_sum(dq2);
  } else {
    float acc = 0.f, acc2 = 0.f;
    if (fp8) {
      uint8_t* out = reinterpret_cast<uint8_t*>(L.rq) + row;
      for (int n = threadIdx.x; n < a.ldN; n += 256) {
        const float r = n < N ? (float)rho[n] : 0.f;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(__fdiv_rn(r, sg), __NV_SATFINITE, __NV_E4M3);
        out[n] = q;
        __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        // one rounding of r - q sg; |fl(e)| (1 + 2^-23) bounds the exact difference
        const float e = __fmul_ru(fabsf(__fmaf_rn(-__half2float(__half(hr)), sg, r)), 1.00000012f);
        acc = __fmaf_ru(e, e, acc);
      }
    } else if (L.split) {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(L.rq) + row;
      __nv_bfloat16* out2 = reinterpret_cast<__nv_bfloat16*>(L.rq2) + row;
      for (int n = threadIdx.x; n < a.ldN; n += 256) {
        const float r = n < N ? (float)rho[n] : 0.f;
        const __nv_bfloat16 q1 = __float2bfloat16_rn(r);
        const float d1 = __fsub_rn(r, __bfloat162float(q1));     // exact
        const __nv_bfloat16 q2 = __float2bfloat16_rn(d1);
        const float r2 = __bfloat162float(q2);
        const float d2 = __fsub_rn(d1, r2);                       // exact
        out[n] = q1;
        out2[n] = q2;
        acc = __fmaf_ru(d2, d2, acc);
        acc2 = __fmaf_ru(r2, r2, acc2);
      }
    } else {
      __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(L.rq) + row;
      for (int n = threadIdx.x; n < a.ldN; n += 256) {
        const float r = n < N ? (float)rho[n] : 0.f;
        const __nv_bfloat16 q = __float2bfloat16_rn(r);
        out[n] = q;
        const float e = __fsub_rn(r, __bfloat162float(q));        // exact
        acc = __fmaf_ru(e, e, acc);
      }
    }
    dq2 = (double)warp_sum_ru(acc);
    r22 = (double)warp_sum_ru(acc2);
  }
  if (lane == 0) {
    s_sum[0][wid] = dq2;
    s_sum[1][wid] = r22;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, t2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      t += s_sum[0][w];
      t2 += s_sum[1][w];
    }
    double dq = sqrt(t) * (1.0 + 1e-12);
    if (L.split) dq += L.c2 * sqrt(t2) * (1.0 + 1e-12);
    a.st[b].dq = dq;
    if (fp8) L.rsig[b] = sg;
    // algorithmic work of the batched correlation of this signal: 2 N K flops per product
    if (a.alg_bytes) atomicAdd(&a.alg_bytes[5], (L.split ? 3.0 : 1.0) * 2.0 * (double)a.dd.N * (double)a.K);
  }
}

// slot_set -1: every signal (the initial pass); otherwise over the slot list of level lvl (-2)
// or of list slot_set.
template <typename VT>
__global__ void __launch_bounds__(256) k_quant_rho(PassArgs<VT> a, int lvl, int fp8, int slot_set = -2) {
  if (slot_set == -1) {
    for (int b = blockIdx.x; b < a.sp.B; b += gridDim.x) {
      quant_rho_signal<VT>(a, lvl, fp8, -1, b);
      __syncthreads();
    }
    return;
  }
  const int set = slot_set == -2 ? lvl : slot_set;
  const int n = a.counters[8 + set];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    quant_rho_signal<VT>(a, lvl, fp8, slot_set, a.tc_list[(int64_t)set * a.sp.B + i]);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Kronecker levels

// Batched FP32 GEMM tile: C[bz](m, n) (+)= sum_{r < R} sum_k A(bz, r, m, k) B(bz, r, k, n).
// The four Kronecker stages instantiate it with their index maps (row-major vectorisation).
enum KronStage { KS_T = 0, KS_G = 1, KS_U = 2, KS_Y = 3 };

template <typename VT, int STAGE>
__global__ void __launch_bounds__(256) k_kron_gemm(PassArgs<VT> a) {
  // batch index: blockIdx.z = b * Rb + r (stages T, U) or b (stages G, Y)
  int b, r = 0;
  const LevelDev* Lp;
  int Rmax = 0;
  {
    int bz = blockIdx.z;
    for (int l = 0; l < a.dd.n_levels; ++l)
      if (a.dd.lv[l].kind == LK_KRON) Rmax = max(Rmax, a.dd.lv[l].R);
    if (STAGE == KS_T || STAGE == KS_U) {
      b = bz / Rmax;
      r = bz % Rmax;
    } else {
      b = bz;
    }
    const SigState& s = a.st[b];
    if (s.done) return;
    Lp = &a.dd.lv[s.level];
    if (Lp->kind != LK_KRON) return;
    if (r >= Lp->R) return;
  }
  const LevelDev& L = *Lp;
  const int N1 = L.N1, K1 = L.K1, N2 = L.N2, K2 = L.K2, R = L.R;
  int M, Nc, Kd;
  if (STAGE == KS_T) { M = K1; Nc = N2; Kd = N1; }
  else if (STAGE == KS_G) { M = K1; Nc = K2; Kd = N2; }
  else if (STAGE == KS_U) { M = N1; Nc = K2; Kd = K1; }
  else { M = N1; Nc = N2; Kd = K2; }
  const int m0 = blockIdx.y * GEMM_T, n0 = blockIdx.x * GEMM_T;
  if (m0 >= M || n0 >= Nc) return;
  const int64_t TK = (int64_t)Rmax * max(K1 * N2, N1 * K2);   // same stride for every signal
  float* Tb = a.Tk + (int64_t)b * TK;
  __shared__ float sA[16][GEMM_T + 4];
  __shared__ float sB[16][GEMM_T + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  const int nr = (STAGE == KS_G || STAGE == KS_Y) ? R : 1;
  for (int rr = 0; rr < nr; ++rr) {
    const int rx = (STAGE == KS_G || STAGE == KS_Y) ? rr : r;
    for (int k0 = 0; k0 < Kd; k0 += 16) {
      // load A tile (16 x 64) and B tile (16 x 64)
      for (int e = threadIdx.x; e < 16 * GEMM_T; e += 256) {
        const int kk = e / GEMM_T, mm = e % GEMM_T;
        const int k = k0 + kk, m = m0 + mm, n = n0 + mm;
        float av = 0.f, bv = 0.f;
        if (k < Kd && m < M) {
          if (STAGE == KS_T) av = L.B[((int64_t)rx * N1 + k) * K1 + m];                       // B_r[n1, k1]
          else if (STAGE == KS_G) av = Tb[((int64_t)rx * K1 + m) * N2 + k];                  // T_r[k1, n2]
          else if (STAGE == KS_U) av = L.B[((int64_t)rx * N1 + m) * K1 + k];                 // B_r[n1, k1]
          else av = Tb[((int64_t)rx * N1 + m) * K2 + k];                                     // U_r[n1, k2]
        }
        if (k < Kd && n < Nc) {
          if (STAGE == KS_T) bv = (float)a.Rho[(int64_t)b * a.ldN + (int64_t)k * N2 + n];    // P[n1, n2]
          else if (STAGE == KS_G) bv = L.C[((int64_t)rx * N2 + k) * K2 + n];                 // C_r[n2, k2]
          else if (STAGE == KS_U) bv = a.Xd[(int64_t)b * a.K + (int64_t)k * K2 + n];         // X[k1, k2]
          else bv = L.C[((int64_t)rx * N2 + n) * K2 + k];                                    // C_r[n2, k2]^T
        }
        sA[kk][mm] = av;
        sB[kk][mm] = bv;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = sA[kk][ty * 4 + i];
          bv[i] = sB[kk][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = __fmaf_rn(av[i], bv[q], acc[i][q]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + q;
      if (m >= M || n >= Nc) continue;
      if (STAGE == KS_T) Tb[((int64_t)r * K1 + m) * N2 + n] = acc[i][q];
      else if (STAGE == KS_G) {
        const int64_t j = (int64_t)m * K2 + n;
        a.Gfull[(int64_t)b * a.K + j] = __fmul_rn(acc[i][q], L.dscale[j]);
      } else if (STAGE == KS_U) Tb[((int64_t)r * N1 + m) * K2 + n] = acc[i][q];
      else a.AZ[(int64_t)b * a.ldN + (int64_t)m * N2 + n] = acc[i][q];
    }
}

// X_b = reshape(d * z_b) for the Kronecker residual (dense scatter of the nonzero list).
template <typename VT>
__global__ void k_kron_scatter(PassArgs<VT> a) {
  const int b = blockIdx.y;
  const SigState& s = a.st[b];
  if (s.done || a.dd.lv[s.level].kind != LK_KRON) return;
  const LevelDev& L = a.dd.lv[s.level];
  float* xd = a.Xd + (int64_t)b * a.K;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.K; j += (int64_t)gridDim.x * blockDim.x)
    xd[j] = 0.f;
  __syncthreads();
  // ordering: the zero fill of this block must precede the writes of every block; use one block
  if (blockIdx.x == 0) {
    for (int q = threadIdx.x; q < s.n_nz; q += blockDim.x) {
      const int32_t j = a.nz_idx[(int64_t)b * a.K + q];
      xd[j] = __fmul_rn((float)a.nz_val[(int64_t)b * a.K + q], L.dscale[j]);
    }
  }
}

// ------------------------------------------------------------------ products of sparse factors

// A~ z for signals on a sparse-factor level: one block per signal, factor after factor
// (S_{J-1} first) over the signal's two scratch vectors, each output entry an FP32 FMA chain
// along one CSR row.  z enters as a dense vector (scatter of its nonzero list); the last stage
// writes A~ z into AZ (zero padding up to ldN), which the residual kernel reads.
template <typename VT>
__global__ void __launch_bounds__(256) k_faust_fwd(PassArgs<VT> a) {
  const int b = blockIdx.x;
  const SigState& s = a.st[b];
  if (s.done) return;
  const LevelDev& L = a.dd.lv[s.level];
  if (L.kind != LK_FAUST) return;
  float* u = a.Fs + (int64_t)b * a.fs_ld;
  float* w = u + a.fs_ld / 2;
  for (int64_t j = threadIdx.x; j < a.K; j += blockDim.x) u[j] = 0.f;
  __syncthreads();
  for (int q = threadIdx.x; q < s.n_nz; q += blockDim.x)
    u[a.nz_idx[(int64_t)b * a.K + q]] = (float)a.nz_val[(int64_t)b * a.K + q];
  __syncthreads();
  for (int f = L.J - 1; f >= 0; --f) {
    const FaustFactor F = L.fac[f];
    float* out = f == 0 ? a.AZ + (int64_t)b * a.ldN : w;
    for (int n = threadIdx.x; n < F.rows; n += blockDim.x) {
      float acc = 0.f;
      for (int p = F.rp[n]; p < F.rp[n + 1]; ++p) acc = __fmaf_rn(F.v[p], u[F.ci[p]], acc);
      out[n] = acc;
    }
    if (f == 0)
      for (int64_t n = F.rows + threadIdx.x; n < a.ldN; n += blockDim.x) out[n] = 0.f;
    __syncthreads();
    float* t = u;
    u = w;
    w = t;
  }
}

// A~^T rho for signals on a sparse-factor level: S_0^T first, through the stored CSR of each
// S_f^T; the last stage writes every atom's correlation into Gfull.
template <typename VT>
__global__ void __launch_bounds__(256) k_faust_adj(PassArgs<VT> a) {
  const int b = blockIdx.x;
  const SigState& s = a.st[b];
  if (s.done) return;
  const LevelDev& L = a.dd.lv[s.level];
  if (L.kind != LK_FAUST) return;
  float* u = a.Fs + (int64_t)b * a.fs_ld;
  float* w = u + a.fs_ld / 2;
  const VT* rho = a.Rho + (int64_t)b * a.ldN;
  for (int n = threadIdx.x; n < a.dd.N; n += blockDim.x) u[n] = (float)rho[n];
  __syncthreads();
  for (int f = 0; f < L.J; ++f) {
    const FaustFactor F = L.fac[f];
    float* out = f == L.J - 1 ? a.Gfull + (int64_t)b * a.K : w;
    for (int k = threadIdx.x; k < F.cols; k += blockDim.x) {
      float acc = 0.f;
      for (int p = F.rpT[k]; p < F.rpT[k + 1]; ++p) acc = __fmaf_rn(F.vT[p], u[F.ciT[p]], acc);
      out[k] = acc;
    }
    __syncthreads();
    float* t = u;
    u = w;
    w = t;
  }
}

// ------------------------------------------------------------------ certificate and outputs

// Full-dictionary certificate (a final pass over every atom with the most precise level):
// gap of the returned point with the stable scaling over all K atoms.
template <typename VT>
__global__ void k_cert_finish(PassArgs<VT> a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.sp.B) return;
  SigState& s = a.st[b];
  if (s.status != LASSO_OK || s.n_kept == 0 || s.iters == 0) return;
  const LevelDev& L = a.dd.lv[a.dd.n_levels - 1];
  // the returned point's residual is the last one computed for this signal
  const double rr = s.c_rr, yr = s.c_yr;
  double m1 = 0.0;
  const int nch = (int)((a.K + a.sp.chunk - 1) / a.sp.chunk);
  for (int c = 0; c < nch; ++c) m1 = fmax(m1, a.part_corr[((int64_t)b * a.nch + c) * 2]);
  const double lam = s.lam, nrho = sqrt(rr);
  const double e = s.c_epsz + residual_bound(L, s.c_kapz, s.c_nnz, nrho, sizeof(VT) == 8, !s.c_res_tight);
  double sp_ = 0.0;
  if (rr > 0.0) {
    const double beta = yr / (lam * rr);
    sp_ = m1 > 0.0 ? fmin(fmax(beta, -1.0 / m1), 1.0 / m1) : beta;
  }
  const double P = 0.5 * rr + lam * s.c_l1;
  const double D = lam * sp_ * yr - 0.5 * lam * lam * sp_ * sp_ * rr;
  const double g = fmax(P - D + nrho * e + 0.5 * e * e, 0.0) / s.yy;
  // the audit recomputes every bound along another rounding path; unsafe screening would show
  // as a gross excess, while a gap certified just below tol may come out a few ulps above it
  if (g > a.sp.tol * (1.0 + 1e-3)) {
    s.status = LASSO_WARN_AUDIT;
    s.gap = fmax(g, s.gap);
  }
}

template <typename VT>
__global__ void k_outputs(PassArgs<VT> a, float* __restrict__ Xf, double* __restrict__ gaps, int32_t* __restrict__ status,
                          int32_t* __restrict__ iters, uint8_t* __restrict__ kept_out) {
  const int b = blockIdx.y;
  const SigState& s = a.st[b];
  if (Xf) {
    const VT* xo = a.Xout + (int64_t)b * a.K;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.K; j += (int64_t)gridDim.x * blockDim.x)
      Xf[(int64_t)b * a.K + j] = (float)xo[j];
  }
  if (kept_out) {
    // the preservation mask is cleared by every rejection; an empty preserved set (lambda >=
    // lambda_max, y = 0) leaves it untouched, hence the n_kept test
    const uint8_t* mk = a.mask + (int64_t)b * a.K;
    const bool any = s.n_kept > 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.K; j += (int64_t)gridDim.x * blockDim.x)
      kept_out[(int64_t)b * a.K + j] = any ? mk[j] : (uint8_t)0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (gaps) gaps[b] = s.gap;
    if (status) status[b] = s.status == LASSO_ST_SATURATED ? LASSO_ERR_MAXITER : s.status;
    if (iters) iters[b] = s.iters;
  }
}

template <typename VT>
__global__ void k_load_y(PassArgs<VT> a, const float* __restrict__ Yf, const double* __restrict__ Yd) {
  const int b = blockIdx.y;
  VT* y = const_cast<VT*>(a.Yw) + (int64_t)b * a.ldN;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < a.ldN; n += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (n < a.dd.N) v = Yf ? (double)Yf[(int64_t)b * a.dd.N + n] : Yd[(int64_t)b * a.dd.N + n];
    y[n] = (VT)v;
  }
}

// ------------------------------------------------------------------ host driver

// Optional step tracing (environment LASSO_TRACE_STEPS=1): after a launch, poll the stream for at
// most 10 s and report on stderr whether the step completed.  Diagnostics only.
static bool trace_steps() {
  static int v = -1;
  if (v < 0) v = getenv("LASSO_TRACE_STEPS") != nullptr;
  return v == 1;
}

static void trace_step(cudaStream_t st, const char* name) {
  if (!trace_steps()) return;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t q = cudaStreamQuery(st);
  while (q == cudaErrorNotReady &&
         std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() < 10.0)
    q = cudaStreamQuery(st);
  fprintf(stderr, "[lasso trace] %-28s %s (%.3f s)\n", name,
          q == cudaSuccess ? "done" : (q == cudaErrorNotReady ? "NOT DONE after 10 s" : cudaGetErrorString(q)),
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
}

int g_num_sms = 0;

static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 132;
  }
  return g_num_sms;
}

struct SolveIO {
  const float* Yf = nullptr;      // device, B x N
  const double* Yd = nullptr;     // device, B x N
  const double* lambdas = nullptr;  // device
  int64_t B = 0;
  double tol = 1e-6;
  lasso_opts opts;
  float* Xf = nullptr;            // device outputs (batch API)
  double* gaps = nullptr;
  int32_t* status = nullptr;
  int32_t* iters = nullptr;
  cudaStream_t stream = nullptr;
  // the solve must certify the FP32 point it returns (second solve of saturated signals)
  bool point_f32 = false;
};

// Events of one pass (profile mode): before residual stage, before correlation, before
// screening, before schedule, end; Kronecker stages are timed between their own events.
constexpr int PASS_EVENTS = 9;

// A tensor-core level of the current solve: its operand tensor maps and scales.
struct TcJob {
  int lvl, fp8;
  TcOperands ops;
  const float* scale;
  float* rsig;
};

template <typename VT>
static void launch_pass(const PassArgs<VT>& pa, cudaStream_t st, bool has_kron, bool has_faust, int corr_grid,
                        size_t corr_smem,
                        cudaEvent_t* ev, const std::vector<TcJob>& tc, int* tc_err, const TcJob* full_job) {
  const int B = pa.sp.B;
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  if (has_kron) {
    // structured residual: X = d * z, U_r = B_r X, A~z = sum_r U_r C_r^T
    const int Rmax = [&] {
      int m = 0;
      for (int l = 0; l < pa.dd.n_levels; ++l)
        if (pa.dd.lv[l].kind == LK_KRON) m = std::max(m, pa.dd.lv[l].R);
      return m;
    }();
    const LevelDev* KL = nullptr;
    for (int l = 0; l < pa.dd.n_levels; ++l)
      if (pa.dd.lv[l].kind == LK_KRON) KL = &pa.dd.lv[l];
    const int N1 = KL->N1, N2 = KL->N2, K2 = KL->K2;
    auto tiles = [](int v) { return (unsigned)((v + GEMM_T - 1) / GEMM_T); };
    k_kron_scatter<VT><<<dim3(1, B), 256, 0, st>>>(pa);
    k_kron_gemm<VT, KS_U><<<dim3(tiles(K2), tiles(N1), B * Rmax), 256, 0, st>>>(pa);
    k_kron_gemm<VT, KS_Y><<<dim3(tiles(N2), tiles(N1), B), 256, 0, st>>>(pa);
  }
  if (has_faust) k_faust_fwd<VT><<<B, 256, 0, st>>>(pa);
  if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
  k_residual<VT><<<B, RES_THREADS, 0, st>>>(pa);
  if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
  if (has_kron) {
    const int Rmax = [&] {
      int m = 0;
      for (int l = 0; l < pa.dd.n_levels; ++l)
        if (pa.dd.lv[l].kind == LK_KRON) m = std::max(m, pa.dd.lv[l].R);
      return m;
    }();
    const LevelDev* KL = nullptr;
    for (int l = 0; l < pa.dd.n_levels; ++l)
      if (pa.dd.lv[l].kind == LK_KRON) KL = &pa.dd.lv[l];
    const int K1 = KL->K1, N2 = KL->N2, K2 = KL->K2;
    auto tiles = [](int v) { return (unsigned)((v + GEMM_T - 1) / GEMM_T); };
    k_kron_gemm<VT, KS_T><<<dim3(tiles(N2), tiles(K1), B * Rmax), 256, 0, st>>>(pa);
    k_kron_gemm<VT, KS_G><<<dim3(tiles(K2), tiles(K1), B), 256, 0, st>>>(pa);
  }
  if (has_faust) k_faust_adj<VT><<<B, 256, 0, st>>>(pa);
  if (ev) cudaEventRecordWithFlags(ev[7], st, cudaEventRecordExternal);
  for (const TcJob& j : tc) {
    k_quant_rho<VT><<<(unsigned)std::min<int64_t>(B, num_sms() * 4), 256, 0, st>>>(pa, j.lvl, j.fp8);
    tc_launch_corr(j.ops, pa.K, B, pa.ldN, j.scale, j.rsig, pa.tc_list + (int64_t)j.lvl * B, pa.counters + 8 + j.lvl,
                   pa.Gfull, tc_err, st);
  }
  if (ev) cudaEventRecordWithFlags(ev[8], st, cudaEventRecordExternal);
  if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
  if constexpr (sizeof(VT) == 4) k_corr_pass<VT><<<corr_grid, CORR_THREADS, 0, st>>>(pa);
  else k_corr<VT, CORR_PASS><<<corr_grid, CORR_THREADS, corr_smem, st>>>(pa);
  if (ev) cudaEventRecordWithFlags(ev[4], st, cudaEventRecordExternal);
  k_eval<VT><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(pa);
  k_screen<VT><<<B, SCREEN_THREADS, 0, st>>>(pa);
  if (pa.sp.full_gap) {
    k_schedule_full<VT><<<1, 1024, 0, st>>>(pa);
    if (full_job) {
      k_quant_rho<VT><<<(unsigned)std::min<int64_t>(B, num_sms() * 4), 256, 0, st>>>(pa, full_job->lvl,
                                                                                 full_job->fp8, FULL_SET);
      tc_launch_corr(full_job->ops, pa.K, B, pa.ldN, full_job->scale, full_job->rsig,
                     pa.tc_list + (int64_t)FULL_SET * B, pa.counters + 8 + FULL_SET, pa.Gfull, tc_err, st);
      k_full_check_tc<VT><<<(unsigned)std::min<int64_t>(B, num_sms() * 4), 256, 0, st>>>(pa, full_job->lvl);
    } else {
      k_full_check<VT><<<corr_grid, CORR_THREADS, 0, st>>>(pa);
    }
    k_full_finish<VT><<<(unsigned)std::min<int64_t>(B, num_sms() * 8), 128, 0, st>>>(pa);
  }
  if (ev) cudaEventRecordWithFlags(ev[5], st, cudaEventRecordExternal);
  k_schedule<VT><<<1, 1024, 0, st>>>(pa, 1);
  if (ev) cudaEventRecordWithFlags(ev[6], st, cudaEventRecordExternal);
}

static int pass_launches(bool has_kron, bool has_faust, bool full_gap, int n_tc, bool tc_full) {
  return (has_kron ? 10 : 5) + (has_faust ? 2 : 0) + (full_gap ? (tc_full ? 5 : 3) : 0) + 2 * n_tc;
}

// ------------------------------------------------------------------ autotuner

// Synthetic exact-level state for timing the correlation pass: every signal keeps n_kept atoms
// spread evenly over the dictionary and has a bounded pseudo-random residual.
template <typename VT>
__global__ void k_tune_state(PassArgs<VT> a, int n_kept) {
  const int b = blockIdx.x;
  int32_t* kp = kept_of(a, b, 0);
  for (int p = threadIdx.x; p < n_kept; p += blockDim.x) kp[p] = (int32_t)(((int64_t)p * a.K) / n_kept);
  VT* rho = a.Rho + (int64_t)b * a.ldN;
  for (int64_t n = threadIdx.x; n < a.ldN; n += blockDim.x)
    rho[n] = n < a.dd.N ? (VT)((float)((uint32_t)(n * 2654435761u + (uint32_t)b * 40503u) >> 22) / 1024.f - 0.5f)
                        : (VT)0;
  if (threadIdx.x == 0) {
    SigState st;
    memset(&st, 0, sizeof(st));
    st.level = a.dd.n_levels - 1;
    st.n_kept = n_kept;
    st.n_chunks = (n_kept + a.sp.chunk - 1) / a.sp.chunk;
    st.lam = 1.0;
    st.nrho_ru = 1.f;
    st.thr_f = 1e-3f;
    st.beta_f = 0.5f;
    a.st[b] = st;
  }
}

// Atom chunk and grid of the FP32 correlation pass for a batch size class: the configuration
// with the shortest time on the synthetic exact-level state (K / 8 preserved atoms per signal),
// measured with CUDA events on the solve's stream; kept per dictionary.
template <typename VT>
static int tune_corr(lasso_dict* d, const PassArgs<VT>& pa0, int64_t B, cudaStream_t st, int* chunk, int* bps) {
  int cls = 0;
  while ((int64_t)1 << cls < B) ++cls;
  auto it = d->corr_tune.find(cls);
  if (it != d->corr_tune.end()) {
    *chunk = it->second.chunk;
    *bps = it->second.bps;
    return LASSO_OK;
  }
  PassArgs<VT> pa = pa0;
  const int I = pa.dd.n_levels - 1;
  pa.dd.lv[I].tc = 0;                       // time the gathered products themselves
  const int n_kept = (int)std::max<int64_t>(32, d->K / 8);
  cudaEvent_t e0, e1;
  LASSO_CUDA_TRY(cudaEventCreate(&e0));
  LASSO_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int bc = 4 * CORR_CHUNK, bb = 8;
  const int chunks[3] = {2 * CORR_CHUNK, 4 * CORR_CHUNK, 8 * CORR_CHUNK};
  const int grids[3] = {4, 8, 16};
  for (int c : chunks) {
    pa.sp.chunk = c;
    k_tune_state<VT><<<(unsigned)B, 256, 0, st>>>(pa, n_kept);
    k_schedule<VT><<<1, 1024, 0, st>>>(pa, 0);
    for (int g : grids) {
      const int grid = num_sms() * g;
      k_corr_pass<VT><<<grid, CORR_THREADS, 0, st>>>(pa);   // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) k_corr_pass<VT><<<grid, CORR_THREADS, 0, st>>>(pa);
      cudaEventRecord(e1, st);
      LASSO_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      LASSO_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bc = c;
        bb = g;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  LASSO_CUDA_TRY(cudaGetLastError());
  lasso_dict::CorrTune& t = d->corr_tune[cls];
  t.chunk = bc;
  t.bps = bb;
  t.exact_ns = 1e6 * (double)best / 3.0 / ((double)B * n_kept);   // per (signal, atom) product
  *chunk = bc;
  *bps = bb;
  return LASSO_OK;
}

// Relative complexity of the tensor-core levels, measured (Section V-A measures RC rather than
// deriving it): the time per signal of the level's batched product over every atom, over the
// time per signal of the exact level's gather over every atom (its per-atom cost from tune_corr).
// Measured once per dictionary and batch size class; a level whose RC the caller set keeps it.
static int tune_tc_rc(lasso_dict* d, PassArgs<float>& pa, const std::vector<const HostLevel*>& order,
                      const std::vector<TcJob>& jobs, int64_t B, cudaStream_t st, int* tc_err) {
  int cls = 0;
  while ((int64_t)1 << cls < B) ++cls;
  auto it = d->corr_tune.find(cls);
  if (it == d->corr_tune.end() || !(it->second.exact_ns > 0.0) || jobs.empty()) return LASSO_OK;
  lasso_dict::CorrTune& t = it->second;
  if ((int)t.rc.size() != pa.dd.n_levels) {
    t.rc.assign(pa.dd.n_levels, -1.0);
    cudaEvent_t e0, e1;
    LASSO_CUDA_TRY(cudaEventCreate(&e0));
    LASSO_CUDA_TRY(cudaEventCreate(&e1));
    for (const TcJob& j : jobs) {
      tc_launch_corr(j.ops, pa.K, B, pa.ldN, j.scale, j.rsig, nullptr, nullptr, pa.Gfull, tc_err, st);   // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2; ++r)
        tc_launch_corr(j.ops, pa.K, B, pa.ldN, j.scale, j.rsig, nullptr, nullptr, pa.Gfull, tc_err, st);
      cudaEventRecord(e1, st);
      LASSO_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      LASSO_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      const double ns_signal = 1e6 * (double)ms / 2.0 / (double)B;
      t.rc[j.lvl] = ns_signal / (t.exact_ns * (double)pa.K);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LASSO_CUDA_TRY(cudaGetLastError());
  }
  for (int l = 0; l < pa.dd.n_levels; ++l)
    if (t.rc[l] > 0.0 && !order[l]->rc_set) pa.dd.lv[l].rc = t.rc[l];
  return LASSO_OK;
}

template <typename VT>
static int run_solve(lasso_dict* d, Workspace* w, const SolveIO& io, lasso_stats* stats) {
  auto t_start = std::chrono::steady_clock::now();
  const lasso_opts& o = io.opts;
  const int64_t B = io.B;
  cudaStream_t st = io.stream ? io.stream : w->stream;
  if (!io.stream) LASSO_CUDA_TRY(cudaStreamSynchronize(0));   // inputs written on the legacy stream
  PassArgs<VT> pa;
  memset(&pa, 0, sizeof(pa));
  std::vector<const HostLevel*> order;
  const bool tc_batch = o.tensor_cores && B >= TC_BN && d->K >= TC_BM;
  bool any_approx = false;
  for (auto& h : d->approx) any_approx |= h.kind == LK_BF16 || h.kind == LK_FP8;
  const bool want_tc = tc_batch && any_approx;
  const bool tc_exact = tc_batch && o.tc_exact && sizeof(VT) == 4 && !o.final_fp64 && d->exact_kind == LK_F32;
  const bool split_lv = tc_batch && o.split_level && !tc_exact && sizeof(VT) == 4 && !o.final_fp64 &&
                        d->exact_kind == LK_F32;
  int rc = build_dict_dev(d, o.final_fp64 != 0, &pa.dd, &order, want_tc, tc_exact, split_lv);
  if (rc) return rc;
  std::vector<TcJob> tc_jobs;
  for (int l = 0; l < pa.dd.n_levels; ++l) {
    LevelDev& L = pa.dd.lv[l];
    if (!L.tc) continue;
    const int fp8 = L.kind == LK_FP8;
    if (!w->rq[l]) {
      if (ws_alloc(&w->rq[l], (size_t)w->B * d->ldN * 2) || ws_alloc((void**)&w->rsig[l], (size_t)w->B * 4))
        return LASSO_ERR_NOMEM;
      LASSO_CUDA_TRY(cudaMemset(w->rq[l], 0, (size_t)w->B * d->ldN * 2));
    }
    if (L.split && !w->rq2[l]) {
      if (ws_alloc(&w->rq2[l], (size_t)w->B * d->ldN * 2)) return LASSO_ERR_NOMEM;
      LASSO_CUDA_TRY(cudaMemset(w->rq2[l], 0, (size_t)w->B * d->ldN * 2));
    }
    L.rq = w->rq[l];
    L.rq2 = L.split ? w->rq2[l] : nullptr;
    L.rsig = w->rsig[l];
    TcJob job;
    job.lvl = l;
    job.fp8 = fp8;
    job.scale = fp8 ? L.scale : nullptr;
    job.rsig = fp8 ? L.rsig : nullptr;
    if (L.split)
      rc = tc_make_operands(d->exact.split1, d->exact.split2, d->K, L.rq, L.rq2, B, d->ldN, 0, &job.ops);
    else
      rc = tc_make_operands(L.data, nullptr, d->K, L.rq, nullptr, B, d->ldN, fp8, &job.ops);
    if (rc) return rc;
    tc_jobs.push_back(job);
  }
  if (!tc_jobs.empty() && !w->Gfull) {
    if (ws_alloc((void**)&w->Gfull, (size_t)w->B * d->K * 4)) return LASSO_ERR_NOMEM;
  }
  bool has_kron = false, has_faust = false;
  int rmax = 0;
  for (int l = 0; l < pa.dd.n_levels; ++l) {
    has_kron |= pa.dd.lv[l].kind == LK_KRON;
    has_faust |= pa.dd.lv[l].kind == LK_FAUST;
    if (pa.dd.lv[l].kind == LK_KRON) rmax = std::max(rmax, pa.dd.lv[l].R);
  }
  if (has_kron && B * rmax > 65535) {
    set_last_error("Kronecker levels: signals x terms above 65535 in one batch", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  pa.sp.tol = io.tol;
  pa.sp.Gamma = o.Gamma;
  pa.sp.tau = o.tau;
  pa.sp.L = d->L;
  pa.sp.inv_L = 1.0 / d->L;
  pa.sp.algo = o.algo;
  pa.sp.rule = o.rule;
  pa.sp.screen_every = std::max(1, o.screen_every);
  pa.sp.max_iter = std::max(1, o.max_iter);
  pa.sp.B = (int)B;
  pa.sp.chunk = B >= 64 ? 4 * CORR_CHUNK : CORR_CHUNK;
  pa.sp.full_gap = o.full_gap ? 1 : 0;
  // FP64 iterates that must certify the FP32 point they return keep that point FP32-representable
  pa.sp.z_f32 = sizeof(VT) == 8 && io.point_f32 ? 1 : 0;
  // saturation of the FP32 iterates on the exact level: 200 passes without a 2 % better
  // certificate (a converging FISTA improves far faster), then the FP64 solve takes over
  pa.sp.stall_passes = sizeof(VT) == 4 && o.fp64_fallback && d->exact_kind == LK_F32 ? 200 : 0;
  // the second solve of saturated signals returns an FP32 point, whose certificate has a floor
  // of its own (reading of the tolerance floor): it stops on the same stall test (status
  // LASSO_ERR_MAXITER with its best certificate) instead of running to the pass limit
  // (FISTA only: ISTA's certificate can plateau for long stretches and still converge)
  if (sizeof(VT) == 8 && io.point_f32 && o.algo == LASSO_FISTA) pa.sp.stall_passes = 2000;
  fill_pass_args(pa, w, d);
  int corr_bps = 8;
  if constexpr (sizeof(VT) == 4) {
    if (o.autotune && B >= 64) {
      int c = 0, g = 0;
      rc = tune_corr<VT>(d, pa, B, st, &c, &g);
      if (rc) return rc;
      pa.sp.chunk = c;
      corr_bps = g;
      rc = tune_tc_rc(d, pa, order, tc_jobs, B, st, w->tc_err);
      if (rc) return rc;
    }
  }
  const size_t vs = sizeof(VT);
  const size_t BK = (size_t)B * d->K;
  LASSO_CUDA_TRY(cudaMemsetAsync(w->X, 0, BK * vs, st));
  LASSO_CUDA_TRY(cudaMemsetAsync(w->Z, 0, BK * vs, st));
  LASSO_CUDA_TRY(cudaMemsetAsync(w->Xout, 0, BK * vs, st));
  LASSO_CUDA_TRY(cudaMemsetAsync(w->Rho, 0, (size_t)B * d->ldN * vs, st));
  LASSO_CUDA_TRY(cudaMemsetAsync(w->part_res, 0, (size_t)B * w->nrb * 16, st));
  k_load_y<VT><<<dim3((unsigned)((d->ldN + 255) / 256), (unsigned)B), 256, 0, st>>>(pa, io.Yf, io.Yd);
  k_init_state<VT><<<(unsigned)B, 256, 0, st>>>(pa, io.lambdas);
  // smem for the staged vector
  size_t corr_smem = 0;
  static bool attr_set[2] = {false, false};
  if (!attr_set[vs == 8]) {
    cudaFuncSetAttribute(k_corr<VT, CORR_PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_corr<VT, CORR_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_corr<VT, CORR_CERT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set[vs == 8] = true;
  }
  const int corr_grid = num_sms() * corr_bps;
  // init: lambda_max and a^T y bounds with the most precise level
  LASSO_CUDA_TRY(cudaMemsetAsync(w->tc_err, 0, 4, st));
  k_schedule<VT><<<1, 1024, 0, st>>>(pa, 0);
  // initial pass: on the tensor cores when a BF16 (else FP8) level runs there, else exact products
  const TcJob* init_job = nullptr;
  for (const TcJob& j : tc_jobs)
    if (!pa.dd.lv[j.lvl].split && (!init_job || (init_job->fp8 && !j.fp8))) init_job = &j;
  if (sizeof(VT) == 4 && init_job) {
    LASSO_CUDA_TRY(cudaMemcpyAsync(w->Rho, w->Yw, (size_t)B * d->ldN * vs, cudaMemcpyDeviceToDevice, st));
    k_quant_rho<VT><<<(unsigned)B, 256, 0, st>>>(pa, init_job->lvl, init_job->fp8, -1);
    tc_launch_corr(init_job->ops, pa.K, B, pa.ldN, init_job->scale, init_job->rsig, nullptr, nullptr, pa.Gfull,
                   w->tc_err, st);
    k_init_tc<VT><<<(unsigned)B, 256, 0, st>>>(pa, init_job->lvl);
  } else {
    k_corr<VT, CORR_INIT><<<corr_grid, CORR_THREADS, corr_smem, st>>>(pa);
  }
  k_init_finish<VT><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(pa, o.lambda_relative);
  pa.sp.corr_grid = corr_grid;
  // the full-dictionary check uses the same tensor-core level when the exact level is FP32 data
  // and that level is BF16: the E4M3 level's bounds (eps_j of a few percent) let most rejected
  // atoms reach the preserved maximum, and each of those is recomputed from its exact row
  const TcJob* full_job = sizeof(VT) == 4 && pa.dd.lv[pa.dd.n_levels - 1].kind == LK_F32 && pa.sp.full_gap &&
                                  init_job && !init_job->fp8
                              ? init_job
                              : nullptr;
  k_schedule<VT><<<1, 1024, 0, st>>>(pa, 1);
  LASSO_CUDA_TRY(cudaGetLastError());
  LASSO_CUDA_TRY(cudaMemsetAsync(w->alg_bytes, 0, 16 * sizeof(double), st));
  // capture k passes
  const int k = std::max(1, o.passes_per_sync);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  LASSO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  std::vector<cudaEvent_t> evs;
  if (o.profile) {
    evs.resize((size_t)k * PASS_EVENTS);
    for (auto& e : evs) LASSO_CUDA_TRY(cudaEventCreate(&e));
  }
  double kms[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < k; ++i)
    launch_pass<VT>(pa, st, has_kron, has_faust, corr_grid, corr_smem, o.profile ? &evs[(size_t)i * PASS_EVENTS] : nullptr,
                    tc_jobs, w->tc_err, full_job);
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess) {
    set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  int64_t replays = 0;
  int result = LASSO_OK;
  bool timed_out = false;
  const int64_t max_replays = (int64_t)pa.sp.max_iter / k + 2;
  LASSO_CUDA_TRY(cudaMemsetAsync(w->counters + 1, 0, 4, st));   // wall-clock stop flag
  while (true) {
    ce = cudaMemcpyAsync(w->h_counters, w->counters, 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
      result = LASSO_ERR_CUDA;
      break;
    }
    if (o.profile && replays > 0) {
      for (int i = 0; i < k; ++i) {
        cudaEvent_t* e = &evs[(size_t)i * PASS_EVENTS];
        float t;
        if (cudaEventElapsedTime(&t, e[0], e[1]) == cudaSuccess) kms[4] += t;
        if (cudaEventElapsedTime(&t, e[1], e[2]) == cudaSuccess) kms[0] += t;
        if (cudaEventElapsedTime(&t, e[2], e[7]) == cudaSuccess) kms[4] += t;
        if (cudaEventElapsedTime(&t, e[3], e[4]) == cudaSuccess) kms[1] += t;
        if (cudaEventElapsedTime(&t, e[4], e[5]) == cudaSuccess) kms[2] += t;
        if (cudaEventElapsedTime(&t, e[5], e[6]) == cudaSuccess) kms[3] += t;
        if (cudaEventElapsedTime(&t, e[7], e[8]) == cudaSuccess) kms[5] += t;
      }
      cudaGetLastError();   // a failed timing query must not leave a sticky error behind
    }
    if (w->h_counters[0] >= B) break;
    if (replays >= max_replays || timed_out) break;
    if (o.time_limit_s > 0.0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      if (el > o.time_limit_s) {
        // one more replay: every live signal takes the flag at its next pass and stops with its
        // current point and certificate (status LASSO_ERR_TIMEOUT)
        result = LASSO_ERR_TIMEOUT;
        timed_out = true;
        ce = cudaMemsetAsync(w->counters + 1, 1, 1, st);
        if (ce != cudaSuccess) {
          set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
          result = LASSO_ERR_CUDA;
          break;
        }
      }
    }
    ce = cudaGraphLaunch(exec, st);
    if (ce != cudaSuccess) {
      set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
      result = LASSO_ERR_CUDA;
      break;
    }
    ++replays;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  for (auto& e : evs) cudaEventDestroy(e);
  if (result == LASSO_ERR_CUDA) return result;
  double hbytes[16] = {0};
  LASSO_CUDA_TRY(cudaMemcpyAsync(hbytes, w->alg_bytes, sizeof(hbytes), cudaMemcpyDeviceToHost, st));
  LASSO_CUDA_TRY(cudaStreamSynchronize(st));
  int64_t launches = 6 + replays * (int64_t)k * pass_launches(has_kron, has_faust, pa.sp.full_gap != 0, (int)tc_jobs.size(), full_job != nullptr);
  {
    int herr = 0;
    LASSO_CUDA_TRY(cudaMemcpy(&herr, w->tc_err, 4, cudaMemcpyDeviceToHost));
    if (herr) {
      set_last_error("tensor-core pipeline wait expired", __FILE__, __LINE__);
      return LASSO_ERR_TIMEOUT;
    }
  }
  if (o.certify_full && result == LASSO_OK) {
    // certificate over every atom (offsets: K / CHUNK items per signal)
    std::vector<int32_t> offs(B + 1);
    const int nch = (int)((d->K + pa.sp.chunk - 1) / pa.sp.chunk);
    for (int64_t b = 0; b <= B; ++b) offs[b] = (int32_t)(b * nch);
    LASSO_CUDA_TRY(cudaMemcpyAsync(w->offsets, offs.data(), (B + 1) * 4, cudaMemcpyHostToDevice, st));
    k_corr<VT, CORR_CERT><<<corr_grid, CORR_THREADS, corr_smem, st>>>(pa);
    k_cert_finish<VT><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(pa);
    LASSO_CUDA_TRY(cudaStreamSynchronize(st));
    launches += 2;
  }
  launches += 1;
  k_outputs<VT><<<dim3(io.Xf || io.opts.kept_mask ? 64 : 1, (unsigned)B), 256, 0, st>>>(pa, io.Xf, io.gaps, io.status,
                                                                                       io.iters, io.opts.kept_mask);
  LASSO_CUDA_TRY(cudaGetLastError());
  LASSO_CUDA_TRY(cudaStreamSynchronize(st));
  if (stats) {
    std::vector<SigState> hs(B);
    LASSO_CUDA_TRY(cudaMemcpy(hs.data(), w->st, B * sizeof(SigState), cudaMemcpyDeviceToHost));
    memset(stats, 0, sizeof(*stats));
    for (int64_t b = 0; b < B; ++b) {
      stats->passes = std::max<int64_t>(stats->passes, hs[b].iters);
      for (int l = 0; l < MAX_LEVELS; ++l) stats->level_passes[l] += hs[b].level_passes[l];
      stats->kept_final += hs[b].n_kept;
    }
    stats->lambda_max = hs[0].lam_max_lb;
    stats->lambda = hs[0].lam;
    stats->launches = launches;
    stats->corr_chunk = pa.sp.chunk;
    stats->corr_blocks_per_sm = corr_bps;
    for (int l = 0; l < pa.dd.n_levels && l < 8; ++l) stats->level_rc[l] = pa.dd.lv[l].rc;
    const int per_pass[6] = {1, 1, pa.sp.full_gap ? 4 : 1, 1, (has_kron ? 5 : 0) + (has_faust ? 2 : 0), 2 * (int)tc_jobs.size()};
    for (int q = 0; q < 6; ++q) {
      stats->kernel_launches[q] = replays * (int64_t)k * per_pass[q];
      stats->kernel_ms[q] = kms[q];
      stats->kernel_bytes[q] = hbytes[q];
    }
    for (int l = 0; l < MAX_LEVELS; ++l) stats->level_atoms[l] = hbytes[8 + l];
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  return result;
}

}  // namespace lasso

using namespace lasso;

void lasso_workspace_free(lasso::Workspace* ws) { free_ws(ws); }

extern "C" void lasso_opts_default(lasso_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->Gamma = 0.5;
  o->algo = LASSO_FISTA;
  o->rule = LASSO_RULE_GAP;
  o->screen_every = 1;
  o->max_iter = 20000;
  o->lambda_relative = 0;
  o->final_fp64 = 0;
  o->certify_full = 0;
  o->passes_per_sync = 8;
  o->tensor_cores = 1;
  o->tau = 1e-9;
  o->time_limit_s = 0.0;
  o->profile = 0;
  o->full_gap = 1;
  o->tc_exact = 0;
  o->split_level = 1;
  o->fp64_fallback = 1;
  o->autotune = 1;
}

// ------------------------------------------------------------------ FP64 second solve

static int solve_common(lasso_dict* d, SolveIO& io, lasso_stats* stats);

__global__ void k_find_saturated(const SigState* __restrict__ st, int64_t B, int32_t* __restrict__ idx,
                                 int32_t* __restrict__ count) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < B && st[b].status == LASSO_ST_SATURATED) idx[atomicAdd(count, 1)] = (int32_t)b;
}

// Rows of the saturated signals (y as given, lambda as resolved) for the second solve.
__global__ void k_gather_saturated(const SigState* __restrict__ st, const float* __restrict__ Yf,
                                   const double* __restrict__ Yd, int64_t N, const int32_t* __restrict__ idx, int n,
                                   float* __restrict__ Ysub, double* __restrict__ lam) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int64_t b = idx[i];
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x)
    Ysub[(int64_t)i * N + c] = Yf ? Yf[b * N + c] : (float)Yd[b * N + c];
  if (threadIdx.x == 0) lam[i] = st[b].lam;
}

__global__ void k_scatter_saturated(const int32_t* __restrict__ idx, int n, int64_t K, const float* __restrict__ Xs,
                                    const double* __restrict__ gs, const int32_t* __restrict__ ss,
                                    const int32_t* __restrict__ is, const uint8_t* __restrict__ ks,
                                    float* __restrict__ X, double* __restrict__ gaps,
                                    int32_t* __restrict__ status, int32_t* __restrict__ iters, uint8_t* __restrict__ kept) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int64_t b = idx[i];
  if (X)
    for (int64_t j = threadIdx.x; j < K; j += blockDim.x) X[b * K + j] = Xs[(int64_t)i * K + j];
  if (kept && ks)
    for (int64_t j = threadIdx.x; j < K; j += blockDim.x) kept[b * K + j] = ks[(int64_t)i * K + j];
  if (threadIdx.x == 0) {
    if (gaps) gaps[b] = gs[i];
    if (status) status[b] = ss[i];
    if (iters) iters[b] += is[i];
  }
}

// Signals whose FP32 iterates saturated on the exact level are solved again from scratch with
// FP64 iterates and the FP64-accumulation rung (as final_fp64 does), with the lambda each one
// was solved for; their outputs replace the FP32 ones.
static int fp64_fallback(lasso_dict* d, Workspace* w, SolveIO& io, lasso_stats* stats) {
  const int64_t B = io.B, N = d->N, K = d->K;
  cudaStream_t st = io.stream ? io.stream : w->stream;
  int32_t *idx = nullptr, *cnt = nullptr, *ss = nullptr, *is = nullptr;
  float *Ys = nullptr, *Xs = nullptr;
  double *lam = nullptr, *gs = nullptr;
  uint8_t* ks = nullptr;
  auto release = [&]() {
    cudaFree(ks);
    cudaFree(idx);
    cudaFree(cnt);
    cudaFree(ss);
    cudaFree(is);
    cudaFree(Ys);
    cudaFree(Xs);
    cudaFree(lam);
    cudaFree(gs);
  };
  if (cudaMalloc(&idx, B * 4) != cudaSuccess || cudaMalloc(&cnt, 4) != cudaSuccess) {
    release();
    return LASSO_ERR_NOMEM;
  }
  int n = 0;
  LASSO_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4, st));
  k_find_saturated<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(w->st, B, idx, cnt);
  LASSO_CUDA_TRY(cudaMemcpyAsync(&n, cnt, 4, cudaMemcpyDeviceToHost, st));
  LASSO_CUDA_TRY(cudaStreamSynchronize(st));
  if (n == 0) {
    release();
    return LASSO_OK;
  }
  if (cudaMalloc(&Ys, (size_t)n * N * 4) != cudaSuccess || cudaMalloc(&lam, (size_t)n * 8) != cudaSuccess ||
      cudaMalloc(&Xs, (size_t)n * K * 4) != cudaSuccess || cudaMalloc(&gs, (size_t)n * 8) != cudaSuccess ||
      cudaMalloc(&ss, (size_t)n * 4) != cudaSuccess || cudaMalloc(&is, (size_t)n * 4) != cudaSuccess ||
      (io.opts.kept_mask && cudaMalloc(&ks, (size_t)n * K) != cudaSuccess)) {
    release();
    return LASSO_ERR_NOMEM;
  }
  k_gather_saturated<<<n, 256, 0, st>>>(w->st, io.Yf, io.Yd, N, idx, n, Ys, lam);
  LASSO_CUDA_TRY(cudaGetLastError());
  LASSO_CUDA_TRY(cudaStreamSynchronize(st));
  SolveIO sub = io;
  sub.Yf = Ys;
  sub.Yd = nullptr;
  sub.lambdas = lam;
  sub.B = n;
  sub.opts.final_fp64 = 1;
  sub.opts.lambda_relative = 0;
  sub.opts.fp64_fallback = 0;
  sub.point_f32 = true;
  sub.Xf = Xs;
  sub.gaps = gs;
  sub.status = ss;
  sub.iters = is;
  sub.opts.kept_mask = ks;
  lasso_stats sst;
  const int rc = solve_common(d, sub, stats ? &sst : nullptr);
  if (rc == LASSO_OK) {
    k_scatter_saturated<<<n, 256, 0, st>>>(idx, n, K, Xs, gs, ss, is, ks, io.Xf, io.gaps, io.status, io.iters,
                                           io.opts.kept_mask);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      release();
      set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
      return LASSO_ERR_CUDA;
    }
    if (stats) {
      stats->passes = std::max(stats->passes, sst.passes);
      for (int l = 0; l < MAX_LEVELS; ++l) stats->level_passes[l] += sst.level_passes[l];
      stats->launches += sst.launches;
      for (int q = 0; q < 6; ++q) {
        stats->kernel_launches[q] += sst.kernel_launches[q];
        stats->kernel_ms[q] += sst.kernel_ms[q];
        stats->kernel_bytes[q] += sst.kernel_bytes[q];
      }
      stats->seconds += sst.seconds;
      stats->fp64_resolved = n;
    }
  }
  release();
  return rc;
}

static int solve_common(lasso_dict* d, SolveIO& io, lasso_stats* stats) {
  if (!d || io.B <= 0 || !(io.tol > 0.0)) return LASSO_ERR_INVALID_ARG;
  if (io.opts.rule < LASSO_RULE_GAP || io.opts.rule > LASSO_RULE_STATIC || io.opts.algo < LASSO_FISTA ||
      io.opts.algo > LASSO_ISTA)
    return LASSO_ERR_INVALID_ARG;
  if (d->ldN > 24576) {
    set_last_error("solve: signals longer than 24576 (padded) entries", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  if (io.B > 65535) {   // per-signal kernels index the batch by gridDim.y
    set_last_error("solve: more than 65535 signals in one call", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  if (!d->prepared) {
    int rc = dict_prepare(d, 0.0);
    if (rc) return rc;
  }
  // An FP32 point cannot carry a certificate much below 1e-7: the duality gap of the dynamic dual
  // point is first order in the point's rounding (about 6e-8 relative), and on the 2048 x 8192
  // batch a quarter of the signals stall above tol = 1e-7.  Tolerances below 5e-7 on an FP32
  // dictionary run the FP64-accumulation rung with FP64 iterates (as final_fp64 does).
  if (d->exact_kind == LK_F32 && io.tol < FP32_TOL_FLOOR && !io.point_f32) io.opts.final_fp64 = 1;
  const bool vt_double = d->exact_kind == LK_F64 || io.opts.final_fp64;
  Workspace* w = nullptr;
  int rc = get_ws(d, io.B, vt_double, &w);
  if (rc) return rc;
  if (vt_double) return run_solve<double>(d, w, io, stats);
  rc = run_solve<float>(d, w, io, stats);
  if (rc != LASSO_OK || !io.opts.fp64_fallback || d->exact_kind != LK_F32) return rc;
  return fp64_fallback(d, w, io, stats);
}

namespace lasso {
void clear_last_error();   // capi.cu
}  // namespace lasso

extern "C" int lasso_solve_batch(lasso_dict* d, const float* d_Y, const double* d_lambdas, int64_t B, double tol,
                                 const lasso_opts* opts, float* d_X, double* d_gaps, int32_t* d_status,
                                 int32_t* d_iters, void* stream, lasso_stats* stats) {
  lasso::clear_last_error();
  if (!d_Y || !d_lambdas || !d_X) return LASSO_ERR_INVALID_ARG;
  SolveIO io;
  io.Yf = d_Y;
  io.lambdas = d_lambdas;
  io.B = B;
  io.tol = tol;
  if (opts) io.opts = *opts;
  else lasso_opts_default(&io.opts);
  io.Xf = d_X;
  io.gaps = d_gaps;
  io.status = d_status;
  io.iters = d_iters;
  io.stream = (cudaStream_t)stream;
  return solve_common(d, io, stats);
}

extern "C" int lasso_solve_batch_host(lasso_dict* d, const float* Y, const double* lambdas, int64_t B, double tol,
                                      const lasso_opts* opts, float* X, double* gaps, int32_t* status,
                                      lasso_stats* stats) {
  lasso::clear_last_error();
  if (!d || !Y || !lambdas || !X || B <= 0) return LASSO_ERR_INVALID_ARG;
  if (B > 65535) {
    set_last_error("solve: more than 65535 signals in one call", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  float *dY = nullptr, *dX = nullptr;
  double *dl = nullptr, *dg = nullptr;
  int32_t* ds = nullptr;
  uint8_t* dk = nullptr;
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_opts_default(&o);
  uint8_t* kept_host = o.kept_mask;
  const size_t BN = (size_t)B * d->N, BK = (size_t)B * d->K;
  int rc = LASSO_OK;
  if (cudaMalloc(&dY, BN * 4) != cudaSuccess || cudaMalloc(&dX, BK * 4) != cudaSuccess ||
      cudaMalloc(&dl, B * 8) != cudaSuccess || cudaMalloc(&dg, B * 8) != cudaSuccess ||
      cudaMalloc(&ds, B * 4) != cudaSuccess || (kept_host && cudaMalloc(&dk, BK) != cudaSuccess)) {
    rc = LASSO_ERR_NOMEM;
  }
  o.kept_mask = dk;
  if (!rc && (cudaMemcpy(dY, Y, BN * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(dl, lambdas, B * 8, cudaMemcpyHostToDevice) != cudaSuccess))
    rc = LASSO_ERR_CUDA;
  if (!rc) rc = lasso_solve_batch(d, dY, dl, B, tol, &o, dX, dg, ds, nullptr, nullptr, stats);
  if (rc == LASSO_OK || rc == LASSO_ERR_MAXITER || rc == LASSO_ERR_TIMEOUT) {
    if (cudaMemcpy(X, dX, BK * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        (gaps && cudaMemcpy(gaps, dg, B * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (status && cudaMemcpy(status, ds, B * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (kept_host && cudaMemcpy(kept_host, dk, BK, cudaMemcpyDeviceToHost) != cudaSuccess))
      rc = LASSO_ERR_CUDA;
  }
  cudaFree(dk);
  cudaFree(dY);
  cudaFree(dX);
  cudaFree(dl);
  cudaFree(dg);
  cudaFree(ds);
  return rc;
}

extern "C" int lasso_solve(lasso_dict* d, const double* y, double lambda, double tol, const lasso_opts* opts,
                           double* x, double* gap, int32_t* kept, int64_t* n_kept, lasso_stats* stats) {
  lasso::clear_last_error();
  if (!d || !y || !x) return LASSO_ERR_INVALID_ARG;
  double *dy = nullptr, *dl = nullptr;
  if (cudaMalloc(&dy, d->N * 8) != cudaSuccess || cudaMalloc(&dl, 8) != cudaSuccess) {
    cudaFree(dy);
    return LASSO_ERR_NOMEM;
  }
  cudaMemcpy(dy, y, d->N * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dl, &lambda, 8, cudaMemcpyHostToDevice);
  SolveIO io;
  io.Yd = dy;
  io.lambdas = dl;
  io.B = 1;
  io.tol = tol;
  if (opts) io.opts = *opts;
  else lasso_opts_default(&io.opts);
  io.opts.kept_mask = nullptr;   // the single solve returns its preserved set as a list
  lasso_stats local;
  int rc = solve_common(d, io, stats ? stats : &local);
  cudaFree(dy);
  cudaFree(dl);
  if (rc != LASSO_OK && rc != LASSO_ERR_MAXITER && rc != LASSO_ERR_TIMEOUT && rc != LASSO_WARN_AUDIT) return rc;
  // the solve's workspace; a signal finished by the FP64 second solve lives in the FP64 one
  const bool vt_double = d->exact_kind == LK_F64 || io.opts.final_fp64;
  Workspace* w = vt_double ? d->ws64 : d->ws;
  if (!w) return LASSO_ERR_CUDA;
  SigState s;
  if (cudaMemcpy(&s, w->st, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return LASSO_ERR_CUDA;
  if (!vt_double && s.status == LASSO_ST_SATURATED && io.opts.fp64_fallback && d->ws64) {
    w = d->ws64;
    if (cudaMemcpy(&s, w->st, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return LASSO_ERR_CUDA;
  }
  if (s.status == LASSO_ST_SATURATED) s.status = LASSO_ERR_MAXITER;
  if (w->vt_double) {
    if (cudaMemcpy(x, w->Xout, d->K * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return LASSO_ERR_CUDA;
  } else {
    std::vector<float> xf(d->K);
    if (cudaMemcpy(xf.data(), w->Xout, d->K * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LASSO_ERR_CUDA;
    for (int64_t j = 0; j < d->K; ++j) x[j] = xf[j];
  }
  if (gap) *gap = s.gap;
  if (n_kept) *n_kept = s.n_kept;
  if (kept && s.n_kept > 0) {
    if (cudaMemcpy(kept, w->kept + (int64_t)s.parity * d->K, s.n_kept * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return LASSO_ERR_CUDA;
  }
  return s.status != LASSO_OK ? s.status : rc;
}

template <typename VT>
__global__ void k_copy_lmax(PassArgs<VT> a, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < a.sp.B) out[b] = a.st[b].lam_max_lb;
}

template <typename VT>
static int run_lambda_max(lasso_dict* d, Workspace* w, const float* Y, int64_t B, double* out, cudaStream_t st) {
  PassArgs<VT> pa;
  memset(&pa, 0, sizeof(pa));
  int rc = build_dict_dev(d, false, &pa.dd, nullptr);
  if (trace_steps()) fprintf(stderr, "[lasso trace] lmax: levels built rc %d\n", rc);
  if (rc) return rc;
  pa.sp.B = (int)B;
  pa.sp.L = 1.0;
  pa.sp.inv_L = 1.0;
  pa.sp.chunk = CORR_CHUNK;
  fill_pass_args(pa, w, d);
  if (trace_steps()) fprintf(stderr, "[lasso trace] lmax: arguments ready\n");
  k_load_y<VT><<<dim3((unsigned)((d->ldN + 255) / 256), (unsigned)B), 256, 0, st>>>(pa, Y, nullptr);
  trace_step(st, "lmax: k_load_y");
  k_init_state<VT><<<(unsigned)B, 256, 0, st>>>(pa, nullptr);
  trace_step(st, "lmax: k_init_state");
  k_schedule<VT><<<1, 1024, 0, st>>>(pa, 0);
  trace_step(st, "lmax: k_schedule");
  k_corr<VT, CORR_INIT><<<num_sms() * 8, CORR_THREADS, 0, st>>>(pa);
  trace_step(st, "lmax: k_corr init");
  k_init_finish<VT><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(pa, 1);
  trace_step(st, "lmax: k_init_finish");
  k_copy_lmax<VT><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(pa, out);
  trace_step(st, "lmax: k_copy_lmax");
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return LASSO_ERR_CUDA;
  }
  return LASSO_OK;
}

extern "C" int lasso_lambda_max(lasso_dict* d, const float* d_Y, int64_t B, double* d_out, void* stream) {
  lasso::clear_last_error();
  if (!d || !d_Y || !d_out || B <= 0) return LASSO_ERR_INVALID_ARG;
  if (B > 65535) {
    set_last_error("lambda_max: more than 65535 signals in one call", __FILE__, __LINE__);
    return LASSO_ERR_UNSUPPORTED;
  }
  const bool vt_double = d->exact_kind == LK_F64;
  Workspace* w = nullptr;
  if (trace_steps()) fprintf(stderr, "[lasso trace] lmax: enter (stream %p)\n", stream);
  int rc = get_ws(d, B, vt_double, &w);
  if (trace_steps()) fprintf(stderr, "[lasso trace] lmax: workspace rc %d\n", rc);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : w->stream;
  if (!stream) LASSO_CUDA_TRY(cudaStreamSynchronize(0));
  if (trace_steps()) fprintf(stderr, "[lasso trace] lmax: legacy stream synchronised\n");
  if (vt_double) return run_lambda_max<double>(d, w, d_Y, B, d_out, st);
  return run_lambda_max<float>(d, w, d_Y, B, d_out, st);
}
