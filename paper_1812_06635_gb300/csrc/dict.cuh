// Host-side dictionary object shared by the library's translation units.
#pragma once

#include <map>

#include <vector>

#include "common.cuh"

namespace lasso {

struct Workspace;   // solver buffers, defined in solver.cu

struct HostLevel {
  int kind = -1;               // LevelKind
  int api_kind = 0;            // lasso_level_kind, or -1 (exact FP64) / -2 (exact FP32)
  int param = 0;               // Kronecker terms
  void* data = nullptr;        // dense payload (K x ldN)
  float* scale = nullptr;      // FP8 scales
  double* eps = nullptr;
  double* kappa = nullptr;
  float* atnorm = nullptr;
  float* epsr32[4] = {nullptr, nullptr, nullptr, nullptr};   // per (iterate precision, tensor cores)
  float* kappa32 = nullptr;
  float* eps32 = nullptr;      // eps_j rounded up to FP32
  // exact FP32 level only: BF16 split a = a1 + a2 + e3 for the tensor-core exact level
  void* split1 = nullptr;
  void* split2 = nullptr;
  double* e3 = nullptr;        // ||a_j - a1_j - a2_j|| (rounded up)
  float* epsr32_split = nullptr;
  double c2 = 0.0;             // max_j ||a2_j|| / kappa_j (rounded up)
  float* dscale = nullptr;     // Kronecker d_j as FP32
  // product of sparse factors: every CSR array in one allocation, the J descriptors on the device
  void* fbuf = nullptr;
  FaustFactor* fac = nullptr;
  int J = 0, fdim = 0;
  int n_fwd = 0, n_adj = 0;    // sum over factors of the longest row of S_f / of S_f^T
  std::vector<FaustFactor> fac_h;   // host copy of the descriptors (device pointers)
  double u = U32, gam_corr = 0.0, gam_res = 0.0, rc = 1.0;
  bool rc_set = false;
  double eps_mean = 0.0, eps_max = 0.0;
  bool owns_data = true;
};

}  // namespace lasso

struct lasso_dict {
  int device = 0;
  int64_t N = 0, K = 0, ldN = 0;
  int exact_kind = lasso::LK_F32;      // LK_F64 or LK_F32
  bool is_kron = false;
  int R = 0, N1 = 0, K1 = 0, N2 = 0, K2 = 0;
  float* Bf = nullptr;                 // R x N1 x K1
  float* Cf = nullptr;                 // R x N2 x K2
  double* d = nullptr;                 // K, FP64 column scale
  double* gramB = nullptr;             // R x R x K1
  double* gramC = nullptr;             // R x R x K2
  double* anorm = nullptr;             // K, exact atom norms (rounded up)
  float* anorm32 = nullptr;            // the same rounded up to FP32
  double anorm_max = 0.0;              // max_j ||a_j||
  int faust_dim = 0;                   // largest factor dimension over the sparse-factor levels
  std::vector<lasso::HostLevel> approx;
  lasso::HostLevel exact;
  lasso::HostLevel rung64;             // FP64-accumulation rung on FP32 exact data (lazy)
  double L = 0.0;
  bool prepared = false;
  // per batch size class (log2 B): the correlation pass's chunk and blocks per SM, the exact level's
  // measured time per (signal, atom) product in ns, and the measured relative complexity of every
  // tensor-core level of the solve's ladder (index of the level; -1 where not measured)
  struct CorrTune {
    int chunk = 0, bps = 0;
    double exact_ns = 0.0;
    std::vector<double> rc;
  };
  std::map<int, CorrTune> corr_tune;
  lasso::Workspace* ws = nullptr;     // FP32-iterate solves
  lasso::Workspace* ws64 = nullptr;   // FP64-iterate solves
};

namespace lasso {

// Level descriptor for kernels.  vt_double: the solve iterates in FP64 (affects the roundings).
LevelDev make_level_dev(const lasso_dict* d, const HostLevel& h, bool vt_double = false, bool tc = false);
// All levels of a solve, coarsest first, exact (or the FP64 rung) last.  tc_levels: run the
// batched BF16 / FP8 correlations on the tensor cores; tc_exact: the exact FP32 level too, in
// its split BF16 form.
// split_level: one more level before the exact one, the split BF16 pair of the exact FP32 atoms
// correlated on the tensor cores (relative complexity SPLIT_RC).
int build_dict_dev(lasso_dict* d, bool final_fp64, DictDev* out, std::vector<const HostLevel*>* order,
                   bool tc_levels = false, bool tc_exact = false, bool split_level = false);
constexpr double SPLIT_RC = 0.02;
// BF16 split of the exact FP32 level and its bounds (computed once).
int ensure_split(lasso_dict* d);
int ensure_rung64(lasso_dict* d);
int dict_prepare(lasso_dict* d, double L_override);

}  // namespace lasso
