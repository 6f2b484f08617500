// Error reporting and build information of the C ABI.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace lasso {

static thread_local char g_last_error[512] = {0};

void set_last_error(const char* msg, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", msg, base ? base + 1 : file, line);
}

}  // namespace lasso

extern "C" const char* lasso_strerror(int status) {
  switch (status) {
    case LASSO_OK: return "ok";
    case LASSO_ERR_INVALID_ARG: return "invalid argument";
    case LASSO_ERR_CUDA: return lasso::g_last_error[0] ? lasso::g_last_error : "CUDA error";
    case LASSO_ERR_NONFINITE: return "non-finite value in the data or the gap";
    case LASSO_ERR_MAXITER: return "iteration limit reached before the tolerance";
    case LASSO_ERR_TIMEOUT: return "time limit reached before the tolerance";
    case LASSO_ERR_UNSUPPORTED: return "unsupported size or option";
    case LASSO_ERR_NOMEM: return "device allocation failed";
    case LASSO_WARN_AUDIT: return "full-dictionary certificate above the tolerance";
  }
  return "unknown status";
}

extern "C" const char* lasso_build_info(void) {
  return "lasso-gb300 sm_103a";
}
