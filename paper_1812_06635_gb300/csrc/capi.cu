// Error reporting and build information of the C ABI.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace lasso {

static thread_local char g_last_error[512] = {0};
static thread_local char g_message[640] = {0};

void set_last_error(const char* msg, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", msg, base ? base + 1 : file, line);
}

// Every status-returning call of the C ABI starts with this, so that the message lasso_strerror
// appends belongs to the most recent call on the thread.
void clear_last_error() { g_last_error[0] = 0; }

}  // namespace lasso

extern "C" const char* lasso_strerror(int status) {
  const char* text = nullptr;
  switch (status) {
    case LASSO_OK: return "ok";
    case LASSO_ERR_INVALID_ARG: text = "invalid argument"; break;
    case LASSO_ERR_CUDA: text = "CUDA error"; break;
    case LASSO_ERR_NONFINITE: text = "non-finite value in the data or the gap"; break;
    case LASSO_ERR_MAXITER: text = "iteration limit reached before the tolerance"; break;
    case LASSO_ERR_TIMEOUT: text = "time limit reached before the tolerance"; break;
    case LASSO_ERR_UNSUPPORTED: text = "unsupported size or option"; break;
    case LASSO_ERR_NOMEM: text = "device allocation failed"; break;
    case LASSO_WARN_AUDIT: text = "full-dictionary certificate above the tolerance"; break;
    default: return "unknown status";
  }
  if (!lasso::g_last_error[0]) return text;
  snprintf(lasso::g_message, sizeof(lasso::g_message), "%s: %s", text, lasso::g_last_error);
  return lasso::g_message;
}

extern "C" const char* lasso_build_info(void) {
  return "lasso-gb300 sm_103a";
}
