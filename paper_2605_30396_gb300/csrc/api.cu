// C-ABI plumbing: error reporting, version, device queries and the status
// word check shared by every entry point.
#include <stdarg.h>
#include <atomic>
#include <stdio.h>

#include "host.hpp"

namespace dlsh {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(static_cast<unsigned long long>(n)); }

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = '\0'; }

int cuda_fail(cudaError_t e, const char* what) {
  return set_error(DLSH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return DLSH_OK;
}

int check_workspace(const void* ws, size_t ws_bytes, size_t need, const char* call) {
  if (need == 0) return DLSH_OK;
  if (ws == nullptr)
    return set_error(DLSH_ERR_WORKSPACE, "%s: workspace is NULL (%zu bytes needed)", call, need);
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return set_error(DLSH_ERR_INVALID_ARG, "%s: workspace must be 256-byte aligned", call);
  if (ws_bytes < need)
    return set_error(DLSH_ERR_WORKSPACE, "%s: workspace has %zu bytes, %zu needed", call, ws_bytes,
                     need);
  return DLSH_OK;
}

int finish(cudaStream_t st, const uint32_t* status_dev, int flags, const char* call) {
  int rc = check_launch(call);
  if (rc != DLSH_OK) return rc;
  if (!(flags & DLSH_FLAG_SYNC)) return DLSH_OK;
  uint32_t word = 0;
  if (status_dev) {
    DLSH_CUDA_TRY(cudaMemcpyAsync(&word, status_dev, sizeof(word), cudaMemcpyDeviceToHost, st),
                  call);
  }
  DLSH_CUDA_TRY(cudaStreamSynchronize(st), call);
  if (word & 1u) return set_error(DLSH_ERR_TIMEOUT, "%s: a device-side wait ran out", call);
  if (word & 2u) return set_error(DLSH_ERR_DEVICE, "%s: a kernel found out-of-range data", call);
  return DLSH_OK;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace dlsh

extern "C" {

const char* dlsh_last_error(void) { return dlsh::g_err; }

int dlsh_version(void) { return 100; }

int dlsh_num_sms(void) { return dlsh::device_sm_count(); }

unsigned long long dlsh_kernel_launches(void) { return dlsh::g_launches.load(); }

}  // extern "C"
