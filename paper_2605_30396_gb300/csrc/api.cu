// C-ABI plumbing: error reporting, version, device queries and the status
// word check shared by every entry point.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

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

// ---- launch choices recorded by the autotuners ----------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, std::vector<int>> g_tune;
static bool g_tune_loaded = false;

// Reads DLSH_AUTOTUNE_CACHE once: lines {"key": "...", "values": [a, b, ...]},
// and the older encoder lines {"K": k, "s": s, "precision": p, "bn": b}.
static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("DLSH_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    char key[128];
    int v[4];
    int K, s, prec, bn;
    const int n = sscanf(line, " {\"key\": \"%127[^\"]\", \"values\": [%d, %d, %d, %d", key, &v[0], &v[1],
                         &v[2], &v[3]);
    if (n >= 2) {
      g_tune[key] = std::vector<int>(v, v + (n - 1));
    } else if (sscanf(line, " {\"K\": %d, \"s\": %d, \"precision\": %d, \"bn\": %d", &K, &s, &prec, &bn) == 4) {
      char k2[128];
      snprintf(k2, sizeof(k2), "encode K=%d s=%d p=%d", K, s, prec);
      g_tune[k2] = std::vector<int>{bn};
    }
  }
  fclose(f);
}

int tune_get(const char* key, int* vals, int n) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return 0;
  for (int i = 0; i < n; ++i) vals[i] = i < static_cast<int>(it->second.size()) ? it->second[i] : 0;
  return 1;
}

void tune_put(const char* key, const int* vals, int n) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  if (n <= 0) g_tune.erase(key);
  else g_tune[key] = std::vector<int>(vals, vals + (n < 4 ? n : 4));
  const char* path = getenv("DLSH_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune) {
    fprintf(f, "{\"key\": \"%s\", \"values\": [", kv.first.c_str());
    for (size_t i = 0; i < kv.second.size(); ++i) fprintf(f, i ? ", %d" : "%d", kv.second[i]);
    fprintf(f, "]}\n");
  }
  fclose(f);
}

}  // namespace dlsh

extern "C" {

const char* dlsh_last_error(void) { return dlsh::g_err; }

int dlsh_version(void) { return 100; }

int dlsh_num_sms(void) { return dlsh::device_sm_count(); }

unsigned long long dlsh_kernel_launches(void) { return dlsh::g_launches.load(); }

}  // extern "C"
