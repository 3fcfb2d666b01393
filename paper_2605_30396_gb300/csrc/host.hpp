// Host-side helpers shared by the C-ABI entry points: thread-local error
// message, CUDA error mapping, workspace carving and the optional synchronous
// status check.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

#include "../../include/dlsh.h"

namespace dlsh {

// Records `code` and a printf-style message for dlsh_last_error(); returns code.
int set_error(int code, const char* fmt, ...);
void clear_error();

// Maps a CUDA runtime error to DLSH_ERR_CUDA with a message naming `what`.
int cuda_fail(cudaError_t e, const char* what);

#define DLSH_CUDA_TRY(expr, what)                            \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::dlsh::cuda_fail(_e, what); \
  } while (0)

// Checks the launch that was just enqueued.
int check_launch(const char* what);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves 256-byte aligned regions out of a caller workspace, or (with base ==
// nullptr) only measures the total.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return align_up(off, 256); }
};

// Validates a workspace pointer/size against the bytes required.
int check_workspace(const void* ws, size_t ws_bytes, size_t need, const char* call);

// With DLSH_FLAG_SYNC: synchronise `st`, read the device status word and map
// it to a status code.  Without: return DLSH_OK (the word stays in the
// workspace for a later check).
int finish(cudaStream_t st, const uint32_t* status_dev, int flags, const char* call);

// Default budget for device-side bounded waits, in SM clock cycles (~2 s).
constexpr long long kWaitBudget = 4000000000LL;

int device_sm_count();

// A value set up once per device, with that device current, and cached for the
// life of the process (function attributes, cooperative grid sizes).  Safe to
// call from several host threads; a failed set-up caches nothing.
template <class T>
class PerDevice {
 public:
  template <class F>
  int get(T* out, F&& init) {
    int dev = 0;
    DLSH_CUDA_TRY(cudaGetDevice(&dev), "dlsh: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDev)
      return set_error(DLSH_ERR_UNSUPPORTED, "dlsh: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(mu_);
    if (!done_[dev]) {
      T v{};
      const int rc = init(v);
      if (rc) return rc;
      val_[dev] = v;
      done_[dev] = true;
    }
    *out = val_[dev];
    return DLSH_OK;
  }

 private:
  static constexpr int kMaxDev = 64;
  std::mutex mu_;
  bool done_[kMaxDev] = {};
  T val_[kMaxDev] = {};
};

// Adds n to the process-wide count of kernels this library has enqueued.
void count_launches(int n);

// Launch choices recorded by the autotuners, keyed by text such as
// "encode K=1024 s=8 p=0", with up to four integer values.  With
// DLSH_AUTOTUNE_CACHE naming a file the table is kept there as JSON lines and
// read back at first use.  tune_get fills vals[0..n) (missing values as 0) and
// returns 1 if the key is known, else 0; tune_put with n <= 0 removes the key.
int tune_get(const char* key, int* vals, int n);
void tune_put(const char* key, const int* vals, int n);

}  // namespace dlsh
