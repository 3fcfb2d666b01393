// Encoder entry point that allocates nothing and needs no caller workspace.
//
// Some callers cannot allocate device memory: plugins whose host application
// owns every device allocation through its own pool, and real-time loops where
// a cudaMalloc (which can synchronise the device) is not allowed.  For them the
// encoder's scratch (padded FP32 dictionary, Gram matrix, packed tensor-core
// operand image, status word) lives in one file-scope device array of fixed
// size, reserved on every GPU that loads this library until the process exits.
#include <mutex>

#include "host.hpp"
#include "internal.hpp"

namespace dlsh {

namespace noalloc {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB: K <= 1024 at any precision and s
constexpr int kMaxDevices = 64;

// Host code must not use this name as a device address: it is a host-side
// stand-in.  The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static std::mutex g_mu;
static void* g_addr[kMaxDevices] = {};

// The device address of g_scratch on the current device: looked up with
// cudaGetSymbolAddress on every call made while the stream is not capturing (so
// a context rebuilt after cudaDeviceReset is seen) and remembered per device;
// while the stream is capturing, the remembered address is used (an error if
// there is none).
static int scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  DLSH_CUDA_TRY(cudaGetDevice(&dev), "dlsh_encode_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_noalloc: device %d out of range", dev);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DLSH_CUDA_TRY(cudaStreamIsCapturing(st, &cs), "dlsh_encode_noalloc: cudaStreamIsCapturing");
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    DLSH_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch), "dlsh_encode_noalloc: cudaGetSymbolAddress");
    if (!p) return set_error(DLSH_ERR_CUDA, "dlsh_encode_noalloc: null scratch address");
    g_addr[dev] = p;
  } else if (!g_addr[dev]) {
    return set_error(DLSH_ERR_INVALID_ARG,
                     "dlsh_encode_noalloc: the first call on device %d must come before any stream "
                     "capture", dev);
  }
  *out = g_addr[dev];
  return DLSH_OK;
}

}  // namespace noalloc
}  // namespace dlsh

extern "C" size_t dlsh_encode_noalloc_max_bytes(void) { return dlsh::noalloc::kScratchBytes; }

extern "C" int dlsh_encode_noalloc(const float* D, int K, int d, const float* X, int64_t N, int s,
                                   float eps, int precision, uint16_t* idx, float* coef,
                                   uint8_t* nnz, float* resid_sq, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_noalloc: d must be 45");
  if (K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_noalloc: K must be in [1, 65535]");
  if (s < 1 || s > 16)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_noalloc: s must be in [1, 16]");
  if (precision < 0 || precision > 4)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_noalloc: unknown precision %d", precision);
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_noalloc: D is NULL");
  if (N < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_noalloc: N < 0");
  if (N > 0 && (!X || !idx || !coef || !nnz))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_noalloc: NULL X/idx/coef/nnz");
  if (!(eps >= 0.f)) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_noalloc: eps < 0");
  const size_t need = encode_ws_bytes(K, s, precision);
  if (need == 0)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_noalloc: K=%d s=%d does not fit", K, s);
  if (need > noalloc::kScratchBytes)
    return set_error(DLSH_ERR_UNSUPPORTED,
                     "dlsh_encode_noalloc: K=%d s=%d precision=%d needs %zu bytes of scratch, "
                     "more than the fixed %zu (use dlsh_encode with a workspace)",
                     K, s, precision, need, noalloc::kScratchBytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  int rc = noalloc::scratch_address(st, &ws);
  if (rc) return rc;
  uint32_t* status = nullptr;
  rc = encode_enqueue(D, K, X, N, s, eps, precision, idx, coef, nnz, resid_sq, ws, st, &status);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_encode_noalloc");
}
