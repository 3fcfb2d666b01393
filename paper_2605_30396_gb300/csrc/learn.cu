// Alternating minimisation of Eq. 1 (Sec. 2.1) on the device, captured into a
// single CUDA graph: D_0 from K chosen signals, then `iters` x {OMP codes,
// MOD update}, a final OMP pass, and the RMSE after every coding pass.  Also
// the paper's CSC storage export (Sec. 2.2).
#include <math.h>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"

namespace dlsh {

namespace learn {

// D_0 row j = X[init_idx[j]] / ||X[init_idx[j]]||; one warp per atom.
__global__ void init_dict_kernel(const float* __restrict__ X, int64_t N,
                                 const int64_t* __restrict__ init_idx, int K,
                                 float* __restrict__ D, uint32_t* status) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= K) return;
  const int64_t i = init_idx[j];
  if (i < 0 || i >= N) {
    if (lane == 0) flag_status(status, ST_BAD_INPUT);
    return;
  }
  const float x0 = X[i * DLSH_D + lane];
  const float x1 = lane < DLSH_D - 32 ? X[i * DLSH_D + 32 + lane] : 0.f;
  double n2 = static_cast<double>(x0) * x0 + static_cast<double>(x1) * x1;
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  if (!(n2 > 0.0)) {
    if (lane == 0) flag_status(status, ST_BAD_INPUT);
    return;
  }
  const double inv = 1.0 / sqrt(n2);
  D[static_cast<size_t>(j) * DLSH_D + lane] = static_cast<float>(x0 * inv);
  if (lane < DLSH_D - 32) D[static_cast<size_t>(j) * DLSH_D + 32 + lane] = static_cast<float>(x1 * inv);
}

// rmse = sqrt(sum resid / (N d)), fixed-order FP64 reduction in one CTA.
__global__ void rmse_kernel(const float* __restrict__ resid, int64_t N, float* __restrict__ out) {
  __shared__ double part[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc += resid[i];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = N > 0 ? static_cast<float>(sqrt(part[0] / (static_cast<double>(N) * DLSH_D))) : 0.f;
}

__global__ void or_status_kernel(uint32_t* dst, const uint32_t* src) {
  if (*src) atomicOr(dst, *src);
}

struct Ws {
  uint32_t* status;
  float* D_a;
  float* D_b;
  float* resid;
  void* enc;
  void* mod;
};

static size_t carve(void* base, int K, int s, int64_t N, int prec, Ws& w) {
  Carver c(base);
  w.status = c.take<uint32_t>(64);
  w.D_a = c.take<float>(static_cast<size_t>(K) * DLSH_D);
  w.D_b = c.take<float>(static_cast<size_t>(K) * DLSH_D);
  w.resid = c.take<float>(N > 0 ? N : 1);
  w.enc = c.take<uint8_t>(encode_ws_bytes(K, s, prec));
  w.mod = c.take<uint8_t>(mod_ws_bytes(K, s, N));
  return c.size();
}

static int enqueue_all(const float* X, int64_t N, int K, int s, float eps, int iters,
                       const int64_t* init_idx, int prec, float* D_out, uint16_t* idx,
                       float* coef, uint8_t* nnz, float* rmse, const Ws& w, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), st), "dlsh_learn: reset");
  init_dict_kernel<<<(K + 7) / 8, 256, 0, st>>>(X, N, init_idx, K, w.D_a, w.status);
  count_launches(1);
  int rc = check_launch("dlsh_learn: init");
  if (rc) return rc;
  float* cur = w.D_a;
  float* nxt = w.D_b;
  for (int it = 0; it <= iters; ++it) {
    uint32_t* est = nullptr;
    rc = encode_enqueue(cur, K, X, N, s, eps, prec, idx, coef, nnz, w.resid, w.enc, st, &est);
    if (rc) return rc;
    or_status_kernel<<<1, 1, 0, st>>>(w.status, est);
    rmse_kernel<<<1, 1024, 0, st>>>(w.resid, N, rmse + it);
    count_launches(2);
    if (it == iters) break;
    uint32_t* mst = nullptr;
    rc = mod_enqueue(X, N, K, idx, coef, nnz, s, cur, w.resid, nxt, w.mod, st, &mst);
    if (rc) return rc;
    or_status_kernel<<<1, 1, 0, st>>>(w.status, mst);
    count_launches(1);
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  DLSH_CUDA_TRY(cudaMemcpyAsync(D_out, cur, sizeof(float) * K * DLSH_D, cudaMemcpyDeviceToDevice, st),
                "dlsh_learn: copy D");
  return check_launch("dlsh_learn: launch");
}

}  // namespace learn

size_t learn_ws_bytes(int K, int s, int64_t N, int prec) {
  learn::Ws w;
  return learn::carve(nullptr, K, s, N, prec, w);
}

namespace csc {

constexpr int CHUNK = 4096;  // signals per CTA (1024 threads x 4)

__global__ void block_sum_kernel(const uint8_t* __restrict__ nnz, int64_t N, int s,
                                 long long* __restrict__ part) {
  __shared__ long long red[1024];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * CHUNK;
  long long acc = 0;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + threadIdx.x * 4 + q;
    if (i < N) acc += nnz[i] > s ? s : nnz[i];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void scan_parts_kernel(long long* part, int nblocks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long run = 0;
    for (int b = 0; b < nblocks; ++b) {
      const long long v = part[b];
      part[b] = run;
      run += v;
    }
    part[nblocks] = run;
  }
}

__global__ void emit_kernel(const uint16_t* __restrict__ idx, const float* __restrict__ coef,
                            const uint8_t* __restrict__ nnz, int64_t N, int s,
                            const long long* __restrict__ part, int nblocks,
                            int64_t* __restrict__ col_ptr, uint16_t* __restrict__ row_idx,
                            float* __restrict__ val) {
  __shared__ long long sc[1024];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * CHUNK + threadIdx.x * 4;
  int nz[4];
  long long local = 0;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + q;
    nz[q] = i < N ? (nnz[i] > s ? s : nnz[i]) : 0;
    local += nz[q];
  }
  sc[threadIdx.x] = local;
  __syncthreads();
  // inclusive Hillis-Steele scan over the 1024 per-thread sums
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = static_cast<int>(threadIdx.x) >= o ? sc[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += v;
    __syncthreads();
  }
  long long c = part[blockIdx.x] + sc[threadIdx.x] - local;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + q;
    if (i < N) {
      col_ptr[i] = c;
      for (int t = 0; t < nz[q]; ++t) {
        row_idx[c + t] = idx[i * s + t];
        val[c + t] = coef[i * s + t];
      }
      c += nz[q];
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) col_ptr[N] = part[nblocks];
}

}  // namespace csc

}  // namespace dlsh

extern "C" {

size_t dlsh_learn_workspace_size(int K, int d, int s, int64_t N, int precision) {
  if (d != DLSH_D || K < 1 || K > 4096 || s < 1 || s > 16 || N < 0 || precision < 0 ||
      precision > 4)
    return 0;
  if (dlsh::encode_ws_bytes(K, s, precision) == 0) return 0;
  return dlsh::learn_ws_bytes(K, s, N, precision);
}

int dlsh_learn_dictionary(const float* X, int64_t N, int d, int K, int s, float eps, int iters,
                          const int64_t* init_idx, int precision, float* D_out, uint16_t* idx,
                          float* coef, uint8_t* nnz, float* rmse, void* ws, size_t ws_bytes,
                          void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_learn_dictionary: d must be 45");
  if (K < 1 || K > 4096)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_learn_dictionary: K must be in [1, 4096]");
  if (s < 1 || s > 16)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_learn_dictionary: s must be in [1, 16]");
  if (precision < 0 || precision > 4)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_learn_dictionary: unknown precision");
  if (iters < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_learn_dictionary: iters < 0");
  if (N < K)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_learn_dictionary: need N >= K signals");
  if (N * s >= (1LL << 31))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_learn_dictionary: N*s must be < 2^31");
  if (!X || !init_idx || !D_out || !idx || !coef || !nnz || !rmse)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_learn_dictionary: NULL array");
  if (!(eps >= 0.f)) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_learn_dictionary: eps < 0");
  const size_t need = dlsh_learn_workspace_size(K, d, s, N, precision);
  if (need == 0)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_learn_dictionary: configuration does not fit");
  int rc = check_workspace(ws, ws_bytes, need, "dlsh_learn_dictionary");
  if (rc) return rc;
  learn::Ws w;
  learn::carve(ws, K, s, N, precision, w);
  cudaStream_t user = static_cast<cudaStream_t>(stream);

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DLSH_CUDA_TRY(cudaStreamIsCapturing(user, &cap), "dlsh_learn_dictionary: capture query");
  if (cap != cudaStreamCaptureStatusNone) {
    // the caller is capturing: become part of the caller's graph
    rc = learn::enqueue_all(X, N, K, s, eps, iters, init_idx, precision, D_out, idx, coef, nnz,
                            rmse, w, user);
    if (rc) return rc;
    return finish(user, w.status, flags & ~DLSH_FLAG_SYNC, "dlsh_learn_dictionary");
  }
  cudaStream_t cs;
  DLSH_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking),
                "dlsh_learn_dictionary: stream");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "dlsh_learn_dictionary: begin capture");
  }
  rc = learn::enqueue_all(X, N, K, s, eps, iters, init_idx, precision, D_out, idx, coef, nnz,
                          rmse, w, cs);
  e = cudaStreamEndCapture(cs, &graph);
  if (rc == DLSH_OK && e != cudaSuccess) rc = cuda_fail(e, "dlsh_learn_dictionary: end capture");
  if (rc == DLSH_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "dlsh_learn_dictionary: instantiate");
  }
  if (rc == DLSH_OK) {
    e = cudaGraphLaunch(exec, user);
    if (e != cudaSuccess) rc = cuda_fail(e, "dlsh_learn_dictionary: graph launch");
  }
  if (exec) cudaGraphExecDestroy(exec);  // freed once the launch completes
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  return finish(user, w.status, flags, "dlsh_learn_dictionary");
}

int dlsh_init_dictionary(const float* X, int64_t N, int d, const int64_t* init_idx, int K,
                         float* D_out, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_init_dictionary: d must be 45");
  if (K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_init_dictionary: K must be in [1, 65535]");
  if (N < 1 || !X || !init_idx || !D_out)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_init_dictionary: NULL array or N < 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  learn::init_dict_kernel<<<(K + 7) / 8, 256, 0, st>>>(X, N, init_idx, K, D_out, nullptr);
  count_launches(1);
  return finish(st, nullptr, flags, "dlsh_init_dictionary");
}

size_t dlsh_csc_workspace_size(int64_t N) {
  if (N < 0) return 0;
  const int64_t nb = (N + dlsh::csc::CHUNK - 1) / dlsh::csc::CHUNK;
  dlsh::Carver c(nullptr);
  c.take<long long>(nb + 1);
  return c.size();
}

int dlsh_csc_from_ell(const uint16_t* idx, const float* coef, const uint8_t* nnz, int64_t N,
                      int s, int64_t* col_ptr, uint16_t* row_idx, float* val, void* ws,
                      size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (N < 0 || s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_csc_from_ell: bad N or s");
  if (!col_ptr || (N > 0 && (!idx || !coef || !nnz || !row_idx || !val)))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_csc_from_ell: NULL array");
  int rc = check_workspace(ws, ws_bytes, dlsh_csc_workspace_size(N), "dlsh_csc_from_ell");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = static_cast<int>((N + csc::CHUNK - 1) / csc::CHUNK);
  long long* part = static_cast<long long*>(ws);
  if (nb == 0) {
    DLSH_CUDA_TRY(cudaMemsetAsync(col_ptr, 0, sizeof(int64_t), st), "dlsh_csc_from_ell: empty");
    return finish(st, nullptr, flags, "dlsh_csc_from_ell");
  }
  csc::block_sum_kernel<<<nb, 1024, 0, st>>>(nnz, N, s, part);
  csc::scan_parts_kernel<<<1, 1, 0, st>>>(part, nb);
  csc::emit_kernel<<<nb, 1024, 0, st>>>(idx, coef, nnz, N, s, part, nb, col_ptr, row_idx, val);
  count_launches(3);
  return finish(st, nullptr, flags, "dlsh_csc_from_ell");
}

}  // extern "C"
