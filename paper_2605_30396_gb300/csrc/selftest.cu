// Self-test of the bounded waits that every pipelined kernel of the library
// relies on.  Each kernel here waits on something that never happens (an
// mbarrier nobody arrives on; a grid barrier one CTA skips), with a short
// budget: the waits must give up, record ST_TIMEOUT in the status word and
// return, leaving the CUDA context usable.  The same helpers
// (mbar_wait, grid_barrier) run in the encoder, the MOD factorisation and the
// fused proposal kernel.
#include "common.cuh"
#include "host.hpp"

namespace dlsh {
namespace selftest {

__global__ void lost_arrival_kernel(uint32_t* status, long long budget) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, budget)) flag_status(status, ST_TIMEOUT);
}

// Cooperative launch: CTA 0 leaves at once and never reaches the barrier.
__global__ void missing_cta_kernel(unsigned* bar, uint32_t* status, long long budget) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, budget, status);
}

}  // namespace selftest
}  // namespace dlsh

extern "C" {

size_t dlsh_selftest_workspace_size(void) { return 256; }

int dlsh_selftest_bounded_wait(int kind, int64_t budget_cycles, void* ws, size_t ws_bytes,
                               void* stream) {
  using namespace dlsh;
  clear_error();
  if (kind != 0 && kind != 1) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_selftest_bounded_wait: kind 0 or 1");
  if (budget_cycles < 1 || budget_cycles > 4000000000LL)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_selftest_bounded_wait: budget out of range");
  int rc = check_workspace(ws, ws_bytes, 256, "dlsh_selftest_bounded_wait");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = static_cast<uint32_t*>(ws);
  unsigned* bar = reinterpret_cast<unsigned*>(static_cast<uint8_t*>(ws) + 64);
  DLSH_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, st), "dlsh_selftest_bounded_wait: reset");
  long long budget = budget_cycles;
  if (kind == 0) {
    selftest::lost_arrival_kernel<<<1, 32, 0, st>>>(status, budget);
  } else {
    void* args[] = {&bar, &status, &budget};
    DLSH_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(selftest::missing_cta_kernel),
                                              dim3(4), dim3(64), args, 0, st),
                  "dlsh_selftest_bounded_wait: launch");
  }
  count_launches(1);
  return finish(st, status, DLSH_FLAG_SYNC, "dlsh_selftest_bounded_wait");
}

}  // extern "C"
