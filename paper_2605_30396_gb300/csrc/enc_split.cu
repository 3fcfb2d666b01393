// The two- and three-tile encoder kernels with selection and solver warps, and
// the alternating two-tile kernel.
#include "encode_core.cuh"

namespace dlsh {
namespace enc {

int launch_alt(const AltArgs& a, int grid, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaFuncSetAttribute(encode_alt_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  encode_alt_kernel<0><<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

template int launch_split<false, 2>(const SplitArgs&, int, cudaStream_t);
template int launch_split<true, 2>(const SplitArgs&, int, cudaStream_t);
template int launch_split<true, 3>(const SplitArgs&, int, cudaStream_t);

}  // namespace enc
}  // namespace dlsh
