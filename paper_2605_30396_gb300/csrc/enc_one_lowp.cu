// The one-tile encoder kernels with BF16 and FP8 correlations (exact top 4 or
// column-quarter winners, re-scored in FP32).
#include "encode_core.cuh"

namespace dlsh {
namespace enc {

template int launch_encode<1, 128, false>(const Args&, int, cudaStream_t);
template int launch_encode<1, 128, true>(const Args&, int, cudaStream_t);
template int launch_encode<2, 128, false>(const Args&, int, cudaStream_t);
template int launch_encode<2, 128, true>(const Args&, int, cudaStream_t);

}  // namespace enc
}  // namespace dlsh
