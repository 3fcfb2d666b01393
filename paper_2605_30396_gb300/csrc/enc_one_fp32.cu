// The one-tile encoder kernels with FP32 correlations: three TF32 products
// with 64- or 128-atom chunks, three FP16 products with 128-atom chunks.
#include "encode_core.cuh"

namespace dlsh {
namespace enc {

template int launch_encode<0, 64, false>(const Args&, int, cudaStream_t);
template int launch_encode<0, 128, false>(const Args&, int, cudaStream_t);
template int launch_encode<OPF16X2, 128, false>(const Args&, int, cudaStream_t);

}  // namespace enc
}  // namespace dlsh
