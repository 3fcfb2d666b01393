// The two-tile encoder kernels on two warp groups (FP32, BF16, FP8).
#include "encode_core.cuh"

namespace dlsh {
namespace enc {

template int launch_pair<0, false>(const PairArgs&, int, cudaStream_t);
template int launch_pair<1, false>(const PairArgs&, int, cudaStream_t);
template int launch_pair<1, true>(const PairArgs&, int, cudaStream_t);
template int launch_pair<2, false>(const PairArgs&, int, cudaStream_t);
template int launch_pair<2, true>(const PairArgs&, int, cudaStream_t);

}  // namespace enc
}  // namespace dlsh
