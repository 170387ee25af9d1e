// FP32 + binary64-fixup instantiation of the pair kernel for the collision times; one
// instantiation per translation unit so that the eight build in parallel.
#include "pair_kernel.cuh"

namespace dem {
namespace pk {
template cudaError_t launch_pairs<0, MODE_CTIME>(const PairArgs &, int, cudaStream_t);
}  // namespace pk
}  // namespace dem
