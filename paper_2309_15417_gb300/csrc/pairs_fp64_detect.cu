// all-binary64 instantiation of the pair kernel for the narrow phase + collision times (dem_detect); one
// instantiation per translation unit so that the eight build in parallel.
#include "pair_kernel.cuh"

namespace dem {
namespace pk {
template cudaError_t launch_pairs<1, MODE_BOTH>(const PairArgs &, int, cudaStream_t);
}  // namespace pk
}  // namespace dem
