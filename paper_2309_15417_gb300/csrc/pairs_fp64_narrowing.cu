// all-binary64 instantiation of the pair kernel for the collision times by the paper's narrowing; one
// instantiation per translation unit so that the eight build in parallel.
#include "pair_kernel.cuh"

namespace dem {
namespace pk {
template cudaError_t launch_pairs<1, MODE_NTIME>(const PairArgs &, int, cudaStream_t);
}  // namespace pk
}  // namespace dem
