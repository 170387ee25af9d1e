// All-binary64 instantiations of the pair kernel (compiled apart from the other
// precision so that the two build in parallel).
#include "pair_kernel.cuh"

namespace dem {
namespace pk {
template cudaError_t launch_pairs<1, MODE_NARROW>(const PairArgs &, int, cudaStream_t);
template cudaError_t launch_pairs<1, MODE_CTIME>(const PairArgs &, int, cudaStream_t);
template cudaError_t launch_pairs<1, MODE_BOTH>(const PairArgs &, int, cudaStream_t);
template cudaError_t launch_pairs<1, MODE_NTIME>(const PairArgs &, int, cudaStream_t);
}  // namespace pk
}  // namespace dem
