// Tensor-core solver for given Gram matrices, instantiated for K = 64 users.
#include "solve_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_solve_tc_k<64>(const SolveTcParams&, int, int, cudaStream_t);
template cudaError_t launch_solve_grouped_k<64>(const SolveTcParams&, int, int, cudaStream_t);
}  // namespace fpcg
