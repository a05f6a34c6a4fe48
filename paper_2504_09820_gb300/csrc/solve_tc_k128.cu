// Tensor-core solver for given Gram matrices, instantiated for K = 128 users.
#include "solve_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_solve_tc_k<128>(const SolveTcParams&, int, int, cudaStream_t);
template cudaError_t launch_solve_grouped_k<128>(const SolveTcParams&, int, int, cudaStream_t);
}  // namespace fpcg
