// Tensor-core solver for given Gram matrices, instantiated for K = 8 users
// (16-wide slots holding diag(A, I)).
#include "solve_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_solve_tc_k<8>(const SolveTcParams&, int, int, cudaStream_t);
template cudaError_t launch_solve_grouped_k<8>(const SolveTcParams&, int, int, cudaStream_t);
}  // namespace fpcg
