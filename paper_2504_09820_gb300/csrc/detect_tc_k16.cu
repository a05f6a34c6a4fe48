// Fused tensor-core detector, instantiated for K = 16 users.
#include "detect_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_detect_tc_k<16>(const DetectTcParams&, int, int, cudaStream_t);
template cudaError_t tc_rem_pool<16>(cudaStream_t, uint8_t**, int**);
}  // namespace fpcg
