// Fused tensor-core detector, instantiated for K = 16 users.
#include "detect_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_detect_tc_k<16>(const DetectTcParams&, int, int, cudaStream_t);
}  // namespace fpcg
