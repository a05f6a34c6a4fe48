// Fused tensor-core detector over several (N, K) classes in one launch,
// block size L = 16 (K = 16, 32 and 64 in one kernel).
#include "detect_tc_impl.cuh"

namespace fpcg {
template cudaError_t launch_detect_tc_multi_l<16>(MultiTcParams&, int, int, int, cudaStream_t);
}  // namespace fpcg
