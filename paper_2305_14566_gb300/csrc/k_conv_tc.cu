// BF16 implicit-GEMM convolution on tcgen05 tensor cores (placeholder until
// the tensor-core kernel lands: reports every shape as unsupported).
#include "omni_internal.cuh"

namespace omni {
bool conv_tc_supported(int, int, int, int) { return false; }
cudaError_t launch_conv_tc(const ConvArgs&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace omni
