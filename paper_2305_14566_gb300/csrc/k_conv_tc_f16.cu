// FP16 instantiation of the tensor-core convolution kernels (conv_tc_impl.cuh).
#define OMNI_TC_F16 1
#include "conv_tc_impl.cuh"
