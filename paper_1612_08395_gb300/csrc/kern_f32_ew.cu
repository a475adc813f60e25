// FP32 instantiation of the elementwise kernels.

#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE_EW(float)
}  // namespace bem
