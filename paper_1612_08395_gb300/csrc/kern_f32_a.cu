// FP32 instantiation of transform pass A for every supported length.
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE_A(float)
}  // namespace bem
