// FP32 instantiation of the convolution passes and elementwise kernels.
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE(float)
template cudaError_t set_smem_attrs<float>(int);
}  // namespace bem
