// FP64 instantiation of transform pass B for every supported length.
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE_B(double)
}  // namespace bem
