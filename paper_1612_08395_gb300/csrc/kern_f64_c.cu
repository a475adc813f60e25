// FP64 instantiation of transform pass C for every supported length.
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE_C(double)
}  // namespace bem
