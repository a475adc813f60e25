// FP64 instantiation of the convolution passes and elementwise kernels, and
// the mixed-precision helpers of the refinement sweep.
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE(double)
template cudaError_t set_smem_attrs<double>(int);

// p64 += dscale * dp on S (FP32 correction), optionally projected onto p >= 0.
__global__ void k_refine_apply(double* p64, const float* dp, double dscale, const uint8_t* S,
                               int project, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (!S[i]) continue;
    double v = p64[i] + dscale * (double)dp[i];
    if (project && v < 0.0) v = 0.0;
    p64[i] = v;
  }
}
void launch_refine_apply(double* p64, const float* dp, double dscale, const uint8_t* S, int project,
                         size_t n, cudaStream_t s) {
  k_refine_apply<<<ew_grid(n), 256, 0, s>>>(p64, dp, dscale, S, project, n);
}

__global__ void k_to_f32_scaled(const double* src, double scale, float* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)(scale * src[i]);
}
void launch_to_f32_scaled(const double* src, double scale, float* dst, size_t n, cudaStream_t s) {
  k_to_f32_scaled<<<ew_grid(n), 256, 0, s>>>(src, scale, dst, n);
}

__global__ void k_to_f32(const double* src, float* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
void launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s) {
  k_to_f32<<<ew_grid(n), 256, 0, s>>>(src, dst, n);
}

__global__ void k_active_set(const double* p, const double* g, uint8_t* S, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    S[i] = (p[i] > 0.0 || g[i] < 0.0) ? 1 : 0;
}
void launch_active_set(const double* p, const double* g, uint8_t* S, size_t n, cudaStream_t s) {
  k_active_set<<<ew_grid(n), 256, 0, s>>>(p, g, S, n);
}
}  // namespace bem
