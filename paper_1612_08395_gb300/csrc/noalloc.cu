// bem_convolve_noalloc: the FP64 stress -> displacement transform for callers
// that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts whose device memory is owned by a
// caching allocator or arena that the library must not bypass (an allocation
// beside such a pool fragments it, or fails once the pool holds the memory),
// and latency-critical loops where cudaMalloc's implicit device-wide
// synchronisation is not allowed.  This entry point allocates nothing: the
// scratch the three transform passes need (the transposed half spectrum W, a
// transposed copy of the kernel spectrum, the twiddle and index tables) lives
// in one file-scope device array of kScratchBytes bytes, which every GPU that
// loads the library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address; its device address is obtained once per device with
// cudaGetSymbolAddress (on the first call made with that device current) and
// passed to the kernels.  That first call also opts the pass kernels into the
// shared memory their launch shapes need (the same once-per-device set-up a
// handle does), so it should come before any stream capture.
//
// Every call shares the array and it keeps the previous call's contents.
// Nothing in it needs clearing: each call writes every element it later reads
// (the spectrum copy, the twiddle and index tables and all of W) before
// reading it.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <mutex>

#include <cuda_runtime.h>

#include "bem.h"
#include "bem_impl.h"

namespace {

constexpr size_t kScratchBytes = 2u << 20;  // 2 MiB: W and the spectrum for grids up to 256 x 256
constexpr int kMaxSide = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

__global__ void k_transpose_spectrum(const double* src, double* dst, int hx, int hyq) {
  // src[ky * hx + kx] (as bem_spectrum writes it) -> dst[kx * hyq + ky]
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  if (kx < hx && ky < hyq) dst[(size_t)kx * hyq + ky] = src[(size_t)ky * hx + kx];
}

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int bem_convolve_noalloc(const double* khat, int Nx, int Ny, double compliance,
                                    const double* p, double* u, void* stream) {
  if (Nx < 2 || Ny < 2 || Nx > kMaxSide || Ny > kMaxSide)
    return bem::set_error(BEM_EINVAL, "bem_convolve_noalloc: Nx and Ny must be in 2..256 (static scratch of 2 MiB)");
  if (!khat || !p || !u || !(compliance > 0.0))
    return bem::set_error(BEM_EINVAL, "bem_convolve_noalloc: NULL array or compliance <= 0");
  if (!on_device(khat) || !on_device(p) || !on_device(u))
    return bem::set_error(BEM_EINVAL, "bem_convolve_noalloc: khat, p and u must be device pointers");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return bem::set_error(BEM_ECUDA, "bem_convolve_noalloc: no usable current device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
      // once per device: the pass kernels' shared-memory opt-in, then the
      // scratch array's device address
      const int rc = bem::device_setup(dev);
      if (rc != BEM_OK) return rc;
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return bem::set_error(BEM_ECUDA, "bem_convolve_noalloc: cudaGetSymbolAddress of the scratch failed");
      }
      g_scratch_dev[dev] = ptr;
    }
    base = g_scratch_dev[dev];
  }
  const int px = pow2_at_least(2 * Nx < 32 ? 32 : 2 * Nx);
  const int py = pow2_at_least(2 * Ny < 32 ? 32 : 2 * Ny);
  const int M = px / 2, hx = M + 1, hyq = py / 2 + 1;
  // scratch layout: W | transposed spectrum | FP64 twiddles | FP32 twiddles
  const size_t ntw = (size_t)M + py + M + 1;
  const size_t w_bytes = sizeof(double) * 2 * (size_t)hx * Ny;
  const size_t k_off = (w_bytes + 255) & ~(size_t)255;
  const size_t t_off = (k_off + sizeof(double) * (size_t)hx * hyq + 255) & ~(size_t)255;
  const size_t t32_off = (t_off + sizeof(double2) * ntw + 255) & ~(size_t)255;
  const size_t g_off = (t32_off + sizeof(float2) * ntw + 255) & ~(size_t)255;
  const size_t g_ints = 2 * bem::kSoEntries + (size_t)M + py;
  if (g_off + sizeof(int) * g_ints > kScratchBytes)
    return bem::set_error(BEM_EINVAL, "bem_convolve_noalloc: grid needs more than the 2 MiB static scratch");

  // launch geometry of the plain FP64 passes: the plan a handle of this grid
  // uses for bem_convolve in FP64
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return bem::set_error(BEM_ECUDA, "bem_convolve_noalloc: cannot query the SM count");
  const bem::Plan pl = bem::default_plan(Nx, Ny, px, py, 8, nsm);
  if (!bem::plan_fits(pl, 8))
    return bem::set_error(BEM_EINVAL, "bem_convolve_noalloc: no launchable plan for this grid");

  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = static_cast<unsigned char*>(base);
  double* khat_t = reinterpret_cast<double*>(scratch + k_off);
  double2* tw64 = reinterpret_cast<double2*>(scratch + t_off);
  float2* tw32 = reinterpret_cast<float2*>(scratch + t32_off);
  int* geo = reinterpret_cast<int*>(scratch + g_off);
  bem::launch_geo_tables(geo, geo + bem::kSoEntries, pl.gA, 8, s);
  bem::launch_geo_tables(geo + bem::kSoEntries + M, geo + 2 * bem::kSoEntries + M, pl.gB, 8, s);
  k_transpose_spectrum<<<dim3((hx + 127) / 128, hyq), 128, 0, s>>>(khat, khat_t, hx, hyq);
  bem::launch_twiddles(tw64, tw32, ilog2i(M), s);
  bem::launch_twiddles(tw64 + M, tw32 + M, ilog2i(py), s);
  bem::launch_split_twiddles(tw64 + M + py, tw32 + M + py, M, s);

  bem::PassArgs<double> a{};
  a.pl = pl;
  a.f.src = p;
  a.f.dst = u;
  a.W = scratch;
  a.rows_w = Ny;
  a.nrows_in = Ny;
  a.ncols_in = Nx;
  a.khat = khat_t;
  a.twA = tw64;
  a.twB = tw64 + M;
  a.twS = tw64 + M + py;
  a.soA = geo;
  a.spA = geo + bem::kSoEntries;
  a.soB = geo + bem::kSoEntries + M;
  a.spB = geo + 2 * bem::kSoEntries + M;
  a.uscale = compliance / ((double)px * (double)py);
  bem::launch_pass_a<double>(a, bem::A_PLAIN, s);
  bem::launch_pass_b<double>(a, bem::B_CONV, s);
  bem::launch_pass_c<double>(a, bem::C_PLAIN, s);
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return bem::set_error(BEM_ECUDA, cudaGetErrorString(e));
  return BEM_OK;
}
