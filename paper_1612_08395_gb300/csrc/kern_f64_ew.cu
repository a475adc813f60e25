// FP64 instantiation of the elementwise kernels and the FP64 helpers of the
// refinement sweep, twiddle and index tables.
#include <algorithm>
#include "conv_kernels.cuh"

namespace bem {
BEM_INSTANTIATE_EW(double)

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

// Stage twiddle tables of a length 2^logL transform, stages in DIF order,
// tables concatenated.  FP32: the table of stage (R, s) holds
// exp(-2 pi i o/(R s)) for o < s (the radix-8 offsets are tw_off8); the
// butterflies form the powers they need.  FP64: the table of stage (R, s)
// holds every power, exp(-2 pi i o q/(R s)) at (q-1) s + o for q = 1..R-1
// (offsets FftC::pow_off; fewer than 2^logL entries in all).  Computed in FP64.
__global__ void k_twiddles(double2* t64, float2* t32, int logL) {
  const int r0 = logL % 3;
  const int L = 1 << logL;
  int off = 0, off64 = 0;
  int R = r0 ? (1 << r0) : 8;
  int s = L / R;
  for (;;) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < s; o += gridDim.x * blockDim.x) {
      double sn, cs;
      sincospi(-2.0 * (double)o / ((double)R * (double)s), &sn, &cs);
      t32[off + o] = make_float2((float)cs, (float)sn);
      for (int q = 1; q < R; ++q) {  // o q < R s: the argument stays in (-2, 0]
        sincospi(-2.0 * (double)(o * q) / ((double)R * (double)s), &sn, &cs);
        t64[off64 + (q - 1) * s + o] = make_double2(cs, sn);
      }
    }
    if (s == 1) break;
    off += s;
    off64 += (R - 1) * s;
    R = 8;
    s /= 8;
  }
}
void launch_twiddles(double2* t64, float2* t32, int logL, cudaStream_t s) {
  k_twiddles<<<64, 256, 0, s>>>(t64, t32, logL);
}

// Stage twiddle tables of the radix-16 column pass of length 2^logL (9 <= logL
// <= 13; other lengths have no such pass and get no table): a leading stage
// of radix R0 = 2^(logL mod 4) (16 if that is 1) and stride s = 2^logL/R0,
// then radix-16 stages; the table of stage (R, s) holds exp(-2 pi i o/(R s))
// for o < s, tables concatenated in DIF order.  Computed in FP64.
__global__ void k_twiddles16(double2* t64, float2* t32, int logL) {
  if (logL < 9 || logL > 13) return;
  const int rb = logL & 3;
  int R = rb ? 1 << rb : 16;
  int s = (1 << logL) / R;
  int off = 0;
  while (s > 1) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < s; o += gridDim.x * blockDim.x) {
      double sn, cs;
      sincospi(-2.0 * (double)o / ((double)R * (double)s), &sn, &cs);
      t64[off + o] = make_double2(cs, sn);
      t32[off + o] = make_float2((float)cs, (float)sn);
    }
    off += s;
    R = 16;
    s /= 16;
  }
}
void launch_twiddles16(double2* t64, float2* t32, int logL, cudaStream_t s) {
  k_twiddles16<<<64, 256, 0, s>>>(t64, t32, logL);
}

// exp(-i pi k / M), k = 0..M: the real-FFT split of a length-2M real transform.
__global__ void k_split_twiddles(double2* t64, float2* t32, int M) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= M; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-(double)k / (double)M, &sn, &cs);
    t64[k] = make_double2(cs, sn);
    t32[k] = make_float2((float)cs, (float)sn);
  }
}
void launch_split_twiddles(double2* t64, float2* t32, int M, cudaStream_t s) {
  k_split_twiddles<<<64, 256, 0, s>>>(t64, t32, M);
}

// Index tables of one transform length: so[ls*8 + r] = swz(r << ls) and
// sp[k] = swz(dig_pos(k)) (see Geo).
__global__ void k_geo_tables(int* so, int* sp, Geo g, int esize) {
  const Swz z{g.sa, g.sb, g.sc, g.sd};
  const int L = 1 << g.logL;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kSoEntries + L; i += gridDim.x * blockDim.x) {
    int x;
    if (i < kSoEntries) {
      const int ls = i >> 3, r = i & 7;
      x = (r << ls) < L ? (r << ls) : 0;
    } else {
      x = dig_pos(i - kSoEntries, g.logL, g.r0);
    }
    const int v = esize == 4 ? swz<float>(x, z) : swz<double>(x, z);
    if (i < kSoEntries) so[i] = v;
    else sp[i - kSoEntries] = v;
  }
}
void launch_geo_tables(int* so, int* sp, Geo g, int esize, cudaStream_t s) {
  k_geo_tables<<<32, 256, 0, s>>>(so, sp, g, esize);
}

// Bounding box of the contact set: first/last row and column holding an
// element of S (atomicMin / atomicMax on sc->band0/band1/col0/col1, which start
// at ny / -1 / nx / -1).
__global__ void k_box(int nx, int ny, const uint8_t* S, Scalars* sc) {
  __shared__ int lo, hi, clo, chi;
  if (threadIdx.x == 0) { lo = ny; hi = -1; clo = nx; chi = -1; }
  __syncthreads();
  const bool vec = (nx & 15) == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0;
  int cmin = nx, cmax = -1;
  for (int row = blockIdx.x; row < ny; row += gridDim.x) {  // the same trip count in every thread
    const uint8_t* r = S + (size_t)row * nx;
    bool any = false;
    if (vec) {
      const uint4* r4 = reinterpret_cast<const uint4*>(r);
      for (int j = threadIdx.x; j < (nx >> 4); j += blockDim.x) {
        const uint4 v = r4[j];
        if ((v.x | v.y | v.z | v.w) != 0u) {
          any = true;
          for (int q = 0; q < 16; ++q)
            if (r[16 * j + q]) { cmin = min(cmin, 16 * j + q); cmax = max(cmax, 16 * j + q); }
        }
      }
    } else {
      for (int j = threadIdx.x; j < nx; j += blockDim.x)
        if (r[j]) { any = true; cmin = min(cmin, j); cmax = max(cmax, j); }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) {
      lo = min(lo, row);
      hi = max(hi, row);
    }
  }
  if (cmax >= 0) { atomicMin(&clo, cmin); atomicMax(&chi, cmax); }
  __syncthreads();
  if (threadIdx.x == 0 && hi >= 0) {
    atomicMin(&sc->band0, lo);
    atomicMax(&sc->band1, hi);
    atomicMin(&sc->col0, clo);
    atomicMax(&sc->col1, chi);
  }
}
// Bounding box of the geometric overlap set {h <= d} (into sc->band0/band1/
// col0/col1, which start at ny / -1 / nx / -1).
__global__ void k_box_overlap(int nx, int ny, const double* __restrict__ h, double d, Scalars* sc) {
  __shared__ int lo, hi, clo, chi;
  if (threadIdx.x == 0) { lo = ny; hi = -1; clo = nx; chi = -1; }
  __syncthreads();
  int cmin = nx, cmax = -1;
  for (int row = blockIdx.x; row < ny; row += gridDim.x) {  // the same trip count in every thread
    const double* r = h + (size_t)row * nx;
    bool any = false;
    for (int j = threadIdx.x; j < nx; j += blockDim.x)
      if (r[j] <= d) { any = true; cmin = min(cmin, j); cmax = max(cmax, j); }
    if (__syncthreads_or(any) && threadIdx.x == 0) {
      lo = min(lo, row);
      hi = max(hi, row);
    }
  }
  if (cmax >= 0) { atomicMin(&clo, cmin); atomicMax(&chi, cmax); }
  __syncthreads();
  if (threadIdx.x == 0 && hi >= 0) {
    atomicMin(&sc->band0, lo);
    atomicMax(&sc->band1, hi);
    atomicMin(&sc->col0, clo);
    atomicMax(&sc->col1, chi);
  }
}
void launch_box_overlap(const Plan& pl, const double* h, double d, Scalars* sc, cudaStream_t s) {
  const int grid = std::min(pl.ny, 2 * pl.nsm);
  k_box_overlap<<<grid, 256, 0, s>>>(pl.nx, pl.ny, h, d, sc);
}

// Copy the box [x0, x0+bx) x [y0, y0+by) of an nx x ny FP64 field, `fill` where
// the box leaves the grid (bx a power of two).
__global__ void k_box_copy64(const double* __restrict__ src, int nx, int ny, int x0, int y0,
                             double* __restrict__ dst, int lbx, int nb, double fill) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int X = x0 + (i & ((1 << lbx) - 1)), Y = y0 + (i >> lbx);
    dst[i] = (X < nx && Y < ny) ? src[(size_t)Y * nx + X] : fill;
  }
}
void launch_box_copy64(const double* src, int nx, int ny, int x0, int y0, double* dst, int bx, int by,
                       double fill, cudaStream_t s) {
  int lbx = 0;
  while ((1 << lbx) < bx) ++lbx;
  const int nb = bx * by;
  k_box_copy64<<<ew_grid((size_t)nb), 256, 0, s>>>(src, nx, ny, x0, y0, dst, lbx, nb, fill);
}

void launch_box(const Plan& pl, const uint8_t* S, Scalars* sc, cudaStream_t s) {
  const int grid = std::min(pl.ny, 2 * pl.nsm);
  k_box<<<grid, 256, 0, s>>>(pl.nx, pl.ny, S, sc);
}

__global__ void k_active_set(const double* p, const double* g, uint8_t* S, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    S[i] = (p[i] > 0.0 || g[i] < 0.0) ? 1 : 0;
}
void launch_active_set(const double* p, const double* g, uint8_t* S, size_t n, cudaStream_t s) {
  k_active_set<<<ew_grid(n), 256, 0, s>>>(p, g, S, n);
}
}  // namespace bem
