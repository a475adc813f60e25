// Influence coefficients K(di, dj) of Eq. 9 in FP64 on the device.
//
//   K(di, dj) = int_{(di-1/2)dx}^{(di+1/2)dx} int_{(dj-1/2)dy}^{(dj+1/2)dy} (a^2+b^2)^-(1+k)/2 db da
//
// Near the singularity (max(di, dj) <= NEAR) K is the corner difference of
//   F(x, y) = int_0^x int_0^y (a^2+b^2)^-(1+k)/2 db da
//           = [ x^(1-k) G(y/x) + y^(1-k) G(x/y) ] / (1-k),
//   G(U)    = int_0^{asinh U} cosh(s)^-k ds,
// obtained by integrating r^-(1+k) r dr exactly along rays from the corner
// (polar coordinates), then u = tan(theta) and u = sinh(s); the remaining
// integrand cosh^-k is smooth, so composite Gauss-Legendre converges fast.
// F is odd in each argument.  Away from the singularity the integrand is
// analytic on the element and tensor Gauss-Legendre rules are used directly,
// with fewer points the farther the element; the distance is counted in units
// of the element's longer side, so elongated elements near the singularity
// take the corner formula.
#include <math.h>
#include <cuda_runtime.h>

#include "bem_impl.h"

namespace bem {

namespace {
constexpr int NG16 = 16;
constexpr int NEAR = 4;
__constant__ double c_x16[16], c_w16[16];
__constant__ double c_x10[10], c_w10[10];
__constant__ double c_x6[6], c_w6[6];
__constant__ double c_x4[4], c_w4[4];

// Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method, starting
// from the Tricomi approximation; P_n and P_n' from the Bonnet recurrence.
void legendre_rule(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 1; i <= n; ++i) {
    double th = pi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
    double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
    double dpn = 0.0;
    for (int it = 0; it < 60; ++it) {
      double pkm1 = 1.0, pk = z;
      for (int kk = 2; kk <= n; ++kk) {
        double pkp1 = ((2.0 * kk - 1.0) * z * pk - (kk - 1.0) * pkm1) / kk;
        pkm1 = pk;
        pk = pkp1;
      }
      dpn = n * (pkm1 - z * pk) / (1.0 - z * z);
      double step = pk / dpn;
      z -= step;
      if (fabs(step) <= 1e-16 * fabs(z) + 1e-300) break;
    }
    x[i - 1] = z;
    w[i - 1] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
}
}  // namespace

int influence_init_nodes() {
  double x[16], w[16];
  legendre_rule(16, x, w);
  if (cudaMemcpyToSymbol(c_x16, x, sizeof(double) * 16) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_w16, w, sizeof(double) * 16) != cudaSuccess) return -1;
  legendre_rule(10, x, w);
  if (cudaMemcpyToSymbol(c_x10, x, sizeof(double) * 10) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_w10, w, sizeof(double) * 10) != cudaSuccess) return -1;
  legendre_rule(6, x, w);
  if (cudaMemcpyToSymbol(c_x6, x, sizeof(double) * 6) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_w6, w, sizeof(double) * 6) != cudaSuccess) return -1;
  legendre_rule(4, x, w);
  if (cudaMemcpyToSymbol(c_x4, x, sizeof(double) * 4) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_w4, w, sizeof(double) * 4) != cudaSuccess) return -1;
  return 0;
}

// G(U) = int_0^{asinh U} cosh(s)^-k ds, composite 16-point Gauss-Legendre
// with panels no longer than 0.5.
__device__ double g_ray(double U, double k) {
  const double S = asinh(U);
  int np = (int)ceil(S / 0.5);
  if (np < 1) np = 1;
  const double hp = S / np;
  double sum = 0.0;
  for (int q = 0; q < np; ++q) {
    const double mid = (q + 0.5) * hp;
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < NG16; ++i) {
      const double x = mid + 0.5 * hp * c_x16[i];
      s += c_w16[i] * exp(-k * log(cosh(x)));
    }
    sum += s;
  }
  return sum * 0.5 * hp;
}

// F(x, y): integral over [0, x] x [0, y], odd in x and in y.
__device__ double f_corner(double x, double y, double k) {
  if (x == 0.0 || y == 0.0) return 0.0;
  const double ax = fabs(x), ay = fabs(y);
  const double v = (pow(ax, 1.0 - k) * g_ray(ay / ax, k) + pow(ay, 1.0 - k) * g_ray(ax / ay, k)) / (1.0 - k);
  return ((x < 0.0) != (y < 0.0)) ? -v : v;
}

template <int NP>
__device__ double tensor_gl(const double* xs, const double* ws, double a0, double a1, double b0,
                            double b1, double expo) {
  const double ca = 0.5 * (a0 + a1), ha = 0.5 * (a1 - a0);
  const double cb = 0.5 * (b0 + b1), hb = 0.5 * (b1 - b0);
  double s = 0.0;
#pragma unroll 1
  for (int i = 0; i < NP; ++i) {
    const double a = ca + ha * xs[i];
    const double a2 = a * a;
    double si = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double b = cb + hb * xs[j];
      si += ws[j] * exp(expo * log(a2 + b * b));
    }
    s += ws[i] * si;
  }
  return s * ha * hb;
}

__global__ void k_influence(double* Kq, int hx, int hy, double dx, double dy, double k) {
  const int di = blockIdx.x * blockDim.x + threadIdx.x;
  const int dj = blockIdx.y;
  if (di >= hx || dj >= hy) return;
  const double a0 = (di - 0.5) * dx, a1 = (di + 0.5) * dx;
  const double b0 = (dj - 0.5) * dy, b1 = (dj + 0.5) * dy;
  // distance class of the element: its index distance, but for elongated
  // elements never more than its physical distance from the singularity in
  // units of its longer side (a long element can reach close to the origin)
  const double ea = fmax(0.0, a0), eb = fmax(0.0, b0), side = fmax(dx, dy);
  const double phys = sqrt(ea * ea + eb * eb) / side + 0.5;
  const double far = fmin((double)(di > dj ? di : dj), phys);
  double v;
  if (far <= NEAR) {
    v = f_corner(a1, b1, k) - f_corner(a0, b1, k) - f_corner(a1, b0, k) + f_corner(a0, b0, k);
  } else {
    const double expo = -0.5 * (1.0 + k);
    if (far <= 12) v = tensor_gl<16>(c_x16, c_w16, a0, a1, b0, b1, expo);
    else if (far <= 40) v = tensor_gl<10>(c_x10, c_w10, a0, a1, b0, b1, expo);
    else if (far <= 200) v = tensor_gl<6>(c_x6, c_w6, a0, a1, b0, b1, expo);
    else v = tensor_gl<4>(c_x4, c_w4, a0, a1, b0, b1, expo);
  }
  Kq[(size_t)dj * hx + di] = v;
}

void launch_influence(double* Kq, int hx, int hy, double dx, double dy, double k, cudaStream_t s) {
  const dim3 block(128), grid((hx + 127) / 128, hy);
  k_influence<<<grid, block, 0, s>>>(Kq, hx, hy, dx, dy, k);
}

}  // namespace bem
