// Shared device helpers: complex arithmetic, shared-memory Stockham FFT,
// FP64 block reductions.  sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bem {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ C<T> mk(T re, T im) { C<T> c; c.x = re; c.y = im; return c; }
template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> mul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C<T> conj(C<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ C<T> scale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by (s*i), s = +-1
template <typename T, int S> __device__ __forceinline__ C<T> mul_si(C<T> a) {
  return S > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// exp(i*pi*x)
__device__ __forceinline__ float2 expipi(float x) { float s, c; sincospif(x, &s, &c); return make_float2(c, s); }
__device__ __forceinline__ double2 expipi(double x) { double s, c; sincospi(x, &s, &c); return make_double2(c, s); }

template <typename T> struct consts;
template <> struct consts<float> { static constexpr float rsqrt2 = 0.70710678118654752440f; };
template <> struct consts<double> { static constexpr double rsqrt2 = 0.70710678118654752440; };

// ---------------------------------------------------------------------------
// Small DFTs in registers.  S = -1: forward (exp(-2 pi i rq/R)), S = +1: inverse.
template <typename T, int S> __device__ __forceinline__ void dft2(C<T>& a, C<T>& b) {
  C<T> t = sub<T>(a, b); a = add<T>(a, b); b = t;
}
template <typename T, int S> __device__ __forceinline__ void dft4(C<T>& v0, C<T>& v1, C<T>& v2, C<T>& v3) {
  C<T> a0 = add<T>(v0, v2), a1 = sub<T>(v0, v2), a2 = add<T>(v1, v3), a3 = mul_si<T, S>(sub<T>(v1, v3));
  v0 = add<T>(a0, a2); v2 = sub<T>(a0, a2); v1 = add<T>(a1, a3); v3 = sub<T>(a1, a3);
}
// v[0..7] -> X[q] in v[q]
template <typename T, int S> __device__ __forceinline__ void dft8(C<T>* v) {
  C<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, S>(e0, e1, e2, e3);
  dft4<T, S>(o0, o1, o2, o3);
  const T r = consts<T>::rsqrt2;
  // w8 = exp(S*2*pi*i/8) = (1 + S i)/sqrt2 ; w8^2 = S i ; w8^3 = (-1 + S i)/sqrt2
  C<T> t1 = mk<T>(r * (o1.x - S * o1.y), r * (o1.y + S * o1.x));
  C<T> t2 = mul_si<T, S>(o2);
  C<T> t3 = mk<T>(r * (-o3.x - S * o3.y), r * (-o3.y + S * o3.x));
  v[0] = add<T>(e0, o0); v[4] = sub<T>(e0, o0);
  v[1] = add<T>(e1, t1); v[5] = sub<T>(e1, t1);
  v[2] = add<T>(e2, t2); v[6] = sub<T>(e2, t2);
  v[3] = add<T>(e3, t3); v[7] = sub<T>(e3, t3);
}

// ---------------------------------------------------------------------------
// Stockham autosort FFT in shared memory, in place (values go through
// registers between two barriers).  One sequence of length L = 2^logL
// (logL >= 3) at `s`; the calling thread is butterfly lane j0 in [0, L/8) of
// that sequence; every thread of the block must call it (it synchronises).
// Each pass moves 8 elements per thread: radix 8, or on the first pass a
// radix-4 (x2) or radix-2 (x4) step when logL is not a multiple of 3.
// Twiddle factors: exp(S*2*pi*i*r*k/(Ns*R)) from one sincospi per butterfly
// and its powers.  Unnormalised in both directions.
template <typename T, int S>
__device__ __forceinline__ void twiddle8(C<T>* v, int k, int NsR) {
  C<T> w1 = expipi((T)(S * 2) * (T)k / (T)NsR);
  C<T> w2 = mul<T>(w1, w1);
  C<T> w3 = mul<T>(w2, w1);
  C<T> w4 = mul<T>(w2, w2);
  v[1] = mul<T>(v[1], w1);
  v[2] = mul<T>(v[2], w2);
  v[3] = mul<T>(v[3], w3);
  v[4] = mul<T>(v[4], w4);
  v[5] = mul<T>(v[5], mul<T>(w4, w1));
  v[6] = mul<T>(v[6], mul<T>(w3, w3));
  v[7] = mul<T>(v[7], mul<T>(w4, w3));
}

template <typename T, int S>
__device__ void fft_smem(C<T>* s, int logL, int j0) {
  const int L = 1 << logL;
  const int L8 = L >> 3;
  int logNs = 0;
  const int rem = logL % 3;
  C<T> v[8];
  if (rem == 1) {  // radix 2, four butterflies, Ns = 1 (no twiddles)
#pragma unroll
    for (int q = 0; q < 4; ++q) { int j = j0 + q * L8; v[2 * q] = s[j]; v[2 * q + 1] = s[j + (L >> 1)]; }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int j = j0 + q * L8;
      dft2<T, S>(v[2 * q], v[2 * q + 1]);
      s[2 * j] = v[2 * q]; s[2 * j + 1] = v[2 * q + 1];
    }
    __syncthreads();
    logNs = 1;
  } else if (rem == 2) {  // radix 4, two butterflies, Ns = 1
    const int L4 = L >> 2;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int j = j0 + q * L8;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[4 * q + r] = s[j + r * L4];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int j = j0 + q * L8;
      dft4<T, S>(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
#pragma unroll
      for (int r = 0; r < 4; ++r) s[4 * j + r] = v[4 * q + r];
    }
    __syncthreads();
    logNs = 2;
  }
  for (; logNs < logL; logNs += 3) {
    const int Ns = 1 << logNs;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = s[j0 + r * L8];
    __syncthreads();
    const int k = j0 & (Ns - 1);
    if (logNs > 0) twiddle8<T, S>(v, k, Ns << 3);
    dft8<T, S>(v);
    const int base = ((j0 >> logNs) << (logNs + 3)) + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) s[base + r * Ns] = v[r];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// FP64 block reduction of NQ values; result valid in thread 0.  `red` must hold
// NQ * (blockDim.x/32) doubles of shared memory.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[q] = x;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q * nw + wid] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nw ? red[q * nw + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[q] = x;
    }
  }
  __syncthreads();
}

// Signal that this block's partials are written; returns true in every thread
// of the block that arrives last.  The counter is reset by that block.
__device__ __forceinline__ bool last_block_arrival(unsigned int* counter, int* flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(counter, 1u);
    *flag_smem = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

}  // namespace bem
