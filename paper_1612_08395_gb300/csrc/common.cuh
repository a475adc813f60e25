// Shared device helpers: complex arithmetic, in-place radix-8 FFT stages in
// shared memory, FP64 block reductions.  sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bem {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

// ---------------------------------------------------------------------------
// Packed FP32 pairs: one instruction for both components (Blackwell f32x2,
// IEEE round-to-nearest like the scalar instructions).
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " add.rn.f32x2 rc, ra, rb;\n mov.b64 {%0, %1}, rc;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rc, ra, rb;\n mov.b64 {%0, %1}, rc;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * (s, s) + c
__device__ __forceinline__ float2 pfma_s(float2 a, float sc, float2 c) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %4};\n"
      " mov.b64 rc, {%5, %6};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(sc), "f"(c.x), "f"(c.y));
  return r;
}
// a * (s, s)
__device__ __forceinline__ float2 pmul_s(float2 a, float sc) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %4};\n"
      " mul.rn.f32x2 rc, ra, rb;\n mov.b64 {%0, %1}, rc;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(sc));
  return r;
}

template <typename T> __device__ __forceinline__ C<T> mk(T re, T im) { C<T> c; c.x = re; c.y = im; return c; }
template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> mul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C<T> conj(C<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ C<T> scale(C<T> a, T s) {
  if constexpr (sizeof(T) == 4) return pmul_s(a, s);
  else return mk<T>(a.x * s, a.y * s);
}
// multiply by (s*i), s = +-1
template <typename T, int S> __device__ __forceinline__ C<T> mul_si(C<T> a) {
  return S > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

template <typename T> struct consts;
template <> struct consts<float> { static constexpr float rsqrt2 = 0.70710678118654752440f; };
template <> struct consts<double> { static constexpr double rsqrt2 = 0.70710678118654752440; };

// ---------------------------------------------------------------------------
// Small DFTs in registers.  S = -1: forward (exp(-2 pi i rq/R)), S = +1: inverse.
template <typename T, int S> __device__ __forceinline__ void dft2(C<T>& a, C<T>& b) {
  C<T> t = sub<T>(a, b); a = add<T>(a, b); b = t;
}
// a +- (S i) d, componentwise (scalar: the swap would cost more than it saves)
template <typename T, int S> __device__ __forceinline__ C<T> add_si(C<T> a, C<T> d) {
  return mk<T>(a.x - S * d.y, a.y + S * d.x);
}
template <typename T, int S> __device__ __forceinline__ C<T> sub_si(C<T> a, C<T> d) {
  return mk<T>(a.x + S * d.y, a.y - S * d.x);
}
template <typename T, int S> __device__ __forceinline__ void dft4(C<T>& v0, C<T>& v1, C<T>& v2, C<T>& v3) {
  if constexpr (sizeof(T) == 4) {
    const float2 a0 = padd(v0, v2), a1 = psub(v0, v2), a2 = padd(v1, v3), d = psub(v1, v3);
    v0 = padd(a0, a2); v2 = psub(a0, a2);
    v1 = add_si<T, S>(a1, d); v3 = sub_si<T, S>(a1, d);
  } else {
    C<T> a0 = add<T>(v0, v2), a1 = sub<T>(v0, v2), a2 = add<T>(v1, v3), a3 = mul_si<T, S>(sub<T>(v1, v3));
    v0 = add<T>(a0, a2); v2 = sub<T>(a0, a2); v1 = add<T>(a1, a3); v3 = sub<T>(a1, a3);
  }
}
// v[0..7] -> X[q] in v[q]
template <typename T, int S> __device__ __forceinline__ void dft8(C<T>* v) {
  C<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, S>(e0, e1, e2, e3);
  dft4<T, S>(o0, o1, o2, o3);
  const T r = consts<T>::rsqrt2;
  if constexpr (sizeof(T) == 4) {
    // w8 o1 = r (o1.x - S o1.y, o1.y + S o1.x); w8^3 o3 = -r (o3.x + S o3.y, o3.y - S o3.x)
    const float2 u1 = mk<T>(o1.x - S * o1.y, o1.y + S * o1.x);
    const float2 u3 = mk<T>(o3.x + S * o3.y, o3.y - S * o3.x);
    v[0] = padd(e0, o0); v[4] = psub(e0, o0);
    v[1] = pfma_s(u1, r, e1); v[5] = pfma_s(u1, -r, e1);
    v[2] = add_si<T, S>(e2, o2); v[6] = sub_si<T, S>(e2, o2);
    v[3] = pfma_s(u3, -r, e3); v[7] = pfma_s(u3, r, e3);
    return;
  }
  // w8 = exp(S*2*pi*i/8) = (1 + S i)/sqrt2 ; w8^2 = S i ; w8^3 = (-1 + S i)/sqrt2
  C<T> t1 = mk<T>(r * (o1.x - S * o1.y), r * (o1.y + S * o1.x));
  C<T> t2 = mul_si<T, S>(o2);
  C<T> t3 = mk<T>(r * (-o3.x - S * o3.y), r * (-o3.y + S * o3.x));
  v[0] = add<T>(e0, o0); v[4] = sub<T>(e0, o0);
  v[1] = add<T>(e1, t1); v[5] = sub<T>(e1, t1);
  v[2] = add<T>(e2, t2); v[6] = sub<T>(e2, t2);
  v[3] = add<T>(e3, t3); v[7] = sub<T>(e3, t3);
}

// 16-point DFT as 4 x 4 (n = n2 + 4 n1, k = k1 + 4 k2): DFT-4 over n1 for
// each n2, twiddles w16^(S n2 k1), DFT-4 over n2 for each k1; v[0..15] ->
// X[q] in v[q].  cos(pi/8) and sin(pi/8) are the twiddle w16's components.
template <typename T, int S> __device__ __forceinline__ void dft16(C<T>* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, S>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  // v[n2 + 4 k1] = Y[n2][k1]
  const T c8 = (T)0.92387953251128675613, s8 = (T)0.38268343236508977173, r = consts<T>::rsqrt2;
  const C<T> w1 = mk<T>(c8, S * s8), w3 = mk<T>(s8, S * c8);
  v[5] = mul<T>(v[5], w1);    // (1,1): w^1
  v[15] = mul<T>(v[15], mk<T>(-c8, -S * s8));  // (3,3): w^9 = -w^1
  v[13] = mul<T>(v[13], w3);  // (1,3): w^3
  v[7] = mul<T>(v[7], w3);    // (3,1): w^3
  // (1,2), (2,1): w^2 = (1 + S i)/sqrt2;  (2,3), (3,2): w^6 = (-1 + S i)/sqrt2;  (2,2): w^4 = S i
  v[9] = mk<T>(r * (v[9].x - S * v[9].y), r * (v[9].y + S * v[9].x));
  v[6] = mk<T>(r * (v[6].x - S * v[6].y), r * (v[6].y + S * v[6].x));
  v[14] = mk<T>(r * (-v[14].x - S * v[14].y), r * (-v[14].y + S * v[14].x));
  v[11] = mk<T>(r * (-v[11].x - S * v[11].y), r * (-v[11].y + S * v[11].x));
  v[10] = mul_si<T, S>(v[10]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4 x 4 index
  C<T> u[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) u[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = u[4 * k1 + k2];
}

// v[q] *= w^q, q = 1..15; each power formed just before it is used, none more
// than four products from w.
template <typename T>
__device__ __forceinline__ void twiddle16(C<T>* v, C<T> w) {
  const C<T> w2 = mul<T>(w, w);
  v[1] = mul<T>(v[1], w);
  v[2] = mul<T>(v[2], w2);
  const C<T> w3 = mul<T>(w2, w);
  v[3] = mul<T>(v[3], w3);
  const C<T> w4 = mul<T>(w2, w2);
  v[4] = mul<T>(v[4], w4);
  const C<T> w5 = mul<T>(w4, w);
  v[5] = mul<T>(v[5], w5);
  v[6] = mul<T>(v[6], mul<T>(w3, w3));
  const C<T> w7 = mul<T>(w4, w3);
  v[7] = mul<T>(v[7], w7);
  const C<T> w8 = mul<T>(w4, w4);
  v[8] = mul<T>(v[8], w8);
  v[9] = mul<T>(v[9], mul<T>(w8, w));
  v[10] = mul<T>(v[10], mul<T>(w5, w5));
  v[11] = mul<T>(v[11], mul<T>(w8, w3));
  v[12] = mul<T>(v[12], mul<T>(w8, w4));
  v[13] = mul<T>(v[13], mul<T>(w8, w5));
  v[14] = mul<T>(v[14], mul<T>(w7, w7));
  v[15] = mul<T>(v[15], mul<T>(w8, w7));
}

// ---------------------------------------------------------------------------
// In-place radix-8 FFT stages in shared memory.
//
// A length L = 2^m transform runs as a decimation-in-frequency (DIF) sequence
// of stages: first one stage of radix R0 = 2^(m mod 3) (if m is not a multiple
// of 3) with stride L/R0, then radix-8 stages with strides ..., 64, 8, 1.  A
// stage of radix R and stride s combines, for butterfly offset o < s in
// group g, the elements g*R*s + o + r*s (r < R) -- each thread reads and
// writes the same R positions, so one barrier between stages suffices.  DIF
// leaves the spectrum in digit-reversed order: frequency k sits at position
// dig_pos(k).  The inverse runs the same stages in the opposite order as
// decimation-in-time (DIT) with conjugate twiddles, taking digit-reversed
// input back to natural order.  Twiddles come from per-stage tables:
// entry o of the stage (R, s) table is exp(-2 pi i o / (R s)); a butterfly
// reads its base twiddle once and forms the powers it needs.
//
// Shared-memory positions go through an XOR swizzle of the low bank bits
// (4 bits for 8-byte elements, 3 bits for 16-byte ones) chosen per length so
// that every stage's accesses, and the digit-reversed reads, avoid bank
// conflicts.
struct Swz {
  int a, b, c, d;
};
template <typename T> __device__ __forceinline__ int swz(int i, const Swz& z);
template <> __device__ __forceinline__ int swz<float>(int i, const Swz& z) {
  return i ^ ((((i >> z.a) ^ (i >> z.b)) & 7) | ((((i >> z.c) ^ (i >> z.d)) & 1) << 3));
}
template <> __device__ __forceinline__ int swz<double>(int i, const Swz& z) {
  return i ^ ((((i >> z.a) ^ (i >> z.b)) & 3) | ((((i >> z.c) ^ (i >> z.d)) & 1) << 2));
}

// Position of frequency k after the DIF stages of a length-2^logL transform.
__host__ __device__ __forceinline__ int dig_pos(int k, int logL, int r0) {
  int p = 0, sh = logL;
  if (r0) {
    sh -= r0;
    p = (k & ((1 << r0) - 1)) << sh;
    k >>= r0;
  }
  while (sh > 0) {
    sh -= 3;
    p |= (k & 7) << sh;
    k >>= 3;
  }
  return p;
}

// Offset of the twiddle table of the radix-8 stage with stride 2^ls.
__host__ __device__ __forceinline__ int tw_off8(int logL, int r0, int ls) {
  const int top = 1 << (logL - r0);
  return (r0 ? top : 0) + (top - (8 << ls)) / 7;
}

// v[q] *= w^q, q = 1..7, with the same products as powers8 but each power
// formed just before it is used (fewer values live at once).
template <typename T>
__device__ __forceinline__ void twiddle8(C<T>* v, C<T> w) {
  const C<T> w2 = mul<T>(w, w);
  v[1] = mul<T>(v[1], w);
  v[2] = mul<T>(v[2], w2);
  const C<T> w3 = mul<T>(w2, w);
  v[3] = mul<T>(v[3], w3);
  const C<T> w4 = mul<T>(w2, w2);
  v[4] = mul<T>(v[4], w4);
  v[5] = mul<T>(v[5], mul<T>(w4, w));
  v[6] = mul<T>(v[6], mul<T>(w3, w3));
  v[7] = mul<T>(v[7], mul<T>(w4, w3));
}

// v[q] *= pw[(q-1) s] (or its conjugate), q = 1..7: the powers read from a
// table instead of formed by multiplication.  The FP64 path uses this: at
// GB300's FP64 rate the six products that form the powers cost more than the
// seven coalesced table loads.
template <typename T, bool CONJ>
__device__ __forceinline__ void twiddle8_pow(C<T>* v, const C<T>* pw, int s) {
#pragma unroll
  for (int q = 1; q < 8; ++q) {
    const C<T> w = __ldg(pw + (q - 1) * s);
    v[q] = mul<T>(v[q], CONJ ? conj<T>(w) : w);
  }
}

template <typename T>
__device__ __forceinline__ void powers8(C<T> w, C<T>* wp) {
  wp[1] = w;
  wp[2] = mul<T>(w, w);
  wp[3] = mul<T>(wp[2], w);
  wp[4] = mul<T>(wp[2], wp[2]);
  wp[5] = mul<T>(wp[4], w);
  wp[6] = mul<T>(wp[3], wp[3]);
  wp[7] = mul<T>(wp[4], wp[3]);
}

// The swizzle is linear over GF(2) (XOR of shifted, masked bits), and within
// a stage the group base and the r * stride term occupy disjoint bits, so
// swz(base + r s) = swz(base) ^ swz(r s).  The eight values swz(r << ls) of
// every stride are precomputed per transform length (table `so`, 8 entries
// per ls = 0..13), leaving one XOR per shared-memory access.

// DIF radix-8 stage with stride 2^ls; thread = butterfly t (t < L/8);
// tw = this stage's twiddle table; so8 = swz(r << ls), r = 0..7.
template <typename T>
__device__ __forceinline__ void dif8(C<T>* buf, int t, int ls, const C<T>* tw, const Swz& z,
                                     const int* so8) {
  const int o = t & ((1 << ls) - 1);
  const int sb = swz<T>(((t >> ls) << (ls + 3)) + o, z);
  const int4 s0 = __ldg(reinterpret_cast<const int4*>(so8));
  const int4 s1 = __ldg(reinterpret_cast<const int4*>(so8) + 1);
  const int ix[8] = {sb ^ s0.x, sb ^ s0.y, sb ^ s0.z, sb ^ s0.w, sb ^ s1.x, sb ^ s1.y, sb ^ s1.z, sb ^ s1.w};
  C<T> v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = buf[ix[r]];
  dft8<T, -1>(v);
  if (ls > 0) {
    C<T> wp[8];
    powers8<T>(__ldg(tw + o), wp);
#pragma unroll
    for (int q = 1; q < 8; ++q) v[q] = mul<T>(v[q], wp[q]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) buf[ix[q]] = v[q];
}

// DIT radix-8 inverse stage with stride 2^ls (conjugate twiddles before the butterfly).
template <typename T>
__device__ __forceinline__ void dit8(C<T>* buf, int t, int ls, const C<T>* tw, const Swz& z,
                                     const int* so8) {
  const int o = t & ((1 << ls) - 1);
  const int sb = swz<T>(((t >> ls) << (ls + 3)) + o, z);
  const int4 s0 = __ldg(reinterpret_cast<const int4*>(so8));
  const int4 s1 = __ldg(reinterpret_cast<const int4*>(so8) + 1);
  const int ix[8] = {sb ^ s0.x, sb ^ s0.y, sb ^ s0.z, sb ^ s0.w, sb ^ s1.x, sb ^ s1.y, sb ^ s1.z, sb ^ s1.w};
  C<T> v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = buf[ix[r]];
  if (ls > 0) {
    C<T> wp[8];
    powers8<T>(conj<T>(__ldg(tw + o)), wp);
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = mul<T>(v[r], wp[r]);
  }
  dft8<T, 1>(v);
#pragma unroll
  for (int q = 0; q < 8; ++q) buf[ix[q]] = v[q];
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (16-byte chunks, L2 only).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
template <typename Cx>
__device__ __forceinline__ void cp_async_cx(Cx* smem, const Cx* gmem) {
  if (sizeof(Cx) == 16) cp_async16(smem, gmem);
  else cp_async8(smem, gmem);
}

// ---------------------------------------------------------------------------
// FP64 block reduction of NQ values; result valid in thread 0.  `red` must hold
// NQ * (blockDim.x/32) doubles of shared memory.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q * nw + wid] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = lane < nw ? red[q * nw + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Debug builds (-DBEM_DEBUG_CHECKS): bounds checks on the index arithmetic of
// the transposed intermediate W.  A failed check sets bit 2 of the handle's
// sticky error word and skips the access (no trap); release builds compile the
// checks away.
#ifdef BEM_DEBUG_CHECKS
__device__ __forceinline__ bool bem_check(bool ok, unsigned int* err) {
  if (!ok && err) atomicOr(err, 2u);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool bem_check(bool, unsigned int*) { return true; }
#endif

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (global -> shared, contiguous, 16-byte aligned and
// sized) that complete on a shared-memory mbarrier.  Waits are bounded: after
// kMbarTries unsuccessful polls, or about a second, the caller gets `false`
// and gives up.
constexpr int kMbarTries = 1 << 20;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Arrive once and expect `bytes` of transactions in the current phase.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 2D tiled TMA load of the box at (x, y) of the tensor map `tmap` (its address
// in global memory) into shared memory (128-byte aligned), completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Order earlier generic-proxy accesses of shared memory before later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Wall-clock bound of one wait (ns of %globaltimer), next to the poll bound.
constexpr unsigned long long kMbarMaxNs = 1000000000ull;
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (int i = 0; i < kMbarTries; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i == 0) t0 = global_ns();
    else if ((i & 255) == 0 && global_ns() - t0 > kMbarMaxNs) return false;
  }
  return false;
}

// Signal that this block's partials are written; returns true in every thread
// of the block that arrives last.  The counter is reset by that block.  Only
// thread 0 writes a block's partials, so only it fences: release before its
// arrival, and, in the last block, acquire before the partials are read (with
// L2 loads, after the barrier that publishes the flag).
__device__ __forceinline__ bool last_block_arrival(unsigned int* counter, int* flag_smem) {
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    const bool last = t == gridDim.x - 1;
    if (last) __threadfence();
    *flag_smem = last ? 1 : 0;
  }
  __syncthreads();
  return *flag_smem != 0;
}

// ---------------------------------------------------------------------------
// Float-float sums for the FP32 path.  GB300 executes FP64 at a small fraction
// of its FP32 rate (about two FP64 operations per clock and SM), so a
// block-wide FP64 shuffle reduction costs over a microsecond per CTA.  The FP32
// path's per-thread values are FP32; their block and grid sums are formed as
// unevaluated pairs hi + lo of floats instead, with Knuth's error-free TwoSum
// for the leading parts (about 44 significant bits, far beyond the inputs), in
// the same fixed order as block_sum, and turned into FP64 once at the end.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float v = s - a.x;
  float e = (a.x - (s - v)) + (b.x - v);  // a.x + b.x = s + e exactly
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 ff_shfl_down(float2 x, int o) {
  return make_float2(__shfl_down_sync(0xffffffffu, x.x, o), __shfl_down_sync(0xffffffffu, x.y, o));
}
__device__ __forceinline__ double ff_to_double(float2 v) { return (double)v.x + (double)v.y; }

// Block reduction of NQ float-float values; result valid in thread 0.  `red`
// must hold NQ * (blockDim.x/32) float2 of shared memory.
template <int NQ>
__device__ __forceinline__ void block_sum_ff(float2 (&v)[NQ], float2* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // the NQ sums advance level by level together (independent chains)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = ff_add(v[q], ff_shfl_down(v[q], o));
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q * nw + wid] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = lane < nw ? red[q * nw + lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = ff_add(v[q], ff_shfl_down(v[q], o));
    }
  }
  __syncthreads();
}

// This CTA's partial sums of the per-thread values acc[0 .. NQ-1] into its
// slot pp (4 doubles).  FP32: float-float pairs (hi, lo) stored in the slot's
// doubles; FP64: doubles.  Read back with grid_sum.
template <typename T, int NQ>
__device__ __forceinline__ void block_partials(const T* acc, double* pp, double* red) {
  if constexpr (sizeof(T) == 4) {
    float2 v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = make_float2((float)acc[q], 0.f);
    block_sum_ff<NQ>(v, reinterpret_cast<float2*>(red));
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) reinterpret_cast<float2*>(pp)[q] = v[q];
    }
  } else {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = (double)acc[q];
    block_sum<NQ>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) pp[q] = v[q];
    }
  }
}

// Sum of the partials that n CTAs wrote with block_partials<T, NQ>, in a fixed
// order (deterministic); result in thread 0, as FP64.  FP32 path: the first
// warp alone (lane l sums partials l, l + 32, ... with all of a round's loads
// in flight, then a shuffle tree), so no barrier; every thread must call it
// in the FP64 path (block reduction).
template <typename T, int NQ>
__device__ __forceinline__ void grid_sum(const double* part, int n, double* s, double* red) {
  if constexpr (sizeof(T) == 4) {
    if (threadIdx.x >= 32) return;
    float2 v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = make_float2(0.f, 0.f);
    constexpr int R = 4;  // partials per lane and round
    for (int b0 = (int)threadIdx.x; b0 < n; b0 += 32 * R) {
      float2 x[R][NQ];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int b = b0 + 32 * r;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          x[r][q] = b < n ? __ldcg(reinterpret_cast<const float2*>(part + 4 * b + q)) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = ff_add(v[q], x[r][q]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = ff_add(v[q], ff_shfl_down(v[q], o));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = ff_to_double(v[q]);
    (void)red;
  } else {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      double x[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = __ldcg(part + 4 * b + q);
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += x[q];
    }
    block_sum<NQ>(v, red);
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = v[q];
  }
}

}  // namespace bem
