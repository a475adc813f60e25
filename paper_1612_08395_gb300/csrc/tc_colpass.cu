// Column pass (pass B of the transform, Eq. 13) on the 5th-generation tensor
// cores: the length-4096 column DFT as matrix products instead of FFT stages.
//
// A length P = 4096 = 64 x 64 column transform is done in the four-step form.
// With n = 64 n1 + n2 and k = k1 + 64 k2 (w_L = exp(-2 pi i / L)):
//   forward  X[k1 + 64 k2] = sum_n2 w64^(n2 k2) w4096^(n2 k1) sum_n1 w64^(n1 k1) x[64 n1 + n2]
// and the inverse through conj(DFT(conj Z)), with the same forward matrices:
//   U[k1][n2] = sum_k2 conj Z[k1 + 64 k2] w64^(n2 k2),  U *= w4096^(n2 k1),
//   z[64 n1 + n2] = conj( sum_k1 U[k1][n2] w64^(n1 k1) ).
// The column holds the zero-padded rows: inputs x[n] vanish for n >= 2048
// (n1 >= 32) and only outputs n < 2048 (n1 < 32) are kept, so the first and
// last products have 32 of 64 complex inputs or outputs.
//
// Each 64-point complex DFT is one real GEMM on tcgen05 (kind::f16, BF16
// operands, FP32 accumulators in TMEM): the complex matrix is expanded to 128 x
// 128 reals, ordered [re 0..31, im 0..31, re 32..63, im 32..63] in both its
// output (N) and input (K) index, so the half-size first and last products are
// the leading 64 rows / columns.  FP32 accuracy comes from splitting every
// operand into three BF16 terms (h + m + l, 24 significant bits) and keeping
// the six products down to 2^-24: h.h + h.m + m.h + h.l + m.m + l.h.
//
// One CTA of 128 threads (4 warps, one TMEM lane quadrant each) owns an SM and
// loops over pairs of columns; the 128 rows of every product are the two
// columns' 64 sub-sequences.  Thread t reads its row of each product's result
// from TMEM; the twiddles and the spectrum multiply run in registers; the next
// product's operand rows go to shared memory as BF16 splits (transposed where
// the next contraction runs over the other index).  One elected thread issues
// the MMAs; completion arrives on an mbarrier (bounded waits).
//
// Used only when enabled (BEM_TC_COLUMN_PASS=1): FP32 column pass of a
// 4096-point torus side over the whole grid (not the fixed-set band).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdlib.h>

#include <mutex>

#include "bem.h"
#include "bem_impl.h"
#include "common.cuh"

namespace bem {
namespace {

constexpr int kTcThreads = 128;
constexpr int kN = 128;            // expanded outputs of a 64-point DFT
constexpr int kK = 128;            // expanded inputs
// Operand layouts: K-major, no swizzle, core matrices of 8 rows x 16 bytes
// (8 BF16).  B (the DFT matrix): core matrices packed, LBO 128 B, SBO 2048 B.
// A (data, written by threads, some rows transposed): LBO 144 B so the 8-value
// chunks of one row fall in distinct banks, SBO = 16 chunks x 144 B.
constexpr unsigned kLboB = 128, kSboB = (kK / 8) * 128;
constexpr unsigned kLboA = 144, kSboA = (kK / 8) * 144;
constexpr unsigned kBytesB = (kN / 8) * kSboB;   // 32 KB per split
constexpr unsigned kBytesA = (128 / 8) * kSboA;  // 36 KB per split
constexpr unsigned kSmemTc = 3 * kBytesB + 3 * kBytesA + 64;

// The expanded DFT64 matrix in BF16 splits, laid out for the B operand, and the
// twiddles w4096^j; built once per device.
__device__ __align__(128) unsigned char g_dft_b[3 * kBytesB];
__device__ float2 g_tw4096[4096];

__host__ __device__ __forceinline__ int dft_index(int o, int part) {  // expanded position of (index, re/im)
  return (o >> 5) * 64 + part * 32 + (o & 31);
}
__device__ __forceinline__ unsigned off_b(int r, int k) {
  return (unsigned)((r >> 3) * kSboB + (k >> 3) * kLboB + (r & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ unsigned off_a(int r, int k) {
  return (unsigned)((r >> 3) * kSboA + (k >> 3) * kLboA + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  r = r - __bfloat162float(m);
  l = __float2bfloat16_rn(r);
}

__global__ void k_tc_tables() {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 4096) {
    double s, c;
    sincospi(-2.0 * i / 4096.0, &s, &c);
    g_tw4096[i] = make_float2((float)c, (float)s);
  }
  if (i < kN * kK) {
    // B[row = output (o, po)][col = input (q, pq)]: out_re = in_re cos + in_im sin,
    // out_im = in_im cos - in_re sin, with angle 2 pi o q / 64
    const int row = i / kK, col = i % kK;
    const int o = (row >> 6) * 32 + (row & 31), po = (row >> 5) & 1;
    const int q = (col >> 6) * 32 + (col & 31), pq = (col >> 5) & 1;
    double s, c;
    sincospi(2.0 * (double)((o * q) & 63) / 64.0, &s, &c);
    double v;
    if (po == 0) v = pq == 0 ? c : s;
    else v = pq == 0 ? -s : c;
    __nv_bfloat16 h, m, l;
    split3((float)v, h, m, l);
    // v rounded to FP32 first: the FP32 column pass uses FP32 twiddles too
    const unsigned off = off_b(row, col);
    *reinterpret_cast<__nv_bfloat16*>(g_dft_b + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(g_dft_b + kBytesB + off) = m;
    *reinterpret_cast<__nv_bfloat16*>(g_dft_b + 2 * kBytesB + off) = l;
  }
}

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(unsigned d, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// D = A . B^T over K = 16 * ksteps, N outputs, six split products per K step:
// the leading product h.h accumulates in TMEM columns [0, 128), the five
// smaller ones in [128, 256) (their rounding is 2^-8 smaller there); the two
// are added in FP32 registers when the row is read.
__device__ __forceinline__ void gemm_issue(unsigned tmem, unsigned sa, unsigned sb, int ksteps, int n) {
  const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
  for (int ks = 0; ks < ksteps; ++ks) {
    const unsigned oa = ks * 2 * kLboA, ob = ks * 2 * kLboB;
    const uint64_t ah = sdesc(sa + oa, kLboA, kSboA), am = sdesc(sa + kBytesA + oa, kLboA, kSboA),
                   al = sdesc(sa + 2 * kBytesA + oa, kLboA, kSboA);
    const uint64_t bh = sdesc(sb + ob, kLboB, kSboB), bm = sdesc(sb + kBytesB + ob, kLboB, kSboB),
                   bl = sdesc(sb + 2 * kBytesB + ob, kLboB, kSboB);
    const unsigned acc = ks > 0 ? 1u : 0u, t2 = tmem + 128u;
    mma_bf16(t2, ah, bl, idesc, acc);
    mma_bf16(t2, am, bm, idesc, 1u);
    mma_bf16(t2, al, bh, idesc, 1u);
    mma_bf16(t2, ah, bm, idesc, 1u);
    mma_bf16(t2, am, bh, idesc, 1u);
    mma_bf16(tmem, ah, bh, idesc, acc);
  }
}

__device__ __forceinline__ bool wait_bar(unsigned bar, unsigned parity) {
  for (int i = 0; i < kMbarTries; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Thread 0 issues a product and commits it; every thread waits for it.  The
// operand writes of all threads are made visible to the tensor core first.
__device__ __forceinline__ bool run_gemm(unsigned tmem, unsigned sa, unsigned sb, int ksteps, int n, unsigned bar,
                                         unsigned& phase) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (threadIdx.x == 0) {
    gemm_issue(tmem, sa, sb, ksteps, n);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
  }
  const bool ok = wait_bar(bar, phase);
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return __syncthreads_and(ok);
}

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// This thread's row of the last product: 64 complex values (index o: re at
// column dft_index(o, 0), im at dft_index(o, 1)).  n = 128 or 64 columns.
__device__ __forceinline__ void read_row(unsigned tmem, int n, float2* z) {
  const unsigned lane = (unsigned)((threadIdx.x >> 5) * 32) << 16;
  float v[32], w[32];
#pragma unroll
  for (int c0 = 0; c0 < 128; c0 += 32) {
    if (c0 >= n) break;
    tmem_ld32(tmem + lane + (unsigned)c0, v);
    tmem_ld32(tmem + lane + 128u + (unsigned)c0, w);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] += w[j];
    // columns c0 .. c0+31: one (o-half, part) block of 32 outputs
    const int ob = (c0 >> 6) * 32, part = (c0 >> 5) & 1;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (part == 0) z[ob + j].x = v[j];
      else z[ob + j].y = v[j];
    }
  }
}

// Write the value (re, im) of input q into row r of the A splits.
__device__ __forceinline__ void put_a(unsigned char* a, int r, int q, float2 x) {
  __nv_bfloat16 h, m, l;
  const unsigned o0 = off_a(r, dft_index(q, 0)), o1 = off_a(r, dft_index(q, 1));
  split3(x.x, h, m, l);
  *reinterpret_cast<__nv_bfloat16*>(a + o0) = h;
  *reinterpret_cast<__nv_bfloat16*>(a + kBytesA + o0) = m;
  *reinterpret_cast<__nv_bfloat16*>(a + 2 * kBytesA + o0) = l;
  split3(x.y, h, m, l);
  *reinterpret_cast<__nv_bfloat16*>(a + o1) = h;
  *reinterpret_cast<__nv_bfloat16*>(a + kBytesA + o1) = m;
  *reinterpret_cast<__nv_bfloat16*>(a + 2 * kBytesA + o1) = l;
}

// Row r of the A splits from 64 consecutive inputs q = 0..63 (own row: 16-byte stores).
__device__ __forceinline__ void put_row(unsigned char* a, int r, const float2* x, int nq) {
#pragma unroll
  for (int q0 = 0; q0 < 64; q0 += 8) {
    if (q0 >= nq) break;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      __nv_bfloat16 hs[8], ms[8], ls[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) split3(part ? x[q0 + j].y : x[q0 + j].x, hs[j], ms[j], ls[j]);
      const unsigned o = off_a(r, dft_index(q0, part));  // 8 consecutive positions, one chunk
      *reinterpret_cast<uint4*>(a + o) = *reinterpret_cast<const uint4*>(hs);
      *reinterpret_cast<uint4*>(a + kBytesA + o) = *reinterpret_cast<const uint4*>(ms);
      *reinterpret_cast<uint4*>(a + 2 * kBytesA + o) = *reinterpret_cast<const uint4*>(ls);
    }
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_pass_b_tc(PassArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem_tc[];
  unsigned char* sb = smem_tc;                   // B splits (the DFT matrix)
  unsigned char* sa = smem_tc + 3 * kBytesB;     // A splits (the data)
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sa + 3 * kBytesA);
  unsigned* tslot = reinterpret_cast<unsigned*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (a.sc != nullptr && a.sc->done) return;
  // the DFT matrix into shared memory (16-byte copies)
  for (int i = tid; i < (int)(3 * kBytesB / 16); i += kTcThreads)
    reinterpret_cast<uint4*>(sb)[i] = reinterpret_cast<const uint4*>(g_dft_b)[i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(su32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;
  const unsigned usa = su32(sa), usb = su32(sb), ubar = su32(bar);
  unsigned phase = 0;
  const int M = a.pl.M, rin = a.rows_w;
  const int hyq = 2049;  // spectrum quarter: ky = 0 .. 2048
  float2* W = reinterpret_cast<float2*>(a.W);
  const int c = tid >> 6, r64 = tid & 63;  // this thread's column of the pair and sub-index
  const int ntask = (M + 2) / 2;
  bool ok = true;
  float2 z[64];
  for (int task = blockIdx.x; task < ntask && ok; task += gridDim.x) {
    const int kx = 2 * task + c;
    const bool live = kx <= M;
    const size_t coff = (size_t)(live ? kx : 0) * rin;
    // product 1: row (c, n2 = r64), inputs n1 < 32: x[64 n1 + n2]
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
      const int y = 64 * n1 + r64;
      z[n1] = (live && y < rin) ? W[coff + y] : make_float2(0.f, 0.f);
    }
    put_row(sa, tid, z, 32);
    ok = run_gemm(tmem, usa, usb, 4, kN, ubar, phase);
    if (!ok) break;
    read_row(tmem, kN, z);  // Y[k1], k1 = 0..63, for n2 = r64
    // twiddle w4096^(n2 k1), then product 2 contracts over n2: row (c, k1), input n2
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int k1 = 0; k1 < 64; ++k1) {
      const float2 w = g_tw4096[(r64 * k1) & 4095];
      const float2 y = z[k1];
      put_a(sa, c * 64 + k1, r64, make_float2(y.x * w.x - y.y * w.y, y.x * w.y + y.y * w.x));
    }
    ok = run_gemm(tmem, usa, usb, 8, kN, ubar, phase);
    if (!ok) break;
    read_row(tmem, kN, z);  // X[k1 + 64 k2], k1 = r64, k2 = 0..63
    // spectrum (real, even in ky), conjugate, product 3 over k2 (own row)
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    const float* kc = a.khat + (size_t)(live ? kx : 0) * hyq;
#pragma unroll
    for (int k2 = 0; k2 < 64; ++k2) {
      const int ky = r64 + 64 * k2;
      const float kf = live ? __ldg(kc + (ky <= 2048 ? ky : 4096 - ky)) : 0.f;
      z[k2] = make_float2(z[k2].x * kf, -z[k2].y * kf);
    }
    put_row(sa, tid, z, 64);
    ok = run_gemm(tmem, usa, usb, 8, kN, ubar, phase);
    if (!ok) break;
    read_row(tmem, kN, z);  // U[k1 = r64][n2], n2 = 0..63
    // twiddle w4096^(n2 k1), product 4 contracts over k1: row (c, n2), input k1
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int n2 = 0; n2 < 64; ++n2) {
      const float2 w = g_tw4096[(r64 * n2) & 4095];
      const float2 y = z[n2];
      put_a(sa, c * 64 + n2, r64, make_float2(y.x * w.x - y.y * w.y, y.x * w.y + y.y * w.x));
    }
    ok = run_gemm(tmem, usa, usb, 8, 64, ubar, phase);
    if (!ok) break;
    read_row(tmem, 64, z);  // S[n1][n2 = r64], n1 < 32
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (live) {
#pragma unroll
      for (int n1 = 0; n1 < 32; ++n1) {
        const int y = 64 * n1 + r64;
        if (y < rin) W[coff + y] = make_float2(z[n1].x, -z[n1].y);
      }
    }
    __syncthreads();  // TMEM reads done before the next product overwrites D
  }
  if (!ok && tid == 0 && a.kerr) atomicOr(a.kerr, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
}

std::mutex g_tc_mu;
bool g_tc_ready[64] = {};

}  // namespace

bool tc_column_pass_enabled() {
  static const bool on = [] {
    const char* e = getenv("BEM_TC_COLUMN_PASS");
    return e && e[0] == '1';
  }();
  return on;
}

// The tensor-core column pass applies to the FP32 transform of a torus whose
// column length is 4096, over the whole grid (no fixed-set band).
bool tc_column_pass_applies(const PassArgs<float>& a) {
  return a.pl.py == 4096 && a.rows_w <= 2048 && !a.use_band && a.khat != nullptr;
}

// Once per device (from the device set-up, outside any capture): the DFT matrix
// and twiddle tables, and the shared-memory opt-in of the pass.
int tc_column_pass_setup() {
  if (!tc_column_pass_enabled()) return BEM_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set_error(BEM_ECUDA, "no device");
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (g_tc_ready[dev]) return BEM_OK;
  k_tc_tables<<<(kN * kK + 255) / 256, 256>>>();
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaFuncSetAttribute(k_pass_b_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc) != cudaSuccess)
    return set_error(BEM_ECUDA, "tensor-core column pass set-up failed");
  g_tc_ready[dev] = true;
  return BEM_OK;
}

int launch_pass_b_tc(const PassArgs<float>& a, cudaStream_t s) {
  k_pass_b_tc<<<a.pl.nsm, kTcThreads, kSmemTc, s>>>(a);
  return BEM_OK;
}

}  // namespace bem
