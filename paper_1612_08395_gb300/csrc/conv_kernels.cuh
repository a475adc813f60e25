// The stress -> displacement transform u = A K*p (Eq. 13) as three passes
// over a zero-padded Px x Py torus, with the conjugate-gradient work fused
// into the first pass's prologue and the last pass's epilogue.
//
//   pass A  rows:    real row of Nx values (zero-padded to Px) -> half
//                    spectrum X[kx], kx = 0..Px/2, via one complex FFT of
//                    length M = Px/2 on (x[2n], x[2n+1]) and the standard
//                    split.  Written transposed: W[kx][iy].
//   pass B  columns: for each kx, DIF FFT of length Py of the Ny values
//                    (zero-padded), multiply by the real spectrum K^(ky, kx)
//                    in digit-reversed order, DIT inverse FFT, keep Ny values,
//                    in place in W.
//   pass C  rows:    complex-to-real inverse of length Px from the half
//                    spectrum, keep Nx values, scale by A/(Px Py), epilogue.
//
// The transform length is a template parameter (dispatched at launch), so
// strides, masks and swizzle constants fold into immediates.  Because
// Px >= 2 Nx and Py >= 2 Ny, the nonzero inputs of every forward transform
// fill its first half and only the first half of every inverse is kept: the
// first forward stage reads just those inputs straight from global memory
// and the last inverse stage computes and writes just those outputs.
// Prologue and epilogue field loads are issued together (gather, then
// compute, then store) so their latencies overlap.
//
// Every kernel that belongs to a CG loop returns at once when the solve's
// `done` flag is set, so a captured chunk of iterations can run past
// convergence at the cost of empty launches.
#pragma once
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "bem_impl.h"
#include "common.cuh"
#include "geo_table.h"

namespace bem {

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < (T)0 ? -x : x; }

// Iterations without halving the best eps before a CG solve is declared stalled.
constexpr int kStall = 200;

// Compile-time description of a length-2^LOGL transform for element type T.
template <typename T, int LOGL>
struct FftC {
  static constexpr int L = 1 << LOGL, L8 = L >> 3, R0 = LOGL % 3;
  static constexpr int LS_TOP = R0 == 0 ? LOGL - 6 : LOGL - R0 - 3;  // largest radix-8 stride below stage 0
  using G = GeoC<(int)sizeof(T), LOGL>;
  static __device__ __forceinline__ int sw(int i) {
    if (sizeof(T) == 4)
      return i ^ ((((i >> G::a) ^ (i >> G::b)) & 7) | ((((i >> G::c) ^ (i >> G::d)) & 1) << 3));
    return i ^ ((((i >> G::a) ^ (i >> G::b)) & 3) | ((((i >> G::c) ^ (i >> G::d)) & 1) << 2));
  }
  // n of element e (0..7) of thread t in stage 0 (the first DIF stage)
  static __device__ __forceinline__ int n0(int t, int e) {
    if (R0 == 0) return t + e * L8;
    if (R0 == 2) return t + (e >> 2) * L8 + (e & 3) * (L >> 2);
    return t + (e >> 1) * L8 + (e & 1) * (L >> 1);
  }
  // whether element e of stage 0 lies in the first half (t < L8 always)
  static __device__ __forceinline__ constexpr bool first_half(int e) {
    return R0 == 0 ? e < 4 : (R0 == 2 ? (e & 3) < 2 : (e & 1) == 0);
  }
  // FP64 tables hold every power a butterfly needs (see twiddle8_pow): offset
  // of the radix-8 stage with stride 2^ls there
  static __device__ __forceinline__ constexpr int pow_off(int ls) {
    return (R0 ? ((1 << R0) - 1) << (LOGL - R0) : 0) + (1 << (LOGL - R0)) - (8 << ls);
  }
  // stage 0 butterflies on the 8 values of a thread (DIF: butterfly, then twiddle)
  static __device__ __forceinline__ void stage0_fwd(C<T>* v, int t, const C<T>* tw) {
    if (R0 == 0) {
      dft8<T, -1>(v);
      if constexpr (sizeof(T) == 8) twiddle8_pow<T, false>(v, tw + t, L8);
      else twiddle8<T>(v, __ldg(tw + t));
    } else if (R0 == 2) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        C<T>* u = v + 4 * i;
        dft4<T, -1>(u[0], u[1], u[2], u[3]);
        if constexpr (sizeof(T) == 8) {
          const C<T>* pw = tw + t + i * L8;
          u[1] = mul<T>(u[1], __ldg(pw)); u[2] = mul<T>(u[2], __ldg(pw + (L >> 2)));
          u[3] = mul<T>(u[3], __ldg(pw + 2 * (L >> 2)));
        } else {
          const C<T> w = __ldg(tw + t + i * L8), w2 = mul<T>(w, w), w3 = mul<T>(w2, w);
          u[1] = mul<T>(u[1], w); u[2] = mul<T>(u[2], w2); u[3] = mul<T>(u[3], w3);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        C<T>* u = v + 2 * i;
        dft2<T, -1>(u[0], u[1]);
        u[1] = mul<T>(u[1], __ldg(tw + t + i * L8));
      }
    }
  }
  // inverse of stage 0 (DIT: conjugate twiddle, then butterfly)
  static __device__ __forceinline__ void stage0_inv(C<T>* v, int t, const C<T>* tw) {
    if (R0 == 0) {
      if constexpr (sizeof(T) == 8) twiddle8_pow<T, true>(v, tw + t, L8);
      else twiddle8<T>(v, conj<T>(__ldg(tw + t)));
      dft8<T, 1>(v);
    } else if (R0 == 2) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        C<T>* u = v + 4 * i;
        if constexpr (sizeof(T) == 8) {
          const C<T>* pw = tw + t + i * L8;
          u[1] = mul<T>(u[1], conj<T>(__ldg(pw))); u[2] = mul<T>(u[2], conj<T>(__ldg(pw + (L >> 2))));
          u[3] = mul<T>(u[3], conj<T>(__ldg(pw + 2 * (L >> 2))));
        } else {
          const C<T> w = conj<T>(__ldg(tw + t + i * L8)), w2 = mul<T>(w, w), w3 = mul<T>(w2, w);
          u[1] = mul<T>(u[1], w); u[2] = mul<T>(u[2], w2); u[3] = mul<T>(u[3], w3);
        }
        dft4<T, 1>(u[0], u[1], u[2], u[3]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        C<T>* u = v + 2 * i;
        u[1] = mul<T>(u[1], conj<T>(__ldg(tw + t + i * L8)));
        dft2<T, 1>(u[0], u[1]);
      }
    }
  }
  // shared-memory index of element e of stage 0 for thread t
  static __device__ __forceinline__ int ix0(int t, int e) { return sw(n0(t, e)); }

  // radix-8 DIF / DIT stage with compile-time stride 2^LS (after unrolling)
  static __device__ __forceinline__ void dif(C<T>* buf, int t, int ls, const C<T>* tw) {
    const int o = t & ((1 << ls) - 1);
    const int sb = sw(((t >> ls) << (ls + 3)) + o);
    C<T> v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = buf[sb ^ sw(r << ls)];
    dft8<T, -1>(v);
    if (ls > 0) {
      if constexpr (sizeof(T) == 8) twiddle8_pow<T, false>(v, tw + pow_off(ls) + o, 1 << ls);
      else twiddle8<T>(v, __ldg(tw + tw_off8(LOGL, R0, ls) + o));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[sb ^ sw(q << ls)] = v[q];
  }
  static __device__ __forceinline__ void dit(C<T>* buf, int t, int ls, const C<T>* tw) {
    const int o = t & ((1 << ls) - 1);
    const int sb = sw(((t >> ls) << (ls + 3)) + o);
    C<T> v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = buf[sb ^ sw(r << ls)];
    if (ls > 0) {
      if constexpr (sizeof(T) == 8) twiddle8_pow<T, true>(v, tw + pow_off(ls) + o, 1 << ls);
      else twiddle8<T>(v, conj<T>(__ldg(tw + tw_off8(LOGL, R0, ls) + o)));
    }
    dft8<T, 1>(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[sb ^ sw(q << ls)] = v[q];
  }
};

// ---------------------------------------------------------------------------
// Pass-A prologue, in two phases: gather the fields of one field index, then
// compute the transform input (with the CG work of the mode) and store.
template <typename T>
struct PIn {
  T p, t, g, r;
  uint8_t s;
};

template <typename T, int MODE>
__device__ __forceinline__ void pro_gather(const PassArgs<T>& a, size_t i, PIn<T>& x) {
  if (MODE == A_PLAIN) {
    x.p = __ldg(a.f.src + i);
  } else if (MODE == A_PK_P) {
    x.p = a.f.p[i]; x.t = a.f.t[i]; x.g = a.f.g[i];
  } else if (MODE == A_PK_T) {
    x.p = a.f.p[i]; x.t = a.f.t[i]; x.g = a.f.g[i];
  } else if (MODE == A_CG_T) {
    x.s = a.f.S[i]; x.t = a.f.t[i]; x.g = a.f.g[i]; x.p = a.f.p[i]; x.r = a.f.r[i];
  }
}

template <typename T> struct V2T;
template <> struct V2T<float> { using type = float2; };
template <> struct V2T<double> { using type = double2; };
template <typename T> using V2 = typename V2T<T>::type;

// The field a prologue mode rewrites with the transform input (null: none).
template <typename T, int MODE>
__device__ __forceinline__ T* pro_out(const PassArgs<T>& a) {
  if (MODE == A_PK_P) return a.f.p;
  if (MODE == A_PK_T || MODE == A_CG_T) return a.f.t;
  return nullptr;
}

// Transform input of one element with the CG work of the mode (the value the
// mode also stores back into pro_out), without the store.
template <typename T, int MODE>
__device__ __forceinline__ T pro_value(PIn<T>& x, bool upd, T tau, T beta, T* acc) {
  if (MODE == A_PLAIN) {
    return x.p;
  } else if (MODE == A_PK_P) {
    T q = x.p;
    if (upd) {
      if (x.p > (T)0) {
        q = x.p - tau * x.t;
        q = q > (T)0 ? q : (T)0;
      }
      if (q == (T)0 && x.g < (T)0) { q = -tau * x.g; acc[2] += (T)1; }
      acc[0] += tabs(q - x.p);
    }
    acc[1] += q;
    return q;
  } else if (MODE == A_PK_T) {
    return x.p > (T)0 ? x.g + beta * x.t : (T)0;
  } else {  // A_CG_T: the previous iteration's update, then the new direction
    if (upd) {
      x.p -= tau * x.t;
      x.g -= tau * x.r;
    }
    return x.s ? x.g + beta * x.t : (T)0;
  }
}

template <typename T, int MODE>
__device__ __forceinline__ T pro_apply(const PassArgs<T>& a, size_t i, const PIn<T>& x, bool upd,
                                       T tau, T beta, T* acc) {
  if (MODE == A_PLAIN) {
    return x.p;
  } else if (MODE == A_PK_P) {
    // Polonsky-Keer steps 7-8: p <- max(p - tau t, 0) on the contact set,
    // then the overlap step p = -tau g where p = 0 and g < 0.
    T q = x.p;
    if (upd) {
      if (x.p > (T)0) {
        q = x.p - tau * x.t;
        q = q > (T)0 ? q : (T)0;
      }
      if (q == (T)0 && x.g < (T)0) { q = -tau * x.g; acc[2] += (T)1; }
      acc[0] += tabs(q - x.p);
      a.f.p[i] = q;
    }
    acc[1] += q;
    return q;
  } else if (MODE == A_PK_T) {
    const T tv = x.p > (T)0 ? x.g + beta * x.t : (T)0;
    a.f.t[i] = tv;
    return tv;
  } else {  // A_CG_T: the previous iteration's update, then the new direction
    T gv = x.g;
    if (upd) {
      a.f.p[i] = x.p - tau * x.t;
      gv = x.g - tau * x.r;
      a.f.g[i] = gv;
    }
    const T tv = x.s ? gv + beta * x.t : (T)0;
    a.f.t[i] = tv;
    return tv;
  }
}

// Split the packed length-M transforms of the rows row0 .. row0+nb-1 (shared
// memory, digit-reversed) into the half spectra X[0..M] and store them
// transposed, W[k][row0 + bb].  With z the packed transform,
//   X[k] = (z[k] + conj z[M-k]) / 2 + w_k (z[k] - conj z[M-k]) / (2i),
// w_k = exp(-i pi k / M), and w_{M-k} = -conj w_k, so one work item computes
// X[k] and X[M-k] from the same two values.  FP32 with an even row count and
// even W rows: each item takes two rows and stores 16 bytes per k.
template <typename T>
__device__ __forceinline__ void split_two(const C<T>* s, int pk, int pm, C<T> w, C<T>& xk, C<T>& xm) {
  const C<T> a = s[pk], b = s[pm];
  {
    const C<T> zm = conj<T>(b);
    const C<T> E = scale<T>(add<T>(a, zm), (T)0.5);
    const C<T> dl = sub<T>(a, zm);
    xk = add<T>(E, mul<T>(w, mk<T>((T)0.5 * dl.y, (T)-0.5 * dl.x)));
  }
  {
    const C<T> zm = conj<T>(a);
    const C<T> E = scale<T>(add<T>(b, zm), (T)0.5);
    const C<T> dl = sub<T>(b, zm);
    xm = add<T>(E, mul<T>(mk<T>(-w.x, w.y), mk<T>((T)0.5 * dl.y, (T)-0.5 * dl.x)));
  }
}
template <typename T, int M>
__device__ __forceinline__ void split_store(const C<T>* sm, int rs, int nb, int lognb, int row0, int nrows,
                                            const int* sp, const C<T>* tws, C<T>* W, int rows_w,
                                            unsigned int* kerr) {
  constexpr int hm = M / 2 + 1;
  const int rows = min(nb, nrows - row0);
  const size_t wlim = (size_t)(M + 1) * rows_w;  // W holds (M+1) rows of rows_w
  if (sizeof(T) == 4 && nb >= 2 && (rows_w & 1) == 0) {
    const int lp = lognb - 1;  // row pairs per group
    for (int idx = threadIdx.x; idx < hm << lp; idx += blockDim.x) {
      const int k = idx >> lp, b0 = 2 * (idx & ((1 << lp) - 1));
      if (b0 >= rows) continue;
      const bool two = b0 + 1 < rows;
      const C<T>* s0 = sm + b0 * rs;
      const C<T>* s1 = s0 + rs;
      C<T> xk0, xm0, xk1 = mk<T>(0, 0), xm1 = mk<T>(0, 0);
      if (k == 0) {
        const C<T> z0 = s0[0];
        xk0 = mk<T>(z0.x + z0.y, (T)0);
        xm0 = mk<T>(z0.x - z0.y, (T)0);
        if (two) {
          const C<T> z1 = s1[0];
          xk1 = mk<T>(z1.x + z1.y, (T)0);
          xm1 = mk<T>(z1.x - z1.y, (T)0);
        }
      } else {
        const int pk = __ldg(sp + k), pm = __ldg(sp + M - k);
        const C<T> w = __ldg(tws + k);
        split_two<T>(s0, pk, pm, w, xk0, xm0);
        if (two) split_two<T>(s1, pk, pm, w, xk1, xm1);
      }
      const int km = k == 0 ? M : M - k;
      C<T>* wk = W + (size_t)k * rows_w + row0 + b0;
      C<T>* wm = W + (size_t)km * rows_w + row0 + b0;
      if (!bem_check((size_t)km * rows_w + row0 + b0 + (two ? 1 : 0) < wlim && row0 + b0 < rows_w, kerr)) continue;
      if (two) {
        *reinterpret_cast<float4*>(wk) = make_float4((float)xk0.x, (float)xk0.y, (float)xk1.x, (float)xk1.y);
        if (km != k) *reinterpret_cast<float4*>(wm) = make_float4((float)xm0.x, (float)xm0.y, (float)xm1.x, (float)xm1.y);
      } else {
        wk[0] = xk0;
        if (km != k) wm[0] = xm0;
      }
    }
    return;
  }
  for (int idx = threadIdx.x; idx < hm << lognb; idx += blockDim.x) {
    const int k = idx >> lognb, bb = idx & (nb - 1);
    if (bb >= rows) continue;
    const C<T>* s = sm + bb * rs;
    C<T> xk, xm;
    if (k == 0) {
      const C<T> z0 = s[0];
      xk = mk<T>(z0.x + z0.y, (T)0);
      xm = mk<T>(z0.x - z0.y, (T)0);
    } else {
      split_two<T>(s, __ldg(sp + k), __ldg(sp + M - k), __ldg(tws + k), xk, xm);
    }
    const int km = k == 0 ? M : M - k;
    if (!bem_check((size_t)km * rows_w + row0 + bb < wlim && row0 + bb < rows_w, kerr)) continue;
    W[(size_t)k * rows_w + row0 + bb] = xk;
    if (km != k) W[(size_t)km * rows_w + row0 + bb] = xm;
  }
}

// Launch bounds of the row passes (A and C): the plan caps their CTAs at
// BEM_MAX_THREADS_A threads except for the longest rows; three resident CTAs
// per SM (registers capped accordingly) hide more of the global latency.
#ifndef BEM_ROW_MIN_BLOCKS
#define BEM_ROW_MIN_BLOCKS 3
#endif
#define BEM_ROW_BOUNDS(LOGL) __launch_bounds__((LOGL) >= 13 ? 1024 : 512, (LOGL) >= 13 ? 1 : BEM_ROW_MIN_BLOCKS)

// ---------------------------------------------------------------------------
// Pass A: nbA rows per CTA, M/8 threads per row.
template <typename T, int MODE, int LOGL>
__global__ void BEM_ROW_BOUNDS(LOGL) k_pass_a(PassArgs<T> a) {
  using Cx = C<T>;
  using F = FftC<T, LOGL>;
  constexpr int L = F::L, L8 = F::L8, M = L;
  constexpr bool HALF = MODE != A_TORUS;  // conv inputs fill the first half only
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[3 * 32];
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != A_PLAIN && MODE != A_TORUS) {
    if (sc->done) return;
  }
  const int nb = a.pl.nbA, lognb = a.pl.lognbA, rs = a.pl.gA.rs;
  const int tid = threadIdx.x;
  const int b = tid >> (LOGL - 3), t = tid & (L8 - 1);
  const int row0 = blockIdx.x * nb;
  const int row = row0 + b;
  const int ncols = a.ncols_in, nrows = a.nrows_in;
  const bool act = row < nrows;
  const int half = (ncols + 1) >> 1;
  Cx* buf = sm + b * rs;
  const Cx* tw = reinterpret_cast<const Cx*>(a.twA);
  T acc[3] = {0, 0, 0};
  bool upd = false;
  T tau = 0, beta = 0;
  if (MODE == A_PK_P || MODE == A_CG_T) { upd = sc->have_tau != 0; tau = (T)sc->tau; }
  if (MODE == A_PK_T || MODE == A_CG_T) beta = (T)sc->beta;
  if (MODE == A_PK_P && blockIdx.x == 0 && tid == 0) sc->nA = gridDim.x;
  const size_t rowoff = (size_t)row * ncols;

  Cx v[8];
  if (MODE == A_TORUS) {
    // K on the even Px x Py torus (spectrum set-up, FP64, all columns)
    const int py = a.pl.py, px = a.pl.px;
    const int ry = row < py - row ? row : py - row;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int n = F::n0(t, e);
      T xv[2] = {0, 0};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = 2 * n + h;
        const int rx = col < px - col ? col : px - col;
        if (act) xv[h] = (T)__ldg(a.kq64 + (size_t)ry * (M + 1) + rx);
      }
      v[e] = mk<T>(xv[0], xv[1]);
    }
  } else {
    PIn<T> in[8][2];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (HALF && !F::first_half(e)) continue;
      const int n = F::n0(t, e);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act && n < half && 2 * n + h < ncols) pro_gather<T, MODE>(a, rowoff + 2 * n + h, in[e][h]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = mk<T>(0, 0);
      if (HALF && !F::first_half(e)) continue;
      const int n = F::n0(t, e);
      T xv[2] = {0, 0};
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act && n < half && 2 * n + h < ncols)
          xv[h] = pro_apply<T, MODE>(a, rowoff + 2 * n + h, in[e][h], upd, tau, beta, acc);
      v[e] = mk<T>(xv[0], xv[1]);
    }
  }
  F::stage0_fwd(v, t, tw);
#pragma unroll
  for (int e = 0; e < 8; ++e) buf[F::ix0(t, e)] = v[e];
  __syncthreads();
#pragma unroll
  for (int ls = F::LS_TOP; ls >= 0; ls -= 3) {
    F::dif(buf, t, ls, tw);
    __syncthreads();
  }
  if (MODE == A_PK_P) block_partials<T, 3>(acc, a.partA + 4 * blockIdx.x, red);
  // split the packed transform into the half spectrum, store transposed
  split_store<T, M>(sm, rs, nb, lognb, row0, nrows, a.spA, reinterpret_cast<const Cx*>(a.twS),
                    reinterpret_cast<Cx*>(a.W), a.rows_w, a.kerr);
}

// ---------------------------------------------------------------------------
// Persistent pass A: each CTA loops over row groups (nbA rows each) and, while
// it transforms one group, its prologue fields for the next group stream into
// shared memory as bulk copies (one per field row).  Used when rows are
// multiples of 16 elements and the fields are 16-byte aligned.
template <int MODE> struct ProStage {
  static constexpr int nT = (MODE == A_PK_P || MODE == A_PK_T) ? 3 : (MODE == A_CG_T ? 4 : (MODE == A_PLAIN ? 1 : 0));
  static constexpr bool S = MODE == A_CG_T;
};
template <typename T, int MODE>
__host__ __device__ constexpr size_t pro_stage_bytes(int nb, int nx) {
  return ((size_t)ProStage<MODE>::nT * sizeof(T) + (ProStage<MODE>::S ? 1 : 0)) * (size_t)nb * nx;
}
template <typename T, int MODE>
__device__ __forceinline__ const T* pro_field(const PassArgs<T>& a, int f) {
  if (MODE == A_PLAIN) return a.f.src;
  if (MODE == A_CG_T) return f == 0 ? a.f.t : (f == 1 ? a.f.g : (f == 2 ? a.f.p : a.f.r));
  return f == 0 ? a.f.p : (f == 1 ? a.f.t : a.f.g);
}
// Thread 0 stages the prologue fields of rows row0 .. row0+rows-1 into shared
// memory: one bulk copy per field row, completing on `bar` (16-byte aligned
// rows: the persistent launch requires nx % 16 == 0 and aligned fields).
template <typename T, int MODE>
__device__ __forceinline__ void pro_prefetch(const PassArgs<T>& a, T* st, uint8_t* ss, int row0, int rows,
                                             int nx, int nb, unsigned long long* bar) {
  if (threadIdx.x != 0) return;
  const unsigned rb = (unsigned)(nx * (int)sizeof(T));
  fence_proxy_async_smem();
  mbar_expect_tx(bar, (unsigned)rows * (ProStage<MODE>::nT * rb + (ProStage<MODE>::S ? (unsigned)nx : 0u)));
#pragma unroll
  for (int f = 0; f < ProStage<MODE>::nT; ++f) {
    const T* src = pro_field<T, MODE>(a, f);
    for (int bb = 0; bb < rows; ++bb)
      bulk_g2s(st + ((size_t)f * nb + bb) * nx, src + (size_t)(row0 + bb) * nx, rb, bar);
  }
  if (ProStage<MODE>::S) {
    for (int bb = 0; bb < rows; ++bb)
      bulk_g2s(ss + (size_t)bb * nx, a.f.S + (size_t)(row0 + bb) * nx, (unsigned)nx, bar);
  }
}
// Both elements of an even column pair (col, col+1) from the staging area.
template <typename T, int MODE>
__device__ __forceinline__ void pro_gather_pair_staged(const T* st, const uint8_t* ss, int b, int col, int nx,
                                                       int nb, PIn<T>& x0, PIn<T>& x1) {
  const size_t j = (size_t)b * nx + col, plane = (size_t)nb * nx;
  const V2<T>* s2 = reinterpret_cast<const V2<T>*>(st + j);
  const size_t p2 = plane / 2;
  if (MODE == A_PLAIN) {
    const V2<T> v = s2[0];
    x0.p = v.x; x1.p = v.y;
  } else if (MODE == A_CG_T) {
    const V2<T> vt = s2[0], vg = s2[p2], vp = s2[2 * p2], vr = s2[3 * p2];
    const uchar2 vs = *reinterpret_cast<const uchar2*>(ss + j);
    x0.t = vt.x; x1.t = vt.y; x0.g = vg.x; x1.g = vg.y; x0.s = vs.x; x1.s = vs.y;
    x0.p = vp.x; x1.p = vp.y; x0.r = vr.x; x1.r = vr.y;
  } else {
    const V2<T> vp = s2[0], vt = s2[p2], vg = s2[2 * p2];
    x0.p = vp.x; x1.p = vp.y; x0.t = vt.x; x1.t = vt.y; x0.g = vg.x; x1.g = vg.y;
  }
}

template <typename T, int MODE>
__device__ __forceinline__ void pro_gather_staged(const T* st, const uint8_t* ss, int b, int col, int nx,
                                                  int nb, PIn<T>& x) {
  const size_t j = (size_t)b * nx + col, plane = (size_t)nb * nx;
  if (MODE == A_PLAIN) { x.p = st[j]; }
  else if (MODE == A_CG_T) {
    x.t = st[j]; x.g = st[plane + j]; x.p = st[2 * plane + j]; x.r = st[3 * plane + j]; x.s = ss[j];
  }
  else { x.p = st[j]; x.t = st[plane + j]; x.g = st[2 * plane + j]; }
}

#ifndef BEM_ROWP_MIN_BLOCKS
#define BEM_ROWP_MIN_BLOCKS 2
#endif
#define BEM_ROWP_BOUNDS(LOGL) __launch_bounds__((LOGL) >= 13 ? 1024 : 512, (LOGL) >= 13 ? 1 : BEM_ROWP_MIN_BLOCKS)

template <typename T, int MODE, int LOGL>
__device__ __forceinline__ void pass_ap_body(const PassArgs<T>& a) {
  using Cx = C<T>;
  using F = FftC<T, LOGL>;
  constexpr int L = F::L, L8 = F::L8, M = L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[3 * 32];
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != A_PLAIN) {
    if (sc->done) return;
  }
  const int nb = a.pl.nbA, lognb = a.pl.lognbA, rs = a.pl.gA.rs;
  const int tid = threadIdx.x;
  const int b = tid >> (LOGL - 3), t = tid & (L8 - 1);
  const int ncols = a.ncols_in, nrows = a.nrows_in;
  const int half = (ncols + 1) >> 1;
  const int G = (nrows + nb - 1) / nb;
  Cx* buf = sm + b * rs;
  T* st = reinterpret_cast<T*>(smem_raw + ((sizeof(Cx) * (size_t)nb * rs + 15) & ~(size_t)15));
  uint8_t* ss = reinterpret_cast<uint8_t*>(st) + (size_t)ProStage<MODE>::nT * sizeof(T) * nb * ncols;
  const Cx* tw = reinterpret_cast<const Cx*>(a.twA);
  const Cx* tws = reinterpret_cast<const Cx*>(a.twS);
  const int* sp = a.spA;
  Cx* W = reinterpret_cast<Cx*>(a.W);
  T acc[3] = {0, 0, 0};
  bool upd = false;
  T tau = 0, beta = 0;
  if (MODE == A_PK_P || MODE == A_CG_T) { upd = sc->have_tau != 0; tau = (T)sc->tau; }
  if (MODE == A_PK_T || MODE == A_CG_T) beta = (T)sc->beta;
  if (MODE == A_PK_P && blockIdx.x == 0 && tid == 0) sc->nA = gridDim.x;

  __shared__ unsigned long long bar;
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  unsigned phase = 0;
  // row groups g0 .. gend-1 (fixed-set CG: the contact band only; the rows of W
  // outside it are not written and pass B treats them as zero)
  int g0 = 0, gend = G;
  if (MODE == A_CG_T && a.use_band) {
    g0 = sc->band0 / nb;
    gend = sc->band1 >= sc->band0 ? sc->band1 / nb + 1 : g0;
  }
  if (MODE == A_PLAIN && a.use_band == 2) {  // a residual whose input lies in rows band_lo .. band_hi
    g0 = a.band_lo / nb;
    gend = a.band_hi >= a.band_lo ? min(a.band_hi / nb + 1, G) : g0;
  }
  int g = g0 + blockIdx.x;
  if (g < gend) pro_prefetch<T, MODE>(a, st, ss, g * nb, min(nb, nrows - g * nb), ncols, nb, &bar);
  for (; g < gend; g += gridDim.x) {
    const int row0 = g * nb, row = row0 + b;
    const bool act = row < nrows;
    const size_t rowoff = (size_t)row * ncols;
    bool ok = mbar_wait(&bar, phase);
    phase ^= 1u;
#ifdef BEM_DEBUG_CHECKS
    // Test hook of debug builds: once per solve whose scalars ask for it, CTA 0
    // of the first CG-loop launch waits (bounded) on a barrier nothing
    // completes; every copy it issued has already landed, so it gives up like a
    // lost copy would.  (A_PLAIN launches carry no scalars.)
    if (MODE != A_PLAIN && sc != nullptr && g == g0 && blockIdx.x == 0) {
      __shared__ unsigned long long never;
      __shared__ int inj;
      if (tid == 0) {
        inj = atomicExch(&sc->inject, 0);
        if (inj) mbar_init(&never, 1);
      }
      __syncthreads();
      if (inj && tid == 0) ok = ok && mbar_wait(&never, 0);
    }
#endif
    if (__syncthreads_or(!ok)) {  // the staged rows never arrived: give up together
      if (tid == 0 && a.kerr) atomicOr(a.kerr, 1u);
      return;
    }
    // ncols is a multiple of 16 here: column pairs (2n, 2n+1) are whole
    PIn<T> in[8][2];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (!F::first_half(e)) continue;
      const int n = F::n0(t, e);
      if (act && n < half) pro_gather_pair_staged<T, MODE>(st, ss, b, 2 * n, ncols, nb, in[e][0], in[e][1]);
    }
    __syncthreads();  // staging consumed: refill it for the next group
    const int gn = g + gridDim.x;
    if (gn < gend) pro_prefetch<T, MODE>(a, st, ss, gn * nb, min(nb, nrows - gn * nb), ncols, nb, &bar);
    Cx v[8];
    T* out = pro_out<T, MODE>(a);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = mk<T>(0, 0);
      if (!F::first_half(e)) continue;
      const int n = F::n0(t, e);
      if (act && n < half) {
        const T x0 = pro_value<T, MODE>(in[e][0], upd, tau, beta, acc);
        const T x1 = pro_value<T, MODE>(in[e][1], upd, tau, beta, acc);
        if (MODE != A_PLAIN) {
          V2<T> o;
          o.x = x0; o.y = x1;
          *reinterpret_cast<V2<T>*>(out + rowoff + 2 * n) = o;
        }
        if (MODE == A_CG_T && upd) {  // p and g after the previous iteration's update
          V2<T> o;
          o.x = in[e][0].p; o.y = in[e][1].p;
          *reinterpret_cast<V2<T>*>(a.f.p + rowoff + 2 * n) = o;
          o.x = in[e][0].g; o.y = in[e][1].g;
          *reinterpret_cast<V2<T>*>(a.f.g + rowoff + 2 * n) = o;
        }
        v[e] = mk<T>(x0, x1);
      }
    }
    F::stage0_fwd(v, t, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e) buf[F::ix0(t, e)] = v[e];
    __syncthreads();
#pragma unroll
    for (int ls = F::LS_TOP; ls >= 0; ls -= 3) {
      F::dif(buf, t, ls, tw);
      __syncthreads();
    }
    split_store<T, M>(sm, rs, nb, lognb, row0, nrows, sp, tws, W, a.rows_w, a.kerr);
  }
  if (MODE == A_PK_P) block_partials<T, 3>(acc, a.partA + 4 * blockIdx.x, red);
}

// One launch of the persistent pass A; and the same over several instances of
// one size class at once (blockIdx.y = instance, each with its own arguments,
// fields, scalars and convergence flag).
template <typename T, int MODE, int LOGL>
__global__ void BEM_ROWP_BOUNDS(LOGL) k_pass_ap(PassArgs<T> a) {
  pass_ap_body<T, MODE, LOGL>(a);
}
template <typename T, int MODE, int LOGL>
__global__ void BEM_ROWP_BOUNDS(LOGL) k_pass_ap_mi(const PassArgs<T>* __restrict__ arr) {
  pass_ap_body<T, MODE, LOGL>(arr[blockIdx.y]);
}

// ---------------------------------------------------------------------------
// Pass B: nbB columns per CTA, Py/8 threads per column; columns kx = 0..M.
#ifndef BEM_COL_MIN_BLOCKS
#define BEM_COL_MIN_BLOCKS 2
#endif
#define BEM_COL_BOUNDS(LOGL) __launch_bounds__((LOGL) >= 13 ? 1024 : 512, (LOGL) >= 13 ? 1 : BEM_COL_MIN_BLOCKS)
template <typename T, int MODE, int LOGL>
__device__ __forceinline__ void pass_b_body(const PassArgs<T>& a) {
  using Cx = C<T>;
  using F = FftC<T, LOGL>;
  constexpr int L = F::L, L8 = F::L8, R0 = F::R0, hyq = (L >> 1) + 1;
  constexpr bool HALF = MODE == B_CONV;  // Ny <= Py/2 rows in, Ny rows out
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  if (MODE == B_CONV && a.sc != nullptr) {
    if (a.sc->done) return;
  }
  const int M = a.pl.M, rin = a.rows_w, rs = a.pl.gB.rs;
  const int tid = threadIdx.x;
  const int c = tid >> (LOGL - 3), t = tid & (L8 - 1);
  const int kx = blockIdx.x * a.pl.nbB + c;
  const bool act = kx <= M;
  Cx* buf = sm + c * rs;
  const Cx* tw = reinterpret_cast<const Cx*>(a.twB);
  const int* sp = a.spB;
  Cx* W = reinterpret_cast<Cx*>(a.W);
  const size_t coff = (size_t)(act ? kx : 0) * rin;
  // rows of W that can be nonzero: all, or the contact band in the fixed-set CG loop
  int ylo = 0, yhi = rin - 1;
  if (MODE == B_CONV && a.use_band) {
    ylo = a.use_band == 2 ? a.band_lo : a.sc->band0;
    yhi = min(a.use_band == 2 ? a.band_hi : a.sc->band1, rin - 1);
  }

  Cx v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    v[e] = mk<T>(0, 0);
    if (HALF && !F::first_half(e)) continue;
    const int y = F::n0(t, e);
    if (act && y >= ylo && y <= yhi && bem_check(coff + y < (size_t)(M + 1) * rin, a.kerr)) v[e] = W[coff + y];
  }
  F::stage0_fwd(v, t, tw);
#pragma unroll
  for (int e = 0; e < 8; ++e) buf[F::ix0(t, e)] = v[e];
  __syncthreads();
#pragma unroll
  for (int ls = F::LS_TOP; ls >= 3; ls -= 3) {
    F::dif(buf, t, ls, tw);
    __syncthreads();
  }
  if (MODE == B_SPECTRUM) {
    F::dif(buf, t, 0, tw);
    __syncthreads();
    if (!act) return;
    for (int ky = t; ky < hyq; ky += L8) {
      const double re = (double)buf[__ldg(sp + ky)].x;
      a.khat64_out[(size_t)kx * hyq + ky] = re;
      a.khat32_out[(size_t)kx * hyq + ky] = (float)re;
    }
    return;
  }
  // last DIF stage (stride 1), spectrum multiply, first DIT stage (stride 1),
  // in registers.  Thread t takes the group holding frequencies t + q L/8.
  {
    const int sp0 = __ldg(sp + t);
    const T* kc = a.khat + (size_t)(act ? kx : 0) * hyq;
    T kf[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int ky = t + q * L8;
      const int kk = ky <= (L >> 1) ? ky : L - ky;
      kf[q] = act ? __ldg(kc + kk) : (T)0;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = buf[sp0 ^ r];
    dft8<T, -1>(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = scale<T>(v[q], kf[q]);
    dft8<T, 1>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[sp0 ^ r] = v[r];
  }
  __syncthreads();
#pragma unroll
  for (int ls = 3; ls <= F::LS_TOP; ls += 3) {
    F::dit(buf, t, ls, tw);
    __syncthreads();
  }
  // last DIT stage (inverse of stage 0), natural order, first half to global
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = buf[F::ix0(t, e)];
  F::stage0_inv(v, t, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (!F::first_half(e)) continue;
      const int y = F::n0(t, e);
      if (y >= ylo && y <= yhi && bem_check(coff + y < (size_t)(M + 1) * rin, a.kerr)) W[coff + y] = v[e];
    }
  }
  (void)R0;
}

template <typename T, int MODE, int LOGL>
__global__ void BEM_COL_BOUNDS(LOGL) k_pass_b(PassArgs<T> a) {
  pass_b_body<T, MODE, LOGL>(a);
}
template <typename T, int MODE, int LOGL>
__global__ void BEM_COL_BOUNDS(LOGL) k_pass_b_mi(const PassArgs<T>* __restrict__ arr) {
  pass_b_body<T, MODE, LOGL>(arr[blockIdx.y]);
}

// ---------------------------------------------------------------------------
// Pass B with radix-16 stages: a length L = 2^LOGL column (512 <= L <= 8192)
// as a leading stage of radix R0 = 2^(LOGL mod 4) (radix 16 when LOGL is a
// multiple of 4) with stride 2^LS0 = L/R0, then radix-16 stages with strides
// 2^(LS0-4), ..., 16, 1.  Thread t (t < L/16) holds the 16 points
// t + e L/16 in the leading stage (the 16/R0 butterflies t + j L/16), so a
// forward transform reads only e < 8 (the nonzero half) and the inverse
// writes only e < 8.  After the stride-1 stage position dig16(k) holds
// frequency k, and the 16 positions of t's last-stage group hold the
// frequencies t + q L/16: thread t multiplies those by the spectrum and runs
// the first inverse stage in registers.  Against the radix-8 pass this takes
// two fewer shared-memory round trips and barriers per transform (4096
// points: four barriers instead of six) and a third fewer twiddle stages.
// The stage table of the leading stage holds exp(-2 pi i o/L), o < 2^LS0;
// that of the radix-16 stage with stride 2^ls holds exp(-2 pi i o/2^(ls+4)),
// o < 2^ls; tables concatenated in DIF order.
template <typename T, int LOGL>
struct Fft16 {
  static_assert(LOGL >= 9 && LOGL <= 13, "radix-16 column pass: 512 to 8192 points");
  static constexpr int L = 1 << LOGL, L16 = L >> 4, RB = LOGL & 3, R0 = RB ? 1 << RB : 16;
  static constexpr int LS0 = LOGL - (RB ? RB : 4);
  using G = GeoR16<(int)sizeof(T), LOGL>;
  static __device__ __forceinline__ int sw(int i) {
    if (sizeof(T) == 4)
      return i ^ ((((i >> G::a) ^ (i >> G::b)) & 7) | ((((i >> G::c) ^ (i >> G::d)) & 1) << 3));
    return i ^ ((((i >> G::a) ^ (i >> G::b)) & 3) | ((((i >> G::c) ^ (i >> G::d)) & 1) << 2));
  }
  // position of frequency k (k < L/16) after the DIF stages: digits of k in
  // the stages' radices, most significant position digit first
  static __device__ __forceinline__ int dig16(int k) {
    int p = (k & (R0 - 1)) << LS0;
    k >>= (RB ? RB : 4);
#pragma unroll
    for (int ls = LS0 - 4; ls >= 0; ls -= 4) {
      p |= (k & 15) << ls;
      k >>= 4;
    }
    return p;
  }
  // table offset of the radix-16 stage with stride 2^ls (ls < LS0)
  static __host__ __device__ constexpr int tw_off(int ls) { return (1 << LS0) + ((1 << LS0) - (1 << (ls + 4))) / 15; }

  static __device__ __forceinline__ void stage0_fwd(C<T>* v, int t, const C<T>* tw) {
    if constexpr (R0 == 16) {
      dft16<T, -1>(v);
      twiddle16<T>(v, __ldg(tw + t));
    } else {
      constexpr int J = 16 / R0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        C<T> u[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) u[r] = v[j + r * J];
        const C<T> w = __ldg(tw + t + j * L16);
        if constexpr (R0 == 8) {
          dft8<T, -1>(u);
          twiddle8<T>(u, w);
        } else if constexpr (R0 == 4) {
          dft4<T, -1>(u[0], u[1], u[2], u[3]);
          const C<T> w2 = mul<T>(w, w);
          u[1] = mul<T>(u[1], w); u[2] = mul<T>(u[2], w2); u[3] = mul<T>(u[3], mul<T>(w2, w));
        } else {
          dft2<T, -1>(u[0], u[1]);
          u[1] = mul<T>(u[1], w);
        }
#pragma unroll
        for (int r = 0; r < R0; ++r) v[j + r * J] = u[r];
      }
    }
  }
  static __device__ __forceinline__ void stage0_inv(C<T>* v, int t, const C<T>* tw) {
    if constexpr (R0 == 16) {
      twiddle16<T>(v, conj<T>(__ldg(tw + t)));
      dft16<T, 1>(v);
    } else {
      constexpr int J = 16 / R0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        C<T> u[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) u[r] = v[j + r * J];
        const C<T> w = conj<T>(__ldg(tw + t + j * L16));
        if constexpr (R0 == 8) {
          twiddle8<T>(u, w);
          dft8<T, 1>(u);
        } else if constexpr (R0 == 4) {
          const C<T> w2 = mul<T>(w, w);
          u[1] = mul<T>(u[1], w); u[2] = mul<T>(u[2], w2); u[3] = mul<T>(u[3], mul<T>(w2, w));
          dft4<T, 1>(u[0], u[1], u[2], u[3]);
        } else {
          u[1] = mul<T>(u[1], w);
          dft2<T, 1>(u[0], u[1]);
        }
#pragma unroll
        for (int r = 0; r < R0; ++r) v[j + r * J] = u[r];
      }
    }
  }
  // radix-16 DIF / DIT stage with stride 2^ls, 4 <= ls < LS0 (in shared memory)
  static __device__ __forceinline__ void dif(C<T>* buf, int t, int ls, const C<T>* tw) {
    const int o = t & ((1 << ls) - 1);
    const int sb = sw(((t >> ls) << (ls + 4)) + o);
    C<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[sb ^ sw(r << ls)];
    dft16<T, -1>(v);
    twiddle16<T>(v, __ldg(tw + tw_off(ls) + o));
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[sb ^ sw(q << ls)] = v[q];
  }
  static __device__ __forceinline__ void dit(C<T>* buf, int t, int ls, const C<T>* tw) {
    const int o = t & ((1 << ls) - 1);
    const int sb = sw(((t >> ls) << (ls + 4)) + o);
    C<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[sb ^ sw(r << ls)];
    twiddle16<T>(v, conj<T>(__ldg(tw + tw_off(ls) + o)));
    dft16<T, 1>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[sb ^ sw(q << ls)] = v[q];
  }
};

// At most 256 threads per CTA (one 8192-point column: 512) and three CTAs per
// SM: 80 registers per thread, which leaves a few bytes of spills; at 128
// registers the pass would run two CTAs per SM.
#define BEM_COL16_BOUNDS(LOGL) __launch_bounds__(BEM_COL16_MAX_THREADS(LOGL), (LOGL) >= 13 ? 1 : 3)
template <typename T, int LOGL>
__device__ __forceinline__ void pass_b16_body(const PassArgs<T>& a) {
  using Cx = C<T>;
  using F = Fft16<T, LOGL>;
  constexpr int L = F::L, L16 = F::L16, hyq = (L >> 1) + 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  if (a.sc != nullptr && a.sc->done) return;
  const int M = a.pl.M, rin = a.rows_w;
  const int tid = threadIdx.x;
  const int c = tid >> (LOGL - 4), t = tid & (L16 - 1);
  const int kx = blockIdx.x * a.pl.nbB + c;
  const bool act = kx <= M;
  Cx* buf = sm + c * L;
  const Cx* tw = reinterpret_cast<const Cx*>(a.twB16);
  Cx* W = reinterpret_cast<Cx*>(a.W);
  const size_t coff = (size_t)(act ? kx : 0) * rin;
  int ylo = 0, yhi = rin - 1;
  if (a.use_band) {
    ylo = a.use_band == 2 ? a.band_lo : a.sc->band0;
    yhi = min(a.use_band == 2 ? a.band_hi : a.sc->band1, rin - 1);
  }

  Cx v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    v[e] = mk<T>(0, 0);
    if (e >= 8) continue;
    const int y = t + e * L16;
    if (act && y >= ylo && y <= yhi && bem_check(coff + y < (size_t)(M + 1) * rin, a.kerr)) v[e] = W[coff + y];
  }
  F::stage0_fwd(v, t, tw);
#pragma unroll
  for (int e = 0; e < 16; ++e) buf[F::sw(t + e * L16)] = v[e];
  __syncthreads();
#pragma unroll
  for (int ls = F::LS0 - 4; ls >= 4; ls -= 4) {
    F::dif(buf, t, ls, tw);
    __syncthreads();
  }
  // stride-1 stage, spectrum multiply and the first inverse stage in registers
  {
    const int gb = F::sw(F::dig16(t));
    const T* kc = a.khat + (size_t)(act ? kx : 0) * hyq;
    T kf[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int ky = t + q * L16;
      const int kk = ky <= (L >> 1) ? ky : L - ky;
      kf[q] = act ? __ldg(kc + kk) : (T)0;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[gb ^ F::sw(r)];
    dft16<T, -1>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = scale<T>(v[q], kf[q]);
    dft16<T, 1>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[gb ^ F::sw(r)] = v[r];
  }
  __syncthreads();
#pragma unroll
  for (int ls = 4; ls <= F::LS0 - 4; ls += 4) {
    F::dit(buf, t, ls, tw);
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = buf[F::sw(t + e * L16)];
  F::stage0_inv(v, t, tw);
  if (act) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int y = t + e * L16;
      if (y >= ylo && y <= yhi && bem_check(coff + y < (size_t)(M + 1) * rin, a.kerr)) W[coff + y] = v[e];
    }
  }
}
template <typename T, int LOGL>
__global__ void BEM_COL16_BOUNDS(LOGL) k_pass_b16(PassArgs<T> a) {
  pass_b16_body<T, LOGL>(a);
}
template <typename T, int LOGL>
__global__ void BEM_COL16_BOUNDS(LOGL) k_pass_b16_mi(const PassArgs<T>* __restrict__ arr) {
  pass_b16_body<T, LOGL>(arr[blockIdx.y]);
}

// Epilogue fields of pass C that are prefetched into shared memory at kernel
// start (their loads then overlap the inverse transform): number of T-typed
// fields and whether the contact set S (one byte per element) is staged.
template <int MODE> struct EpiStage {
  static constexpr int nT = (MODE == C_PK_G || MODE == C_CG_R) ? 2 : (MODE == C_CG_G || MODE == C_GAP) ? 1 : 0;
  static constexpr bool S = MODE == C_CG_R || MODE == C_CG_G;
  static constexpr bool any = nT > 0 || S;
};
// Bytes of that staging area for nb rows of nx elements.
template <typename T, int MODE>
__host__ __device__ constexpr size_t epi_stage_bytes(int nb, int nx) {
  return ((size_t)EpiStage<MODE>::nT * sizeof(T) + (EpiStage<MODE>::S ? 1 : 0)) * (size_t)nb * nx;
}

// ---------------------------------------------------------------------------
// Pass C epilogue, in two phases like the prologue.
template <typename T>
struct EIn {
  T c, p, t, g;
  uint8_t s;
};

template <typename T, int MODE>
__device__ __forceinline__ void epi_gather(const PassArgs<T>& a, size_t i, EIn<T>& x) {
  if (MODE == C_PK_G) {
    x.c = a.f.c[i]; x.p = a.f.p[i];
  } else if (MODE == C_PK_R) {
    x.p = a.f.p[i]; x.t = a.f.t[i]; x.g = a.f.g[i];
  } else if (MODE == C_CG_R) {
    x.s = a.f.S[i]; x.t = a.f.t[i]; x.g = a.f.g[i];
  } else if (MODE == C_CG_G) {
    x.s = a.f.S[i]; x.c = a.f.c[i];
  } else if (MODE == C_GAP) {
    x.c = a.f.c[i];
  }
}

// Gather from the shared-memory staging area: T fields [f][b][col], then S [b][col].
template <typename T, int MODE>
__device__ __forceinline__ void epi_gather_staged(const T* st, const uint8_t* ss, int b, int col, int nx,
                                                  int nb, EIn<T>& x) {
  const size_t j = (size_t)b * nx + col, plane = (size_t)nb * nx;
  if (MODE == C_PK_G) { x.c = st[j]; x.p = st[plane + j]; }
  else if (MODE == C_CG_R) { x.t = st[j]; x.g = st[plane + j]; x.s = ss[j]; }
  else if (MODE == C_CG_G) { x.c = st[j]; x.s = ss[j]; }
  else if (MODE == C_GAP) { x.c = st[j]; }
}

// The field an epilogue mode writes (null: none) and the value it writes.
template <typename T, int MODE>
__device__ __forceinline__ T* epi_out(const PassArgs<T>& a) {
  if (MODE == C_PLAIN) return a.f.dst;
  if (MODE == C_PK_G || MODE == C_CG_G || MODE == C_GAP) return a.f.g;
  if (MODE == C_CG_R) return a.f.r;
  return nullptr;
}
template <typename T, int MODE>
__device__ __forceinline__ T epi_value(T u, const EIn<T>& x, T* acc) {
  if (MODE == C_PLAIN) {
    return u;
  } else if (MODE == C_PK_G) {
    const T gv = u + x.c;
    if (x.p > (T)0) { acc[0] += gv * gv; acc[1] += (T)1; }
    return gv;
  } else if (MODE == C_PK_R) {
    if (x.p > (T)0) { acc[0] += x.g * x.t; acc[1] += u * x.t; }
    return (T)0;
  } else if (MODE == C_CG_R) {
    const T rv = x.s ? u : (T)0;
    acc[0] += rv * x.t;
    acc[1] += rv * x.g;
    acc[2] += rv * rv;
    acc[3] += x.g * x.g;
    return rv;
  } else if (MODE == C_CG_G) {
    if (x.s) {
      const T gv = u + x.c;
      acc[0] += gv * gv;
      acc[1] += x.c * x.c;
      return gv;
    }
    return (T)0;
  } else {  // C_GAP
    return u + x.c;
  }
}
template <typename T, int MODE>
__device__ __forceinline__ void epi_gather_pair_staged(const T* st, const uint8_t* ss, int b, int col, int nx,
                                                       int nb, EIn<T>& x0, EIn<T>& x1) {
  const size_t j = (size_t)b * nx + col, plane = (size_t)nb * nx;
  const V2<T>* s2 = reinterpret_cast<const V2<T>*>(st + j);
  if (MODE == C_PK_G) {
    const V2<T> vc = s2[0], vp = s2[plane / 2];
    x0.c = vc.x; x1.c = vc.y; x0.p = vp.x; x1.p = vp.y;
  } else if (MODE == C_CG_R) {
    const V2<T> vt = s2[0], vg = s2[plane / 2];
    const uchar2 vs = *reinterpret_cast<const uchar2*>(ss + j);
    x0.t = vt.x; x1.t = vt.y; x0.g = vg.x; x1.g = vg.y; x0.s = vs.x; x1.s = vs.y;
  } else if (MODE == C_CG_G) {
    const V2<T> vc = s2[0];
    const uchar2 vs = *reinterpret_cast<const uchar2*>(ss + j);
    x0.c = vc.x; x1.c = vc.y; x0.s = vs.x; x1.s = vs.y;
  } else if (MODE == C_GAP) {
    const V2<T> vc = s2[0];
    x0.c = vc.x; x1.c = vc.y;
  }
}

template <typename T, int MODE>
__device__ __forceinline__ void epi_apply(const PassArgs<T>& a, size_t i, T u, const EIn<T>& x, T* acc) {
  if (MODE == C_PLAIN) {
    a.f.dst[i] = u;
  } else if (MODE == C_PK_G) {
    const T gv = u + x.c;
    a.f.g[i] = gv;
    if (x.p > (T)0) { acc[0] += gv * gv; acc[1] += (T)1; }
  } else if (MODE == C_PK_R) {
    if (x.p > (T)0) { acc[0] += x.g * x.t; acc[1] += u * x.t; }
  } else if (MODE == C_CG_R) {
    const T rv = x.s ? u : (T)0;
    a.f.r[i] = rv;
    acc[0] += rv * x.t;
    acc[1] += rv * x.g;
    acc[2] += rv * rv;
    acc[3] += x.g * x.g;
  } else if (MODE == C_CG_G) {
    if (x.s) {
      const T gv = u + x.c;
      a.f.g[i] = gv;
      acc[0] += gv * gv;
      acc[1] += x.c * x.c;
    } else {
      a.f.g[i] = (T)0;
    }
  } else if (MODE == C_GAP) {
    a.f.g[i] = u + x.c;
  }
}

// Count a CG iteration; past the cap the solve ends unconverged (a device-side
// bound on the batched while-loop graph whatever the iteration's outcome).
__device__ __forceinline__ void count_loop(Scalars* sc) {
  sc->loops += 1;
  if (!sc->done && sc->loops >= sc->max_loops) { sc->status = SC_NOCONV; sc->done = 1; }
}

// Scalar work of the last CTA of a pass-C launch (FP64): the Polonsky-Keer
// stopping test and beta after the gap pass, tau after the r pass, tau or the
// initial residual of the fixed-set CG.
// Scalars the fixed-set r pass's last CTA needs, read when every CTA starts
// (their loads then are off the critical path at the end) by thread 32, so
// that thread 0 issues the staging copies at once; barriers of the pass order
// the shared-memory copy before the last CTA's thread 0 reads it.
struct CgPre {
  double stop2;
  int iter, max_iter, loops, max_loops;
};
__device__ __forceinline__ void cg_pre_load(const Scalars* sc, CgPre* pre) {
  if (threadIdx.x != (blockDim.x > 32 ? 32u : 0u)) return;
  pre->stop2 = sc->stop2;
  pre->iter = sc->iter;
  pre->max_iter = sc->max_iter;
  pre->loops = sc->loops;
  pre->max_loops = sc->max_loops;
}

template <typename T, int MODE>
__device__ __forceinline__ void pass_c_finalize(Scalars* sc, const double (&s2)[4], const double (&s3)[3],
                                                const CgPre& pre) {
  if (MODE == C_PK_G) {
    sc->cnt_c = 0;
    const double G = s2[0], nic = s2[1];
    int done = 0;
    if (sc->have_tau) {
      sc->sum_dp = s3[0];
      sc->sum_p = s3[1];
      sc->n_ol = s3[2];
      sc->iter += 1;
      const double eps = s3[1] > 0.0 ? s3[0] / s3[1] : 0.0;
      sc->eps = eps;
      sc->delta = s3[2] > 0.0 ? 0.0 : 1.0;
      if (!isfinite(eps) || !isfinite(G)) { sc->status = SC_NUMERIC; done = 1; }
      else if (eps < sc->tol) done = 1;
      else if (sc->iter >= sc->max_iter) { sc->status = SC_NOCONV; done = 1; }
      // rounding floor: no new minimum of eps for kStall iterations ends the solve
      if (!done) {
        if (sc->iter == 1 || eps < 0.5 * sc->eps_min) { sc->eps_min = eps; sc->it_min = sc->iter; }
        else if (sc->iter - sc->it_min > kStall) { sc->status = SC_STALL; done = 1; }
      }
    }
    sc->n_ic = nic;
    sc->G = G;
    if (!done) {
      if (nic == 0.0 || G == 0.0) { done = 1; }
      else { sc->beta = sc->delta * G / sc->G_old; sc->G_old = G; }
    }
    if (done) sc->done = 1;
  } else if (MODE == C_PK_R) {
    sc->cnt_a = 0;
    const double sgt = s2[0], srt = s2[1];
    if (!isfinite(sgt) || !isfinite(srt)) { sc->status = SC_NUMERIC; sc->done = 1; }
    else if (srt == 0.0) { sc->done = 1; }
    else if (!(sgt > 0.0) || srt < 0.0) {
      // finite precision lost the conjugacy (tau would be <= 0 and the overlap
      // step p = -tau g would go negative): skip this update and restart the
      // directions from the gap (delta = 0)
      sc->have_tau = 0;
      sc->delta = 0.0;
    } else { sc->tau = sgt / srt; sc->have_tau = 1; }
    count_loop(sc);
  } else if (MODE == C_CG_R) {
    // The residual g here has every update so far applied (pass A applies the
    // previous iteration's), so |g|^2 = G decides convergence exactly.  Else the
    // step tau = G / (t . r), and the next residual's norm
    // |g - tau r|^2 = G - 2 tau g.r + tau^2 |r|^2 from this pass's sums gives
    // beta = |g - tau r|^2 / G and the stopping test after this update: if it
    // passes, the solve ends with the update pending (applied by cg_finish),
    // else the next pass A applies p -= tau t, g -= tau r, t = g + beta t.
    // The stopping tests compare squares; the scalars this needs are read
    // before any is written, so their loads overlap.
    const double stop2 = pre.stop2;
    const int iter = pre.iter, max_iter = pre.max_iter, loops = pre.loops + 1, max_loops = pre.max_loops;
    const double str = s2[0], sgr = s2[1], srr = s2[2], G = s2[3];
    int done = 0, status = SC_OK, have = 0;
    double tau = 0.0, beta = 0.0, gn = G;
    if (!isfinite(str) || !isfinite(G) || !isfinite(sgr) || !isfinite(srr)) {
      status = SC_NUMERIC;
      done = 1;
    } else if (G <= stop2 || str <= 0.0) {
      done = 1;
    } else if (iter >= max_iter) {
      status = SC_NOCONV;
      done = 1;
    } else {
      tau = G / str;
      gn = G - 2.0 * tau * sgr + tau * tau * srr;
      if (gn < 0.0) gn = 0.0;
      beta = gn / G;
      have = 1;
      if (gn <= stop2) done = 1;  // converged once this update is applied
    }
    if (!done && loops >= max_loops) {  // the device-side loop bound (count_loop)
      status = SC_NOCONV;
      done = 1;
    }
    sc->loops = loops;
    sc->cnt_a = 0;
    sc->str = str;
    sc->G = gn;
    sc->have_tau = have;
    if (have) {
      sc->tau = tau;
      sc->beta = beta;
      sc->iter = iter + 1;
    }
    if (status != SC_OK) sc->status = status;
    if (done) sc->done = 1;
  } else if (MODE == C_CG_G) {
    sc->cnt_a = 0;
    const double G = s2[0];
    double bn = sqrt(s2[1]);
    if (bn == 0.0) bn = 1.0;
    sc->G = G;
    sc->bnorm = bn;
    sc->beta = 0.0;
    sc->iter = 0;
    sc->eps = sqrt(G) / bn;
    sc->stop2 = (sc->tol * bn) * (sc->tol * bn);  // stop once |g|^2 <= (tol |b|)^2
    if (!isfinite(G)) { sc->status = SC_NUMERIC; sc->done = 1; }
    else if (G <= sc->stop2) sc->done = 1;
  }
}

template <typename T, int MODE, int LOGL>
__global__ void BEM_ROW_BOUNDS(LOGL) k_pass_c(PassArgs<T> a) {
  using Cx = C<T>;
  using F = FftC<T, LOGL>;
  constexpr int L = F::L, L8 = F::L8, M = L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[4 * 32];
  __shared__ int lastflag;
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != C_PLAIN && MODE != C_GAP) {
    if (sc->done) return;
  }
  __shared__ CgPre pre;
  if (MODE == C_CG_R) cg_pre_load(sc, &pre);
  const int nb = a.pl.nbA, lognb = a.pl.lognbA, rs = a.pl.gA.rs;
  const int nx = a.pl.nx, ny = a.pl.ny;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int b = tid >> (LOGL - 3), t = tid & (L8 - 1);
  const int row0 = blockIdx.x * nb;
  const Cx* W = reinterpret_cast<const Cx*>(a.W);
  const Cx* tws = reinterpret_cast<const Cx*>(a.twS);
  const Cx* tw = reinterpret_cast<const Cx*>(a.twA);
  const int* sp = a.spA;
  // prefetch the epilogue fields of this CTA's rows (if rows are 16-byte multiples)
  constexpr bool kStage = EpiStage<MODE>::any;
  const bool staged = kStage && (nx & 15) == 0 && row0 + nb <= ny;
  T* st = reinterpret_cast<T*>(smem_raw + ((sizeof(Cx) * (size_t)nb * rs + 15) & ~(size_t)15));
  uint8_t* ss = reinterpret_cast<uint8_t*>(st) + (size_t)EpiStage<MODE>::nT * sizeof(T) * nb * nx;
  if (staged) {
    const int cpr = nx * (int)sizeof(T) / 16;  // 16-byte chunks per row of a T field
#pragma unroll
    for (int f = 0; f < EpiStage<MODE>::nT; ++f) {
      const T* src = (MODE == C_PK_G) ? (f == 0 ? a.f.c : a.f.p) : (MODE == C_CG_R ? (f == 0 ? a.f.t : a.f.g) : a.f.c);
      for (int q = tid; q < cpr * nb; q += nthr) {
        const int bb = q / cpr, ch = q - bb * cpr;
        cp_async16(reinterpret_cast<char*>(st + ((size_t)f * nb + bb) * nx) + 16 * ch,
                   reinterpret_cast<const char*>(src + (size_t)(row0 + bb) * nx) + 16 * ch);
      }
    }
    if (EpiStage<MODE>::S) {
      const int cps = nx / 16;
      for (int q = tid; q < cps * nb; q += nthr) {
        const int bb = q / cps, ch = q - bb * cps;
        cp_async16(ss + (size_t)bb * nx + 16 * ch, a.f.S + (size_t)(row0 + bb) * nx + 16 * ch);
      }
    }
    cp_async_commit();
  }
  // rebuild the packed half-length spectrum, scattered to digit-reversed
  // positions: Z[k] = E + i O, E = X[k] + conj X[M-k], O = (X[k] - conj X[M-k]) e^{+i pi k/M}.
  // Each thread handles up to NP pairs (k, M-k); all loads are issued first.
  {
    constexpr int hm = (M >> 1) + 1;
    const int total = hm << lognb;
    constexpr int NP = 5;  // ceil((M/2 + 1) nb / (nb M/8)) for M >= 16
    Cx xk[NP], xm[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int idx = tid + j * nthr;
      xk[j] = mk<T>(0, 0);
      xm[j] = mk<T>(0, 0);
      if (idx < total) {
        const int k = idx >> lognb, rw = row0 + (idx & (nb - 1));
        if (rw < ny) {
          if (bem_check(k <= M && rw < a.rows_w, a.kerr)) {
            xk[j] = W[(size_t)k * a.rows_w + rw];
            xm[j] = W[(size_t)(M - k) * a.rows_w + rw];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int idx = tid + j * nthr;
      if (idx >= total) continue;
      const int k = idx >> lognb, bb = idx & (nb - 1);
      Cx* s = sm + bb * rs;
      const Cx wk = conj<T>(__ldg(tws + k));
      {
        const Cx E = add<T>(xk[j], conj<T>(xm[j]));
        const Cx O = mul<T>(sub<T>(xk[j], conj<T>(xm[j])), wk);
        s[__ldg(sp + k)] = add<T>(E, mul_si<T, 1>(O));
      }
      if (k != 0 && k != M - k) {
        const Cx wm = mk<T>(-wk.x, wk.y);  // exp(+i pi (M-k)/M) = -conj(wk)
        const Cx E = add<T>(xm[j], conj<T>(xk[j]));
        const Cx O = mul<T>(sub<T>(xm[j], conj<T>(xk[j])), wm);
        s[__ldg(sp + M - k)] = add<T>(E, mul_si<T, 1>(O));
      }
    }
  }
  __syncthreads();
  Cx* buf = sm + b * rs;
#pragma unroll
  for (int ls = 0; ls <= F::LS_TOP; ls += 3) {
    F::dit(buf, t, ls, tw);
    __syncthreads();
  }
  // last DIT stage: natural-order outputs z[n] = (x[2n], x[2n+1]) * Px; the
  // epilogue fields are gathered first so their loads overlap the stage
  const T us = (T)a.uscale;
  T acc[4] = {0, 0, 0, 0};
  const int row = row0 + b;
  const bool act = row < ny;
  const size_t rowoff = (size_t)row * nx;
  const int half = (nx + 1) >> 1;
  EIn<T> ein[8][2];
  if (staged) {
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (!F::first_half(e)) continue;
      const int n = F::n0(t, e);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act && n < half && 2 * n + h < nx)
          epi_gather_staged<T, MODE>(st, ss, b, 2 * n + h, nx, nb, ein[e][h]);
    }
  } else if (MODE != C_PLAIN) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (!F::first_half(e)) continue;
      const int n = F::n0(t, e);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (act && n < half && 2 * n + h < nx) epi_gather<T, MODE>(a, rowoff + 2 * n + h, ein[e][h]);
    }
  }
  Cx v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = buf[F::ix0(t, e)];
  F::stage0_inv(v, t, tw);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if (!F::first_half(e)) continue;
    const int n = F::n0(t, e);
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (act && n < half && 2 * n + h < nx)
        epi_apply<T, MODE>(a, rowoff + 2 * n + h, us * (h ? v[e].y : v[e].x), ein[e][h], acc);
  }
  if (MODE == C_PLAIN || MODE == C_GAP) return;
  constexpr int NQ = MODE == C_CG_R ? 4 : 2;
  block_partials<T, NQ>(acc, a.partC + 4 * blockIdx.x, red);
  if (!last_block_arrival(MODE == C_PK_G ? &sc->cnt_c : &sc->cnt_a, &lastflag)) return;
  double s2[4] = {0, 0, 0, 0};
  grid_sum<T, NQ>(a.partC, gridDim.x, s2, red);
  double s3[3] = {0, 0, 0};
  if (MODE == C_PK_G) grid_sum<T, 3>(a.partA, __ldcg(&sc->nA), s3, red);
  if (tid != 0) return;
  pass_c_finalize<T, MODE>(sc, s2, s3, pre);
}

// ---------------------------------------------------------------------------
// Persistent pass C: each CTA loops over row groups; the strided W rows of the
// next group stream into shared memory with cp.async and its epilogue fields
// as bulk copies (one per field row, on an mbarrier) while the current group
// is transformed.  Used when rows are multiples of 16 elements.
template <typename T, int MODE, int LOGL>
__device__ __forceinline__ void pass_cp_body(const PassArgs<T>& a) {
  using Cx = C<T>;
  using F = FftC<T, LOGL>;
  constexpr int L = F::L, L8 = F::L8, M = L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[4 * 32];
  __shared__ int lastflag;
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != C_PLAIN && MODE != C_GAP) {
    if (sc->done) return;
  }
  __shared__ CgPre pre;
  if (MODE == C_CG_R) cg_pre_load(sc, &pre);
  const int nb = a.pl.nbA, lognb = a.pl.lognbA, rs = a.pl.gA.rs;
  const int nx = a.pl.nx, ny = a.pl.ny;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int b = tid >> (LOGL - 3), t = tid & (L8 - 1);
  const int G = (ny + nb - 1) / nb;
  const Cx* W = reinterpret_cast<const Cx*>(a.W);
  const Cx* tws = reinterpret_cast<const Cx*>(a.twS);
  const Cx* tw = reinterpret_cast<const Cx*>(a.twA);
  const int* sp = a.spA;
  Cx* buf = sm + b * rs;
  // shared memory: transform rows | W staging [w_stage_rows(M) x nb] | epilogue staging
  const size_t off_w = pass_c_w_offset(sizeof(Cx) * (size_t)nb * rs);
  Cx* wst = reinterpret_cast<Cx*>(smem_raw + off_w);
  const size_t off_e = off_w + ((sizeof(Cx) * (size_t)w_stage_rows(M) * nb + 15) & ~(size_t)15);
  T* st = reinterpret_cast<T*>(smem_raw + off_e);
  uint8_t* ss = reinterpret_cast<uint8_t*>(st) + (size_t)EpiStage<MODE>::nT * sizeof(T) * nb * nx;

  // W of a row group by TMA: thread 0 issues one 2D box load per w_box_rows(M)
  // rows of W (nb complex values of each), completing on wbar
  __shared__ unsigned long long wbar;
  unsigned wphase = 0;
  const bool tma = a.tmW != nullptr;
  auto prefetch_w = [&](int gg) {
    const int r0 = gg * nb, rows = min(nb, ny - r0);
    if (tma) {
      if (tid == 0) {
        constexpr int bo = w_box_rows(M), nload = w_stage_rows(M) / bo;
        fence_proxy_async_smem();
        mbar_expect_tx(&wbar, (unsigned)(nload * bo * nb * (int)sizeof(Cx)));
        for (int j = 0; j < nload; ++j) tma_load_2d(wst + (size_t)j * bo * nb, a.tmW, 2 * r0, j * bo, &wbar);
      }
      return;
    }
    if (sizeof(Cx) == 8 && nb >= 2 && rows == nb && (a.rows_w & 1) == 0) {
      // FP32 and an even number of full rows: 16-byte chunks of two rows
      const int lh = lognb - 1;
      for (int q = tid; q < (M + 1) << lh; q += nthr) {
        const int k = q >> lh, j = q & ((1 << lh) - 1);
        if (bem_check(r0 + 2 * j + 1 < a.rows_w, a.kerr))
          cp_async16(wst + (k << lognb) + 2 * j, W + (size_t)k * a.rows_w + r0 + 2 * j);
      }
    } else {
      for (int q = tid; q < (M + 1) << lognb; q += nthr) {
        const int k = q >> lognb, bb = q & (nb - 1);
        if (bb < rows && bem_check(r0 + bb < a.rows_w, a.kerr))
          cp_async_cx<Cx>(wst + q, W + (size_t)k * a.rows_w + r0 + bb);
      }
    }
    cp_async_commit();
  };
  // epilogue fields: thread 0 issues one bulk copy per field row, completing on ebar
  __shared__ unsigned long long ebar;
  if (tid == 0) {
    mbar_init(&ebar, 1);
    if (tma) mbar_init(&wbar, 1);
  }
  __syncthreads();
  unsigned ephase = 0;
  auto prefetch_e = [&](int gg) {
    if (tid != 0) return;
    const int r0 = gg * nb, rows = min(nb, ny - r0);
    const unsigned rb = (unsigned)(nx * (int)sizeof(T));
    fence_proxy_async_smem();
    mbar_expect_tx(&ebar, (unsigned)rows * (EpiStage<MODE>::nT * rb + (EpiStage<MODE>::S ? (unsigned)nx : 0u)));
#pragma unroll
    for (int f = 0; f < EpiStage<MODE>::nT; ++f) {
      const T* src = (MODE == C_PK_G) ? (f == 0 ? a.f.c : a.f.p) : (MODE == C_CG_R ? (f == 0 ? a.f.t : a.f.g) : a.f.c);
      for (int bb = 0; bb < rows; ++bb)
        bulk_g2s(st + ((size_t)f * nb + bb) * nx, src + (size_t)(r0 + bb) * nx, rb, &ebar);
    }
    if (EpiStage<MODE>::S) {
      for (int bb = 0; bb < rows; ++bb)
        bulk_g2s(ss + (size_t)bb * nx, a.f.S + (size_t)(r0 + bb) * nx, (unsigned)nx, &ebar);
    }
  };

  const T us = (T)a.uscale;
  T acc[4] = {0, 0, 0, 0};
  const int half = (nx + 1) >> 1;
  // row groups g0 .. gend-1 (fixed-set CG: the contact band only; r = 0 outside it)
  int g0 = 0, gend = G;
  if (MODE == C_CG_R && a.use_band) {
    g0 = sc->band0 / nb;
    gend = sc->band1 >= sc->band0 ? sc->band1 / nb + 1 : g0;
  }
  if (MODE == C_GAP && a.use_band == 2) {  // the residual on rows band_lo .. band_hi only
    g0 = a.band_lo / nb;
    gend = a.band_hi >= a.band_lo ? min(a.band_hi / nb + 1, G) : g0;
  }
  int g = g0 + blockIdx.x;
  if (g < gend) {
    prefetch_w(g);
    if (EpiStage<MODE>::any) prefetch_e(g);
  }
  for (; g < gend; g += gridDim.x) {
    const int row0 = g * nb;
    if (tma) {  // W of this group
      const bool ok = mbar_wait(&wbar, wphase);
      wphase ^= 1u;
      if (__syncthreads_or(!ok)) {  // it never arrived: give up together
        if (tid == 0 && a.kerr) atomicOr(a.kerr, 1u);
        return;
      }
    } else {
      cp_async_wait_all();  // W of this group
      __syncthreads();
    }
    // rebuild the packed half-length spectrum from the staged W rows
#pragma unroll 2
    for (int idx = tid; idx < ((M >> 1) + 1) << lognb; idx += nthr) {
      const int k = idx >> lognb, bb = idx & (nb - 1);
      const Cx xk = wst[(k << lognb) + bb], xm = wst[((M - k) << lognb) + bb];
      Cx* s = sm + bb * rs;
      const Cx wk = conj<T>(__ldg(tws + k));
      {
        const Cx E = add<T>(xk, conj<T>(xm));
        const Cx O = mul<T>(sub<T>(xk, conj<T>(xm)), wk);
        s[__ldg(sp + k)] = add<T>(E, mul_si<T, 1>(O));
      }
      if (k != 0 && k != M - k) {
        const Cx wm = mk<T>(-wk.x, wk.y);
        const Cx E = add<T>(xm, conj<T>(xk));
        const Cx O = mul<T>(sub<T>(xm, conj<T>(xk)), wm);
        s[__ldg(sp + M - k)] = add<T>(E, mul_si<T, 1>(O));
      }
    }
    __syncthreads();  // W staging consumed
    const int gn = g + gridDim.x;
    if (gn < gend) prefetch_w(gn);
#pragma unroll
    for (int ls = 0; ls <= F::LS_TOP; ls += 3) {
      F::dit(buf, t, ls, tw);
      __syncthreads();
    }
    if (EpiStage<MODE>::any) {  // epilogue fields of this group
      const bool ok = mbar_wait(&ebar, ephase);
      ephase ^= 1u;
      if (__syncthreads_or(!ok)) {  // they never arrived: give up together
        cp_async_wait_all();
        if (tid == 0 && a.kerr) atomicOr(a.kerr, 1u);
        return;
      }
    }
    const int row = row0 + b;
    const bool act = row < ny;
    const size_t rowoff = (size_t)row * nx;
    // nx is a multiple of 16 here: column pairs (2n, 2n+1) are whole
    EIn<T> ein[8][2];
    if (MODE != C_PLAIN) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (!F::first_half(e)) continue;
        const int n = F::n0(t, e);
        if (act && n < half) {
          if (EpiStage<MODE>::any) {
            epi_gather_pair_staged<T, MODE>(st, ss, b, 2 * n, nx, nb, ein[e][0], ein[e][1]);
          } else {
            epi_gather<T, MODE>(a, rowoff + 2 * n, ein[e][0]);
            epi_gather<T, MODE>(a, rowoff + 2 * n + 1, ein[e][1]);
          }
        }
      }
    }
    Cx v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = buf[F::ix0(t, e)];
    F::stage0_inv(v, t, tw);
    T* out = epi_out<T, MODE>(a);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (!F::first_half(e)) continue;
      const int n = F::n0(t, e);
      if (act && n < half) {
        V2<T> o;
        o.x = epi_value<T, MODE>(us * v[e].x, ein[e][0], acc);
        o.y = epi_value<T, MODE>(us * v[e].y, ein[e][1], acc);
        if (MODE != C_PK_R) *reinterpret_cast<V2<T>*>(out + rowoff + 2 * n) = o;
      }
    }
    __syncthreads();  // epilogue staging and transform rows consumed
    if (gn < gend && EpiStage<MODE>::any) prefetch_e(gn);
  }
  cp_async_wait_all();
  if (MODE == C_PLAIN || MODE == C_GAP) return;
  constexpr int NQ = MODE == C_CG_R ? 4 : 2;
  block_partials<T, NQ>(acc, a.partC + 4 * blockIdx.x, red);
  if (!last_block_arrival(MODE == C_PK_G ? &sc->cnt_c : &sc->cnt_a, &lastflag)) return;
  double s2[4] = {0, 0, 0, 0};
  grid_sum<T, NQ>(a.partC, gridDim.x, s2, red);
  double s3[3] = {0, 0, 0};
  if (MODE == C_PK_G) grid_sum<T, 3>(a.partA, __ldcg(&sc->nA), s3, red);
  if (tid != 0) return;
  pass_c_finalize<T, MODE>(sc, s2, s3, pre);
}

template <typename T, int MODE, int LOGL>
__global__ void BEM_ROWP_BOUNDS(LOGL) k_pass_cp(PassArgs<T> a) {
  pass_cp_body<T, MODE, LOGL>(a);
}
template <typename T, int MODE, int LOGL>
__global__ void BEM_ROWP_BOUNDS(LOGL) k_pass_cp_mi(const PassArgs<T>* __restrict__ arr) {
  pass_cp_body<T, MODE, LOGL>(arr[blockIdx.y]);
}

// ---------------------------------------------------------------------------
// Elementwise kernels (grid-stride, FP64 partials per CTA, last block reduces).

template <typename T>
__global__ void k_pk_init(int n, const double* __restrict__ h64, double d, T* __restrict__ c,
                          T* __restrict__ p, T* __restrict__ t, int warm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double cv = h64[i] - d;
    c[i] = (T)cv;
    if (!warm) p[i] = cv < 0.0 ? (T)1e-3 : (T)0;
    t[i] = (T)0;
  }
}

// Contact-box sub-grid: gather p, c, S of the box (zero outside the grid), and
// scatter p back (in-grid elements only).  bx is a power of two.
template <typename T>
__global__ void k_box_gather(const T* __restrict__ p, const T* __restrict__ c, const uint8_t* __restrict__ S,
                             int nx, int ny, int x0, int y0, T* __restrict__ bp, T* __restrict__ bc,
                             uint8_t* __restrict__ bS, int lbx, int nb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int X = x0 + (i & ((1 << lbx) - 1)), Y = y0 + (i >> lbx);
    const bool in = X < nx && Y < ny;
    const size_t src = in ? (size_t)Y * nx + X : 0;
    bp[i] = in ? p[src] : (T)0;
    bc[i] = in ? c[src] : (T)0;
    bS[i] = in ? S[src] : (uint8_t)0;
  }
}
template <typename T>
__global__ void k_box_scatter(const T* __restrict__ bp, T* __restrict__ p, int nx, int ny, int x0, int y0,
                              int lbx, int nb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int X = x0 + (i & ((1 << lbx) - 1)), Y = y0 + (i >> lbx);
    if (X < nx && Y < ny) p[(size_t)Y * nx + X] = bp[i];
  }
}

// The update a fixed-set CG solve ends with when its stopping test passed on
// the predicted |g - tau r|^2 (pass C leaves it pending): p -= tau t,
// g -= tau r on the contact band (t and r vanish off the set).
template <typename T>
__global__ void k_cg_finish(int nx, Fields<T> f, const Scalars* sc) {
  if (!sc->have_tau) return;
  const T tau = (T)sc->tau;
  const size_t off = (size_t)sc->band0 * nx;
  const size_t n = sc->band1 >= sc->band0 ? (size_t)(sc->band1 - sc->band0 + 1) * nx : 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    f.p[off + i] -= tau * f.t[off + i];
    f.g[off + i] -= tau * f.r[off + i];
  }
}

// Loop condition of a while-loop graph over several instances: run the body
// again while any instance's solve is not done.
template <typename T>
__global__ void k_batch_ctl(const PassArgs<T>* __restrict__ arr, int n, unsigned long long cond) {
  int live = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) live |= !(*(volatile int*)&arr[i].sc->done);
  live = __syncthreads_or(live);
  if (threadIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, live ? 1u : 0u);
}

// Detach every element of S with tensile stress -p > p_crit (Eq. 24).
template <typename T>
__global__ void k_detach(int n, Fields<T> f, double* part, Scalars* sc) {
  __shared__ double red[3 * 32];
  __shared__ int lastflag;
  const T pc = (T)sc->pcrit;
  T cnt = 0, ns = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (f.S[i]) {
      if (-f.p[i] > pc) { f.S[i] = 0; f.p[i] = (T)0; cnt += (T)1; }
      else ns += (T)1;
    }
  }
  double v[2] = {(double)cnt, (double)ns};
  block_sum<2>(v, red);
  if (threadIdx.x == 0) { part[4 * blockIdx.x] = v[0]; part[4 * blockIdx.x + 1] = v[1]; }
  if (!last_block_arrival(&sc->cnt_r, &lastflag)) return;
  double s[2];
  grid_sum<double, 2>(part, gridDim.x, s, red);
  if (threadIdx.x != 0) return;
  sc->cnt_r = 0;
  sc->n_ol = s[0];
  sc->n_ic = s[1];
}

// Final statistics: out[0] = sum p, out[1] = #contact, out[2] = max |g| on
// contact, out[3] = max(-g) off contact.  Contact = S if use_set else p > 0.
template <typename T>
__global__ void k_stats(int n, const T* p, const T* g, const uint8_t* S, int use_set, double* part,
                        unsigned int* counter, double* out) {
  __shared__ double red[3 * 32];
  __shared__ double redm[2][32];
  __shared__ int lastflag;
  double sp = 0, cnt = 0, m1 = 0, m2 = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double pv = (double)p[i];
    const bool in = use_set ? (S[i] != 0) : (pv > 0.0);
    sp += pv;
    if (in) { cnt += 1.0; if (g) m1 = fmax(m1, fabs((double)g[i])); }
    else if (g) m2 = fmax(m2, -(double)g[i]);
  }
  double v[2] = {sp, cnt};
  // max reductions
  for (int o = 16; o > 0; o >>= 1) {
    m1 = fmax(m1, __shfl_down_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_down_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) { redm[0][threadIdx.x >> 5] = m1; redm[1][threadIdx.x >> 5] = m2; }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    double a1 = 0, a2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a1 = fmax(a1, redm[0][w]); a2 = fmax(a2, redm[1][w]); }
    double* pp = part + 4 * blockIdx.x;
    pp[0] = v[0]; pp[1] = v[1]; pp[2] = a1; pp[3] = a2;
  }
  if (!last_block_arrival(counter, &lastflag)) return;
  // fixed-order parallel reduction of the per-CTA partials
  double s0 = 0, s1 = 0, x1 = 0, x2 = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    s0 += __ldcg(part + 4 * b); s1 += __ldcg(part + 4 * b + 1);
    x1 = fmax(x1, __ldcg(part + 4 * b + 2)); x2 = fmax(x2, __ldcg(part + 4 * b + 3));
  }
  for (int o = 16; o > 0; o >>= 1) {
    x1 = fmax(x1, __shfl_down_sync(0xffffffffu, x1, o));
    x2 = fmax(x2, __shfl_down_sync(0xffffffffu, x2, o));
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { redm[0][threadIdx.x >> 5] = x1; redm[1][threadIdx.x >> 5] = x2; }
  double v2[2] = {s0, s1};
  block_sum<2>(v2, red);
  if (threadIdx.x == 0) {
    double a1 = 0, a2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a1 = fmax(a1, redm[0][w]); a2 = fmax(a2, redm[1][w]); }
    out[0] = v2[0]; out[1] = v2[1]; out[2] = a1; out[3] = a2;
    *counter = 0;
  }
}

template <typename T>
__global__ void k_convert_in(const double* src, T* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}
template <typename T>
__global__ void k_convert_out(const T* src, double* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}
template <typename T>
__global__ void k_offset(const double* h64, double d, T* c, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c[i] = (T)(h64[i] - d);
}
template <typename T>
__global__ void k_set_from_p(const T* p, uint8_t* S, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    S[i] = p[i] > (T)0 ? 1 : 0;
}
template <typename T>
__global__ void k_mask_field(T* x, const uint8_t* S, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!S[i]) x[i] = (T)0;
}

// ---------------------------------------------------------------------------
// Host launchers: dispatch on the transform length.

#define BEM_LOGL_CASES_A(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)
#define BEM_LOGL_CASES_B(X) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)

// Resident CTAs per SM of a kernel at a launch shape (cached per shape).
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple((const void*)kernel, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  if (n < 1) n = 1;
  cache[key] = n;
  return n;
}

#ifndef BEM_PERSISTENT
#define BEM_PERSISTENT 1
#endif

inline bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// The persistent row passes stage whole field rows with 16-byte bulk copies.
template <typename T, int MODE>
bool pro_fields_aligned(const PassArgs<T>& a) {
  if (MODE == A_PLAIN) return aligned16(a.f.src);
  return aligned16(a.f.p) && aligned16(a.f.t) && aligned16(a.f.g) && aligned16(a.f.S) &&
         (MODE != A_CG_T || aligned16(a.f.r));
}
template <typename T>
bool epi_fields_aligned(const PassArgs<T>& a) {
  return aligned16(a.f.c) && aligned16(a.f.p) && aligned16(a.f.t) && aligned16(a.f.S) && aligned16(a.W) &&
         aligned16(a.f.dst) && aligned16(a.f.g) && aligned16(a.f.r);
}

template <typename T, int MODE>
void launch_a_mode(const PassArgs<T>& a, cudaStream_t s) {
  const dim3 block(a.pl.threadsA);
  const int groups = (a.nrows_in + a.pl.nbA - 1) / a.pl.nbA;
  if (BEM_PERSISTENT && MODE != A_TORUS && (a.ncols_in & 15) == 0 && pro_fields_aligned<T, MODE>(a)) {
    const size_t smem = ((a.pl.smemA + 15) & ~(size_t)15) + pro_stage_bytes<T, MODE>(a.pl.nbA, a.ncols_in);
    switch (a.pl.gA.logL) {
#define BEM_CASE(LG)                                                                        \
  case LG: {                                                                                \
    const int occ = resident_ctas(k_pass_ap<T, MODE, LG>, a.pl.threadsA, smem);            \
    const int grid = std::min(groups, a.pl.nsm * occ);                                      \
    k_pass_ap<T, MODE, LG><<<grid, block, smem, s>>>(a);                                    \
  } break;
      BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
    }
    return;
  }
  const dim3 grid(groups);
  switch (a.pl.gA.logL) {
#define BEM_CASE(LG) case LG: k_pass_a<T, MODE, LG><<<grid, block, a.pl.smemA, s>>>(a); break;
    BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  }
}
#define BEM_LOGL_CASES_B16(X) X(9) X(10) X(11) X(12) X(13)
template <typename T, int MODE>
void launch_b_mode(const PassArgs<T>& a, cudaStream_t s) {
  const dim3 grid(a.pl.gridB), block(a.pl.threadsB);
  if (MODE == B_CONV && a.pl.radixB == 16) {
    switch (a.pl.gB.logL) {
#define BEM_CASE(LG) case LG: k_pass_b16<T, LG><<<grid, block, a.pl.smemB, s>>>(a); break;
      BEM_LOGL_CASES_B16(BEM_CASE)
#undef BEM_CASE
    }
    return;
  }
  switch (a.pl.gB.logL) {
#define BEM_CASE(LG) case LG: k_pass_b<T, MODE, LG><<<grid, block, a.pl.smemB, s>>>(a); break;
    BEM_LOGL_CASES_B(BEM_CASE)
#undef BEM_CASE
  }
}
template <typename T, int MODE>
void launch_c_mode(const PassArgs<T>& a, cudaStream_t s) {
  const dim3 block(a.pl.threadsA);
  const int groups = a.pl.gridA;
  if (BEM_PERSISTENT && (a.pl.nx & 15) == 0 && epi_fields_aligned<T>(a)) {
    const size_t smem = pass_c_smem(a.pl.smemC, a.pl.M, a.pl.nbA, (int)sizeof(C<T>),
                                    epi_stage_bytes<T, MODE>(a.pl.nbA, a.pl.nx));
    switch (a.pl.gA.logL) {
#define BEM_CASE(LG)                                                                        \
  case LG: {                                                                                \
    const int occ = resident_ctas(k_pass_cp<T, MODE, LG>, a.pl.threadsA, smem);            \
    const int grid = std::min(groups, a.pl.nsm * occ);                                      \
    k_pass_cp<T, MODE, LG><<<grid, block, smem, s>>>(a);                                    \
  } break;
      BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
    }
    return;
  }
  const dim3 grid(groups);
  const size_t smem = ((a.pl.smemC + 15) & ~(size_t)15) + epi_stage_bytes<T, MODE>(a.pl.nbA, a.pl.nx);
  switch (a.pl.gA.logL) {
#define BEM_CASE(LG) case LG: k_pass_c<T, MODE, LG><<<grid, block, smem, s>>>(a); break;
    BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  }
}

// Several-instance launches (blockIdx.y = instance).  Every instance has the
// plan `a0` has (one size class); each keeps the grid.x its single launch
// would have, so its partial sums, and so its results, are the same bitwise.
template <typename T, int MODE>
void launch_a_mode_mi(const PassArgs<T>& a0, const PassArgs<T>* arr, int n, cudaStream_t s) {
  const dim3 block(a0.pl.threadsA);
  const int groups = (a0.nrows_in + a0.pl.nbA - 1) / a0.pl.nbA;
  const size_t smem = ((a0.pl.smemA + 15) & ~(size_t)15) + pro_stage_bytes<T, MODE>(a0.pl.nbA, a0.ncols_in);
  switch (a0.pl.gA.logL) {
#define BEM_CASE(LG)                                                                        \
  case LG: {                                                                                \
    const int occ = resident_ctas(k_pass_ap<T, MODE, LG>, a0.pl.threadsA, smem);           \
    const dim3 grid(std::min(groups, a0.pl.nsm * occ), n);                                  \
    k_pass_ap_mi<T, MODE, LG><<<grid, block, smem, s>>>(arr);                               \
  } break;
    BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  }
}
template <typename T, int MODE>
void launch_c_mode_mi(const PassArgs<T>& a0, const PassArgs<T>* arr, int n, cudaStream_t s) {
  const dim3 block(a0.pl.threadsA);
  const int groups = a0.pl.gridA;
  const size_t smem = pass_c_smem(a0.pl.smemC, a0.pl.M, a0.pl.nbA, (int)sizeof(C<T>),
                                  epi_stage_bytes<T, MODE>(a0.pl.nbA, a0.pl.nx));
  switch (a0.pl.gA.logL) {
#define BEM_CASE(LG)                                                                        \
  case LG: {                                                                                \
    const int occ = resident_ctas(k_pass_cp<T, MODE, LG>, a0.pl.threadsA, smem);           \
    const dim3 grid(std::min(groups, a0.pl.nsm * occ), n);                                  \
    k_pass_cp_mi<T, MODE, LG><<<grid, block, smem, s>>>(arr);                               \
  } break;
    BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  }
}
template <typename T>
void launch_pass_a_mi(const PassArgs<T>& a0, int mode, const PassArgs<T>* arr, int n, cudaStream_t s) {
  if (mode == A_PK_P) launch_a_mode_mi<T, A_PK_P>(a0, arr, n, s);
  else if (mode == A_PK_T) launch_a_mode_mi<T, A_PK_T>(a0, arr, n, s);
  else if (mode == A_CG_T) launch_a_mode_mi<T, A_CG_T>(a0, arr, n, s);
}
template <typename T>
void launch_pass_b_mi(const PassArgs<T>& a0, const PassArgs<T>* arr, int n, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (n == 1 && tc_column_pass_enabled() && tc_column_pass_applies(a0)) {
      launch_pass_b_tc(a0, s);
      return;
    }
  }
  const dim3 grid(a0.pl.gridB, n), block(a0.pl.threadsB);
  if (a0.pl.radixB == 16) {
    switch (a0.pl.gB.logL) {
#define BEM_CASE(LG) case LG: k_pass_b16_mi<T, LG><<<grid, block, a0.pl.smemB, s>>>(arr); break;
      BEM_LOGL_CASES_B16(BEM_CASE)
#undef BEM_CASE
    }
    return;
  }
  switch (a0.pl.gB.logL) {
#define BEM_CASE(LG) case LG: k_pass_b_mi<T, B_CONV, LG><<<grid, block, a0.pl.smemB, s>>>(arr); break;
    BEM_LOGL_CASES_B(BEM_CASE)
#undef BEM_CASE
  }
}
template <typename T>
void launch_pass_c_mi(const PassArgs<T>& a0, int mode, const PassArgs<T>* arr, int n, cudaStream_t s) {
  if (mode == C_PK_G) launch_c_mode_mi<T, C_PK_G>(a0, arr, n, s);
  else if (mode == C_PK_R) launch_c_mode_mi<T, C_PK_R>(a0, arr, n, s);
  else if (mode == C_CG_R) launch_c_mode_mi<T, C_CG_R>(a0, arr, n, s);
}
template <typename T>
void launch_batch_ctl(const PassArgs<T>* arr, int n, unsigned long long cond, cudaStream_t s) {
  k_batch_ctl<T><<<1, 256, 0, s>>>(arr, n, cond);
}

template <typename T>
void launch_pass_a(const PassArgs<T>& a, int mode, cudaStream_t s) {
  switch (mode) {
    case A_PLAIN: launch_a_mode<T, A_PLAIN>(a, s); break;
    case A_PK_P: launch_a_mode<T, A_PK_P>(a, s); break;
    case A_PK_T: launch_a_mode<T, A_PK_T>(a, s); break;
    case A_CG_T: launch_a_mode<T, A_CG_T>(a, s); break;
    case A_TORUS:
      if constexpr (sizeof(T) == 8) launch_a_mode<T, A_TORUS>(a, s);
      break;
  }
}
template <typename T>
void launch_pass_b(const PassArgs<T>& a, int mode, cudaStream_t s) {
  if (mode == B_SPECTRUM) {
    launch_b_mode<T, B_SPECTRUM>(a, s);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (tc_column_pass_enabled() && tc_column_pass_applies(a)) {
      launch_pass_b_tc(a, s);
      return;
    }
  }
  launch_b_mode<T, B_CONV>(a, s);
}
template <typename T>
void launch_pass_c(const PassArgs<T>& a, int mode, cudaStream_t s) {
  switch (mode) {
    case C_PLAIN: launch_c_mode<T, C_PLAIN>(a, s); break;
    case C_PK_G: launch_c_mode<T, C_PK_G>(a, s); break;
    case C_PK_R: launch_c_mode<T, C_PK_R>(a, s); break;
    case C_CG_R: launch_c_mode<T, C_CG_R>(a, s); break;
    case C_CG_G: launch_c_mode<T, C_CG_G>(a, s); break;
    case C_GAP: launch_c_mode<T, C_GAP>(a, s); break;
  }
}

// Opt every pass kernel into the largest dynamic shared memory the SM allows
// next to its static reduction scratch (227 KB per block in total).  `bytes`
// caps the request.  Returns the first failure.
template <typename K>
cudaError_t set_smem_max(K kernel, int bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int lim = 227 * 1024 - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes < lim ? bytes : lim);
}
#define BEM_ATTR(fn) \
  if ((r = set_smem_max(fn, bytes)) != cudaSuccess && e == cudaSuccess) e = r;
template <typename T>
cudaError_t set_smem_attrs_a(int bytes) {
  cudaError_t e = cudaSuccess, r;
#define BEM_CASE(LG)                          \
  BEM_ATTR((k_pass_a<T, A_PLAIN, LG>))        \
  BEM_ATTR((k_pass_a<T, A_PK_P, LG>))         \
  BEM_ATTR((k_pass_a<T, A_PK_T, LG>))         \
  BEM_ATTR((k_pass_a<T, A_CG_T, LG>))         \
  BEM_ATTR((k_pass_ap<T, A_PLAIN, LG>))       \
  BEM_ATTR((k_pass_ap<T, A_PK_P, LG>))        \
  BEM_ATTR((k_pass_ap<T, A_PK_T, LG>))        \
  BEM_ATTR((k_pass_ap<T, A_CG_T, LG>))        \
  BEM_ATTR((k_pass_ap_mi<T, A_PK_P, LG>))     \
  BEM_ATTR((k_pass_ap_mi<T, A_PK_T, LG>))     \
  BEM_ATTR((k_pass_ap_mi<T, A_CG_T, LG>))     \
  if constexpr (sizeof(T) == 8) { BEM_ATTR((k_pass_a<T, A_TORUS, LG>)) }
  BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  return e;
}
template <typename T>
cudaError_t set_smem_attrs_b(int bytes) {
  cudaError_t e = cudaSuccess, r;
#define BEM_CASE(LG) \
  BEM_ATTR((k_pass_b<T, B_CONV, LG>)) BEM_ATTR((k_pass_b<T, B_SPECTRUM, LG>)) BEM_ATTR((k_pass_b_mi<T, B_CONV, LG>))
  BEM_LOGL_CASES_B(BEM_CASE)
#undef BEM_CASE
#define BEM_CASE(LG) BEM_ATTR((k_pass_b16<T, LG>)) BEM_ATTR((k_pass_b16_mi<T, LG>))
  BEM_LOGL_CASES_B16(BEM_CASE)
#undef BEM_CASE
  return e;
}
template <typename T>
cudaError_t set_smem_attrs_c(int bytes) {
  cudaError_t e = cudaSuccess, r;
#define BEM_CASE(LG)                          \
  BEM_ATTR((k_pass_c<T, C_PLAIN, LG>))        \
  BEM_ATTR((k_pass_c<T, C_PK_G, LG>))         \
  BEM_ATTR((k_pass_c<T, C_PK_R, LG>))         \
  BEM_ATTR((k_pass_c<T, C_CG_R, LG>))         \
  BEM_ATTR((k_pass_c<T, C_CG_G, LG>))         \
  BEM_ATTR((k_pass_c<T, C_GAP, LG>))          \
  BEM_ATTR((k_pass_cp<T, C_PLAIN, LG>))       \
  BEM_ATTR((k_pass_cp<T, C_PK_G, LG>))        \
  BEM_ATTR((k_pass_cp<T, C_PK_R, LG>))        \
  BEM_ATTR((k_pass_cp<T, C_CG_R, LG>))        \
  BEM_ATTR((k_pass_cp<T, C_CG_G, LG>))        \
  BEM_ATTR((k_pass_cp<T, C_GAP, LG>))         \
  BEM_ATTR((k_pass_cp_mi<T, C_PK_G, LG>))     \
  BEM_ATTR((k_pass_cp_mi<T, C_PK_R, LG>))     \
  BEM_ATTR((k_pass_cp_mi<T, C_CG_R, LG>))
  BEM_LOGL_CASES_A(BEM_CASE)
#undef BEM_CASE
  return e;
}
#undef BEM_ATTR

static inline int ew_grid(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
void launch_pk_init(const Plan& pl, const double* h64, double d, T* c, T* p, T* t, int warm,
                    int ngrid, cudaStream_t s) {
  k_pk_init<T><<<ngrid, 256, 0, s>>>(pl.nx * pl.ny, h64, d, c, p, t, warm);
}
template <typename T>
void launch_box_gather(const T* p, const T* c, const uint8_t* S, int nx, int ny, int x0, int y0, T* bp, T* bc,
                       uint8_t* bS, int bx, int by, cudaStream_t s) {
  int lbx = 0;
  while ((1 << lbx) < bx) ++lbx;
  const int nb = bx * by;
  k_box_gather<T><<<ew_grid((size_t)nb), 256, 0, s>>>(p, c, S, nx, ny, x0, y0, bp, bc, bS, lbx, nb);
}
template <typename T>
void launch_box_scatter(const T* bp, T* p, int nx, int ny, int x0, int y0, int bx, int by, cudaStream_t s) {
  int lbx = 0;
  while ((1 << lbx) < bx) ++lbx;
  const int nb = bx * by;
  k_box_scatter<T><<<ew_grid((size_t)nb), 256, 0, s>>>(bp, p, nx, ny, x0, y0, lbx, nb);
}
template <typename T>
void launch_cg_finish(const Plan& pl, Fields<T> f, const Scalars* sc, int ngrid, cudaStream_t s) {
  k_cg_finish<T><<<ngrid, 256, 0, s>>>(pl.nx, f, sc);
}
template <typename T>
void launch_detach(const Plan& pl, Fields<T> f, double* part, Scalars* sc, int ngrid,
                   cudaStream_t s) {
  k_detach<T><<<ngrid, 256, 0, s>>>(pl.nx * pl.ny, f, part, sc);
}
template <typename T>
void launch_stats(const Plan& pl, const T* p, const T* g, const uint8_t* S, int use_set,
                  double* part, double* out, int ngrid, cudaStream_t s) {
  // the counter lives right after the partials (4*ngrid doubles)
  unsigned int* counter = reinterpret_cast<unsigned int*>(part + 4 * ngrid);
  k_stats<T><<<ngrid, 256, 0, s>>>(pl.nx * pl.ny, p, g, S, use_set, part, counter, out);
}
template <typename T>
void launch_convert_in(const double* src, T* dst, size_t n, cudaStream_t s) {
  k_convert_in<T><<<ew_grid(n), 256, 0, s>>>(src, dst, n);
}
template <typename T>
void launch_convert_out(const T* src, double* dst, size_t n, cudaStream_t s) {
  k_convert_out<T><<<ew_grid(n), 256, 0, s>>>(src, dst, n);
}
template <typename T>
void launch_offset(const double* h64, double d, T* c, size_t n, cudaStream_t s) {
  k_offset<T><<<ew_grid(n), 256, 0, s>>>(h64, d, c, n);
}
template <typename T>
void launch_set_from_p(const T* p, uint8_t* S, size_t n, cudaStream_t s) {
  k_set_from_p<T><<<ew_grid(n), 256, 0, s>>>(p, S, n);
}
template <typename T>
void launch_mask_field(T* x, const uint8_t* S, size_t n, cudaStream_t s) {
  k_mask_field<T><<<ew_grid(n), 256, 0, s>>>(x, S, n);
}

#define BEM_INSTANTIATE_A(T)                                                                   \
  template void launch_pass_a<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pass_a_mi<T>(const PassArgs<T>&, int, const PassArgs<T>*, int, cudaStream_t); \
  template cudaError_t set_smem_attrs_a<T>(int);
#define BEM_INSTANTIATE_B(T)                                                                   \
  template void launch_pass_b<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pass_b_mi<T>(const PassArgs<T>&, const PassArgs<T>*, int, cudaStream_t); \
  template cudaError_t set_smem_attrs_b<T>(int);
#define BEM_INSTANTIATE_C(T)                                                                   \
  template void launch_pass_c<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pass_c_mi<T>(const PassArgs<T>&, int, const PassArgs<T>*, int, cudaStream_t); \
  template cudaError_t set_smem_attrs_c<T>(int);
#define BEM_INSTANTIATE_EW(T)                                                                  \
  template void launch_pk_init<T>(const Plan&, const double*, double, T*, T*, T*, int, int,    \
                                  cudaStream_t);                                               \
  template void launch_box_gather<T>(const T*, const T*, const uint8_t*, int, int, int, int, T*, T*, \
                                     uint8_t*, int, int, cudaStream_t);                         \
  template void launch_box_scatter<T>(const T*, T*, int, int, int, int, int, int, cudaStream_t); \
  template void launch_detach<T>(const Plan&, Fields<T>, double*, Scalars*, int, cudaStream_t); \
  template void launch_cg_finish<T>(const Plan&, Fields<T>, const Scalars*, int, cudaStream_t); \
  template void launch_stats<T>(const Plan&, const T*, const T*, const uint8_t*, int, double*, \
                                double*, int, cudaStream_t);                                   \
  template void launch_convert_in<T>(const double*, T*, size_t, cudaStream_t);                \
  template void launch_convert_out<T>(const T*, double*, size_t, cudaStream_t);               \
  template void launch_offset<T>(const double*, double, T*, size_t, cudaStream_t);            \
  template void launch_set_from_p<T>(const T*, uint8_t*, size_t, cudaStream_t);               \
  template void launch_mask_field<T>(T*, const uint8_t*, size_t, cudaStream_t);                \
  template void launch_batch_ctl<T>(const PassArgs<T>*, int, unsigned long long, cudaStream_t);

}  // namespace bem
