// The stress -> displacement transform u = A K*p (Eq. 13) as three passes
// over a zero-padded Px x Py torus, with the conjugate-gradient work fused
// into the first pass's prologue and the last pass's epilogue.
//
//   pass A  rows:    real row of Nx values (zero-padded to Px) -> half
//                    spectrum X[kx], kx = 0..Px/2, via one complex FFT of
//                    length Px/2 on (x[2n], x[2n+1]) and the standard split.
//                    Written transposed: W[kx][iy].
//   pass B  columns: for each kx, forward FFT of length Py of the Ny values
//                    (zero-padded), multiply by the real spectrum K^(ky, kx),
//                    inverse FFT, keep Ny values, in place in W.  Columns 0
//                    and Px/2 are real and ride together in one complex FFT.
//   pass C  rows:    complex-to-real inverse of length Px from the half
//                    spectrum, keep Nx values, scale by A/(Px Py), epilogue.
//
// Every kernel that belongs to a CG loop returns at once when the solve's
// `done` flag is set, so a captured chunk of iterations can run past
// convergence at the cost of empty launches.
#pragma once
#include "bem_impl.h"
#include "common.cuh"

namespace bem {

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < (T)0 ? -x : x; }

// Iterations without halving the best eps before a CG solve is declared stalled.
constexpr int kStall = 200;

// Sum per-CTA partials in a fixed order (deterministic); result in thread 0.
template <int NQ>
__device__ __forceinline__ void sum_partials(const double* part, int n, double (&v)[NQ], double* red) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += __ldcg(part + 4 * b + q);
  }
  block_sum<NQ>(v, red);
}

// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(1024) k_pass_a(PassArgs<T> a) {
  using Cx = C<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[3 * 32];
  Cx* buf = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != A_PLAIN && MODE != A_TORUS) {
    if (sc->done) return;
  }
  const int M = a.pl.M, logM = a.pl.logM, nb = a.pl.nbA;
  const int row0 = blockIdx.x * nb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ncols = a.ncols_in, nrows = a.nrows_in;
  const int half = (ncols + 1) >> 1;
  T acc0 = 0, acc1 = 0, acc2 = 0;
  bool upd = false;
  T tau = 0, beta = 0;
  if (MODE == A_PK_P) { upd = sc->have_tau != 0; tau = (T)sc->tau; }
  if (MODE == A_PK_T || MODE == A_CG_T) beta = (T)sc->beta;

  for (int idx = tid; idx < nb * M; idx += nthr) {
    const int b = idx >> logM, n = idx & (M - 1);
    const int row = row0 + b;
    T xv[2] = {0, 0};
    if (row < nrows && n < half) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = 2 * n + e;
        if (col >= ncols) continue;
        const size_t i = (size_t)row * ncols + col;
        T x = 0;
        if (MODE == A_PLAIN) {
          x = a.f.src[i];
        } else if (MODE == A_PK_P) {
          const T pv = a.f.p[i];
          T q = pv;
          if (upd) {
            if (pv > (T)0) {
              q = pv - tau * a.f.t[i];
              q = q > (T)0 ? q : (T)0;
            }
            const T gv = a.f.g[i];
            if (q == (T)0 && gv < (T)0) { q = -tau * gv; acc2 += (T)1; }
            acc0 += tabs(q - pv);
            a.f.p[i] = q;
          }
          acc1 += q;
          x = q;
        } else if (MODE == A_PK_T) {
          const T tv = a.f.p[i] > (T)0 ? a.f.g[i] + beta * a.f.t[i] : (T)0;
          a.f.t[i] = tv;
          x = tv;
        } else if (MODE == A_CG_T) {
          const T tv = a.f.S[i] ? a.f.g[i] + beta * a.f.t[i] : (T)0;
          a.f.t[i] = tv;
          x = tv;
        } else if (MODE == A_TORUS) {
          const int py = a.pl.py, px = a.pl.px;
          const int ry = row < py - row ? row : py - row;
          const int rx = col < px - col ? col : px - col;
          x = (T)a.kq64[(size_t)ry * (M + 1) + rx];
        }
        xv[e] = x;
      }
    }
    buf[(b << logM) + n] = mk<T>(xv[0], xv[1]);
  }
  __syncthreads();
  {
    const int per = M >> 3;
    const int b = tid / per, j0 = tid - b * per;
    fft_smem<T, -1>(buf + (b << logM), logM, j0);
  }
  if (MODE == A_PK_P) {
    double v[3] = {(double)acc0, (double)acc1, (double)acc2};
    block_sum<3>(v, red);
    if (tid == 0) {
      double* pp = a.partA + 4 * blockIdx.x;
      pp[0] = v[0]; pp[1] = v[1]; pp[2] = v[2];
    }
  }
  // split the packed transform into the half spectrum and store transposed
  const T invM = (T)1 / (T)M;
  Cx* W = reinterpret_cast<Cx*>(a.W);
  for (int idx = tid; idx < (M + 1) * nb; idx += nthr) {
    const int k = idx / nb, b = idx - k * nb;
    const int row = row0 + b;
    if (row >= nrows) continue;
    const Cx* s = buf + (b << logM);
    Cx X;
    if (k == 0 || k == M) {
      const Cx z0 = s[0];
      X = mk<T>(k == 0 ? z0.x + z0.y : z0.x - z0.y, (T)0);
    } else {
      const Cx zk = s[k], zm = conj<T>(s[M - k]);
      const Cx E = scale<T>(add<T>(zk, zm), (T)0.5);
      const Cx dlt = sub<T>(zk, zm);
      const Cx O = mk<T>((T)0.5 * dlt.y, (T)-0.5 * dlt.x);  // (zk - zm) / (2i)
      X = add<T>(E, mul<T>(expipi(-(T)k * invM), O));
    }
    W[(size_t)k * a.rows_w + row] = X;
  }
}

// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(1024) k_pass_b(PassArgs<T> a) {
  using Cx = C<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx* buf = reinterpret_cast<Cx*>(smem_raw);
  if (MODE == B_CONV && a.sc != nullptr) {
    if (a.sc->done) return;
  }
  const int Py = a.pl.py, logPy = a.pl.logPy, nb = a.pl.nbB, M = a.pl.M;
  const int rin = a.rows_w;
  const int col0 = blockIdx.x * nb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  Cx* W = reinterpret_cast<Cx*>(a.W);
  for (int idx = tid; idx < nb * Py; idx += nthr) {
    const int c = idx >> logPy, y = idx & (Py - 1);
    const int kx = col0 + c;
    Cx v = mk<T>(0, 0);
    if (kx < M && y < rin) {
      if (kx == 0) v = mk<T>(W[y].x, W[(size_t)M * rin + y].x);
      else v = W[(size_t)kx * rin + y];
    }
    buf[(c << logPy) + y] = v;
  }
  __syncthreads();
  const int per = Py >> 3;
  const int bseq = tid / per, j0 = tid - bseq * per;
  fft_smem<T, -1>(buf + (bseq << logPy), logPy, j0);
  const int hy = Py >> 1, hyq = hy + 1;
  if (MODE == B_SPECTRUM) {
    for (int idx = tid; idx < nb * hyq; idx += nthr) {
      const int c = idx / hyq, ky = idx - c * hyq;
      const int kx = col0 + c;
      if (kx >= M) continue;
      const Cx* s = buf + (c << logPy);
      const Cx v1 = s[ky], v2 = s[(Py - ky) & (Py - 1)];
      if (kx == 0) {
        const double re0 = 0.5 * ((double)v1.x + (double)v2.x);  // Re (v1 + conj v2)/2
        const double reM = 0.5 * ((double)v1.y + (double)v2.y);  // Re (v1 - conj v2)/(2i)
        a.khat64_out[ky] = re0;
        a.khat64_out[(size_t)M * hyq + ky] = reM;
        a.khat32_out[ky] = (float)re0;
        a.khat32_out[(size_t)M * hyq + ky] = (float)reM;
      } else {
        a.khat64_out[(size_t)kx * hyq + ky] = (double)v1.x;
        a.khat32_out[(size_t)kx * hyq + ky] = (float)v1.x;
      }
    }
    return;
  }
  // multiply by the real, even spectrum; pairs (ky, Py-ky) handled together
  for (int idx = tid; idx < nb * hyq; idx += nthr) {
    const int c = idx / hyq, ky = idx - c * hyq;
    const int kx = col0 + c;
    if (kx >= M) continue;
    Cx* s = buf + (c << logPy);
    const int ky2 = (Py - ky) & (Py - 1);
    if (kx == 0) {
      const Cx v1 = s[ky], v2 = s[ky2];
      const T k0 = a.khat[ky], kM = a.khat[(size_t)M * hyq + ky];
      // v = A + iB with A, B the spectra of columns 0 and M
      const Cx Av = scale<T>(add<T>(v1, conj<T>(v2)), (T)0.5);
      const Cx dd = sub<T>(v1, conj<T>(v2));
      const Cx Bv = mk<T>((T)0.5 * dd.y, (T)-0.5 * dd.x);
      const Cx n1 = add<T>(scale<T>(Av, k0), mul_si<T, 1>(scale<T>(Bv, kM)));
      const Cx n2 = add<T>(scale<T>(conj<T>(Av), k0), mul_si<T, 1>(scale<T>(conj<T>(Bv), kM)));
      s[ky] = n1;
      if (ky2 != ky) s[ky2] = n2;
    } else {
      const T kf = a.khat[(size_t)kx * hyq + ky];
      s[ky] = scale<T>(s[ky], kf);
      if (ky2 != ky) s[ky2] = scale<T>(s[ky2], kf);
    }
  }
  __syncthreads();
  fft_smem<T, 1>(buf + (bseq << logPy), logPy, j0);
  for (int idx = tid; idx < nb * rin; idx += nthr) {
    const int c = idx / rin, y = idx - c * rin;
    const int kx = col0 + c;
    if (kx >= M) continue;
    const Cx v = buf[(c << logPy) + y];
    if (kx == 0) {
      W[y] = mk<T>(v.x, (T)0);
      W[(size_t)M * rin + y] = mk<T>(v.y, (T)0);
    } else {
      W[(size_t)kx * rin + y] = v;
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(1024) k_pass_c(PassArgs<T> a) {
  using Cx = C<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[3 * 32];
  __shared__ int lastflag;
  Cx* buf = reinterpret_cast<Cx*>(smem_raw);
  Scalars* sc = a.sc;
  if (MODE != C_PLAIN && MODE != C_GAP) {
    if (sc->done) return;
  }
  const int M = a.pl.M, logM = a.pl.logM, nb = a.pl.nbA, ld = M + 1;
  const int nx = a.pl.nx, ny = a.pl.ny;
  const int row0 = blockIdx.x * nb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const Cx* W = reinterpret_cast<const Cx*>(a.W);
  for (int idx = tid; idx < (M + 1) * nb; idx += nthr) {
    const int k = idx / nb, b = idx - k * nb;
    const int row = row0 + b;
    buf[b * ld + k] = row < ny ? W[(size_t)k * a.rows_w + row] : mk<T>(0, 0);
  }
  __syncthreads();
  // rebuild the packed half-length spectrum: Z[k] = E + i O with
  // E = X[k] + conj X[M-k],  O = (X[k] - conj X[M-k]) exp(+2 pi i k / Px)
  const T invM = (T)1 / (T)M;
  const int hm = (M >> 1) + 1;
  for (int idx = tid; idx < nb * hm; idx += nthr) {
    const int b = idx / hm, k = idx - b * hm;
    Cx* s = buf + b * ld;
    const Cx xk = s[k], xm = s[M - k];
    const Cx wk = expipi((T)k * invM);
    {
      const Cx E = add<T>(xk, conj<T>(xm));
      const Cx O = mul<T>(sub<T>(xk, conj<T>(xm)), wk);
      s[k] = add<T>(E, mul_si<T, 1>(O));
    }
    if (k != 0 && k != M - k) {
      const Cx wm = mk<T>(-wk.x, wk.y);  // exp(+2 pi i (M-k)/Px) = -conj(wk)
      const Cx E = add<T>(xm, conj<T>(xk));
      const Cx O = mul<T>(sub<T>(xm, conj<T>(xk)), wm);
      s[M - k] = add<T>(E, mul_si<T, 1>(O));
    }
  }
  __syncthreads();
  {
    const int per = M >> 3;
    const int b = tid / per, j0 = tid - b * per;
    fft_smem<T, 1>(buf + b * ld, logM, j0);
  }
  const T us = (T)a.uscale;
  T acc0 = 0, acc1 = 0;
  T beta_unused = 0;
  (void)beta_unused;
  for (int idx = tid; idx < nb * M; idx += nthr) {
    const int b = idx >> logM, n = idx & (M - 1);
    const int row = row0 + b;
    if (row >= ny) continue;
    const Cx z = buf[b * ld + n];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = 2 * n + e;
      if (col >= nx) continue;
      const size_t i = (size_t)row * nx + col;
      const T u = us * (e ? z.y : z.x);
      if (MODE == C_PLAIN) {
        a.f.dst[i] = u;
      } else if (MODE == C_PK_G) {
        const T gv = u + a.f.c[i];
        a.f.g[i] = gv;
        if (a.f.p[i] > (T)0) { acc0 += gv * gv; acc1 += (T)1; }
      } else if (MODE == C_PK_R) {
        if (a.f.p[i] > (T)0) {
          const T tv = a.f.t[i];
          acc0 += a.f.g[i] * tv;
          acc1 += u * tv;
        }
      } else if (MODE == C_CG_R) {
        const T rv = a.f.S[i] ? u : (T)0;
        a.f.r[i] = rv;
        acc0 += rv * a.f.t[i];
      } else if (MODE == C_CG_G) {
        if (a.f.S[i]) {
          const T cv = a.f.c[i];
          const T gv = u + cv;
          a.f.g[i] = gv;
          acc0 += gv * gv;
          acc1 += cv * cv;
        } else {
          a.f.g[i] = (T)0;
        }
      } else if (MODE == C_GAP) {
        a.f.g[i] = u + a.f.c[i];
      }
    }
  }
  if (MODE == C_PLAIN || MODE == C_GAP) return;
  double v[2] = {(double)acc0, (double)acc1};
  block_sum<2>(v, red);
  if (tid == 0) {
    double* pp = a.partC + 4 * blockIdx.x;
    pp[0] = v[0]; pp[1] = v[1];
  }
  if (!last_block_arrival(MODE == C_PK_G ? &sc->cnt_c : &sc->cnt_a, &lastflag)) return;
  double s2[2];
  sum_partials<2>(a.partC, gridDim.x, s2, red);
  double s3[3] = {0, 0, 0};
  if (MODE == C_PK_G) sum_partials<3>(a.partA, gridDim.x, s3, red);
  if (tid != 0) return;
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
    else { sc->tau = sgt / srt; sc->have_tau = 1; }
  } else if (MODE == C_CG_R) {
    sc->cnt_a = 0;
    const double str = s2[0];
    sc->str = str;
    if (!isfinite(str)) { sc->status = SC_NUMERIC; sc->done = 1; }
    else if (str <= 0.0) { sc->done = 1; }
    else sc->tau = sc->G / str;
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
    if (!isfinite(G)) { sc->status = SC_NUMERIC; sc->done = 1; }
    else if (sqrt(G) <= sc->tol * bn) sc->done = 1;
  }
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

template <typename T>
__global__ void k_cg_update(int n, Fields<T> f, double* part, Scalars* sc) {
  __shared__ double red[3 * 32];
  __shared__ int lastflag;
  if (sc->done) return;
  const T tau = (T)sc->tau;
  T acc = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T tv = f.t[i], rv = f.r[i];
    f.p[i] -= tau * tv;
    const T gv = f.g[i] - tau * rv;
    f.g[i] = gv;
    acc += gv * gv;
  }
  double v[1] = {(double)acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[4 * blockIdx.x] = v[0];
  if (!last_block_arrival(&sc->cnt_e, &lastflag)) return;
  double s[1];
  sum_partials<1>(part, gridDim.x, s, red);
  if (threadIdx.x != 0) return;
  sc->cnt_e = 0;
  const double Gn = s[0];
  sc->iter += 1;
  sc->eps = sqrt(Gn) / sc->bnorm;
  if (!isfinite(Gn)) { sc->status = SC_NUMERIC; sc->done = 1; return; }
  if (sqrt(Gn) <= sc->tol * sc->bnorm) sc->done = 1;
  else if (sc->iter >= sc->max_iter) { sc->status = SC_NOCONV; sc->done = 1; }
  sc->beta = Gn / sc->G;
  sc->G = Gn;
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
  sum_partials<2>(part, gridDim.x, s, red);
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
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, x1 = 0, x2 = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      s0 += __ldcg(part + 4 * b); s1 += __ldcg(part + 4 * b + 1);
      x1 = fmax(x1, __ldcg(part + 4 * b + 2)); x2 = fmax(x2, __ldcg(part + 4 * b + 3));
    }
    out[0] = s0; out[1] = s1; out[2] = x1; out[3] = x2;
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
// Host launchers

template <typename T>
void launch_pass_a(const PassArgs<T>& a, int mode, cudaStream_t s) {
  const dim3 grid((a.nrows_in + a.pl.nbA - 1) / a.pl.nbA), block(a.pl.threadsA);
  switch (mode) {
    case A_PLAIN: k_pass_a<T, A_PLAIN><<<grid, block, a.pl.smemA, s>>>(a); break;
    case A_PK_P: k_pass_a<T, A_PK_P><<<grid, block, a.pl.smemA, s>>>(a); break;
    case A_PK_T: k_pass_a<T, A_PK_T><<<grid, block, a.pl.smemA, s>>>(a); break;
    case A_CG_T: k_pass_a<T, A_CG_T><<<grid, block, a.pl.smemA, s>>>(a); break;
    case A_TORUS:
      if constexpr (sizeof(T) == 8) k_pass_a<T, A_TORUS><<<grid, block, a.pl.smemA, s>>>(a);
      break;
  }
}

template <typename T>
void launch_pass_b(const PassArgs<T>& a, int mode, cudaStream_t s) {
  const dim3 grid(a.pl.gridB), block(a.pl.threadsB);
  if (mode == B_SPECTRUM) k_pass_b<T, B_SPECTRUM><<<grid, block, a.pl.smemB, s>>>(a);
  else k_pass_b<T, B_CONV><<<grid, block, a.pl.smemB, s>>>(a);
}

template <typename T>
void launch_pass_c(const PassArgs<T>& a, int mode, cudaStream_t s) {
  const dim3 grid(a.pl.gridA), block(a.pl.threadsA);
  switch (mode) {
    case C_PLAIN: k_pass_c<T, C_PLAIN><<<grid, block, a.pl.smemC, s>>>(a); break;
    case C_PK_G: k_pass_c<T, C_PK_G><<<grid, block, a.pl.smemC, s>>>(a); break;
    case C_PK_R: k_pass_c<T, C_PK_R><<<grid, block, a.pl.smemC, s>>>(a); break;
    case C_CG_R: k_pass_c<T, C_CG_R><<<grid, block, a.pl.smemC, s>>>(a); break;
    case C_CG_G: k_pass_c<T, C_CG_G><<<grid, block, a.pl.smemC, s>>>(a); break;
    case C_GAP: k_pass_c<T, C_GAP><<<grid, block, a.pl.smemC, s>>>(a); break;
  }
}

// Opt every pass kernel into `bytes` of dynamic shared memory (the static
// reduction scratch counts against the same 227 KB per block, so the request
// is sized to what the plans need).  Returns the first failure.
template <typename T>
cudaError_t set_smem_attrs(int bytes) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess, r;
#define BEM_ATTR(fn) if ((r = cudaFuncSetAttribute(fn, at, bytes)) != cudaSuccess && e == cudaSuccess) e = r
  BEM_ATTR((k_pass_a<T, A_PLAIN>));
  BEM_ATTR((k_pass_a<T, A_PK_P>));
  BEM_ATTR((k_pass_a<T, A_PK_T>));
  BEM_ATTR((k_pass_a<T, A_CG_T>));
  if constexpr (sizeof(T) == 8) BEM_ATTR((k_pass_a<T, A_TORUS>));
  BEM_ATTR((k_pass_b<T, B_CONV>));
  BEM_ATTR((k_pass_b<T, B_SPECTRUM>));
  BEM_ATTR((k_pass_c<T, C_PLAIN>));
  BEM_ATTR((k_pass_c<T, C_PK_G>));
  BEM_ATTR((k_pass_c<T, C_PK_R>));
  BEM_ATTR((k_pass_c<T, C_CG_R>));
  BEM_ATTR((k_pass_c<T, C_CG_G>));
  BEM_ATTR((k_pass_c<T, C_GAP>));
#undef BEM_ATTR
  return e;
}

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
void launch_cg_update(const Plan& pl, Fields<T> f, double* part, Scalars* sc, int ngrid,
                      cudaStream_t s) {
  k_cg_update<T><<<ngrid, 256, 0, s>>>(pl.nx * pl.ny, f, part, sc);
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

#define BEM_INSTANTIATE(T)                                                                     \
  template void launch_pass_a<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pass_b<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pass_c<T>(const PassArgs<T>&, int, cudaStream_t);                      \
  template void launch_pk_init<T>(const Plan&, const double*, double, T*, T*, T*, int, int,    \
                                  cudaStream_t);                                               \
  template void launch_cg_update<T>(const Plan&, Fields<T>, double*, Scalars*, int,            \
                                    cudaStream_t);                                             \
  template void launch_detach<T>(const Plan&, Fields<T>, double*, Scalars*, int, cudaStream_t); \
  template void launch_stats<T>(const Plan&, const T*, const T*, const uint8_t*, int, double*, \
                                double*, int, cudaStream_t);                                   \
  template void launch_convert_in<T>(const double*, T*, size_t, cudaStream_t);                \
  template void launch_convert_out<T>(const T*, double*, size_t, cudaStream_t);               \
  template void launch_offset<T>(const double*, double, T*, size_t, cudaStream_t);            \
  template void launch_set_from_p<T>(const T*, uint8_t*, size_t, cudaStream_t);               \
  template void launch_mask_field<T>(T*, const uint8_t*, size_t, cudaStream_t);

}  // namespace bem
