/*
 * Oracle numerics in plain C (FP64).  TEST INFRASTRUCTURE ONLY: nothing on the
 * product path may link, load or call this file.  It shares no code with the
 * CUDA library; the two are built separately and compared in tests.
 *
 * What lives here, each written from its definition and nothing more:
 *   - oracle_K_table: influence coefficients K(di,dj) of Eq. 9 (the integrand
 *     of Eqs. 6/8 with the squares that Eq. 9 restores), by a global adaptive
 *     2D cubature over the element, split at the axes so that the integrable
 *     r^-(1+k) singularity only ever sits at a corner of a sub-rectangle.
 *   - oracle_c1_quad: the dimensionless coefficient c1(k) of Eq. 23 (uncorrected),
 *     using the exact reduction of the 4-fold integral over two unit squares
 *     to 4*int_0^1 int_0^1 (1-u)(1-v)(u^2+v^2)^-(1+k)/2 du dv (the difference of
 *     two independent uniform variables on [0,1] has the triangle density 1-|s|).
 *   - oracle_direct_conv / oracle_direct_conv_at: the matrix product of Eq. 7/12,
 *     u_ij = sum_{i'j'} K(i-i', j-j') p_i'j', summed directly, O(N^4).
 *
 * The cubature: tensor Gauss-Legendre rules of 8 and 16 points per axis (nodes
 * by Newton iteration on the Legendre recurrence); the 16x16 value is kept and
 * |Q16 - Q8| is its error estimate; the region with the largest estimate is
 * split into four until the summed estimate meets the tolerance.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NG_LO 8
#define NG_HI 16

static double gl_x_lo[NG_LO], gl_w_lo[NG_LO], gl_x_hi[NG_HI], gl_w_hi[NG_HI];
static int gl_ready = 0;

/* Gauss-Legendre nodes/weights on [-1,1]: Newton on P_n(x) = 0, with P_n
 * from the three-term recurrence j P_j = (2j-1) x P_{j-1} - (j-1) P_{j-2}. */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; i++) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; j++) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      dp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void gl_init(void) {
  if (gl_ready) return;
  gauss_legendre(NG_LO, gl_x_lo, gl_w_lo);
  gauss_legendre(NG_HI, gl_x_hi, gl_w_hi);
  gl_ready = 1;
}

/* integrand: (a^2+b^2)^(-(1+k)/2), optionally times (1-a)(1-b) for c1 */
typedef struct {
  double expo;   /* -(1+k)/2 */
  int triangle;  /* multiply by (1-a)(1-b) */
} integrand_t;

static inline double f_eval(const integrand_t *f, double a, double b) {
  double v = pow(a * a + b * b, f->expo);
  if (f->triangle) v *= (1.0 - a) * (1.0 - b);
  return v;
}

typedef struct {
  double a0, a1, b0, b1, val, err;
} region_t;

static void rule(const integrand_t *f, region_t *r) {
  double ca = 0.5 * (r->a0 + r->a1), ha = 0.5 * (r->a1 - r->a0);
  double cb = 0.5 * (r->b0 + r->b1), hb = 0.5 * (r->b1 - r->b0);
  double qh = 0.0, ql = 0.0;
  for (int i = 0; i < NG_HI; i++) {
    double a = ca + ha * gl_x_hi[i], s = 0.0;
    for (int j = 0; j < NG_HI; j++) s += gl_w_hi[j] * f_eval(f, a, cb + hb * gl_x_hi[j]);
    qh += gl_w_hi[i] * s;
  }
  for (int i = 0; i < NG_LO; i++) {
    double a = ca + ha * gl_x_lo[i], s = 0.0;
    for (int j = 0; j < NG_LO; j++) s += gl_w_lo[j] * f_eval(f, a, cb + hb * gl_x_lo[j]);
    ql += gl_w_lo[i] * s;
  }
  r->val = qh * ha * hb;
  r->err = fabs(qh - ql) * ha * hb;
}

/* binary max-heap on err */
typedef struct {
  region_t *v;
  int n, cap;
} heap_t;

static int heap_push(heap_t *h, region_t r) {
  if (h->n == h->cap) {
    int nc = h->cap ? 2 * h->cap : 64;
    region_t *nv = (region_t *)realloc(h->v, (size_t)nc * sizeof(region_t));
    if (!nv) return -1;
    h->v = nv;
    h->cap = nc;
  }
  int i = h->n++;
  h->v[i] = r;
  while (i > 0) {
    int p = (i - 1) / 2;
    if (h->v[p].err >= h->v[i].err) break;
    region_t t = h->v[p];
    h->v[p] = h->v[i];
    h->v[i] = t;
    i = p;
  }
  return 0;
}

static region_t heap_pop(heap_t *h) {
  region_t top = h->v[0];
  h->v[0] = h->v[--h->n];
  int i = 0;
  for (;;) {
    int l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && h->v[l].err > h->v[m].err) m = l;
    if (r < h->n && h->v[r].err > h->v[m].err) m = r;
    if (m == i) break;
    region_t t = h->v[m];
    h->v[m] = h->v[i];
    h->v[i] = t;
    i = m;
  }
  return top;
}

/* Global adaptive cubature over a list of starting rectangles.  Returns the
 * integral; *err_out gets the summed error estimate; returns NAN on failure. */
static double cubature(const integrand_t *f, const region_t *start, int nstart, double rel_tol,
                       double abs_tol, int max_regions, double *err_out) {
  heap_t h = {0, 0, 0};
  double val = 0.0, err = 0.0;
  for (int i = 0; i < nstart; i++) {
    region_t r = start[i];
    if (r.a1 <= r.a0 || r.b1 <= r.b0) continue;
    rule(f, &r);
    val += r.val;
    err += r.err;
    if (heap_push(&h, r)) { free(h.v); return NAN; }
  }
  int count = h.n;
  while (h.n > 0 && err > fmax(abs_tol, rel_tol * fabs(val)) && count < max_regions) {
    region_t r = heap_pop(&h);
    val -= r.val;
    err -= r.err;
    double am = 0.5 * (r.a0 + r.a1), bm = 0.5 * (r.b0 + r.b1);
    region_t c[4] = {{r.a0, am, r.b0, bm, 0, 0}, {am, r.a1, r.b0, bm, 0, 0},
                     {r.a0, am, bm, r.b1, 0, 0}, {am, r.a1, bm, r.b1, 0, 0}};
    for (int i = 0; i < 4; i++) {
      rule(f, &c[i]);
      val += c[i].val;
      err += c[i].err;
      if (heap_push(&h, c[i])) { free(h.v); return NAN; }
    }
    count += 4;
  }
  /* re-sum the kept regions to shed the rounding of the running updates */
  double v2 = 0.0, e2 = 0.0;
  for (int i = 0; i < h.n; i++) { v2 += h.v[i].val; e2 += h.v[i].err; }
  free(h.v);
  if (err_out) *err_out = e2;
  return v2;
}

/* split [lo,hi] at 0 when it straddles it; returns number of pieces (1 or 2) */
static int split_at_zero(double lo, double hi, double *pl, double *ph) {
  if (lo < 0.0 && hi > 0.0) {
    pl[0] = lo; ph[0] = 0.0;
    pl[1] = 0.0; ph[1] = hi;
    return 2;
  }
  pl[0] = lo; ph[0] = hi;
  return 1;
}

/* K over a<-[a0,a1], b<-[b0,b1] of (a^2+b^2)^(-(1+k)/2) (Eq. 9). */
double oracle_K_rect(double k, double a0, double a1, double b0, double b1, double rel_tol,
                     double *err_out) {
  gl_init();
  integrand_t f = {-0.5 * (1.0 + k), 0};
  double al[2], ah[2], bl[2], bh[2];
  int na = split_at_zero(a0, a1, al, ah), nb = split_at_zero(b0, b1, bl, bh);
  region_t st[4];
  int ns = 0;
  for (int i = 0; i < na; i++)
    for (int j = 0; j < nb; j++) {
      region_t r = {al[i], ah[i], bl[j], bh[j], 0, 0};
      st[ns++] = r;
    }
  return cubature(&f, st, ns, rel_tol, 0.0, 400000, err_out);
}

/* Influence table: out[dj*nx + di] = K(di, dj) for 0<=di<nx, 0<=dj<ny, element
 * sizes dx, dy: the integral over a in [(di-1/2)dx,(di+1/2)dx],
 * b in [(dj-1/2)dy,(dj+1/2)dy] (Eq. 9, limits p,q,m,n).  Returns 0 or -1. */
int oracle_K_table(double k, double dx, double dy, int nx, int ny, double rel_tol, double *out) {
  gl_init();
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (long idx = 0; idx < (long)nx * ny; idx++) {
    int di = (int)(idx % nx), dj = (int)(idx / nx);
    double v = oracle_K_rect(k, (di - 0.5) * dx, (di + 0.5) * dx, (dj - 0.5) * dy, (dj + 0.5) * dy,
                             rel_tol, NULL);
    if (!(v == v)) bad = 1;
    out[idx] = v;
  }
  return bad ? -1 : 0;
}

/* Uncorrected c1(k) of Eq. 23 via the triangle-density reduction. */
double oracle_c1_quad(double k, double rel_tol, double *err_out) {
  gl_init();
  integrand_t f = {-0.5 * (1.0 + k), 1};
  region_t st[1] = {{0.0, 1.0, 0.0, 1.0, 0, 0}};
  double e = 0.0;
  double v = cubature(&f, st, 1, rel_tol, 0.0, 400000, &e);
  if (err_out) *err_out = 4.0 * e;
  return 4.0 * v;
}

/* Direct sum of Eq. 7: u[iy*nx+ix] = sum_{jy,jx} Kq[|iy-jy|*kstride + |ix-jx|] p[jy*nx+jx].
 * Kq holds K(di,dj) for 0<=di<nx, 0<=dj<ny at Kq[dj*kstride+di]. */
void oracle_direct_conv(int nx, int ny, const double *Kq, int kstride, const double *p, double *u) {
#pragma omp parallel for schedule(static)
  for (long o = 0; o < (long)nx * ny; o++) {
    int iy = (int)(o / nx), ix = (int)(o % nx);
    double s = 0.0;
    for (int jy = 0; jy < ny; jy++) {
      const double *krow = Kq + (size_t)abs(iy - jy) * kstride;
      const double *prow = p + (size_t)jy * nx;
      for (int jx = 0; jx < nx; jx++) s += krow[abs(ix - jx)] * prow[jx];
    }
    u[o] = s;
  }
}

/* Same sum at npts selected output indices (flat iy*nx+ix). */
void oracle_direct_conv_at(int nx, int ny, const double *Kq, int kstride, const double *p,
                           int npts, const long *pts, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < npts; q++) {
    int iy = (int)(pts[q] / nx), ix = (int)(pts[q] % nx);
    double s = 0.0;
    for (int jy = 0; jy < ny; jy++) {
      const double *krow = Kq + (size_t)abs(iy - jy) * kstride;
      const double *prow = p + (size_t)jy * nx;
      for (int jx = 0; jx < nx; jx++) s += krow[abs(ix - jx)] * prow[jx];
    }
    out[q] = s;
  }
}
