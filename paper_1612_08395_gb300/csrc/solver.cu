// Host orchestration of the solver: handle set-up (influence table and
// spectrum), the constrained and fixed-set conjugate-gradient loops as chunks
// of captured CUDA graphs, the adhesive detach loop, the FP64 refinement
// sweep, load-unload sweeps, and the C ABI of include/bem.h.
#include <math.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <vector>
#include <string>

#include <cuda.h>  // CUtensorMap (the encoder comes from the driver entry point)

#include "bem.h"
#include "bem_impl.h"
#include "geo_table.h"

namespace bem {
template <typename T> cudaError_t set_smem_attrs_a(int bytes);
template <typename T> cudaError_t set_smem_attrs_b(int bytes);
template <typename T> cudaError_t set_smem_attrs_c(int bytes);

Geo make_geo(int logL, int rows, int esize) {
  const GeoRow& r = (esize == 4 ? kGeo8 : kGeo16)[logL - 3];
  int lr = 0;
  while ((1 << lr) < rows) ++lr;
  if (lr > 6) lr = 6;
  Geo g{};
  g.logL = logL;
  g.r0 = logL % 3;
  g.sa = r.a; g.sb = r.b; g.sc = r.c; g.sd = r.d;
  g.rs = (1 << logL) + (rows > 1 ? r.pad[lr] : 0);
  return g;
}
}

using namespace bem;

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA, "%s: %s (%s:%d)",   \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
  } while (0)

#define CKR(call)                  \
  do {                             \
    int r_ = (call);               \
    if (r_ != BEM_OK) return r_;   \
  } while (0)

namespace {

// CTAs per SM of the grid-stride elementwise kernels (CG update, statistics, detach)
#ifndef BEM_EW_CTAS_PER_SM
#define BEM_EW_CTAS_PER_SM 2
#endif
#ifndef BEM_CHUNK
#define BEM_CHUNK 8
#endif
constexpr int kChunk = BEM_CHUNK;  // CG iterations per captured graph launch
// CG iterations per body of the while-loop graph of batched loops
#ifndef BEM_LOOP_BODY
#define BEM_LOOP_BODY 4
#endif
constexpr int kLoopBody = BEM_LOOP_BODY;

// Threads per CTA of the row passes (rows per CTA x M/8); 512 keeps two CTAs
// resident per SM at the passes' register use.
#ifndef BEM_MAX_THREADS_A
#define BEM_MAX_THREADS_A 512
#endif

template <typename T> struct PrecFields {
  T *p = nullptr, *g = nullptr, *t = nullptr, *r = nullptr, *c = nullptr;
  bool ready = false;
  cudaGraphExec_t pk_graph[2] = {nullptr, nullptr}, cg_graph[2] = {nullptr, nullptr};  // [timed]
};

int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }
int pow2_at_least(int v) { int p = 1; while (p < v) p <<= 1; return p; }

// Small grids: fewer rows (columns) per CTA until a pass has about two CTAs
// per SM, keeping at least two warps per CTA -- otherwise a 128^2 grid runs
// its passes on a handful of SMs and every CG iteration is latency-bound.
constexpr int kMinThreads = 64;
constexpr int kCtasPerSm = 2;

// The plan for given rows per CTA of the row passes (nbA), columns per CTA of
// the column pass (nbB) and radix of the column pass's stages (8 or 16).
Plan plan_with(int nx, int ny, int px, int py, int esize, int nsm, int nbA, int nbB, int radixB = 8) {
  Plan pl{};
  pl.nx = nx; pl.ny = ny; pl.px = px; pl.py = py;
  pl.M = px / 2;
  const int logM = ilog2(pl.M), logPy = ilog2(py);
  pl.nbA = nbA;
  pl.lognbA = ilog2(nbA);
  pl.gA = make_geo(logM, nbA, esize);
  pl.threadsA = nbA * (pl.M / 8);
  pl.gridA = (ny + nbA - 1) / nbA;
  pl.smemA = (size_t)nbA * pl.gA.rs * 2 * esize;
  pl.smemC = pl.smemA;
  pl.nbB = nbB;
  pl.radixB = radixB;
  pl.gB = make_geo(logPy, nbB, esize);
  pl.threadsB = nbB * (py / radixB);
  pl.gridB = (pl.M + 1 + nbB - 1) / nbB;
  // the radix-16 pass needs no row pad (its swizzle spreads every access)
  pl.smemB = (size_t)nbB * (radixB == 16 ? py : pl.gB.rs) * 2 * esize;
  pl.nsm = nsm;
  return pl;
}

// Whether a plan's shapes are launchable: whole warps, the kernels' launch
// bounds, and shared memory (with the persistent passes' staging) in budget.
bool shape_fits(const Plan& pl, int esize) {
  const int logM = ilog2(pl.M), logPy = ilog2(pl.py);
  const int capA = logM >= 13 ? 1024 : 512;
  const int capB = pl.radixB == 16 ? BEM_COL16_MAX_THREADS(logPy) : logPy >= 13 ? 1024 : 512;
  if (pl.nbA < 1 || pl.nbA > 64 || pl.nbB < 1 || pl.nbB > 64) return false;
  if (pl.threadsA < 64 || pl.threadsA > capA || (pl.threadsA & 31)) return false;
  if (pl.threadsB < 64 || pl.threadsB > capB || (pl.threadsB & 31)) return false;
  // radix-16 column pass: FP32, 512 to 8192 points (whole warps per column)
  if (pl.radixB != 8 && (pl.radixB != 16 || esize != 4 || logPy < 9 || logPy > 13)) return false;
  const size_t lim = 200 * 1024, rows = (size_t)pl.nbA * pl.nx;
  if (pl.smemA + (4 * (size_t)esize + 1) * rows + 16 > lim) return false;
  if (pass_c_smem(pl.smemC, pl.M, pl.nbA, 2 * esize, (2 * (size_t)esize + 1) * rows) + 32 > lim) return false;
  if (pl.smemB > lim) return false;
  return true;
}

// Columns per CTA of the column pass: about 256 threads per CTA, and for small
// grids about two CTAs per SM.
int default_cols_b(int M, int py, int esize, int nsm, int radix) {
  const int tb = py / radix;
  int nbb = 256 / tb;
  if (nbb < 1) nbb = 1;
  while (nbb > 1 && (size_t)nbb * (py + 32) * 2 * esize > 128 * 1024) nbb >>= 1;
  while (nbb > 1 && (nbb / 2) * tb >= kMinThreads && (M + nbb) / nbb < kCtasPerSm * nsm) nbb >>= 1;
  return nbb;
}

// Radix of the column pass before tuning: radix-8 stages, or the radix-16
// pass where BEM_RADIX_B=16 asks for it and it applies (FP32, 512 to 8192
// points); the FP32 autotuner chooses between them per grid size.
int forced_radix_b() {
  const char* env = getenv("BEM_RADIX_B");
  const int r = env ? atoi(env) : 0;
  return r == 8 || r == 16 ? r : 0;
}
int default_radix_b(int py, int esize) {
  const int logPy = ilog2(py);
  if (forced_radix_b() == 16 && esize == 4 && logPy >= 9 && logPy <= 13) return 16;
  return 8;
}

// Default shapes: about 256 threads per CTA, rows of W written in 32-byte
// segments, and for small grids about two CTAs per SM.
Plan make_plan(int nx, int ny, int px, int py, int esize, int nsm) {
  const int M = px / 2;
  const int tr = M / 8;
  int nb = 256 / tr;
  const int sector = 32 / (2 * esize);  // rows per CTA for 32-byte segments of W
  if (nb < sector) nb = sector;
  if (nb < 1) nb = 1;
  while (nb > 1 && nb * tr > BEM_MAX_THREADS_A) nb >>= 1;
  while (nb > 1 && (size_t)nb * (M + 32) * 2 * esize > 128 * 1024) nb >>= 1;
  while (nb > 1 && (nb / 2) * tr >= kMinThreads && (ny + nb - 1) / nb < kCtasPerSm * nsm) nb >>= 1;
  const int radix = default_radix_b(py, esize);
  return plan_with(nx, ny, px, py, esize, nsm, nb, default_cols_b(M, py, esize, nsm, radix), radix);
}

}  // namespace

namespace bem {
Plan default_plan(int nx, int ny, int px, int py, int esize, int nsm) {
  return make_plan(nx, ny, px, py, esize, nsm);
}
bool plan_fits(const Plan& pl, int esize) { return shape_fits(pl, esize); }

// Once per device and process, with that device current: opt every pass kernel
// into the shared memory it may ask for, and upload the quadrature nodes.
int device_setup(int dev) {
  static std::mutex init_mu;
  static bool init_done[64] = {};
  std::lock_guard<std::mutex> lk(init_mu);
  if (dev < 0 || dev >= 64) return fail(BEM_ECUDA, "device index %d unsupported", dev);
  if (init_done[dev]) return BEM_OK;
  const int smem_max = 227 * 1024;
  cudaError_t ea = set_smem_attrs_a<float>(smem_max);
  if (ea == cudaSuccess) ea = set_smem_attrs_b<float>(smem_max);
  if (ea == cudaSuccess) ea = set_smem_attrs_c<float>(smem_max);
  if (ea == cudaSuccess) ea = set_smem_attrs_a<double>(smem_max);
  if (ea == cudaSuccess) ea = set_smem_attrs_b<double>(smem_max);
  if (ea == cudaSuccess) ea = set_smem_attrs_c<double>(smem_max);
  if (ea != cudaSuccess) return fail(BEM_ECUDA, "shared-memory opt-in failed: %s", cudaGetErrorString(ea));
  if (influence_init_nodes() != 0) return fail(BEM_ECUDA, "quadrature nodes upload failed");
  const int rc = tc_column_pass_setup();
  if (rc != BEM_OK) return rc;
  init_done[dev] = true;
  return BEM_OK;
}
}  // namespace bem

struct bem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Plan plan32{}, plan64{};
  int nx = 0, ny = 0, px = 0, py = 0;
  double dx = 0, dy = 0, k = 0, nu = 0, E0 = 0, c0 = 0, alpha = 0, A = 0;
  double* kq64 = nullptr;
  int* geo = nullptr;       // index tables: [A32 | B32 | A64 | B64], each so (112) + sp (L)
  double2* tw64 = nullptr;  // [length-M stages | length-Py stages | split], FP64
  float2* tw32 = nullptr;   // the same, FP32
  double* khat64 = nullptr;
  float* khat32 = nullptr;
  void* W = nullptr;
  double* h64 = nullptr;    // profile
  double* io64 = nullptr;   // FP64 staging / FP64 pressure of the refinement
  double* io64b = nullptr;  // second FP64 staging
  uint8_t* S = nullptr;
  double* part = nullptr;   // per-CTA partials (A)
  double* partC = nullptr;  // per-CTA partials (C)
  double* partE = nullptr;  // per-CTA partials (elementwise kernels)
  double* stats = nullptr;  // 4 doubles + stats partials
  int stats_ngrid = 0;
  int ew_ngrid = 0;
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned
  double* stats_host = nullptr;  // pinned
  PrecFields<float> f32;
  PrecFields<double> f64;
  size_t bytes = 0;
  unsigned long long launches = 0;
  bool timing = false;          // BEM_FLAG_TIME_PASSES for the current call
  cudaEvent_t ev[2][4] = {};    // [pk/cg][A start, B start, C start, C end]
  double pass_ms[3] = {0, 0, 0};
  long long pass_count[2] = {0, 0};
  double pass_bytes[3] = {0, 0, 0};  // algorithmic bytes / flops of the timed launches
  double pass_flops[3] = {0, 0, 0};
  // Contact-box sub-contexts (smaller tori for fixed-set solves whose contact
  // set fits a box of at most half their size); they share the parent's stream.
  bool is_sub = false, own_stream = true;
  std::vector<bem_ctx*> subs;
  // CG loops join this batcher when set (concurrent solves of the server)
  bem::LoopBatcher* batcher = nullptr;
  cudaEvent_t ev_ready = nullptr;  // this context's work before its batched loop
  // Tensor maps of W for pass C's TMA staging, [FP32, FP64] views with the
  // plan's rows per CTA (device memory; null where TMA does not apply)
  void* tmw[2] = {nullptr, nullptr};
  bool tmw_ok[2] = {false, false};
};

static int create_ctx(int Nx, int Ny, double dx, double dy, double k, double nu, double E0, double c0,
                      bem_ctx* parent, bem_ctx** out);

namespace {

template <typename T> PrecFields<T>& fields_of(bem_ctx* h);
template <> PrecFields<float>& fields_of<float>(bem_ctx* h) { return h->f32; }
template <> PrecFields<double>& fields_of<double>(bem_ctx* h) { return h->f64; }
template <typename T> const Plan& plan_of(bem_ctx* h);
template <> const Plan& plan_of<float>(bem_ctx* h) { return h->plan32; }
template <> const Plan& plan_of<double>(bem_ctx* h) { return h->plan64; }
template <typename T> const T* khat_of(bem_ctx* h);
template <> const float* khat_of<float>(bem_ctx* h) { return h->khat32; }
template <> const double* khat_of<double>(bem_ctx* h) { return h->khat64; }

int dmalloc(bem_ctx* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(BEM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  h->bytes += bytes;
  return BEM_OK;
}

template <typename T>
int ensure_fields(bem_ctx* h) {
  PrecFields<T>& f = fields_of<T>(h);
  if (f.ready) return BEM_OK;
  const size_t n = (size_t)h->nx * h->ny;
  CKR(dmalloc(h, (void**)&f.p, n * sizeof(T)));
  CKR(dmalloc(h, (void**)&f.g, n * sizeof(T)));
  CKR(dmalloc(h, (void**)&f.t, n * sizeof(T)));
  CKR(dmalloc(h, (void**)&f.r, n * sizeof(T)));
  CKR(dmalloc(h, (void**)&f.c, n * sizeof(T)));
  CK(cudaMemsetAsync(f.p, 0, n * sizeof(T), h->stream));
  CK(cudaMemsetAsync(f.g, 0, n * sizeof(T), h->stream));
  CK(cudaMemsetAsync(f.t, 0, n * sizeof(T), h->stream));
  CK(cudaMemsetAsync(f.r, 0, n * sizeof(T), h->stream));
  f.ready = true;
  return BEM_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The tensor map of W for pass C's TMA staging in precision es (4 or 8): W as
// (M+1) rows of 2 ny reals, boxes of 2 nb reals x w_box_rows(M) rows, zero fill
// past the ends.  TMA wants 16-byte strides and box rows, so FP32 needs an even
// ny and an even nb; where that fails (or TMA is unavailable) the map stays off
// and pass C stages W with cp.async.  BEM_TMA=0 switches it off.
int update_w_map(bem_ctx* h, int es, int nb) {
  const int i = es == 8 ? 1 : 0;
  h->tmw_ok[i] = false;
  static const bool on = [] {
    const char* e = getenv("BEM_TMA");
    return !(e && e[0] == '0');
  }();
  EncodeTiledFn enc = tensor_map_encoder();
  if (!on || !enc) return BEM_OK;
  if (es == 4 && ((h->ny & 1) || (nb & 1))) return BEM_OK;
  const int M = h->px / 2;
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * h->ny, (cuuint64_t)M + 1};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * h->ny * es};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * nb), (cuuint32_t)w_box_rows(M)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->W,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return BEM_OK;  // not representable: stay on cp.async
  if (!h->tmw[i]) {
    if (cudaMalloc(&h->tmw[i], sizeof(CUtensorMap)) != cudaSuccess) {
      cudaGetLastError();
      h->tmw[i] = nullptr;
      return BEM_OK;
    }
    h->bytes += sizeof(CUtensorMap);
  }
  // ordered before every later launch on the handle's stream
  CK(cudaMemcpyAsync(h->tmw[i], &m, sizeof m, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->tmw_ok[i] = true;
  return BEM_OK;
}

template <typename T>
PassArgs<T> make_args(bem_ctx* h) {
  PassArgs<T> a{};
  a.pl = plan_of<T>(h);
  PrecFields<T>& pf = fields_of<T>(h);
  a.f.p = pf.p; a.f.g = pf.g; a.f.t = pf.t; a.f.r = pf.r; a.f.c = pf.c; a.f.S = h->S;
  a.W = h->W;
  a.rows_w = h->ny;
  a.nrows_in = h->ny;
  a.ncols_in = h->nx;
  a.khat = khat_of<T>(h);
  const size_t M = h->px / 2, P = h->py;
  if constexpr (sizeof(T) == 8) {
    a.twA = h->tw64; a.twB = h->tw64 + M; a.twS = h->tw64 + M + P; a.twB16 = h->tw64 + M + P + M + 1;
  } else {
    a.twA = h->tw32; a.twB = h->tw32 + M; a.twS = h->tw32 + M + P; a.twB16 = h->tw32 + M + P + M + 1;
  }
  const int* gt = h->geo + (sizeof(T) == 8 ? 2 * kSoEntries + M + P : 0);
  a.soA = gt;
  a.spA = gt + kSoEntries;
  a.soB = gt + kSoEntries + M;
  a.spB = gt + 2 * kSoEntries + M;
  a.uscale = h->A / ((double)h->px * (double)h->py);
  a.partA = h->part;
  a.partC = h->partC;
  a.tmW = h->tmw_ok[sizeof(T) == 8 ? 1 : 0] ? h->tmw[sizeof(T) == 8 ? 1 : 0] : nullptr;
  a.sc = h->sc;
  a.kerr = &h->sc->kerr;
  return a;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy n doubles from a host or device pointer to the device buffer dst.
int upload(bem_ctx* h, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->stream));
  return BEM_OK;
}
int download(bem_ctx* h, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                     is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  return BEM_OK;
}

int device_error(bem_ctx* h) {
  const unsigned e = h->sc_host->kerr;
  // reported once: clear the word so the next solve on this handle starts clean
  h->sc_host->kerr = 0;
  cudaMemsetAsync(&h->sc->kerr, 0, sizeof(unsigned), h->stream);
  cudaStreamSynchronize(h->stream);
  if (e & 2u) return fail(BEM_ECUDA, "a debug bounds check failed in a kernel (error bits %#x)", e);
  return fail(BEM_ETIMEOUT, "a kernel gave up waiting for its own asynchronous copies (error bits %#x)", e);
}

int read_scalars(bem_ctx* h) {
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->sc_host->kerr) return device_error(h);
  return BEM_OK;
}

int init_scalars(bem_ctx* h, double tol, int max_iter, double pcrit) {
  Scalars s{};
  s.tol = tol;
  s.max_iter = max_iter;
  s.G_old = 1.0;
  s.delta = 0.0;
  s.bnorm = 1.0;
  s.pcrit = pcrit;
  s.max_loops = max_iter + 64;  // the device-driven loop's bound
  s.band0 = h->ny;  // empty box until k_box runs
  s.band1 = -1;
  s.col0 = h->nx;
  s.col1 = -1;
  s.kerr = h->sc_host->kerr;
#ifdef BEM_DEBUG_CHECKS
  // test hook: BEM_INJECT_WAIT_TIMEOUT=1 makes the solve's first persistent
  // pass A launch run a bounded wait out (reported as BEM_ETIMEOUT)
  const char* inj = getenv("BEM_INJECT_WAIT_TIMEOUT");
  s.inject = inj && inj[0] == '1';
#endif
  *h->sc_host = s;
  // every member but the sticky error word
  CK(cudaMemcpyAsync(h->sc, h->sc_host, offsetof(Scalars, kerr), cudaMemcpyHostToDevice, h->stream));
  // the host copy is reused for reads; make sure the upload has consumed it
  CK(cudaStreamSynchronize(h->stream));
  return BEM_OK;
}

// u = A K*x for one field of type T (x -> dst), plain passes.
template <typename T>
void conv_plain(bem_ctx* h, const T* x, T* dst, cudaStream_t s) {
  PassArgs<T> a = make_args<T>(h);
  a.f.src = x;
  a.f.dst = dst;
  a.sc = nullptr;
  launch_pass_a<T>(a, A_PLAIN, s);
  launch_pass_b<T>(a, B_CONV, s);
  launch_pass_c<T>(a, C_PLAIN, s);
  h->launches += 3;
}

// A launch failed while capturing: report it (the caller ends the capture).
#define CAPTURE_CHECK(what)                                                                  \
  do {                                                                                       \
    cudaError_t le_ = cudaPeekAtLastError();                                                 \
    if (le_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                    \
      return fail(BEM_ECUDA, "capture: %s failed: %s", what, cudaGetErrorString(le_));      \
    }                                                                                        \
  } while (0)

// The passes of `iters` CG iterations, captured on the handle's stream; with
// `ev`, event records around the three passes of the first iteration.
// Rows of a multiple of 16 elements (the persistent row passes): the CG loop
// may join a batch of several instances.
bool loop_batchable(const bem_ctx* h) { return (h->nx & 15) == 0; }

template <typename T>
int capture_iterations(bem_ctx* h, bool pk, int iters, cudaEvent_t* ev) {
  PassArgs<T> a = make_args<T>(h);
  a.use_band = pk ? 0 : 1;  // fixed-set CG: only the contact band's rows
  for (int it = 0; it < iters; ++it) {
    const bool mark = ev && it == 0;
    if (mark) cudaEventRecordWithFlags(ev[0], h->stream, cudaEventRecordExternal);
    CAPTURE_CHECK("event 0");
    launch_pass_a<T>(a, pk ? A_PK_P : A_CG_T, h->stream);
    CAPTURE_CHECK("pass A");
    if (mark) cudaEventRecordWithFlags(ev[1], h->stream, cudaEventRecordExternal);
    launch_pass_b<T>(a, B_CONV, h->stream);
    CAPTURE_CHECK("pass B");
    if (mark) cudaEventRecordWithFlags(ev[2], h->stream, cudaEventRecordExternal);
    launch_pass_c<T>(a, pk ? C_PK_G : C_CG_R, h->stream);
    CAPTURE_CHECK("pass C");
    if (mark) cudaEventRecordWithFlags(ev[3], h->stream, cudaEventRecordExternal);
    CAPTURE_CHECK("event 3");
    if (pk) {
      launch_pass_a<T>(a, A_PK_T, h->stream);
      CAPTURE_CHECK("pass A (t)");
      launch_pass_b<T>(a, B_CONV, h->stream);
      CAPTURE_CHECK("pass B (t)");
      launch_pass_c<T>(a, C_PK_R, h->stream);
      CAPTURE_CHECK("pass C (t)");
    }
    // fixed-set CG: the update of p and g is applied by the next pass A
  }
  return BEM_OK;
}

// A chunk of kChunk CG iterations as one graph; with `timed`, event records
// around the three passes of its first iteration (BEM_FLAG_TIME_PASSES).
template <typename T>
int capture_chunk(bem_ctx* h, bool pk, bool timed, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaEvent_t* ev = h->ev[pk ? 0 : 1];
  if (timed && !ev[0])
    for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&ev[i]));
  CK(cudaGetLastError());
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = capture_iterations<T>(h, pk, kChunk, timed ? ev : nullptr);
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc != BEM_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc != BEM_OK ? rc : fail(BEM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(BEM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return BEM_OK;
}

// Algorithmic bytes and flops of one launch of each pass (A, B, C) on `rows`
// grid rows, for element size es: field reads and writes of the mode, W
// written / read / rewritten, the spectrum quarter; FFT flops 5 L log2 L per
// complex transform of length L, halved for a pruned half.
void add_pass_work(bem_ctx* h, bool pk, int rows, int es) {
  const double nx = h->nx, M = h->px / 2, P = h->py, cx = 2.0 * es;
  const double W = cx * (M + 1) * rows;
  // fixed-set CG: pass A reads p, g, t, r, S and writes p, g, t; pass C reads
  // t, g, S and writes r
  const double fa = pk ? 4.0 * es : 7.0 * es + 1, fc = pk ? 3.0 * es : 3.0 * es + 1;
  h->pass_bytes[0] += fa * nx * rows + W;
  h->pass_bytes[1] += 2 * W + es * (M + 1) * (P / 2 + 1);
  h->pass_bytes[2] += W + fc * nx * rows;
  const double fm = 5 * M * log2(M), fp = 5 * P * log2(P);
  h->pass_flops[0] += rows * (0.5 * fm + 20 * M);
  h->pass_flops[1] += (M + 1) * (fp + 8 * P);
  h->pass_flops[2] += rows * (0.5 * fm + 20 * M);
}

}  // namespace

// ---------------------------------------------------------------------------
// Batching of CG loops across concurrent solves.
namespace bem {

struct LoopReq {
  bem_ctx* h = nullptr;
  bool pk = false;
  int es = 4;
  PassArgs<float> a32{};
  PassArgs<double> a64{};
  bool done = false;
  bool solo = false;  // no other loop of its size class was waiting: run it alone
  int rc = BEM_OK;
};

struct LoopBatcher {
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;     // threads inside a solve (they may join)
  bool leading = false;
  std::vector<LoopReq*> waiting;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  struct Entry {
    cudaGraphExec_t exec = nullptr;
    void* d_args = nullptr;
  };
  std::map<std::vector<int>, Entry> graphs;  // size class + instance count
  long long launches = 0, instances = 0;     // batched loop graphs launched, loops they carried
};

LoopBatcher* batcher_create() {
  LoopBatcher* b = new LoopBatcher();
  cudaGetDevice(&b->device);
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return nullptr;
  }
  return b;
}

void batcher_destroy(LoopBatcher* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.d_args) cudaFree(kv.second.d_args);
  }
  cudaEventDestroy(b->ev);
  cudaStreamDestroy(b->stream);
  delete b;
}

void batcher_enter(LoopBatcher* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  b->active++;
}

void batcher_leave(LoopBatcher* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  b->active--;
  b->cv.notify_all();  // the waiting loops may now be all there are
}

void batcher_stats(LoopBatcher* b, long long* launches, long long* instances) {
  std::lock_guard<std::mutex> lk(b->mu);
  *launches += b->launches;
  *instances += b->instances;
}

void attach_batcher(::bem_ctx* h, LoopBatcher* b) {
  h->batcher = b;
  for (::bem_ctx* c : h->subs) attach_batcher(c, b);
}

}  // namespace bem

namespace {

// Size class of a loop request: requests with equal keys share every launch
// shape, so one several-instance launch per pass serves them all.
std::vector<int> loop_key(const LoopReq& r) {
  const Plan& pl = r.es == 4 ? r.a32.pl : r.a64.pl;
  return {r.es, r.pk ? 1 : 0, pl.nx, pl.ny, pl.px, pl.py, pl.nbA, pl.nbB, pl.radixB, r.h->ew_ngrid};
}

// The while-loop graph of n instances of one size class: kLoopBody iterations
// of several-instance passes, then the condition kernel (any instance live).
template <typename T>
int capture_loop_mi(LoopBatcher* b, const PassArgs<T>& a0, bool pk, int n, const PassArgs<T>* arr,
                    cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(b->stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(BEM_ECUDA, "batched loop graph set-up failed: %s", cudaGetErrorString(e));
  }
  for (int it = 0; it < kLoopBody; ++it) {
    if (pk) {
      launch_pass_a_mi<T>(a0, A_PK_P, arr, n, b->stream);
      launch_pass_b_mi<T>(a0, arr, n, b->stream);
      launch_pass_c_mi<T>(a0, C_PK_G, arr, n, b->stream);
      launch_pass_a_mi<T>(a0, A_PK_T, arr, n, b->stream);
      launch_pass_b_mi<T>(a0, arr, n, b->stream);
      launch_pass_c_mi<T>(a0, C_PK_R, arr, n, b->stream);
    } else {
      launch_pass_a_mi<T>(a0, A_CG_T, arr, n, b->stream);
      launch_pass_b_mi<T>(a0, arr, n, b->stream);
      launch_pass_c_mi<T>(a0, C_CG_R, arr, n, b->stream);
    }
  }
  launch_batch_ctl<T>(arr, n, (unsigned long long)cond, b->stream);
  const cudaError_t le = cudaPeekAtLastError();
  cudaGraph_t body_out = nullptr;
  e = cudaStreamEndCapture(b->stream, &body_out);
  if (le != cudaSuccess || e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return fail(BEM_ECUDA, "batched loop capture failed: %s", cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(BEM_ECUDA, "batched loop instantiate failed: %s", cudaGetErrorString(e));
  return BEM_OK;
}

// Launch one size class's requests as one graph on the batcher's stream, after
// each instance's earlier work; each instance's stream then waits for it.
template <typename T>
int launch_group(LoopBatcher* b, std::vector<LoopReq*>& g, const std::vector<int>& key) {
  const int n = (int)g.size();
  std::vector<PassArgs<T>> host(n);
  for (int i = 0; i < n; ++i) {
    host[i] = sizeof(T) == 4 ? *reinterpret_cast<const PassArgs<T>*>(&g[i]->a32)
                             : *reinterpret_cast<const PassArgs<T>*>(&g[i]->a64);
    CK(cudaStreamWaitEvent(b->stream, g[i]->h->ev_ready, 0));
  }
  std::vector<int> gk = key;
  gk.push_back(n);
  LoopBatcher::Entry& en = b->graphs[gk];
  if (!en.d_args) CK(cudaMalloc(&en.d_args, sizeof(PassArgs<T>) * (size_t)n));
  if (!en.exec) {
    CKR(capture_loop_mi<T>(b, host[0], g[0]->pk, n,
                           reinterpret_cast<const PassArgs<T>*>(en.d_args), &en.exec));
  }
  // pageable source: the copy is staged before the call returns
  CK(cudaMemcpyAsync(en.d_args, host.data(), sizeof(PassArgs<T>) * (size_t)n, cudaMemcpyHostToDevice, b->stream));
  CK(cudaGraphLaunch(en.exec, b->stream));
  b->launches += 1;
  b->instances += n;
  CK(cudaEventRecord(b->ev, b->stream));
  for (LoopReq* r : g) CK(cudaStreamWaitEvent(r->h->stream, b->ev, 0));
  return BEM_OK;
}

int launch_batch(LoopBatcher* b, std::vector<LoopReq*>& reqs) {
  std::map<std::vector<int>, std::vector<LoopReq*>> groups;
  for (LoopReq* r : reqs) groups[loop_key(*r)].push_back(r);
  for (auto& kv : groups) {
    if (kv.second.size() == 1) {  // nothing to share a launch with: the solve runs its own loop
      kv.second[0]->solo = true;
      continue;
    }
    const int rc = kv.first[0] == 4 ? launch_group<float>(b, kv.second, kv.first)
                                    : launch_group<double>(b, kv.second, kv.first);
    if (rc != BEM_OK) return rc;
  }
  return BEM_OK;
}

// The solve's CG loop as part of a batch: join, and either wait for a leader or
// lead: take every waiting request once all solves in flight wait (or after a
// short wait for the rest) and launch them.
int run_loop_batched(bem_ctx* h, bool pk, int es, bool* solo) {
  LoopBatcher* b = h->batcher;
  LoopReq r;
  r.h = h;
  r.pk = pk;
  r.es = es;
  if (es == 4) {
    r.a32 = make_args<float>(h);
    r.a32.use_band = pk ? 0 : 1;
  } else {
    r.a64 = make_args<double>(h);
    r.a64.use_band = pk ? 0 : 1;
  }
  if (!h->ev_ready) CK(cudaEventCreateWithFlags(&h->ev_ready, cudaEventDisableTiming));
  CK(cudaEventRecord(h->ev_ready, h->stream));
  const int loops0 = h->sc_host->loops;
  {
    std::unique_lock<std::mutex> lk(b->mu);
    b->waiting.push_back(&r);
    b->cv.notify_all();
    const auto t0 = std::chrono::steady_clock::now();
    while (!r.done) {
      const bool all_in = (int)b->waiting.size() >= b->active;
      const bool waited = std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(200);
      if (!b->leading && !b->waiting.empty() && (all_in || waited)) {
        b->leading = true;
        std::vector<LoopReq*> take;
        take.swap(b->waiting);
        lk.unlock();
        const int rc = launch_batch(b, take);
        lk.lock();
        for (LoopReq* q : take) {
          q->rc = rc;
          q->done = true;
        }
        b->leading = false;
        b->cv.notify_all();
      } else {
        b->cv.wait_for(lk, std::chrono::microseconds(50));
      }
    }
  }
  if (r.rc != BEM_OK) return r.rc;
  *solo = r.solo;
  if (r.solo) return BEM_OK;
  CKR(read_scalars(h));
  const int ran = h->sc_host->loops - loops0 + 1;
  h->launches += (unsigned long long)((ran + kLoopBody - 1) / kLoopBody) * kLoopBody * (pk ? 6 : 3);
  if (!h->sc_host->done) return fail(BEM_ECUDA, "a batched CG loop stopped before the solve was done");
  return BEM_OK;
}

// Under BEM_FLAG_TIME_PASSES every kTimeEvery-th chunk (the first of each
// solve included) runs the graph with event-record nodes; the others run the
// plain graph, so the sampling costs little of the time it measures.
constexpr int kTimeEvery = 4;

// Run chunks of the captured loop until the device sets `done` (or, batched
// with other solves, the several-instance loop graph).
int run_loop(bem_ctx* h, cudaGraphExec_t g, cudaGraphExec_t g_timed, int max_iter, bool pk, int es) {
  // batched with other solves: rows of a multiple of 16 elements (the
  // persistent row passes), no pass timing
  if (h->batcher && !h->timing && loop_batchable(h)) {
    bool solo = false;
    const int rc = run_loop_batched(h, pk, es, &solo);
    if (rc != BEM_OK || !solo) return rc;
  }
  const int max_launch = max_iter / kChunk + 2;
  for (int l = 0; l < max_launch; ++l) {
    const bool timed = h->timing && l % kTimeEvery == 0;
    CK(cudaGraphLaunch(timed ? g_timed : g, h->stream));
    h->launches += (unsigned long long)kChunk * (pk ? 6 : 3);
    CKR(read_scalars(h));
    if (timed) {
      cudaEvent_t* ev = h->ev[pk ? 0 : 1];
      for (int i = 0; i < 3; ++i) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        h->pass_ms[i] += ms;
      }
      h->pass_count[0] += 1;
      int rows = h->ny;
      if (!pk) {
        h->pass_count[1] += 1;
        const int b0 = h->sc_host->band0, b1 = h->sc_host->band1;
        rows = b1 >= b0 ? b1 - b0 + 1 : 0;
      }
      add_pass_work(h, pk, rows, es);
    }
    if (h->sc_host->done) return BEM_OK;
  }
  return BEM_OK;
}

struct StepOut {
  int iterations = 0;
  double eps = 0;
  int status = BEM_OK;
  int stalls = 0;  // CG solves that ended on the stall guard above their tolerance
};

// SC_STALL (eps stopped falling: the arithmetic's rounding floor) counts as
// converged; final_eps reports where it stopped and the result counts it in
// `stalled`.
int map_status(int sc_status) {
  if (sc_status == SC_NOCONV) return BEM_ENOCONV;
  if (sc_status == SC_NUMERIC) return BEM_ENUMERIC;
  return BEM_OK;
}

int pick_sub(bem_ctx* h, bem_ctx** out);
template <typename T>
int pk_in_box(bem_ctx* h, bem_ctx* sub, double d, double tol, int max_iter, bool warm, StepOut* so);

// Non-adhesive solve at depth d in precision T (Sec. 2.1, Polonsky-Keer CG).
template <typename T>
int run_pk(bem_ctx* h, double d, double tol, int max_iter, bool warm, StepOut* so) {
  CKR(ensure_fields<T>(h));
  PrecFields<T>& pf = fields_of<T>(h);
  if (!h->is_sub) {
    CKR(init_scalars(h, tol, max_iter, 0.0));
    launch_box_overlap(plan_of<T>(h), h->h64, d, h->sc, h->stream);
    h->launches += 1;
    CKR(read_scalars(h));
    bem_ctx* sub = nullptr;
    CKR(pick_sub(h, &sub));
    if (sub) return pk_in_box<T>(h, sub, d, tol, max_iter, warm, so);
  }
  if (!pf.pk_graph[0]) CKR(capture_chunk<T>(h, true, false, &pf.pk_graph[0]));
  if (h->timing && !pf.pk_graph[1]) CKR(capture_chunk<T>(h, true, true, &pf.pk_graph[1]));
  launch_pk_init<T>(plan_of<T>(h), h->h64, d, pf.c, pf.p, pf.t, warm ? 1 : 0, h->ew_ngrid, h->stream);
  h->launches += 1;
  CKR(init_scalars(h, tol, max_iter, 0.0));
  CKR(run_loop(h, pf.pk_graph[0], pf.pk_graph[1], max_iter, true, (int)sizeof(T)));
  so->iterations += h->sc_host->iter;
  so->eps = h->sc_host->eps;
  if (h->sc_host->status != SC_OK) so->status = map_status(h->sc_host->status);
  if (h->sc_host->status == SC_STALL) so->stalls += 1;
  return BEM_OK;
}

// The sub-context whose torus is the smallest power-of-two size holding the
// contact box twice over in each direction (so the zero padding of the box is
// at least as large as the box, as the method's padding of the whole grid is),
// or null when that is not smaller than this context's torus.  Created on
// first use: its influence coefficients are the sub-table of this context's
// (they depend only on the element offsets), its spectrum is its own.
int pick_sub(bem_ctx* h, bem_ctx** out) {
  *out = nullptr;
  const Scalars& s = *h->sc_host;
  if (s.band1 < s.band0 || s.col1 < s.col0) return BEM_OK;
  const int bw = s.col1 - s.col0 + 1, bh = s.band1 - s.band0 + 1;
  const int qx = pow2_at_least(2 * bw < 32 ? 32 : 2 * bw), qy = pow2_at_least(2 * bh < 32 ? 32 : 2 * bh);
  if (qx > h->px || qy > h->py || (size_t)qx * qy >= (size_t)h->px * h->py) return BEM_OK;
  for (bem_ctx* c : h->subs)
    if (c->px == qx && c->py == qy) { *out = c; return BEM_OK; }
  bem_ctx* c = nullptr;
  // BEM_INJECT_SUB_FAILURE=1 makes every sub-context creation fail as an
  // allocation failure would (host-side fault injection for the fallback below)
  const char* inj = getenv("BEM_INJECT_SUB_FAILURE");
  const int rc = inj && inj[0] == '1'
                     ? fail(BEM_ENOMEM, "sub-context allocation failed (injected)")
                     : create_ctx(qx / 2, qy / 2, h->dx, h->dy, h->k, h->nu, h->E0, h->c0, h, &c);
  if (rc != BEM_OK) {
    // no room for the smaller torus (or it failed to set up): the whole grid gives
    // the same result, so carry on there
    g_err.clear();
    cudaGetLastError();
    return BEM_OK;
  }
  h->subs.push_back(c);
  *out = c;
  return BEM_OK;
}

template <typename T>
int run_fixed_cg(bem_ctx* h, double tol, int max_iter, double pcrit, StepOut* so);
template <typename T>
int run_pk(bem_ctx* h, double d, double tol, int max_iter, bool warm, StepOut* so);

// Move a sub-context's launch count, pass timings and work into this context,
// and the solve's outcome into this context's host scalars.
void absorb_sub(bem_ctx* h, bem_ctx* sub) {
  h->launches += sub->launches;
  sub->launches = 0;
  for (int i = 0; i < 3; ++i) {
    h->pass_ms[i] += sub->pass_ms[i];
    h->pass_bytes[i] += sub->pass_bytes[i];
    h->pass_flops[i] += sub->pass_flops[i];
    sub->pass_ms[i] = sub->pass_bytes[i] = sub->pass_flops[i] = 0;
  }
  h->pass_count[0] += sub->pass_count[0];
  h->pass_count[1] += sub->pass_count[1];
  sub->pass_count[0] = sub->pass_count[1] = 0;
  h->sc_host->iter = sub->sc_host->iter;
  h->sc_host->eps = sub->sc_host->eps;
  h->sc_host->status = sub->sc_host->status;
  h->sc_host->done = sub->sc_host->done;
}

// The non-adhesive solve on the box of the geometric overlap set {h <= d}.
// Pressures are non-negative and the influence coefficients positive, so the
// deflection u = A K*p is non-negative and the gap u + h - d >= h - d: no
// element with h > d can carry pressure.  The Polonsky-Keer iteration on a
// sub-grid holding that set is therefore the iteration on the whole grid
// (outside it p stays 0 and g > 0).  Sub-grid elements beyond the grid get a
// height far above any depth.  Afterwards p is scattered back and the gap of
// the whole grid is formed with one full transform.
template <typename T>
int pk_in_box(bem_ctx* h, bem_ctx* sub, double d, double tol, int max_iter, bool warm, StepOut* so) {
  const int x0 = h->sc_host->col0, y0 = h->sc_host->band0;
  const size_t n = (size_t)h->nx * h->ny;
  PrecFields<T>& pf = fields_of<T>(h);
  CKR(ensure_fields<T>(sub));
  PrecFields<T>& bf = fields_of<T>(sub);
  launch_box_copy64(h->h64, h->nx, h->ny, x0, y0, sub->h64, sub->nx, sub->ny, 1.0e6, h->stream);
  launch_box_gather<T>(pf.p, pf.c, h->S, h->nx, h->ny, x0, y0, bf.p, bf.c, sub->S, sub->nx, sub->ny, h->stream);
  h->launches += 2;
  sub->timing = h->timing;
  StepOut bo;
  CKR(run_pk<T>(sub, d, tol, max_iter, warm, &bo));
  CK(cudaMemsetAsync(pf.p, 0, n * sizeof(T), h->stream));
  launch_box_scatter<T>(bf.p, pf.p, h->nx, h->ny, x0, y0, sub->nx, sub->ny, h->stream);
  launch_offset<T>(h->h64, d, pf.c, n, h->stream);
  PassArgs<T> a = make_args<T>(h);
  a.f.src = pf.p;
  a.sc = nullptr;
  launch_pass_a<T>(a, A_PLAIN, h->stream);
  launch_pass_b<T>(a, B_CONV, h->stream);
  launch_pass_c<T>(a, C_GAP, h->stream);
  h->launches += 5;
  absorb_sub(h, sub);
  so->iterations += bo.iterations;
  so->eps = bo.eps;
  so->stalls += bo.stalls;
  if (bo.status != BEM_OK) so->status = bo.status;
  return BEM_OK;
}

// The fixed-set solve on the contact box: the operator restricted to S only
// couples elements of S, all inside the box, so solving on a sub-grid placed
// at the box origin (with the same element size and coefficients) gives the
// same result as solving on the whole grid.  p outside S is zero either way.
template <typename T>
int fixed_cg_in_box(bem_ctx* h, bem_ctx* sub, double tol, int max_iter, double pcrit, StepOut* so) {
  const int x0 = h->sc_host->col0, y0 = h->sc_host->band0;
  PrecFields<T>& pf = fields_of<T>(h);
  CKR(ensure_fields<T>(sub));
  PrecFields<T>& bf = fields_of<T>(sub);
  launch_mask_field<T>(pf.p, h->S, (size_t)h->nx * h->ny, h->stream);
  launch_box_gather<T>(pf.p, pf.c, h->S, h->nx, h->ny, x0, y0, bf.p, bf.c, sub->S, sub->nx, sub->ny, h->stream);
  sub->timing = h->timing;
  StepOut bo;
  const int rc = run_fixed_cg<T>(sub, tol, max_iter, pcrit, &bo);
  if (rc != BEM_OK) return rc;
  launch_box_scatter<T>(bf.p, pf.p, h->nx, h->ny, x0, y0, sub->nx, sub->ny, h->stream);
  h->launches += 3;
  absorb_sub(h, sub);
  so->iterations += bo.iterations;
  so->eps = bo.eps;
  so->stalls += bo.stalls;
  if (bo.status != BEM_OK) so->status = bo.status;
  return BEM_OK;
}

// Fixed-set CG: A (K x)_S + c_S = 0, x = 0 off S, from the current x = f.p.
template <typename T>
int run_fixed_cg(bem_ctx* h, double tol, int max_iter, double pcrit, StepOut* so) {
  CKR(ensure_fields<T>(h));
  PrecFields<T>& pf = fields_of<T>(h);
  CKR(init_scalars(h, tol, max_iter, pcrit));
  launch_box(plan_of<T>(h), h->S, h->sc, h->stream);
  h->launches += 1;
  if (!h->is_sub) {
    CKR(read_scalars(h));
    bem_ctx* sub = nullptr;
    CKR(pick_sub(h, &sub));
    if (sub) return fixed_cg_in_box<T>(h, sub, tol, max_iter, pcrit, so);
  }
  if (!pf.cg_graph[0]) CKR(capture_chunk<T>(h, false, false, &pf.cg_graph[0]));
  if (h->timing && !pf.cg_graph[1]) CKR(capture_chunk<T>(h, false, true, &pf.cg_graph[1]));
  const size_t n = (size_t)h->nx * h->ny;
  launch_mask_field<T>(pf.p, h->S, n, h->stream);
  launch_mask_field<T>(pf.t, h->S, n, h->stream);
  PassArgs<T> a = make_args<T>(h);
  a.f.src = pf.p;
  launch_pass_a<T>(a, A_PLAIN, h->stream);
  launch_pass_b<T>(a, B_CONV, h->stream);
  launch_pass_c<T>(a, C_CG_G, h->stream);
  h->launches += 5;
  CKR(read_scalars(h));
  if (!h->sc_host->done) {
    CKR(run_loop(h, pf.cg_graph[0], pf.cg_graph[1], max_iter, false, (int)sizeof(T)));
    if (h->sc_host->have_tau) {
      Fields<T> f = a.f;
      launch_cg_finish<T>(a.pl, f, h->sc, h->ew_ngrid, h->stream);
      h->launches += 1;
    }
    so->eps = sqrt(std::max(h->sc_host->G, 0.0)) / h->sc_host->bnorm;
  } else {
    so->eps = h->sc_host->eps;
  }
  so->iterations += h->sc_host->iter;
  if (h->sc_host->status != SC_OK) so->status = map_status(h->sc_host->status);
  if (h->sc_host->status == SC_STALL) so->stalls += 1;
  return BEM_OK;
}

template <typename T>
int detach(bem_ctx* h, double pcrit, double* ndetached) {
  PrecFields<T>& pf = fields_of<T>(h);
  Fields<T> f{};
  f.p = pf.p;
  f.S = h->S;
  h->sc_host->pcrit = pcrit;
  CK(cudaMemcpyAsync(&h->sc->pcrit, &pcrit, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  launch_detach<T>(plan_of<T>(h), f, h->partE, h->sc, h->ew_ngrid, h->stream);
  h->launches += 1;
  CKR(read_scalars(h));
  *ndetached = h->sc_host->n_ol;
  return BEM_OK;
}

template <typename T>
int collect(bem_ctx* h, const T* p, const T* g, int use_set, bem_result* r) {
  launch_stats<T>(plan_of<T>(h), p, g, h->S, use_set, h->stats + 8, h->stats, h->stats_ngrid,
                  h->stream);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->stats_host, h->stats, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&h->sc_host->kerr, &h->sc->kerr, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->sc_host->kerr) return device_error(h);
  const double cell = h->dx * h->dy;
  r->force = cell * h->stats_host[0];
  r->contact_count = (int)h->stats_host[1];
  r->area = cell * h->stats_host[1];
  r->contact_radius = sqrt(r->area / 3.14159265358979323846);
  r->max_gap_violation = fmax(h->stats_host[2], h->stats_host[3]);
  return BEM_OK;
}

// FP64 gap of the FP64 pressure in io64: g64 = A K p64 + h - d  (into f64.g).
// With rows band_lo <= band_hi holding every nonzero p64, the transform works
// on those rows only and g64 is formed there only (its other rows keep what
// they held): the adhesive refinement needs the residual on the held set alone.
int gap64(bem_ctx* h, double d, int band_lo = 0, int band_hi = -1) {
  CKR(ensure_fields<double>(h));
  PrecFields<double>& f = h->f64;
  const size_t n = (size_t)h->nx * h->ny;
  launch_offset<double>(h->h64, d, f.c, n, h->stream);
  PassArgs<double> a = make_args<double>(h);
  a.f.src = h->io64;
  a.sc = nullptr;
  if (band_hi >= band_lo && band_lo >= 0 && band_hi < h->ny) {
    a.use_band = 2;
    a.band_lo = band_lo;
    a.band_hi = band_hi;
  }
  launch_pass_a<double>(a, A_PLAIN, h->stream);
  launch_pass_b<double>(a, B_CONV, h->stream);
  launch_pass_c<double>(a, C_GAP, h->stream);
  h->launches += 4;
  return BEM_OK;
}

// Largest |x| over S (use_set) -- via the statistics kernel.
int max_abs_on_set(bem_ctx* h, const double* x, double* out) {
  bem_result tmp{};
  CKR(collect<double>(h, h->io64, x, 1, &tmp));
  *out = h->stats_host[2];
  return BEM_OK;
}

// FP64-residual refinement of the FP32 solution (precision BEM_PREC_FP32_REFINE).
// io64 holds the FP64 pressure.  Each sweep computes the FP64 gap g64 of it
// (one FP64 convolution), chooses the set S, solves A K dp + g64 = 0 on S with
// the FP32 fixed-set CG, and adds dp.  Non-adhesive: S = {p > 0} U {g < 0} and
// p is projected onto p >= 0 after the update; adhesive: S is held and tension
// is allowed.  Stops when max_S |g64| <= tol64 * max_S |h - d|.  Adhesive:
// rows band_lo .. band_hi hold S (when band_lo <= band_hi), and the FP64 gap
// is formed on them only.
int refine_here(bem_ctx* h, double d, bool adhesive, int sweeps, double tol64, double tol32, StepOut* so,
                int band_lo = 0, int band_hi = -1) {
  const size_t n = (size_t)h->nx * h->ny;
  for (int s = 0; s < sweeps; ++s) {
    if (adhesive) CKR(gap64(h, d, band_lo, band_hi));
    else CKR(gap64(h, d));
    if (!adhesive) { launch_active_set(h->io64, h->f64.g, h->S, n, h->stream); h->launches += 1; }
    double res = 0, scale = 0;
    CKR(max_abs_on_set(h, h->f64.g, &res));
    CKR(max_abs_on_set(h, h->f64.c, &scale));
    if (res <= tol64 * scale || !(res > 0)) break;
    // the FP32 correction solves for dp / res so its data are O(1) in FP32
    launch_to_f32_scaled(h->f64.g, 1.0 / res, h->f32.c, n, h->stream);
    h->launches += 1;
    CK(cudaMemsetAsync(h->f32.p, 0, n * sizeof(float), h->stream));
    CK(cudaMemsetAsync(h->f32.t, 0, n * sizeof(float), h->stream));
    StepOut cg;
    CKR(run_fixed_cg<float>(h, tol32, 2000, 0.0, &cg));
    so->iterations += cg.iterations;
    so->stalls += cg.stalls;
    if (h->sc_host->status == SC_NUMERIC) { so->status = BEM_ENUMERIC; break; }
    launch_refine_apply(h->io64, h->f32.p, res, h->S, adhesive ? 0 : 1, n, h->stream);
    h->launches += 1;
  }
  return BEM_OK;
}

// The refinement on the smallest torus holding the set it works on: the held
// set S (adhesive: the residual matters only on S, and p vanishes off it) or
// the overlap set {h <= d} (non-adhesive: the active set {p > 0} U {g < 0}
// lies inside it, since g >= h - d).  The FP64 pressure, the profile and S
// are gathered into the sub-context and the pressure is scattered back.
int refine(bem_ctx* h, double d, bool adhesive, int sweeps, double tol64, double tol32, StepOut* so) {
  if (!h->is_sub) {
    CKR(init_scalars(h, 0.0, 0, 0.0));  // an empty box to collect into
    if (adhesive) launch_box(h->plan64, h->S, h->sc, h->stream);
    else launch_box_overlap(h->plan64, h->h64, d, h->sc, h->stream);
    h->launches += 1;
    CKR(read_scalars(h));
    // rows of the held set (adhesive): its box, in this grid and at the sub-grid's origin
    const int b0 = h->sc_host->band0, b1 = h->sc_host->band1;
    bem_ctx* sub = nullptr;
    CKR(pick_sub(h, &sub));
    if (sub) {
      const int x0 = h->sc_host->col0, y0 = h->sc_host->band0;
      CKR(ensure_fields<double>(sub));
      CKR(ensure_fields<float>(sub));
      launch_box_gather<double>(h->io64, h->io64, h->S, h->nx, h->ny, x0, y0, sub->io64, sub->io64b, sub->S,
                                sub->nx, sub->ny, h->stream);
      launch_box_copy64(h->h64, h->nx, h->ny, x0, y0, sub->h64, sub->nx, sub->ny, 1.0e6, h->stream);
      sub->timing = h->timing;
      CKR(refine_here(sub, d, adhesive, sweeps, tol64, tol32, so, 0, b1 - b0));
      launch_box_scatter<double>(sub->io64, h->io64, h->nx, h->ny, x0, y0, sub->nx, sub->ny, h->stream);
      h->launches += 3;
      absorb_sub(h, sub);
      return BEM_OK;
    }
    return refine_here(h, d, adhesive, sweeps, tol64, tol32, so, b0, b1);
  }
  return refine_here(h, d, adhesive, sweeps, tol64, tol32, so);
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner (FP32 passes).  The first context of each grid size
// times the plain transform with the default shapes and with half and twice
// the rows per CTA of the row passes and the columns per CTA of the column
// pass, and keeps the fastest of each (a change needs a 3% gain, so timing
// noise keeps the default).  The choice is kept for the process, and the lock
// is held while timing, so every context of a size uses the same shapes.
struct ShapeKey {
  int nx, ny, px, py, radix_req;  // radix_req: the column-pass radix BEM_RADIX_B fixes (0: none)
  bool operator<(const ShapeKey& o) const {
    return nx != o.nx ? nx < o.nx : ny != o.ny ? ny < o.ny : px != o.px ? px < o.px : py != o.py ? py < o.py
                                                                                      : radix_req < o.radix_req;
  }
};
std::mutex g_tune_mu;
struct Tuned {
  int nbA, nbB, radixB;
};
std::map<ShapeKey, Tuned> g_tuned;

int set_plan32(bem_ctx* h, const Plan& pl) {
  h->plan32 = pl;
  CKR(update_w_map(h, 4, pl.nbA));
  int* g32 = h->geo;
  const int M = h->px / 2;
  launch_geo_tables(g32, g32 + kSoEntries, pl.gA, 4, h->stream);
  launch_geo_tables(g32 + kSoEntries + M, g32 + 2 * kSoEntries + M, pl.gB, 4, h->stream);
  return BEM_OK;
}

// Device milliseconds of passes A, B, C (summed over `reps` plain transforms).
int time_passes32(bem_ctx* h, int reps, double ms[3]) {
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&ev[i]));
  ms[0] = ms[1] = ms[2] = 0;
  PassArgs<float> a = make_args<float>(h);
  a.f.src = h->f32.p;
  a.f.dst = h->f32.g;
  a.sc = nullptr;
  int rc = BEM_OK;
  for (int it = 0; it < reps + 2 && rc == BEM_OK; ++it) {  // two untimed warm-up transforms
    cudaEventRecord(ev[0], h->stream);
    launch_pass_a<float>(a, A_PLAIN, h->stream);
    cudaEventRecord(ev[1], h->stream);
    launch_pass_b<float>(a, B_CONV, h->stream);
    cudaEventRecord(ev[2], h->stream);
    launch_pass_c<float>(a, C_PLAIN, h->stream);
    cudaEventRecord(ev[3], h->stream);
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) { rc = BEM_ECUDA; break; }
    if (it < 2) continue;
    for (int i = 0; i < 3; ++i) {
      float t = 0;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t;
    }
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (rc != BEM_OK) return fail(rc, "autotuner timing failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += 3 * (unsigned long long)(reps + 2);
  return BEM_OK;
}

int autotune32(bem_ctx* h) {
  const char* env = getenv("BEM_AUTOTUNE");
  if (env && env[0] == '0') return BEM_OK;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const ShapeKey key{h->nx, h->ny, h->px, h->py, forced_radix_b()};
  const Plan base = h->plan32;
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    const Tuned& u = it->second;
    if (u.nbA != base.nbA || u.nbB != base.nbB || u.radixB != base.radixB)
      CKR(set_plan32(h, plan_with(h->nx, h->ny, h->px, h->py, 4, base.nsm, u.nbA, u.nbB, u.radixB)));
    return BEM_OK;
  }
  CKR(ensure_fields<float>(h));
  // Candidates: the default shapes, half and twice the rows per CTA of the row
  // passes, half and twice the columns per CTA of the column pass, and the
  // column pass in the other radix (8 or 16) at its default columns per CTA
  // and half and twice that (unless BEM_RADIX_B fixes the radix).  Each is
  // timed in three interleaved rounds and keeps its fastest round, so that a
  // slow round (clock ramp, another process) cannot pick a shape.
  struct Cand { int nbA, nbB, radixB; double t[3]; };
  std::vector<Cand> cand;
  auto fits = [&](int nbA, int nbB, int radixB) {
    return nbA >= 1 && nbB >= 1 &&
           shape_fits(plan_with(h->nx, h->ny, h->px, h->py, 4, base.nsm, nbA, nbB, radixB), 4);
  };
  cand.push_back({base.nbA, base.nbB, base.radixB, {1e30, 1e30, 1e30}});
  for (int nb : {base.nbA / 2, base.nbA * 2})
    if (fits(nb, base.nbB, base.radixB)) cand.push_back({nb, base.nbB, base.radixB, {1e30, 1e30, 1e30}});
  for (int nb : {base.nbB / 2, base.nbB * 2})
    if (fits(base.nbA, nb, base.radixB)) cand.push_back({base.nbA, nb, base.radixB, {1e30, 1e30, 1e30}});
  if (!forced_radix_b()) {
    const int other = base.radixB == 8 ? 16 : 8;
    const int nbo = default_cols_b(h->px / 2, h->py, 4, base.nsm, other);
    for (int nb : {nbo, nbo / 2, nbo * 2})
      if (fits(base.nbA, nb, other)) cand.push_back({base.nbA, nb, other, {1e30, 1e30, 1e30}});
  }
  constexpr int reps = 6, rounds = 3;
  for (int r = 0; r < rounds; ++r) {
    for (Cand& c : cand) {
      CKR(set_plan32(h, plan_with(h->nx, h->ny, h->px, h->py, 4, base.nsm, c.nbA, c.nbB, c.radixB)));
      double t[3];
      CKR(time_passes32(h, reps, t));
      for (int q = 0; q < 3; ++q) c.t[q] = std::min(c.t[q], t[q]);
    }
  }
  // a change needs a 3% gain over the default shapes
  int bestA = base.nbA, bestB = base.nbB, bestR = base.radixB;
  double tAC = cand[0].t[0] + cand[0].t[2], tB = cand[0].t[1];
  for (size_t c = 1; c < cand.size(); ++c) {
    const Cand& x = cand[c];
    if (x.nbB == base.nbB && x.radixB == base.radixB && x.t[0] + x.t[2] < 0.97 * tAC) {
      tAC = x.t[0] + x.t[2];
      bestA = x.nbA;
    }
    if (x.nbA == base.nbA && x.t[1] < 0.97 * tB) {
      tB = x.t[1];
      bestB = x.nbB;
      bestR = x.radixB;
    }
  }
  CKR(set_plan32(h, plan_with(h->nx, h->ny, h->px, h->py, 4, base.nsm, bestA, bestB, bestR)));
  CK(cudaStreamSynchronize(h->stream));
  g_tuned[key] = {bestA, bestB, bestR};
  return BEM_OK;
}

int validate_ptr(const void* p, const char* name) {
  if (!p) return fail(BEM_EINVAL, "%s must not be NULL", name);
  return BEM_OK;
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" const char* bem_last_error(void) { return g_err.c_str(); }

namespace bem {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}

extern "C" int bem_create(int Nx, int Ny, double dx, double dy, double k, double nu, double E0,
                          double c0, bem_handle* out) {
  g_err.clear();
  if (!out) return fail(BEM_EINVAL, "out must not be NULL");
  return create_ctx(Nx, Ny, dx, dy, k, nu, E0, c0, nullptr, out);
}

// A context for an Nx x Ny grid.  With a parent (a contact-box sub-context of
// it): the parent's stream, and the influence coefficients copied from the
// parent's table (offsets 0..Px/2 x 0..Py/2 of this torus are a sub-block).
static int create_ctx(int Nx, int Ny, double dx, double dy, double k, double nu, double E0, double c0,
                      bem_ctx* parent, bem_ctx** out) {
  if (Nx < 2 || Ny < 2 || Nx > 4096 || Ny > 4096)
    return fail(BEM_EINVAL, "grid %dx%d outside 2..4096", Nx, Ny);
  if (!(dx > 0) || !(dy > 0)) return fail(BEM_EINVAL, "element sizes must be > 0");
  if (!(k > -1.0 && k < 1.0)) return fail(BEM_EINVAL, "k=%g outside (-1, 1)", k);
  if (!(nu > -1.0 && nu <= 0.5)) return fail(BEM_EINVAL, "nu=%g outside (-1, 0.5]", nu);
  if (!(E0 > 0) || !(c0 > 0)) return fail(BEM_EINVAL, "E0 and c0 must be > 0");
  const double alpha = bem_alpha(k, nu);
  if (!(alpha > 0) || !isfinite(alpha)) return fail(BEM_EINVAL, "alpha(k=%g, nu=%g) undefined (beta^2 <= 0)", k, nu);

  bem_ctx* h = new bem_ctx();
  auto cleanup = [&](int rc) { bem_destroy(h); return rc; };
  if (cudaGetDevice(&h->device) != cudaSuccess) return cleanup(fail(BEM_ECUDA, "no CUDA device"));
  if (parent) {
    h->is_sub = true;
    h->own_stream = false;
    h->stream = parent->stream;
    h->batcher = parent->batcher;
  } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
    return cleanup(fail(BEM_ECUDA, "stream creation failed"));
  }
  {
    const int rc0 = device_setup(h->device);
    if (rc0 != BEM_OK) return cleanup(rc0);
  }
  h->nx = Nx; h->ny = Ny; h->dx = dx; h->dy = dy; h->k = k; h->nu = nu; h->E0 = E0; h->c0 = c0;
  h->alpha = alpha;
  h->A = alpha * (1.0 - nu * nu) * pow(c0, k) / E0;  // Eq. 12
  h->px = pow2_at_least(2 * Nx < 32 ? 32 : 2 * Nx);
  h->py = pow2_at_least(2 * Ny < 32 ? 32 : 2 * Ny);
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || nsm < 1)
      return cleanup(fail(BEM_ECUDA, "cannot query the SM count"));
    h->plan32 = make_plan(Nx, Ny, h->px, h->py, 4, nsm);
    h->plan64 = make_plan(Nx, Ny, h->px, h->py, 8, nsm);
  }
  const int M = h->px / 2, hyq = h->py / 2 + 1;
  const size_t n = (size_t)Nx * Ny;
  int rc;
  if ((rc = dmalloc(h, (void**)&h->kq64, sizeof(double) * (size_t)hyq * (M + 1)))) return cleanup(rc);
  // [length-M stages | length-Py stages | split | radix-16 length-Py stages]
  const size_t ntw = (size_t)M + h->py + M + 1 + h->py;
  if ((rc = dmalloc(h, (void**)&h->tw64, sizeof(double2) * ntw))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->tw32, sizeof(float2) * ntw))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->geo, sizeof(int) * 2 * (2 * kSoEntries + M + h->py)))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->khat64, sizeof(double) * (size_t)hyq * (M + 1)))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->khat32, sizeof(float) * (size_t)hyq * (M + 1)))) return cleanup(rc);
  if ((rc = dmalloc(h, &h->W, sizeof(double) * 2 * (size_t)(M + 1) * Ny))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->h64, sizeof(double) * n))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->io64, sizeof(double) * n))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->io64b, sizeof(double) * n))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->S, n))) return cleanup(rc);
  const int gmax = Ny;  // per-CTA partials come from row groups: at most one per row, for any shape
  if ((rc = dmalloc(h, (void**)&h->part, sizeof(double) * 4 * (size_t)gmax))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->partC, sizeof(double) * 4 * (size_t)gmax))) return cleanup(rc);
  h->ew_ngrid = (int)((n + 255) / 256 < (size_t)BEM_EW_CTAS_PER_SM * h->plan32.nsm
                          ? (n + 255) / 256 : (size_t)BEM_EW_CTAS_PER_SM * h->plan32.nsm);
  if (h->ew_ngrid < 1) h->ew_ngrid = 1;
  if ((rc = dmalloc(h, (void**)&h->partE, sizeof(double) * 4 * (size_t)h->ew_ngrid))) return cleanup(rc);
  h->stats_ngrid = h->ew_ngrid;
  if ((rc = dmalloc(h, (void**)&h->stats, sizeof(double) * (8 + 4 * (size_t)h->stats_ngrid + 8)))) return cleanup(rc);
  if ((rc = dmalloc(h, (void**)&h->sc, sizeof(Scalars)))) return cleanup(rc);
  if (cudaMallocHost((void**)&h->sc_host, sizeof(Scalars)) != cudaSuccess ||
      cudaMallocHost((void**)&h->stats_host, 8 * sizeof(double)) != cudaSuccess)
    return cleanup(fail(BEM_ENOMEM, "pinned allocation failed"));
  memset(h->sc_host, 0, sizeof(Scalars));
  if (cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->stats, 0, sizeof(double) * (8 + 4 * (size_t)h->stats_ngrid + 8), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->S, 0, n, h->stream) != cudaSuccess)
    return cleanup(fail(BEM_ECUDA, "memset failed"));

  {
    int* g32 = h->geo;
    int* g64 = h->geo + 2 * kSoEntries + M + h->py;
    launch_geo_tables(g32, g32 + kSoEntries, h->plan32.gA, 4, h->stream);
    launch_geo_tables(g32 + kSoEntries + M, g32 + 2 * kSoEntries + M, h->plan32.gB, 4, h->stream);
    launch_geo_tables(g64, g64 + kSoEntries, h->plan64.gA, 8, h->stream);
    launch_geo_tables(g64 + kSoEntries + M, g64 + 2 * kSoEntries + M, h->plan64.gB, 8, h->stream);
  }
  launch_twiddles(h->tw64, h->tw32, ilog2(M), h->stream);
  launch_twiddles(h->tw64 + M, h->tw32 + M, ilog2(h->py), h->stream);
  launch_split_twiddles(h->tw64 + M + h->py, h->tw32 + M + h->py, M, h->stream);
  launch_twiddles16(h->tw64 + M + h->py + M + 1, h->tw32 + M + h->py + M + 1, ilog2(h->py), h->stream);
  // a1: influence coefficients on the offsets 0..Px/2, 0..Py/2 (Eq. 9)
  if (parent) {
    const size_t pw = (size_t)parent->px / 2 + 1;
    if (cudaMemcpy2DAsync(h->kq64, sizeof(double) * (M + 1), parent->kq64, sizeof(double) * pw,
                          sizeof(double) * (M + 1), hyq, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return cleanup(fail(BEM_ECUDA, "influence sub-table copy failed"));
  } else {
    launch_influence(h->kq64, M + 1, hyq, dx, dy, k, h->stream);
  }
  // spectrum of the even torus extension (Eq. 13: FFT(K)), FP64, once
  {
    void* Wspec = nullptr;
    if (cudaMalloc(&Wspec, sizeof(double) * 2 * (size_t)(M + 1) * h->py) != cudaSuccess)
      return cleanup(fail(BEM_ENOMEM, "spectrum workspace allocation failed"));
    PassArgs<double> a{};
    a.pl = h->plan64;
    a.twA = h->tw64; a.twB = h->tw64 + M; a.twS = h->tw64 + M + h->py;
    const int* g64 = h->geo + 2 * kSoEntries + M + h->py;
    a.soA = g64; a.spA = g64 + kSoEntries;
    a.soB = g64 + kSoEntries + M; a.spB = g64 + 2 * kSoEntries + M;
    a.W = Wspec;
    a.rows_w = h->py;
    a.nrows_in = h->py;
    a.ncols_in = h->px;
    a.kq64 = h->kq64;
    a.khat64_out = h->khat64;
    a.khat32_out = h->khat32;
    launch_pass_a<double>(a, A_TORUS, h->stream);
    launch_pass_b<double>(a, B_SPECTRUM, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaFree(Wspec);
    if (e != cudaSuccess) return cleanup(fail(BEM_ECUDA, "spectrum set-up failed: %s", cudaGetErrorString(e)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(fail(BEM_ECUDA, "set-up kernels failed: %s", cudaGetErrorString(e)));
  if ((rc = update_w_map(h, 4, h->plan32.nbA)) || (rc = update_w_map(h, 8, h->plan64.nbA))) return cleanup(rc);
  if ((rc = autotune32(h))) return cleanup(rc);
  *out = h;
  return BEM_OK;
}

extern "C" void bem_destroy(bem_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (bem_ctx* c : h->subs) bem_destroy(c);
  h->subs.clear();
  auto fr = [](void* p) { if (p) cudaFree(p); };
  for (int t = 0; t < 2; ++t)
    for (cudaGraphExec_t g : {h->f32.pk_graph[t], h->f32.cg_graph[t], h->f64.pk_graph[t], h->f64.cg_graph[t]})
      if (g) cudaGraphExecDestroy(g);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j)
      if (h->ev[i][j]) cudaEventDestroy(h->ev[i][j]);
  if (h->ev_ready) cudaEventDestroy(h->ev_ready);
  fr(h->tmw[0]); fr(h->tmw[1]);
  fr(h->kq64); fr(h->geo); fr(h->tw64); fr(h->tw32); fr(h->khat64); fr(h->khat32); fr(h->W); fr(h->h64); fr(h->io64); fr(h->io64b);
  fr(h->S); fr(h->part); fr(h->partC); fr(h->partE); fr(h->stats); fr(h->sc);
  fr(h->f32.p); fr(h->f32.g); fr(h->f32.t); fr(h->f32.r); fr(h->f32.c);
  fr(h->f64.p); fr(h->f64.g); fr(h->f64.t); fr(h->f64.r); fr(h->f64.c);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->stats_host) cudaFreeHost(h->stats_host);
  if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" int bem_get_info(bem_handle h, bem_info* info) {
  if (!h || !info) return fail(BEM_EINVAL, "NULL argument");
  info->Nx = h->nx; info->Ny = h->ny; info->Px = h->px; info->Py = h->py;
  info->dx = h->dx; info->dy = h->dy; info->k = h->k; info->nu = h->nu; info->E0 = h->E0; info->c0 = h->c0;
  info->alpha = h->alpha; info->compliance = h->A; info->device_bytes = h->bytes;
  info->rows_per_cta = h->plan32.nbA;
  info->cols_per_cta = h->plan32.nbB;
  info->col_radix = h->plan32.radixB;
  for (const bem_ctx* c : h->subs) info->device_bytes += c->bytes;
  info->kernel_launches = h->launches;
  return BEM_OK;
}

extern "C" int bem_set_material(bem_handle h, double nu, double E0, double c0) {
  if (!h) return fail(BEM_EINVAL, "NULL handle");
  if (!(nu > -1.0 && nu <= 0.5)) return fail(BEM_EINVAL, "nu=%g outside (-1, 0.5]", nu);
  if (!(E0 > 0) || !(c0 > 0)) return fail(BEM_EINVAL, "E0 and c0 must be > 0");
  const double alpha = bem_alpha(h->k, nu);
  if (!(alpha > 0) || !isfinite(alpha)) return fail(BEM_EINVAL, "alpha(k=%g, nu=%g) undefined", h->k, nu);
  const double A = alpha * (1.0 - nu * nu) * pow(c0, h->k) / E0;
  if (A == h->A && nu == h->nu && E0 == h->E0 && c0 == h->c0) return BEM_OK;
  h->nu = nu; h->E0 = E0; h->c0 = c0; h->alpha = alpha; h->A = A;
  // the captured CG graphs carry A/(Px Py) as a kernel argument: recapture lazily
  CK(cudaStreamSynchronize(h->stream));
  for (int t = 0; t < 2; ++t) {
    for (cudaGraphExec_t* g : {&h->f32.pk_graph[t], &h->f32.cg_graph[t], &h->f64.pk_graph[t], &h->f64.cg_graph[t]})
      if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
  }
  for (bem_ctx* c : h->subs) CKR(bem_set_material(c, nu, E0, c0));
  return BEM_OK;
}

extern "C" int bem_pass_work(bem_handle h, double bytes[3], double flops[3]) {
  if (!h || !bytes || !flops) return fail(BEM_EINVAL, "NULL argument");
  const double n = h->pass_count[0] > 0 ? (double)h->pass_count[0] : 1.0;
  for (int i = 0; i < 3; ++i) {
    bytes[i] = h->pass_bytes[i] / n;
    flops[i] = h->pass_flops[i] / n;
  }
  return BEM_OK;
}

extern "C" int bem_pass_times(bem_handle h, double ms[3], long long count[2], int reset) {
  if (!h || !ms || !count) return fail(BEM_EINVAL, "NULL argument");
  for (int i = 0; i < 3; ++i) ms[i] = h->pass_ms[i];
  count[0] = h->pass_count[0];
  count[1] = h->pass_count[1];
  if (reset) {
    for (int i = 0; i < 3; ++i) h->pass_ms[i] = 0;
    h->pass_count[0] = h->pass_count[1] = 0;
    for (int i = 0; i < 3; ++i) h->pass_bytes[i] = h->pass_flops[i] = 0;
  }
  return BEM_OK;
}

extern "C" int bem_influence_table(bem_handle h, double* out) {
  if (!h) return fail(BEM_EINVAL, "NULL handle");
  CKR(validate_ptr(out, "out"));
  const size_t cnt = (size_t)(h->px / 2 + 1) * (h->py / 2 + 1);
  CKR(download(h, out, h->kq64, cnt));
  CK(cudaStreamSynchronize(h->stream));
  return BEM_OK;
}

__global__ void k_transpose_quarter(const double* src, double* dst, int hx, int hyq) {
  // src[kx*hyq + ky] -> dst[ky*hx + kx]
  const int kx = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  if (kx < hx && ky < hyq) dst[(size_t)ky * hx + kx] = src[(size_t)kx * hyq + ky];
}

extern "C" int bem_spectrum(bem_handle h, double* out) {
  if (!h) return fail(BEM_EINVAL, "NULL handle");
  CKR(validate_ptr(out, "out"));
  const int hx = h->px / 2 + 1, hyq = h->py / 2 + 1;
  double* tmp = nullptr;
  CK(cudaMallocAsync((void**)&tmp, sizeof(double) * (size_t)hx * hyq, h->stream));
  k_transpose_quarter<<<dim3((hx + 127) / 128, hyq), 128, 0, h->stream>>>(h->khat64, tmp, hx, hyq);
  int rc = download(h, out, tmp, (size_t)hx * hyq);
  cudaFreeAsync(tmp, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

extern "C" int bem_convolve(bem_handle h, int precision, const double* p, double* u) {
  if (!h) return fail(BEM_EINVAL, "NULL handle");
  CKR(validate_ptr(p, "p"));
  CKR(validate_ptr(u, "u"));
  const size_t n = (size_t)h->nx * h->ny;
  CKR(upload(h, h->io64, p, n));
  if (precision == BEM_PREC_FP64) {
    conv_plain<double>(h, h->io64, h->io64b, h->stream);
  } else if (precision == BEM_PREC_FP32) {
    CKR(ensure_fields<float>(h));
    launch_convert_in<float>(h->io64, h->f32.p, n, h->stream);
    conv_plain<float>(h, h->f32.p, h->f32.g, h->stream);
    launch_convert_out<float>(h->f32.g, h->io64b, n, h->stream);
  } else {
    return fail(BEM_EINVAL, "precision %d not supported by bem_convolve", precision);
  }
  CKR(download(h, u, h->io64b, n));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return BEM_OK;
}

namespace {

struct SolveCfg {
  int precision = BEM_PREC_FP32;
  double tol = 0;
  int max_iter = 20000;
  int sweeps = 3;
  int flags = 0;
  cudaStream_t user = nullptr;
};

int parse_opts(const bem_opts* o, SolveCfg* c) {
  if (o) {
    if (o->precision < BEM_PREC_FP64 || o->precision > BEM_PREC_FP32_REFINE)
      return fail(BEM_EINVAL, "unknown precision %d", o->precision);
    if (o->tol < 0 || o->max_iter < 0 || o->refine_sweeps < 0)
      return fail(BEM_EINVAL, "negative option");
    c->precision = o->precision;
    c->tol = o->tol;
    if (o->max_iter > 0) c->max_iter = o->max_iter;
    if (o->refine_sweeps > 0) c->sweeps = o->refine_sweeps;
    c->user = (cudaStream_t)o->stream;
    c->flags = o->flags;
  }
  if (c->tol == 0) c->tol = c->precision == BEM_PREC_FP64 ? 1e-10 : 1e-6;
  return BEM_OK;
}

// One non-adhesive step in the configured precision; leaves the FP64 pressure
// in io64 and fills r.
int step_nonadhesive(bem_ctx* h, const SolveCfg& cfg, double d, bool warm, bem_result* r) {
  const size_t n = (size_t)h->nx * h->ny;
  StepOut so;
  if (cfg.precision == BEM_PREC_FP64) {
    CKR(run_pk<double>(h, d, cfg.tol, cfg.max_iter, warm, &so));
    CKR(collect<double>(h, h->f64.p, h->f64.g, 0, r));
    CK(cudaMemcpyAsync(h->io64, h->f64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    CKR(run_pk<float>(h, d, cfg.tol, cfg.max_iter, warm, &so));
    launch_convert_out<float>(h->f32.p, h->io64, n, h->stream);
    h->launches += 1;
    if (cfg.precision == BEM_PREC_FP32_REFINE) {
      CKR(refine(h, d, false, cfg.sweeps, 1e-13, cfg.tol, &so));
      CKR(gap64(h, d));
      CKR(collect<double>(h, h->io64, h->f64.g, 0, r));
      // keep the FP32 warm start in step with the refined pressure
      launch_to_f32(h->io64, h->f32.p, n, h->stream);
      h->launches += 1;
    } else {
      CKR(collect<float>(h, h->f32.p, h->f32.g, 0, r));
    }
  }
  r->iterations = so.iterations;
  r->final_eps = so.eps;
  r->detach_rounds = 0;
  r->status = so.status;
  r->stalled = so.stalls;
  r->depth = d;
  return BEM_OK;
}

// One adhesive pull-off step at depth d on the current set S (Sec. 3.1).
template <typename T>
int step_adhesive_t(bem_ctx* h, const SolveCfg& cfg, double d, double pcrit, bem_result* r) {
  const size_t n = (size_t)h->nx * h->ny;
  PrecFields<T>& pf = fields_of<T>(h);
  StepOut so;
  int rounds = 0;
  launch_offset<T>(h->h64, d, pf.c, n, h->stream);
  h->launches += 1;
  const double tol = cfg.precision == BEM_PREC_FP64 ? 1e-12 : cfg.tol;
  for (;;) {
    CKR(run_fixed_cg<T>(h, tol, cfg.max_iter, pcrit, &so));
    if (cfg.precision == BEM_PREC_FP32_REFINE) {
      launch_convert_out<float>(h->f32.p, h->io64, n, h->stream);
      CKR(refine(h, d, true, cfg.sweeps, 1e-13, cfg.tol, &so));
      launch_to_f32(h->io64, h->f32.p, n, h->stream);
      launch_offset<float>(h->h64, d, h->f32.c, n, h->stream);
      h->launches += 3;
    }
    double nd = 0;
    CKR(detach<T>(h, pcrit, &nd));
    if (nd == 0) break;
    ++rounds;
  }
  // true gap of the final state (for the off-contact check)
  if (cfg.precision == BEM_PREC_FP32_REFINE) {
    // io64 holds the refined pressure; the last round detached nothing
    CKR(gap64(h, d));
    CKR(collect<double>(h, h->io64, h->f64.g, 1, r));
  } else {
    PassArgs<T> a = make_args<T>(h);
    a.f.src = pf.p;
    a.sc = nullptr;
    launch_offset<T>(h->h64, d, pf.c, n, h->stream);
    launch_pass_a<T>(a, A_PLAIN, h->stream);
    launch_pass_b<T>(a, B_CONV, h->stream);
    launch_pass_c<T>(a, C_GAP, h->stream);
    CKR(collect<T>(h, pf.p, pf.g, 1, r));
    launch_convert_out<T>(pf.p, h->io64, n, h->stream);
    h->launches += 5;
  }
  r->iterations = so.iterations;
  r->final_eps = so.eps;
  r->detach_rounds = rounds;
  r->status = so.status;
  r->stalled = so.stalls;
  r->depth = d;
  return BEM_OK;
}

int run_sweep(bem_ctx* h, const double* profile, const double* d_steps, int nsteps, double dgamma,
              const bem_opts* opts, bem_result* per_step, double* final_pressure,
              const double* p_state = nullptr, const uint8_t* S_state = nullptr) {
  g_err.clear();
  if (!h) return fail(BEM_EINVAL, "NULL handle");
  CKR(validate_ptr(profile, "profile"));
  CKR(validate_ptr(d_steps, "d_steps"));
  CKR(validate_ptr(per_step, "per_step"));
  if (nsteps < 1) return fail(BEM_EINVAL, "nsteps must be >= 1");
  SolveCfg cfg;
  CKR(parse_opts(opts, &cfg));
  const bool adhesive = dgamma > 0;
  for (int i = 0; i < nsteps; ++i)
    if (!isfinite(d_steps[i])) return fail(BEM_EINVAL, "depth %d is not finite", i);
  double pcrit = 0;
  if (adhesive) {
    if (fabs(h->dx - h->dy) > 1e-12 * h->dx)
      return fail(BEM_EINVAL, "adhesive contact needs square elements (Eq. 24)");
    for (int i = 1; i < nsteps; ++i)
      if (d_steps[i] > d_steps[i - 1]) return fail(BEM_EINVAL, "adhesive depths must not increase");
    pcrit = bem_p_crit(h->k, h->nu, h->E0, h->c0, dgamma, h->dx);
    if (!isfinite(pcrit)) return fail(BEM_EINVAL, "p_crit undefined for k=%g (Table 1 covers |k| <= 0.9)", h->k);
  }
  const size_t n = (size_t)h->nx * h->ny;
  h->timing = (cfg.flags & BEM_FLAG_TIME_PASSES) != 0;
  cudaEvent_t ev = nullptr;
  if (cfg.user) {
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, cfg.user));
    CK(cudaStreamWaitEvent(h->stream, ev, 0));
  }
  CKR(upload(h, h->h64, profile, n));
  int first_bad = BEM_OK;
  bool warm = false;  // a sweep starts from the initial guess, unless it resumes a state
  const bool resume = p_state != nullptr;
  if (resume) {
    // the state a previous sweep ended in: the pressure it returned (and, when
    // adhesive, its held contact set), in the form the next step starts from
    if (adhesive && !S_state) return fail(BEM_EINVAL, "resuming an adhesive sweep needs the contact set");
    CKR(upload(h, h->io64, p_state, n));
    if (cfg.precision == BEM_PREC_FP64) {
      CKR(ensure_fields<double>(h));
      CK(cudaMemcpyAsync(h->f64.p, h->io64, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CKR(ensure_fields<float>(h));
      launch_to_f32(h->io64, h->f32.p, n, h->stream);
      h->launches += 1;
    }
    if (adhesive) {
      CK(cudaMemcpyAsync(h->S, S_state, n, is_device_ptr(S_state) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         h->stream));
    } else {
      bem_result st{};
      CKR(collect<double>(h, h->io64, h->io64, 0, &st));
      warm = st.force > 0;  // as after the step that produced the state
    }
  }
  for (int i = 0; i < nsteps; ++i) {
    bem_result r{};
    if (!adhesive || (i == 0 && !resume)) {
      CKR(step_nonadhesive(h, cfg, d_steps[i], warm, &r));
      warm = r.force > 0;
      if (adhesive) {
        if (cfg.precision == BEM_PREC_FP64) launch_set_from_p<double>(h->f64.p, h->S, n, h->stream);
        else launch_set_from_p<double>(h->io64, h->S, n, h->stream);
        if (cfg.precision != BEM_PREC_FP64) launch_to_f32(h->io64, h->f32.p, n, h->stream);
        h->launches += 2;
      }
    } else {
      if (cfg.precision == BEM_PREC_FP64) CKR(step_adhesive_t<double>(h, cfg, d_steps[i], pcrit, &r));
      else CKR(step_adhesive_t<float>(h, cfg, d_steps[i], pcrit, &r));
    }
    per_step[i] = r;
    if (r.status != BEM_OK && first_bad == BEM_OK) first_bad = r.status;
    if (r.status == BEM_ENUMERIC) break;
  }
  if (final_pressure) CKR(download(h, final_pressure, h->io64, n));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  if (ev) {
    CK(cudaEventRecord(ev, h->stream));
    CK(cudaStreamWaitEvent(cfg.user, ev, 0));
    cudaEventDestroy(ev);
  }
  if (first_bad != BEM_OK) fail(first_bad, "solve finished with status %d", first_bad);
  return first_bad;
}

}  // namespace

extern "C" int bem_sweep(bem_handle h, const double* profile, const double* d_steps, int nsteps,
                         double dgamma, const bem_opts* opts, bem_result* per_step,
                         double* final_pressure) {
  return run_sweep(h, profile, d_steps, nsteps, dgamma, opts, per_step, final_pressure);
}

extern "C" int bem_sweep_from(bem_handle h, const double* profile, const double* d_steps, int nsteps,
                              double dgamma, const bem_opts* opts, const double* p_state,
                              const unsigned char* S_state, bem_result* per_step, double* final_pressure) {
  g_err.clear();
  if (!p_state) return fail(BEM_EINVAL, "p_state must not be NULL");
  return run_sweep(h, profile, d_steps, nsteps, dgamma, opts, per_step, final_pressure, p_state, S_state);
}

extern "C" int bem_contact_set(bem_handle h, unsigned char* S_out) {
  g_err.clear();
  if (!h || !S_out) return fail(BEM_EINVAL, "NULL argument");
  const size_t n = (size_t)h->nx * h->ny;
  CK(cudaMemcpyAsync(S_out, h->S, n, is_device_ptr(S_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BEM_OK;
}

extern "C" int bem_solve(bem_handle h, const double* profile, double d, double dgamma,
                         double d_preload, const bem_opts* opts, double* pressure_out,
                         bem_result* res) {
  if (!res) return fail(BEM_EINVAL, "res must not be NULL");
  if (dgamma > 0) {
    if (!(d_preload >= d)) return fail(BEM_EINVAL, "d_preload must be >= d");
    double ds[2] = {d_preload, d};
    bem_result rr[2];
    int rc = run_sweep(h, profile, ds, 2, dgamma, opts, rr, pressure_out);
    *res = rr[1];
    res->iterations += rr[0].iterations;
    return rc;
  }
  double ds[1] = {d};
  return run_sweep(h, profile, ds, 1, 0.0, opts, res, pressure_out);
}
