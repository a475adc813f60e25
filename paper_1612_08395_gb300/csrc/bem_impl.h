// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct bem_ctx;

namespace bem {

// One FFT length of the plan: 2^logL points, first DIF stage radix 2^r0
// (r0 = logL mod 3; 0 means radix 8), shared-memory swizzle and the row
// stride (in elements) of each transform's region in shared memory.
struct Geo {
  int logL, r0;
  int sa, sb, sc, sd;
  int rs;
};

// Per-length index tables on the device (int32):
//   so[ls * 8 + r] = swz(r << ls), ls = 0..13     (112 entries)
//   sp[k]          = swz(dig_pos(k)), k < 2^logL  (digit-reversed, swizzled)
constexpr int kSoEntries = 112;
void launch_geo_tables(int* so, int* sp, Geo g, int esize, cudaStream_t s);

// Launch geometry of the three convolution passes for one handle.
//   ny, nx: field rows and columns;  Px, Py: torus sides (powers of two
//   >= 2 Nx, 2 Ny, at least 32);  M = Px/2 (complex row-FFT length).
//   W: intermediate spectrum, M+1 rows (kx = 0..M) of `ny` complex values --
//   row kx holds column kx of the row transforms, so the column pass reads
//   contiguous memory.
struct Plan {
  int nx, ny, px, py, M;
  Geo gA;     // length M: row transforms of passes A and C
  Geo gB;     // length Py: column transforms of pass B
  int nbA;    // field rows per CTA in passes A and C (power of two)
  int lognbA;
  int nbB;    // spectrum columns per CTA in pass B
  int radixB; // pass B (convolution mode): radix-8 stages (Py/8 threads per
              // column) or radix-16 stages (Py/16 threads, 512 <= Py <= 8192)
  int gridA;  // = ceil(ny / nbA)
  int gridB;  // = ceil((M + 1) / nbB)
  int threadsA, threadsB;
  size_t smemA, smemB, smemC;
  int nsm;    // SMs of the device (persistent launches size their grids by it)
};

// Largest CTA of the radix-16 column pass for a length-2^LOGL column.
#define BEM_COL16_MAX_THREADS(LOGL) ((LOGL) >= 13 ? 512 : 256)

// Device-resident scalar state of one CG solve (FP64 throughout).
struct Scalars {
  double tol;        // stopping tolerance
  double tau, beta, delta, G, G_old, eps, bnorm, pcrit;
  double sum_p, sum_dp, n_ol, n_ic, str, eps_min;
  double stop2;      // fixed-set CG: stop once |g|^2 <= stop2 = (tol |b|)^2
  int max_iter, iter, done, status, have_tau, it_min;
  int nA;        // CTAs of the last pass A launch (its partials feed pass C)
  // Debug builds only: 1 = the first persistent pass A launch of the solve
  // waits on a barrier that nothing completes (tests the bounded wait)
  int inject;
  // Rows band0 .. band1 and columns col0 .. col1 hold every element of the
  // fixed contact set S (band0 > band1: S is empty); written by k_box at the
  // start of a fixed-set solve.
  int band0, band1, col0, col1;
  // CG iterations counted on the device, and the cap after which the solve
  // stops unconverged (the bound of the batched while-loop graph).
  int loops, max_loops;
  unsigned int cnt_a, cnt_c, cnt_r;  // last-block arrival counters
  // Sticky device error bits (kept across solves: init_scalars does not copy
  // this member); 1 = a kernel gave up waiting for its own asynchronous copies,
  // 2 = a bounds check of a debug build (-DBEM_DEBUG_CHECKS) failed.
  unsigned int kerr, pad2;
};

enum { SC_OK = 0, SC_NOCONV = 1, SC_NUMERIC = 2, SC_STALL = 3 };

// Pass A (row real-to-complex FFT) prologue modes.
enum PassAMode {
  A_PLAIN = 0,  // x = src
  A_PK_P = 1,   // Polonsky-Keer update of p (steps 7-8), partials sum|dp|, sum p, #overlap
  A_PK_T = 2,   // t = (p > 0) ? g + beta t : 0
  A_CG_T = 3,   // fixed-set CG: p -= tau t, g -= tau r (the previous step, if any), t = S ? g + beta t : 0
  A_TORUS = 4   // x = K on the even torus (spectrum set-up, FP64)
};
// Pass C (row complex-to-real FFT) epilogue modes.
enum PassCMode {
  C_PLAIN = 0,  // dst = u
  C_PK_G = 1,   // g = u + c; partial sum_{p>0} g^2, #(p>0); last block: eps, delta, beta
  C_PK_R = 2,   // partials sum_{p>0} g t, sum_{p>0} r t; last block: tau
  C_CG_R = 3,   // r = S ? u : 0 (stored); partials t.r, g.r, r.r, g.g; last block: stop test, tau, beta
  C_CG_G = 4,   // g = S ? u + c : 0; partials sum g^2, sum_S c^2; last block: G, bnorm
  C_GAP = 5     // g = u + c (no mask) -- FP64 residual of the refinement
};
enum PassBMode { B_CONV = 0, B_SPECTRUM = 1 };

template <typename T>
struct Fields {
  T* p;        // pressure
  T* g;        // gap / residual
  T* t;        // CG direction
  T* r;        // A K t
  T* c;        // offset h - d (or a residual offset)
  uint8_t* S;  // fixed contact set (adhesive / refinement)
  const T* src;  // A_PLAIN source
  T* dst;        // C_PLAIN destination
};

template <typename T>
struct PassArgs {
  Plan pl;
  Fields<T> f;
  void* W;              // C<T>[(M+1) * rows_w]
  int rows_w;           // row length of W (= ny, or Py for the spectrum)
  int nrows_in;         // rows fed to pass A (= ny, or Py for the torus)
  int ncols_in;         // columns fed to pass A (= nx, or Px for the torus)
  const double* kq64;   // A_TORUS: influence quarter, (Py/2+1) x (M+1)
  const T* khat;        // B_CONV: spectrum quarter, transposed: [kx][ky], ky <= Py/2
  const void* twA;      // stage twiddle tables, length M (C<T>)
  const void* twB;      // stage twiddle tables, length Py (C<T>)
  const void* twB16;    // stage twiddle tables of the radix-16 column pass, length Py (C<T>)
  const void* twS;      // exp(-i pi k / M), k = 0..M (C<T>): real-FFT split
  const int* soA;       // index tables of length M and Py (see Geo)
  const int* spA;
  const int* soB;
  const int* spB;
  double* khat64_out;   // B_SPECTRUM outputs ([kx][ky])
  float* khat32_out;
  double uscale;        // pass C: A / (Px Py)
  double* partA;        // per-CTA partials, 4 per CTA
  double* partC;
  Scalars* sc;
  unsigned int* kerr;   // sticky error word (may be null: errors then go unreported)
  int use_band;         // 1: fixed-set CG loop, the passes work on rows sc->band0 .. band1
                        // only; 2: the plain transform of the FP64 residual (A_PLAIN,
                        // B_CONV, C_GAP) works on rows band_lo .. band_hi only
  int band_lo, band_hi; // use_band = 2: rows holding every nonzero input; the outputs of
                        // the other rows are left unwritten
  // Tensor map (device memory) of W as (M+1) rows of 2 rows_w reals with boxes
  // of 2 nbA reals x w_box rows: the persistent pass C stages a row group's W
  // columns with 2D TMA loads.  Null: 16-byte cp.async instead.
  const void* tmW;
};

// Rows of W per box of the TMA staging, and rows of pass C's W staging area
// (whole boxes: the last box of a long transform reads past row M, zero-filled).
__host__ __device__ constexpr int w_box_rows(int M) { return M + 1 <= 256 ? M + 1 : 256; }
__host__ __device__ constexpr int w_stage_rows(int M) {
  return (M + 1 + w_box_rows(M) - 1) / w_box_rows(M) * w_box_rows(M);
}
// Dynamic shared memory of the persistent pass C: transform rows (128-byte
// aligned end, the TMA destination follows) | W staging | epilogue staging.
__host__ __device__ constexpr size_t pass_c_w_offset(size_t smemC) { return (smemC + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t pass_c_smem(size_t smemC, int M, int nb, int cx_bytes, size_t epi_bytes) {
  return pass_c_w_offset(smemC) + (((size_t)cx_bytes * w_stage_rows(M) * nb + 15) & ~(size_t)15) + epi_bytes;
}

template <typename T> void launch_pass_a(const PassArgs<T>& a, int mode, cudaStream_t s);
template <typename T> void launch_pass_b(const PassArgs<T>& a, int mode, cudaStream_t s);
template <typename T> void launch_pass_c(const PassArgs<T>& a, int mode, cudaStream_t s);

// The same passes over n instances of one size class at once (blockIdx.y =
// instance); a0 is any of them (its plan, row and column counts), arr the
// device array of all n instances' arguments.  Only the CG-loop modes and the
// persistent row passes (rows of a multiple of 16 elements) are provided.
template <typename T> void launch_pass_a_mi(const PassArgs<T>& a0, int mode, const PassArgs<T>* arr, int n,
                                            cudaStream_t s);
template <typename T> void launch_pass_b_mi(const PassArgs<T>& a0, const PassArgs<T>* arr, int n, cudaStream_t s);
template <typename T> void launch_pass_c_mi(const PassArgs<T>& a0, int mode, const PassArgs<T>* arr, int n,
                                            cudaStream_t s);
// Sets the while-loop condition `cond` to "some instance is not done".
template <typename T> void launch_batch_ctl(const PassArgs<T>* arr, int n, unsigned long long cond, cudaStream_t s);

// Column pass on the tensor cores (tc_colpass.cu): an opt-in experiment
// (BEM_TC_COLUMN_PASS=1) for the FP32 column pass of a 4096-point column over
// the whole grid; tc_column_pass_applies tells whether a launch qualifies.
bool tc_column_pass_enabled();
bool tc_column_pass_applies(const PassArgs<float>& a);
int launch_pass_b_tc(const PassArgs<float>& a, cudaStream_t s);
int tc_column_pass_setup();  // once per device, when enabled

// Elementwise kernels.
template <typename T> void launch_pk_init(const Plan& pl, const double* h64, double d, T* c, T* p,
                                          T* t, int warm, int ngrid, cudaStream_t s);
// The pending last update of a fixed-set CG solve (if pass C left one).
template <typename T> void launch_cg_finish(const Plan& pl, Fields<T> f, const Scalars* sc, int ngrid,
                                            cudaStream_t s);
void launch_box(const Plan& pl, const uint8_t* S, Scalars* sc, cudaStream_t s);
void launch_box_overlap(const Plan& pl, const double* h, double d, Scalars* sc, cudaStream_t s);
void launch_box_copy64(const double* src, int nx, int ny, int x0, int y0, double* dst, int bx, int by,
                       double fill, cudaStream_t s);
// Copy the box [x0, x0+bx) x [y0, y0+by) of the nx x ny fields p, c, S into
// bx x by sub-grid fields (zero where the box leaves the grid), and back for p.
template <typename T> void launch_box_gather(const T* p, const T* c, const uint8_t* S, int nx, int ny, int x0,
                                             int y0, T* bp, T* bc, uint8_t* bS, int bx, int by, cudaStream_t s);
template <typename T> void launch_box_scatter(const T* bp, T* p, int nx, int ny, int x0, int y0, int bx, int by,
                                              cudaStream_t s);
template <typename T> void launch_detach(const Plan& pl, Fields<T> f, double* part, Scalars* sc,
                                         int ngrid, cudaStream_t s);
template <typename T> void launch_stats(const Plan& pl, const T* p, const T* g, const uint8_t* S,
                                        int use_set, double* part, double* out, int ngrid,
                                        cudaStream_t s);
template <typename T> void launch_convert_in(const double* src, T* dst, size_t n, cudaStream_t s);
template <typename T> void launch_convert_out(const T* src, double* dst, size_t n, cudaStream_t s);
template <typename T> void launch_offset(const double* h64, double d, T* c, size_t n, cudaStream_t s);
template <typename T> void launch_set_from_p(const T* p, uint8_t* S, size_t n, cudaStream_t s);
template <typename T> void launch_mask_field(T* x, const uint8_t* S, size_t n, cudaStream_t s);
void launch_refine_apply(double* p64, const float* dp, double dscale, const uint8_t* S, int project,
                         size_t n, cudaStream_t s);
void launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s);
void launch_to_f32_scaled(const double* src, double scale, float* dst, size_t n, cudaStream_t s);
// S = (p > 0) or (g < 0): active set of the refinement sweep.
void launch_active_set(const double* p, const double* g, uint8_t* S, size_t n, cudaStream_t s);

// The default launch plan of a grid (the one bem_create gives a handle) and
// whether a plan's shapes are launchable (warps, launch bounds, shared memory).
Plan default_plan(int nx, int ny, int px, int py, int esize, int nsm);
bool plan_fits(const Plan& pl, int esize);
// Once per device (with it current): shared-memory opt-ins of the pass kernels
// and the quadrature nodes.  Returns BEM_OK or a BEM_E* code with the message set.
int device_setup(int dev);

// Batching of CG loops across solves that run concurrently in one process (the
// request server): a thread whose solve reaches its CG loop joins the batcher;
// the loops of all solves waiting at that moment run as one while-loop graph
// per size class, every pass launched once over all of them (blockIdx.y =
// instance), each instance stopping at its own convergence.  Results are
// bitwise those of the solve run alone.
struct LoopBatcher;
LoopBatcher* batcher_create();               // on the current device
void batcher_destroy(LoopBatcher* b);
void batcher_enter(LoopBatcher* b);          // a thread starts a solve that may join
void batcher_leave(LoopBatcher* b);          // ... and ends it
void attach_batcher(::bem_ctx* h, LoopBatcher* b);  // a handle's loops (and its sub-contexts') join b
// Adds the batched loop graphs launched so far and the solves' loops they carried.
void batcher_stats(LoopBatcher* b, long long* launches, long long* instances);

// Record `msg` as the thread's last error and return `code`.
int set_error(int code, const char* msg);

// Twiddle tables of one FFT length (stage tables, 2^logL entries reserved) and
// of the real-FFT split (M+1 entries), FP64 and FP32 copies.
void launch_twiddles(double2* t64, float2* t32, int logL, cudaStream_t s);
void launch_split_twiddles(double2* t64, float2* t32, int M, cudaStream_t s);
void launch_twiddles16(double2* t64, float2* t32, int logL, cudaStream_t s);
// Geometry (swizzle, first-stage radix, row stride) of a length-2^logL
// transform with `rows` transforms per CTA, for elements of esize bytes.
Geo make_geo(int logL, int rows, int esize);

// Influence coefficients (FP64): Kq[dj*(hx) + di], 0 <= di < hx, 0 <= dj < hy.
int influence_init_nodes();
void launch_influence(double* Kq, int hx, int hy, double dx, double dy, double k, cudaStream_t s);


}  // namespace bem
