/*
 * bem.h -- C ABI of the GB300 (sm_103a) boundary element solver for normal
 * non-adhesive and adhesive contact of a power-law graded elastic half-space,
 * E(z) = E0 (z/c0)^k with -1 < k < 1 (Li & Popov, arXiv 1612.08395).
 *
 * Conventions shared by every entry point
 *   - Grid: Nx x Ny square-or-rectangular elements of sides dx, dy; fields are
 *     row-major arrays of Ny rows of Nx doubles, element (iy, ix) at iy*Nx+ix.
 *     Element centres are x_i = (i - Nx/2 + 1/2) dx (domain centre on a node).
 *   - Sign: pressure p > 0 is compressive; the gap is g = A (K*p) + h - d with
 *     A = alpha(k,nu) (1-nu^2) c0^k / E0 (Eqs. 2, 7, 12) and h >= 0 the height
 *     of the indenter above its lowest point, d the indentation depth.
 *   - Pointers: every array argument may be a host pointer or a CUDA device
 *     pointer on the handle's device; the library tells them apart with
 *     cudaPointerGetAttributes.  The caller owns all buffers passed in; the
 *     handle owns its own device memory and stream.
 *   - Errors: functions return BEM_OK (0) or a negative BEM_E* code and set a
 *     thread-local message readable with bem_last_error().  No entry point
 *     aborts the process or traps the GPU; device-side waits are bounded.
 *   - Threads: one handle must not be used by two host threads at once.
 *     Distinct handles are independent.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BEM_OK 0
#define BEM_EINVAL (-1)   /* bad argument: k, nu, sizes, depths, pointers      */
#define BEM_ENOMEM (-2)   /* device or pinned allocation failed                 */
#define BEM_ENOCONV (-3)  /* CG hit max_iter; results are the last iterate      */
#define BEM_ENUMERIC (-4) /* NaN/Inf met in a reduction                         */
#define BEM_ETIMEOUT (-5) /* a bounded device-side wait gave up                 */
#define BEM_ECUDA (-6)    /* a CUDA runtime call failed, or (debug builds with
                             BEM_DEBUG_CHECKS) a kernel's bounds check failed  */
#define BEM_ECANCELED (-7) /* a server job was cancelled before it started       */

/* Arithmetic of the transform and the fields.  BEM_PREC_FP64: everything in
 * FP64 (the plain path).  BEM_PREC_FP32: FFT passes and fields in FP32, CG
 * scalars and all reductions in FP64.  BEM_PREC_FP32_REFINE: FP32 solve, then
 * FP64-residual refinement sweeps on the final contact set. */
#define BEM_PREC_FP64 0
#define BEM_PREC_FP32 1
#define BEM_PREC_FP32_REFINE 2

/* Record CUDA events around the three transform passes of the first CG
 * iteration of every fourth captured chunk of 8 iterations, the first chunk of
 * every solve included (read back with bem_pass_times). */
#define BEM_FLAG_TIME_PASSES 1

typedef struct bem_ctx *bem_handle;

typedef struct {
  double tol;         /* stopping tolerance; 0 = default 1e-10 (FP64) / 1e-6 (FP32) */
  int max_iter;       /* CG iteration cap per solve; 0 = default 20000               */
  int precision;      /* BEM_PREC_*                                                  */
  int refine_sweeps;  /* FP32_REFINE: max refinement sweeps; 0 = default 3           */
  int flags;          /* BEM_FLAG_* bits, 0 = none                                   */
  void *stream;       /* cudaStream_t to order work after; NULL = handle's own      */
} bem_opts;

typedef struct {
  double force;             /* F = dx dy sum p  (Sec. 3.1: "sum of pressures")    */
  double area;              /* dx dy * number of elements in contact              */
  double contact_radius;    /* sqrt(area / pi)                                     */
  double final_eps;         /* last CG stopping measure                            */
  double max_gap_violation; /* max over contact of |g|, and of -g off contact      */
  double depth;             /* d of this solve                                     */
  int iterations;           /* CG iterations (all rounds of this step)             */
  int detach_rounds;        /* adhesive: detach-and-resolve rounds                 */
  int contact_count;        /* elements in contact                                 */
  int status;               /* BEM_OK or BEM_ENOCONV / BEM_ENUMERIC                */
  int stalled;              /* CG solves of this step that stopped because their
                               stopping measure found no new minimum for 200
                               iterations (the arithmetic's rounding floor) while
                               still above the tolerance; counted as converged    */
} bem_result;

/* ---------------------------------------------------------------------------
 * bem_create: validate, compute A (Eqs. 2-4, 12), tabulate the influence
 * coefficients K(di, dj) of Eq. 9 for 0 <= di <= Px/2, 0 <= dj <= Py/2 in FP64
 * on the device, wrap them evenly onto the Px x Py torus (Px, Py = powers of two
 * >= 2 Nx, 2 Ny, at least 32), and take its spectrum (Eq. 13: FFT(K)), kept as
 * the real quarter in FP64 and FP32.
 *   Nx, Ny : 2..4096;  dx, dy > 0;  -1 < k < 1;  -1 < nu <= 0.5 with
 *   beta(k,nu)^2 > 0 (Eq. 4);  E0 > 0;  c0 > 0;  out != NULL.
 * The handle creates its own non-blocking stream on the current device.
 * Returns BEM_EINVAL, BEM_ENOMEM or BEM_ECUDA on failure (*out untouched).
 * The first handle of each grid size in a process times a few launch shapes
 * of the FP32 transform passes (rows per CTA of the row passes, columns per
 * CTA of the column pass; a few milliseconds) and keeps the fastest for every
 * later handle of that size (bem_get_info reports them).  BEM_AUTOTUNE=0 in
 * the environment keeps the default shapes. */
int bem_create(int Nx, int Ny, double dx, double dy, double k, double nu, double E0, double c0,
               bem_handle *out);

void bem_destroy(bem_handle h);

/* Thread-local text of the last error ("" if none). */
const char *bem_last_error(void);

/* ---------------------------------------------------------------------------
 * Non-adhesive (dgamma <= 0): solve the contact problem p >= 0, g >= 0,
 * p g = 0 at depth d by the constrained conjugate-gradient method (Sec. 2.1,
 * Polonsky & Keer), each iteration applying u = A K*p as the zero-padded FFT
 * convolution of Eq. 13.
 * Adhesive (dgamma > 0, Sec. 3.1): preload non-adhesively to d_preload (>= d),
 * then hold the contact area, solve for p at depth d, detach every element with
 * tensile stress -p > p_crit (Eq. 24, corrected c1 of Table 1), and repeat
 * until none detaches.  Requires dx == dy (Eq. 24 is for square elements).
 *   profile      : Nx*Ny heights h >= 0 (host or device)
 *   opts         : NULL for defaults
 *   pressure_out : Nx*Ny FP64 pressures, may be NULL
 *   res          : must not be NULL
 * Returns BEM_OK, BEM_ENOCONV (res filled), BEM_ENUMERIC, BEM_EINVAL, BEM_ECUDA. */
int bem_solve(bem_handle h, const double *profile, double d, double dgamma, double d_preload,
              const bem_opts *opts, double *pressure_out, bem_result *res);

/* ---------------------------------------------------------------------------
 * Load-unload sweep over nsteps depths (Figs. 3b, 6, 7): each step starts from
 * the previous step's pressures.  dgamma <= 0: every step is a non-adhesive
 * solve.  dgamma > 0: step 0 is the non-adhesive preload at d_steps[0] and steps
 * 1.. are adhesive pull-off steps (Sec. 3.1 algorithm); d_steps must then be
 * non-increasing and dx == dy.  per_step[nsteps] receives one result per step;
 * final_pressure (Nx*Ny, may be NULL) the last step's pressures.
 * Returns the first non-OK status met (remaining steps still run unless the
 * error is BEM_EINVAL / BEM_ECUDA / BEM_ENUMERIC). */
int bem_sweep(bem_handle h, const double *profile, const double *d_steps, int nsteps,
              double dgamma, const bem_opts *opts, bem_result *per_step, double *final_pressure);

/* ---------------------------------------------------------------------------
 * Checkpoint and resume of a sweep.  The state a sweep ends in is the pressure
 * it returns in final_pressure and, for an adhesive sweep (Sec. 3.1), the held
 * contact set.  bem_contact_set copies that set (Nx*Ny bytes, 1 = held, host or
 * device memory) after bem_sweep / bem_sweep_from / bem_solve.
 * bem_sweep_from continues a sweep from such a state: the same arguments as
 * bem_sweep plus p_state (Nx*Ny FP64, required) and S_state (required when
 * dgamma > 0, ignored otherwise).  An adhesive resume starts directly with the
 * held-set step at d_steps[0] (no preload); a non-adhesive one warm-starts from
 * p_state as the interrupted sweep would have.  With the same precision, a sweep
 * split into two calls at any step gives the results of the single call,
 * bitwise.  Returns as bem_sweep; BEM_EINVAL if a required state is NULL. */
int bem_sweep_from(bem_handle h, const double *profile, const double *d_steps, int nsteps, double dgamma,
                   const bem_opts *opts, const double *p_state, const unsigned char *S_state,
                   bem_result *per_step, double *final_pressure);
int bem_contact_set(bem_handle h, unsigned char *S_out);

/* ---------------------------------------------------------------------------
 * Request server: many independent solves in flight on the current device.
 *
 * bem_server_create starts nworkers host threads; each runs one job at a time
 * on its own CUDA stream, so up to nworkers solves overlap on the GPU.  A job
 * is admitted when its device-memory footprint fits hbm_budget_bytes next to
 * the running jobs and the cached handles; a job that does not fit yet lets
 * later jobs that do fit go first, and idle cached handles are evicted least
 * recently used first.  Handles (influence spectra) are cached by
 * (Nx, Ny, dx, dy, k) and reused with bem_set_material for nu, E0, c0.
 * Results are deterministic: a job's outputs do not depend on what else runs.
 *
 * bem_job: the arguments of one bem_sweep (a single solve is nsteps = 1; an
 * adhesive solve is {d_preload, d}).  The job struct is copied on submit; the
 * arrays it points to (profile, d_steps, per_step, final_pressure) belong to
 * the caller and must stay valid until the job's completion is polled.
 * opts.stream is ignored (each worker uses its handle's stream).
 * bem_server_submit: BEM_EINVAL on bad arguments, BEM_ENOMEM if the job alone
 *   exceeds the budget.
 * bem_server_poll: moves up to max completion records into out, waiting up to
 *   wait_ms for the first; returns how many.  Times are seconds since create.
 * bem_server_cancel: removes the job with this tag if it is still queued (not
 *   started); its completion record then carries BEM_ECANCELED.  Returns BEM_OK
 *   when cancelled, BEM_EINVAL when no queued job has the tag (already running,
 *   finished or unknown).
 * bem_server_pending: jobs queued or running.
 * bem_server_bytes: device bytes accounted to cached and running handles.
 * bem_server_loop_stats: CG-loop batching so far.  Jobs running at the same
 *   time on one device share their CG loops: when a job's solve reaches its
 *   loop it joins the loops waiting at that moment (all jobs in flight, or
 *   those that arrived within 200 us), and the loops of one size class (grid,
 *   torus, launch shapes, precision and loop kind) run as one while-loop graph
 *   in which every transform pass is a single launch over all of them, each
 *   instance stopping at its own convergence (its CTAs return at once when it
 *   is done).  *launches = such graphs launched, *loops = the solves' loops they
 *   carried.  Results are bitwise those of the job run alone.
 *   BEM_BATCH_LOOPS=0 in the environment makes every job run its own loops.
 * bem_server_footprint: the bytes admission reserves for a job on an Nx x Ny
 *   grid (a handle after FP32 and FP64 solves plus its set-up workspace);
 *   0 for a grid outside 2..4096.
 * bem_server_destroy: finishes the queued jobs, then frees everything. */
typedef struct {
  int Nx, Ny;
  double dx, dy, k, nu, E0, c0;
  const double *profile;
  const double *d_steps;
  int nsteps;
  double dgamma;
  bem_opts opts;
  bem_result *per_step;
  double *final_pressure;
  long long tag;
} bem_job;

typedef struct {
  long long tag;
  int status;
  double t_submit, t_start, t_end;
  int device;  /* CUDA device the job ran on (-1: cancelled before it started) */
} bem_completion;

typedef struct bem_server *bem_server_handle;

/* bem_server_create: nworkers workers on the current device.
 * bem_server_create_on: workers_per_device workers on each of the ndev listed
 *   devices, each device with its own budget of hbm_budget_per_device bytes and
 *   its own handle cache.  A job runs wholly on one device (independent solves
 *   need no exchange between devices); bem_server_place decides which. */
int bem_server_create(int nworkers, size_t hbm_budget_bytes, bem_server_handle *out);
int bem_server_create_on(int ndev, const int *devices, int workers_per_device,
                         size_t hbm_budget_per_device, bem_server_handle *out);

/* Placement of one job across devices (host-only; the server calls it for
 * every queued job, and it is exported so the policy can be checked without a
 * GPU).  views[i] describes device i: its budget, the bytes accounted to it
 * (running jobs and cached handles), of those the bytes of idle cached handles
 * that may be evicted (evictable) and, when it holds an idle cached handle for
 * the job's spectrum key, that handle's bytes (has_cached, cached_bytes), and
 * its idle workers.  A device qualifies when it has an idle worker and the job
 * (need bytes, less its cached handle's) fits its budget once idle handles are
 * evicted.  Among those it prefers one with a cached handle, then the one with
 * the most budget left after the job, then the lower index.  Returns the
 * device's position in views, or -1 when none qualifies now. */
typedef struct {
  size_t budget, used, evictable, cached_bytes;
  int idle_workers, has_cached;
} bem_device_view;
int bem_server_place(int ndev, const bem_device_view *views, size_t need);
int bem_server_submit(bem_server_handle s, const bem_job *job);
int bem_server_poll(bem_server_handle s, bem_completion *out, int max, int wait_ms);
int bem_server_cancel(bem_server_handle s, long long tag);
int bem_server_pending(bem_server_handle s);
size_t bem_server_bytes(bem_server_handle s);
int bem_server_loop_stats(bem_server_handle s, long long *launches, long long *loops);
size_t bem_server_footprint(int Nx, int Ny);
void bem_server_destroy(bem_server_handle s);

/* ---------------------------------------------------------------------------
 * Building blocks, exposed for verification.
 *
 * bem_influence_table: copy the FP64 influence coefficients K(di, dj) of Eq. 9
 *   (integral of (a^2+b^2)^-(1+k)/2 over the element at offset (di, dj)) into
 *   out[dj*(Px/2+1) + di], 0 <= di <= Px/2, 0 <= dj <= Py/2.
 * bem_spectrum: copy the FP64 real quarter of FFT(K) on the Px x Py torus into
 *   out[ky*(Px/2+1) + kx], 0 <= kx <= Px/2, 0 <= ky <= Py/2 (unnormalised).
 * bem_convolve: u = A K*p (Eq. 7 via Eq. 13) for one Nx*Ny field, in the given
 *   precision (BEM_PREC_FP64 or BEM_PREC_FP32); p and u are FP64 arrays. */
int bem_influence_table(bem_handle h, double *out);
int bem_spectrum(bem_handle h, double *out);
int bem_convolve(bem_handle h, int precision, const double *p, double *u);

typedef struct {
  int Nx, Ny, Px, Py;
  double dx, dy, k, nu, E0, c0;
  double alpha;      /* Eq. 3                                        */
  double compliance; /* A = alpha (1-nu^2) c0^k / E0 (Eq. 12)         */
  size_t device_bytes; /* device memory held by the handle            */
  unsigned long long kernel_launches; /* kernels launched by this handle so far */
  int rows_per_cta;     /* FP32 row passes: grid rows per CTA            */
  int cols_per_cta;     /* FP32 column pass: columns per CTA             */
  int col_radix;        /* FP32 column pass: radix of its FFT stages (8 or 16) */
} bem_info;

int bem_get_info(bem_handle h, bem_info *info);

/* Change nu, E0, c0 of a handle (k, the grid and the influence spectrum stay):
 * only the prefactor A of Eq. 12 depends on them.  Same validation as
 * bem_create; BEM_EINVAL leaves the handle unchanged. */
int bem_set_material(bem_handle h, double nu, double E0, double c0);

/* Accumulated device time of the transform passes recorded under
 * BEM_FLAG_TIME_PASSES: ms[0..2] = total milliseconds of passes A (row FFT and
 * CG prologue), B (column FFT, spectrum multiply, inverse column FFT) and C
 * (inverse row FFT and CG epilogue), count[0] = number of timed iterations,
 * count[1] = of those, iterations of the fixed-set loop.  reset != 0 clears the
 * totals after reading.  Events are timed on the handle's stream, the stream
 * the passes run on. */
int bem_pass_times(bem_handle h, double ms[3], long long count[2], int reset);

/* Average algorithmic work of one timed launch of each pass (A, B, C), over
 * the launches counted by bem_pass_times (read it before a reset): bytes[i] =
 * the fields the pass's mode reads and writes, the intermediate W and (pass B)
 * the spectrum quarter; flops[i] = 5 L log2 L per complex FFT of length L,
 * halved where half the inputs are zero or half the outputs are dropped.  The
 * counts follow the torus and rows each launch worked on: in the fixed-set CG
 * of the adhesive algorithm (Sec. 3.1) the passes touch only the rows between
 * the first and last row of the contact set, and a solve whose contact set
 * fits a box of at most half the torus runs on a smaller torus (the operator
 * restricted to the set couples only elements of the set). */
int bem_pass_work(bem_handle h, double bytes[3], double flops[3]);

/* ---------------------------------------------------------------------------
 * bem_convolve_noalloc: u = A K*p in FP64 for callers that must not allocate
 * device memory.  The paper has no counterpart; this is a service of the
 * library.  Callers that cannot call cudaMalloc -- hosts whose device memory
 * belongs to a caching allocator or arena they must not bypass, loops that
 * cannot afford cudaMalloc's device-wide synchronisation -- get the same
 * transform as bem_convolve(FP64) without a handle and without any
 * allocation: its scratch is a 2 MiB static device array that every GPU
 * loading the library holds until exit.
 *   khat       : device pointer, the FP64 spectrum quarter exactly as
 *                bem_spectrum writes it for a handle of the same Nx, Ny
 *                ((Py/2+1) rows of Px/2+1 values)
 *   Nx, Ny     : 2..256
 *   compliance : A = alpha (1-nu^2) c0^k / E0 (bem_get_info().compliance)
 *   p, u       : device pointers to Nx*Ny FP64 fields (input, output)
 *   stream     : cudaStream_t to run on (NULL = legacy default stream)
 * The call is asynchronous on `stream` and uses the launch shapes a handle of
 * the same grid uses.  Its first call on a device does a one-time set-up with
 * that device current: it opts the transform kernels into the shared memory
 * they need (as bem_create does) and looks up the static array's device
 * address; make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents: calls whose work overlaps
 * on the GPU race and must be serialised by the caller.  Returns BEM_EINVAL
 * for sizes beyond the maximum, host pointers or NULL arguments, BEM_ECUDA on
 * a set-up or launch failure. */
int bem_convolve_noalloc(const double *khat, int Nx, int Ny, double compliance, const double *p,
                         double *u, void *stream);

/* ---------------------------------------------------------------------------
 * Host-only helpers (no GPU needed).
 * bem_alpha: alpha(k, nu) of Eq. 3 (NaN outside the valid range).
 * bem_c1_corrected: corrected c1(k) of Table 1 for -0.9 <= k <= 0.9; between
 *   grid points a natural cubic spline of ln c1 (NaN outside).
 * bem_p_crit: critical tensile stress of Eq. 24 for square elements of side
 *   delta, work of adhesion dgamma (NaN on invalid input). */
double bem_alpha(double k, double nu);
double bem_c1_corrected(double k);
double bem_p_crit(double k, double nu, double E0, double c0, double dgamma, double delta);

#ifdef __cplusplus
}
#endif
#endif /* BEM_GB300_H */
