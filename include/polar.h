/* polar.h -- C ABI of the GB300 library for the implicit theta-weighted step on the
 * radius-angle-time mesh of the unit disk.
 *
 * The library advances  u_t + L u = f  on the unit disk in polar coordinates, with
 * Dirichlet data on r = 1, by the adjustable Crank-Nicolson scheme of Eq. (2.5)
 * (parabolic equation, Section 2.1) and of Section 3.2.1 (continuity equation).
 * The paper's weight a multiplies the OLD time level; this interface takes the
 * implicit weight  theta = 1 - a  (theta = 1/2 is Crank-Nicolson).  One step solves
 *
 *     (I/dt + theta L) U^{k+1} = (I/dt - (1-theta) L) U^k + theta F^{k+1} + (1-theta) F^k
 *
 * where F^k collects the source f(t_k) and the Dirichlet data g(t_k) of the ring
 * r = 1 (Eqs. 2.9, 2.11, 2.12; Section 3.2.3).
 *
 * Vector layout at this interface (the unknown ordering of Eq. 2.12): N = m*n + 1
 * doubles; element 0 is the origin, element 1 + j*m + (i-1) is the node
 * (r_i, theta_j), i = 1..m, j = 0..n-1.  Radial lines are contiguous.
 *
 * Spatial operators (Section 3.2):
 *  - POLAR_SCHEME_CONSERVATIVE: control-volume form.  Every face flux
 *    (diffusion D grad u and first-order upwinded drift v u) is shared by the two
 *    cells of the face, so the discrete mass balance is exact.  With v = 0 the ring
 *    rows are those of Section 3.2.1 (Section 2.1 when D = 1) and the origin row is
 *    the control-volume row of Section 3.2.2 (the Swarztrauber-Sweet row of
 *    Section 2.1 when D = 1 and the angles are uniform).
 *  - POLAR_SCHEME_PAPER: the printed stencils of Section 3.2.1 (scalar E at nodes,
 *    forward differences) and the printed origin row of Section 3.2.2.
 *
 * Every function returns 0 (POLAR_OK) or a negative error code; nothing throws across
 * the interface and polar_last_error() returns a message for the calling thread.
 * All GPU work runs on the CUDA stream given in polar_mesh_desc; the library has no
 * CPU fallback: without a usable CUDA device every call that needs one returns
 * POLAR_ECUDA.
 */
#ifndef POLAR_H
#define POLAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  POLAR_OK = 0,
  POLAR_EINVAL = -1,     /* bad argument; detected before any GPU work           */
  POLAR_ENOMEM = -2,     /* device allocation failed                             */
  POLAR_ECUDA = -3,      /* CUDA runtime error, or no device                     */
  POLAR_ENOCONV = -4,    /* solver did not reach the tolerance; state unchanged  */
  POLAR_ENONFINITE = -5, /* NaN/Inf in an input or in the solver; state unchanged */
  POLAR_ESTATE = -7      /* call out of order (e.g. step before set_coeffs)      */
};

enum { POLAR_SCHEME_CONSERVATIVE = 0, POLAR_SCHEME_PAPER = 1 };
enum { POLAR_FP64 = 0, POLAR_MIXED = 1 };   /* solver arithmetic                     */
enum { POLAR_HOST = 0, POLAR_DEVICE = 1 };  /* where a caller's pointer lives         */

typedef struct polar_ctx polar_ctx;

/* Device-memory hooks (memory management of the library; the paper has no counterpart).
 * alloc returns a device pointer to at least `bytes` bytes on the current device, aligned
 * to 256 bytes and usable by work on `stream` (the cudaStream_t of the context), or NULL
 * when it cannot; free gives back a pointer alloc returned, after every use of it on
 * `stream` has been enqueued.  `user` is the alloc_user of the mesh descriptor.  A binding
 * passes its framework's allocator here (e.g. the PyTorch caching allocator), so the
 * library's buffers come out of the framework's memory pool. */
typedef void* (*polar_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*polar_free_fn)(void* ptr, void* stream, void* user);

/* Mesh of Sections 2.1 / 3.1.  The caller owns r and theta; they are copied. */
typedef struct {
  int32_t nr;            /* m >= 2 unknown rings r_1..r_m                              */
  int32_t ntheta;        /* 4 <= n <= 16384 angles theta_0..theta_{n-1}                 */
  const double* r;       /* host, m+2 values, r[0] = 0 < r[1] < ... < r[m+1] = 1        */
  const double* theta;   /* host, n values, 0 <= theta[0] < ... < theta[n-1] < theta[0] + 2 pi */
  int32_t scheme;        /* POLAR_SCHEME_*                                              */
  int32_t precision;     /* POLAR_FP64 or POLAR_MIXED                                   */
  void* stream;          /* cudaStream_t for all work (NULL = legacy default stream)    */
  polar_alloc_fn alloc;  /* device allocations of the context; NULL: cudaMalloc         */
  polar_free_fn free;    /* required when alloc is set; NULL with alloc NULL: cudaFree  */
  void* alloc_user;      /* passed to alloc and free                                    */
} polar_mesh_desc;

/* polar_mesh_create: validates the mesh (strictly increasing r with r[0] = 0 and
 * r[m+1] = 1; strictly increasing theta spanning less than 2 pi; m >= 2; 4 <= n <= 16384,
 * the longest ring the line solves handle: up to 16 CTAs of a thread-block cluster per
 * ring; m n <= 2^31) and allocates every device buffer of the context on the current
 * device through desc->alloc (cudaMalloc when NULL), the multigrid levels included.
 * Later calls allocate through the same hook: polar_set_coeffs (source fields, on first
 * use) and polar_advance / polar_batch_advance (a schedule longer than any before it).
 * polar_mesh_destroy returns every buffer through desc->free (cudaFree when NULL).
 * Errors: POLAR_EINVAL (bad mesh or alloc without free, nothing allocated),
 * POLAR_ENOMEM (an allocation failed or was not 256-byte aligned; what was allocated is
 * freed), POLAR_ECUDA.  On success *out owns the buffers until polar_mesh_destroy. */
int polar_mesh_create(const polar_mesh_desc* desc, polar_ctx** out);
int polar_mesh_destroy(polar_ctx* ctx);

/* Coefficients of the equation (Eq. 2.1 / Eq. 3.1) and its data, in the face
 * layouts below; `memory` says whether ALL pointers are host or device pointers.
 * Arrays are copied; the caller keeps ownership.
 *   d_rface  (m+1)*n  D at radial faces (r_{i+1/2}, theta_j), i = 0..m, index j*(m+1)+i;
 *                     NULL means D = d_const everywhere.
 *   d_tface  m*n      D at angular faces (r_i, theta_{j+1/2}), i = 1..m, index j*m+(i-1),
 *                     theta_{n-1/2} halfway between theta_{n-1} and theta_0 + 2 pi;
 *                     NULL means D = d_const.
 *   v_rface  (m+1)*n  radial drift velocity (mu E_r) at radial faces, or NULL (no drift)
 *   v_tface  m*n      angular drift velocity (mu E_theta) at angular faces, or NULL
 *   e_node   N        scalar E at nodes (PAPER scheme only), or NULL (E = 0)
 *   b        N        reaction b >= 0 at nodes, or NULL (b = b_const)
 *   d0                D at the origin (PAPER scheme only)
 *   nsrc     Q in [0, 4] separable terms: f(t) = sum_q w_q(t) src[q], g(t) = sum_q w_q(t) bnd[q]
 *   src[q]   N        node values of the q-th source field (origin first)
 *   bnd[q]   n        values of the q-th Dirichlet field on r = 1 at theta_j
 * Errors: POLAR_EINVAL (NULL where an array is required, nsrc out of range),
 * POLAR_ENONFINITE (NaN or Inf in any array), POLAR_ECUDA. */
typedef struct {
  int32_t memory;
  const double* d_rface;
  const double* d_tface;
  const double* v_rface;
  const double* v_tface;
  const double* e_node;
  const double* b;
  double d_const;
  double b_const;
  double d0;
  int32_t nsrc;
  const double* src[4];
  const double* bnd[4];
} polar_coeffs;
int polar_set_coeffs(polar_ctx* ctx, const polar_coeffs* coeffs);

/* State U (N values in the interface layout) and its time t.  set copies in,
 * get copies out; `memory` says where u lives.  get before set -> POLAR_ESTATE. */
int polar_set_state(polar_ctx* ctx, const double* u, double t, int32_t memory);
int polar_get_state(polar_ctx* ctx, double* u, double* t, int32_t memory);

/* How a step is solved.  The new level X starts from U; the FP64 residual of the implicit
 * system is formed, and while its Jacobi-scaled max norm exceeds tol the residual (scaled
 * by its max norm) is handed to an inner Krylov solve whose correction is added to X in
 * FP64.  The inner solve is preconditioned by one V-cycle of a multigrid that coarsens
 * the radius only, smooths whole rings (periodic tridiagonal solves) and eliminates the
 * odd rings' radial couplings exactly.  It is conjugate gradients when the assembled
 * operator is symmetric (the conservative scheme without drift), BiCGStab otherwise.
 * POLAR_FP64 runs everything in FP64 (one inner solve normally suffices); POLAR_MIXED
 * runs the inner solve (vectors, operator, V-cycle) in FP32 and the residual and update
 * in FP64, and after a sweep that gains less than a factor 10 (FP32 cannot resolve rows
 * whose couplings exceed their row sums by about 1/eps32, e.g. long rings next to the
 * origin), or an FP32 solve that breaks down or reaches max_iter, finishes the step with
 * the FP64 inner solve (FP64 vectors, operator, V-cycle and ring factors, the factors
 * formed when first needed for the step's dt and theta).  Both paths stop at the same
 * FP64 tolerance.
 *
 * Separable operators -- uniform angles and ring coefficients that do not depend on the
 * angle (D, b and a radial drift depending on r only; the parabolic equation of
 * Section 2.1) -- have a direct inner solve instead: the discrete Fourier transform along
 * theta diagonalises the periodic angular coupling, each Fourier mode is one tridiagonal
 * system in r, and the origin row couples to the mean mode only (the Swarztrauber-Sweet
 * structure of Section 2.1).  It runs in FP64 in both precisions (O(N log n)); one
 * refinement sweep normally reaches the tolerance.  polar_set_coeffs detects
 * separability (coefficients equal across angles to 1e-9 relative, angular couplings
 * equal on both sides; the direct solve uses the coefficients of angle 0 and the FP64
 * refinement absorbs the difference); the transform holds rings of n <= 8192 angles when n is a power
 * of two, n <= 4096 otherwise.
 *
 * Solver controls (NULL -> defaults).
 *   tol         stop when max_i |r_i| / A_ii <= tol * max_i |U_i|, r = e - A U
 *               (Jacobi-scaled residual of the implicit system); default 1e-14
 *   max_iter    Krylov iterations per solve (FP64) or per inner solve (MIXED); default 500
 *   max_refine  outer refinement sweeps (FP64 residual evaluations); default 12
 *   inner_tol   reduction of the Jacobi-scaled max norm max_i |r_i| / A_ii that each FP32
 *               inner solve of the MIXED path reaches; default 1e-5.  Every inner solve
 *               (both paths) also goes at least as far as the outer test still needs:
 *               a tenth of tol * max_i |U_i| after its correction.
 *   method      POLAR_SOLVE_AUTO (default): the direct solve when the operator is
 *               separable, else the Krylov solve; POLAR_SOLVE_KRYLOV; POLAR_SOLVE_DIRECT
 *               (POLAR_EINVAL when the operator is not separable). */
enum { POLAR_SOLVE_AUTO = 0, POLAR_SOLVE_KRYLOV = 1, POLAR_SOLVE_DIRECT = 2 };
typedef struct {
  double tol;
  int32_t max_iter;
  int32_t max_refine;
  double inner_tol;
  int32_t method;
  int32_t reserved;
} polar_solver_opts;

/* 1 when the operator set by the last polar_set_coeffs is separable (the direct solve
 * applies), 0 when it is not, POLAR_ESTATE before polar_set_coeffs. */
int polar_is_separable(const polar_ctx* ctx);

typedef struct {
  int32_t iters;         /* Krylov iterations of all inner solves                     */
  int32_t refinements;   /* FP64 residual evaluations (one more than the inner solves) */
  int32_t status;        /* POLAR_OK or the error of this step                        */
  int32_t fp64_iters;    /* MIXED: of iters, those of FP64 inner solves, which the step
                            switches to once a sweep of FP32 refinement gains less than
                            a factor 10 (or an FP32 solve breaks down or hits
                            max_iter); 0 for FP64                                     */
  double scaled_resid;   /* final max |r_i| / A_ii / max |U_i|                        */
} polar_step_stats;

/* One theta-step of length dt from the current state (Eq. 2.5 / Section 3.2.1):
 * w_old[q] = w_q(t), w_new[q] = w_q(t + dt) weight the nsrc source/boundary fields.
 * theta in (0, 1], dt > 0.  On success U and t advance; on failure they keep their
 * values.  Errors: POLAR_EINVAL, POLAR_ESTATE (no coefficients or state),
 * POLAR_ENOCONV, POLAR_ENONFINITE, POLAR_ECUDA.  stats may be NULL. */
int polar_step(polar_ctx* ctx, double dt, double theta, const double* w_old,
               const double* w_new, const polar_solver_opts* opts, polar_step_stats* stats);

/* nsteps consecutive steps over the time levels t[0..nsteps] (t[0] must equal the
 * current time to 1e-12 relative; t strictly increasing: variable dt_k of Section 3.1).
 * w is (nsteps+1) x nsrc row-major: w[k*nsrc + q] = w_q(t[k]).  Stops at the first
 * failing step, whose index is recorded in the stats (stats has nsteps entries or is
 * NULL; entries after a failure have status POLAR_ESTATE). */
int polar_advance(polar_ctx* ctx, int32_t nsteps, const double* t, double theta,
                  const double* w, const polar_solver_opts* opts, polar_step_stats* stats);

/* Batched execution of independent instances (parameter sweeps, mesh-tuning studies):
 * each instance is an ordinary context (own mesh, coefficients, state, precision) on the
 * same device.  polar_batch_create records the contexts (the caller keeps ownership and
 * must keep them alive); polar_batch_advance advances every instance over its own
 * schedule of nsteps steps: t[i] holds nsteps+1 levels of instance i (t[i][0] its current
 * time), theta[i] its implicit weight, w[i] its (nsteps+1) x nsrc source weights (w may be
 * NULL when no instance has sources).  One CUDA graph advances every instance by one step
 * and is launched nsteps times on `stream`.  The instances are sorted by size into up to
 * 8 groups of about equal total points; each group's step is a parallel branch of the
 * graph, in which each kernel class runs as one launch per phase over the blocks of every
 * active instance of the group -- each instance keeps the
 * block partition of its own launches, so its result equals that of advancing it alone
 * bit for bit -- and the refinement and Krylov loops run while any instance still needs
 * them.  Per-instance masks, rewritten on the device wherever instances start or stop
 * (step start, refinement decisions, Krylov iterations), leave the finished instances out
 * of a launch's work.  Launches whose block or cluster shape differs between instances
 * (ring-solve tiles, coarsest-level solves) run once per shape.  count <= 1024.
 * The graph is rebuilt when a context changed.  stats
 * (count x nsteps, instance-major) or NULL.  An instance stops at its first failing step
 * (state kept at its last committed level, later entries POLAR_ESTATE); the others go on.
 * Returns the first error of any instance.  Contexts must not be stepped concurrently
 * from elsewhere while the batch runs. */
typedef struct polar_batch polar_batch;
int polar_batch_create(polar_ctx* const* ctxs, int32_t count, void* stream, polar_batch** out);
int polar_batch_destroy(polar_batch* batch);
int polar_batch_advance(polar_batch* batch, int32_t nsteps, const double* const* t,
                        const double* theta, const double* const* w,
                        const polar_solver_opts* opts, polar_step_stats* stats);
/* Number of CUDA kernels the batch's step graphs have launched (counted from the steps'
 * sweep and iteration counts). */
int64_t polar_batch_kernel_launches(const polar_batch* batch);

/* Steady problem L U = f (Eq. 2.1 / Eq. 3.1 without the time derivative): one solve of
 * the implicit system with alpha = 0 and theta = 1, f and the Dirichlet data the sources
 * weighted by w (nsrc values; NULL when nsrc = 0), started from the current state, which
 * it replaces; the time is unchanged.  L must be nonsingular (Dirichlet data on r = 1
 * make the diffusion operator so).  stats (one entry) or NULL.  Errors as polar_advance. */
int polar_solve_steady(polar_ctx* ctx, const double* w, const polar_solver_opts* opts,
                       polar_step_stats* stats);

/* Face drift of a potential: v = -mobility grad u of the context's current state u, the
 * radial component at the radial faces ((m+1) n values, layout of v_rface: (u_{i+1,j} -
 * u_{i,j}) / (r_{i+1} - r_i), u_{0,j} the origin, u_{m+1,j} = g_j) and the angular one at
 * the angular faces (m n values, layout of v_tface: (u_{i,j+1} - u_{i,j}) / (r_i
 * (theta_{j+1} - theta_j)), periodic).  g: n values of u on r = 1.  `memory` says where
 * g, v_rface and v_tface live.  Errors: POLAR_EINVAL, POLAR_ESTATE (no state), POLAR_ECUDA. */
int polar_face_drift(polar_ctx* ctx, double mobility, const double* g, double* v_rface,
                     double* v_tface, int32_t memory);

/* Electron-hole drift-diffusion with a self-consistent field (the carrier pair of
 * Section 3.1, both obeying Eq. 3.1, and the Poisson coupling of the outlook in
 * Section 4).  Three contexts on one mesh (conservative scheme, coefficients and states
 * set): the potential phi, whose operator is -div(eps grad phi) (D = eps, no drift) and
 * two of whose source fields (slots src_electrons, src_holes) the step fills with the
 * carrier densities, and the electrons and holes, whose drift the step sets to
 * v_c = -mobility[c] grad phi (e.g. mobility = -mu_n for electrons, +mu_p for holes);
 * their other coefficients stay as set.  One polar_gummel_step advances the pair from
 * t[0] to t[1] by Gummel's iteration: phi from the current densities
 * (polar_solve_steady, sources weighted by w_phi), the drifts from phi
 * (the face-drift kernel; the carriers' operators and multigrid hierarchies re-assembled
 * on the device, after which they take the Krylov inner solve), both carriers one
 * theta-step from their state at t[0] with that drift held over the step (one 2-instance
 * polar_batch; w[c] holds 2 x nsrc weights of carrier c at t[0] and t[1]); repeated
 * until max|phi_j - phi_{j-1}| / max|phi_j| <= tol (the absolute change when phi_j = 0),
 * at most max_iter potential solves.  With depth d > 0 the potential that sets the next
 * drift is Anderson's extrapolation x = g - sum_a gamma_a (dX_a + dF_a) over the last d
 * differences of the iterates x and residuals f = g - x (g the new potential), gamma the
 * least-squares fit of f by dF (normal equations by Cholesky, the oldest difference
 * dropped while a pivot is not above 1e-13 of the largest diagonal entry); it converges
 * in fewer solves, and at couplings where plain Gummel does not.  The carriers then hold
 * t[1]'s densities and phi the potential of those densities.  The object's device buffers
 * (3 N doubles, plus (3 + 2 d) N with depth d > 0, from the potential's allocator; each
 * carrier's face D, reaction and drift faces from its own) are freed with those contexts;
 * destroy the object before any of its contexts.  The carriers' face D and reaction are
 * those set when the object was created.
 * Errors: POLAR_EINVAL (mismatched meshes or scheme, bad slots, mobility, tol, max_iter
 * or depth), POLAR_ESTATE (coefficients or states missing), POLAR_ENOCONV (max_iter
 * reached: the carriers hold the last iterate), errors of the solves. */
typedef struct {
  double mobility[2];      /* electrons, holes: v_c = -mobility[c] grad phi            */
  int32_t src_electrons;   /* source slots of the potential filled with the densities  */
  int32_t src_holes;
  double tol;              /* on max|phi_j - phi_{j-1}| / max|phi_j|                   */
  int32_t max_iter;        /* potential solves per step                                */
  int32_t depth;           /* Anderson acceleration depth, 0 (plain Gummel) .. 5       */
} polar_gummel_desc;
typedef struct {
  int32_t iters;                /* potential solves of the step                        */
  int32_t status;
  double change;                /* the last max|phi_j - phi_{j-1}| / max|phi_j|         */
  polar_step_stats phi;         /* the last potential solve                            */
  polar_step_stats carrier[2];  /* the last step of the electrons and of the holes     */
} polar_gummel_stats;
typedef struct polar_gummel polar_gummel;
int polar_gummel_create(polar_ctx* phi, polar_ctx* electrons, polar_ctx* holes,
                        const polar_gummel_desc* desc, polar_gummel** out);
int polar_gummel_step(polar_gummel* g, const double* t, double theta, const double* const* w,
                      const double* w_phi, const polar_solver_opts* opts,
                      polar_gummel_stats* stats);
int polar_gummel_destroy(polar_gummel* g);

/* y = (alpha I + beta L) x for one vector x with homogeneous Dirichlet data
 * (g = 0): the matrix-free operator every kernel of the step is built on.
 * x and y hold N doubles in the interface layout, both on the host or both on the
 * device as `memory` says.  Used to check the operator against an assembled matrix. */
int polar_apply_operator(polar_ctx* ctx, double alpha, double beta, const double* x,
                         double* y, int32_t memory);

/* polar_apply_rows_noalloc: y = alpha x + beta L x for a 5-point polar operator given row
 * by row, for callers that cannot allocate device memory -- embedders whose device memory
 * is a fixed budget they hand out themselves, or pipelines that must not call cudaMalloc /
 * cudaFree between kernels (both may synchronise the device).  It needs no context and
 * allocates nothing.
 * The paper has no counterpart: this is a memory-management variant of
 * polar_apply_operator for operators the caller holds itself.
 *   m >= 2, 4 <= n <= 16384 (larger n: POLAR_EINVAL).
 *   R, W, E, S, N: device arrays of m n + 1 doubles in the interface layout (origin first,
 *     then node (r_i, theta_j) at 1 + j m + (i - 1)).  Row (i, j) of L is
 *       R x_ij + W (x_{i-1,j} - x_ij) + E (x_{i+1,j} - x_ij) + S (x_{i,j-1} - x_ij)
 *         + N (x_{i,j+1} - x_ij)
 *     with x_{0,j} = x_0 (the origin), x_{m+1,j} = 0 and j periodic; entry 0 of W, E, S, N
 *     is not read.
 *   o: device array of n doubles; the origin row is R[0] x_0 + sum_j o_j (x_{1,j} - x_0).
 *   x, y: device arrays of m n + 1 doubles; their ranges must not overlap (POLAR_EINVAL).
 *   stream: the cudaStream_t to enqueue on (NULL: legacy default stream).
 * Asynchronous: it returns once the work is enqueued (launch errors are reported).
 * Its only scratch is a fixed 128 KB array in device memory that the library reserves on
 * every device it is loaded on, until the process exits: the origin row's sum over the n
 * angles is staged there.  Every call shares that array, so calls that may overlap on the
 * GPU (different streams, or several host threads) race; serialise them.  Each call looks
 * up the array's address on the current device (the first call on a device is its set-up);
 * make that first call before any stream capture begins (a first call made during a
 * capture returns POLAR_ESTATE). */
int polar_apply_rows_noalloc(int32_t m, int32_t n, const double* R, const double* W,
                             const double* E, const double* S, const double* N,
                             const double* o, double alpha, double beta, const double* x,
                             double* y, void* stream);

/* Number of CUDA kernels this context has launched since creation. */
int64_t polar_kernel_launches(const polar_ctx* ctx);

/* Per-kernel timing for roofline measurements (not part of the method).
 * polar_timing_enable(ctx, 1) clears the counters and brackets every later launch of
 * the step's kernels with two CUDA events on the context's stream; 0 turns it off.
 * polar_timing_query returns, for kernel class `index` (0, 1, ... in order of first
 * launch; POLAR_EINVAL past the last), its name (NUL-terminated, truncated to
 * name_len), the number of timed launches, their summed device time in ms and the
 * summed algorithmic bytes of those launches (the words each launch must read and
 * write per grid point times the points it covers).  Querying synchronises the
 * stream.  Any output pointer may be NULL. */
int polar_timing_enable(polar_ctx* ctx, int32_t on);
int polar_timing_query(polar_ctx* ctx, int32_t index, char* name, size_t name_len,
                       int64_t* launches, double* total_ms, double* bytes);
/* The summed arithmetic of kernel class `index`'s timed launches: flops per point as the
 * kernel's source performs them (an FMA counts two; 0 for classes without a model) times
 * the points each launch covers.  POLAR_EINVAL past the last class. */
int polar_timing_flops(polar_ctx* ctx, int32_t index, double* flops);

const char* polar_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POLAR_H */
