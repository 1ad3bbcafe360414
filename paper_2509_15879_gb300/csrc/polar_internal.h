// Internal declarations shared by the host orchestration (polar_api.cu) and the
// kernels (polar_kernels.cu, polar_mg.cu).  Nothing here is part of the C ABI.
//
// Every vector of the solver lives in the "split-parity" layout of its multigrid
// level (m rings, n angles):
//   [0, kOrig)                          origin at 0, the rest zero padding
//   odd block   odd0 + j*ldo + k        ring 2k+1 (k < no = (m+1)/2), angle j
//   even block  even0 + j*lde + k       ring 2k+2 (k < ne = m/2),     angle j
// Radial lines stay contiguous within each parity block (one line of odd rings, one of
// even rings per angle), ldo/lde are multiples of 8 so every line starts on a 64-byte
// boundary, and padding entries are kept at zero by every kernel that writes a vector.
// The ring-by-ring (zebra) relaxation of the multigrid smoother touches one parity
// block at a time, so its loads use every byte of every sector, and the even block of
// a level holds exactly the rings that form the next coarser level.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace polar {

constexpr int kOrig = 8;

struct Shape {
  int m, n;        // rings, angles
  int no, ne;      // odd / even ring counts
  int ldo, lde;    // padded line lengths of the two blocks
  size_t odd0, even0, nv;
  __host__ __device__ size_t at(int i, int j) const {  // ring i in 1..m, angle j
    return (i & 1) ? odd0 + (size_t)j * ldo + (size_t)(i >> 1)
                   : even0 + (size_t)j * lde + (size_t)((i >> 1) - 1);
  }
};

inline Shape make_shape(int m, int n) {
  Shape s;
  s.m = m;
  s.n = n;
  s.no = (m + 1) / 2;
  s.ne = m / 2;
  s.ldo = (s.no + 7) & ~7;
  s.lde = (s.ne + 7) & ~7;
  s.odd0 = kOrig;
  s.even0 = s.odd0 + (size_t)n * s.ldo;
  s.nv = s.even0 + (size_t)n * s.lde;
  return s;
}

// One multigrid level of S = alpha V + beta (V L), the theta-step matrix scaled by
// the control volumes (Section 3.2; alpha = 1/dt, beta = theta).  Static parts come
// from the coefficients (V L in difference form, see polar_api.cu); the per-step parts
// (diag, line factors, origin scalars) are refreshed whenever alpha or beta change.
//   (S x)_ij = diag x_ij + beta (w x_{i-1,j} + e x_{i+1,j} + s x_{i,j-1} + nn x_{i,j+1})
//   (S x)_0  = diag0 x_0 + beta sum_j o_j x_{1,j}
// with x_{0,j} = x_0 and x_{m+1,j} = 0 (homogeneous Dirichlet ring).
template <typename T>
struct LevelView {
  Shape sh;
  // static (V L), nv each; o has n entries
  const T* vol;
  const T* rs;   // row sums of V L (reaction and drift divergence)
  const T* w;
  const T* e;
  const T* s;
  const T* nn;
  const T* o;
  const T* ia;   // interpolation weights of the odd rings from the coarser level:
  const T* ib;   //   x_{2k+1} = ia x_{2k} + ib x_{2k+2} (x_0 = origin, x_{m+1} = 0)
  // per step
  T* diag;       // nv: alpha vol + beta (rs - w - e - s - nn)
  T* rsum;       // nv, level 0 of the FP32 path: alpha vol + beta rs (row sums of S)
  double* dinv;  // nv, level 0 of the FP64 view: 1 / diag (the FP64 residual's Jacobi
                 //   scaling, formed once per step so that no kernel divides per point)
  T* fl;         // line factors of every ring's periodic angular line, nv each
  T* fui;
  T* fcu;
  T* fq;
  T* fring;      // 2 per ring, ring order (odd rings, then even): vf, 1/(1 + v.q)
  T* fz;         // n: coarsest level only, T_1^{-1} (beta w_1)
  double* sc;    // scalars: [0] diag0, [1] coarsest Schur denominator of the FP32 factors,
                 //          [2] sum_j o_j (static), [3] vol0, [4] rs0 (static),
                 //          [5] alpha vol0 + beta rs0, [6] Schur denominator, FP64 factors
};

// Scalars of one Krylov solve, kept on the device so that no iteration needs the host.
struct KrylovScalars {
  double rho, alpha, omega, beta;
  double rr0, rr, tol2;
  double dot[4];
  int done;        // 0 running, 1 converged, 2 breakdown, 3 non-finite, 4 iteration limit
  int iters;
  int max_iter;
  int pad0;
  double rmax;     // refinement reductions: max |r_i|, max |r_i| / S_ii, max |x_i|
  double smax;
  double xmax;
  unsigned int counter;
  unsigned int pad1;
  // step state of the device-side refinement loop (graph mode)
  int failed;      // 0, or the POLAR_* error code of this step
  int sweeps;      // FP64 residual evaluations
  int iters_total; // Krylov iterations of all inner solves
  int converged;
  double scaled;   // last Jacobi-scaled residual max |r_i| / S_ii / max |x_i|
  int halt;        // a step of the current schedule failed: the later ones are skipped
  int pad2;
  double sm_tol;   // inner solve: stop when max_i |r_i| / S_ii of its residual is below
  double sm;       //   sm_tol (sm: the last value)
  // mixed path: the FP32 refinement stalls where the FP32 operator cannot resolve the
  // correction (stiff rings); the rest of the step then takes FP64 Krylov solves over
  // the FP32 V-cycle
  int use64;       // 1: the remaining sweeps of this step use the FP64 Krylov solve
  int inner_done;  // `done` of the last inner solve
  double prev_scaled;
  int iters64;     // Krylov iterations of this step spent in FP64 Krylov solves
  int step_on;     // batched execution: this instance runs the current step (not halted)
  int refine_on;   // batched execution: this instance takes the current refinement sweep
  int sticky64;    // mixed path: steps left that start with the FP64 solve (set when a
                   //   step had to switch to it; the FP32 solve is tried again after)
  double sm_best;  // FP32 inner solve: best Jacobi-scaled residual so far and the
  int sm_best_it;  //   iteration that last halved it (no halving in kStallIters: stall)
  int pad3;
};

// An FP32 inner solve whose Jacobi-scaled residual has not halved in this many iterations
// has stalled (the step then switches to the FP64 solve); a switch makes this many
// following steps of the context start with the FP64 solve.
constexpr int kStallIters = 20;
constexpr int kStickySteps = 8;

// Result of one step of a device-side schedule (graph mode).
struct StepOut {
  int iters;       // Krylov iterations of all inner solves
  int sweeps;      // FP64 residual evaluations
  int status;      // POLAR_OK, the step's error, or POLAR_ESTATE if skipped
  int iters64;     // of iters: FP64 Krylov iterations of the mixed path's fallback
  double scaled;   // final Jacobi-scaled residual
};

// Parameters of one theta-step, read by the kernels from device memory (the first two
// entries are the Params of the level kernels).
struct StepParams {
  double alpha;      // 1 / dt
  double beta;       // theta
  double omt;        // 1 - theta
  double cf[4];      // source weights of both levels
  double cg[4];      // Dirichlet weights of both levels (negated)
  double tol;        // refinement tolerance on the Jacobi-scaled residual
  double inner_tol;  // relative residual reduction of each inner solve
  int max_iter;
  int max_refine;
  int do_refresh;    // the per-step refresh runs only when alpha or beta changed
  int mixed;         // 1: the context's inner solves are FP32 (mixed path)
};

// Conditional-node handle of a CUDA graph (0: not in a graph).
using CondHandle = unsigned long long;

// ---- batched execution (many instances, one launch per kernel class and phase)
// A batched launch serves a list of slots, one per instance it covers: slot s works on
// argument table entry s, instance `inst` of the batch, whose own launch would use a grid of
// vg blocks.  Which instances are active is read from a mask (one int per batch instance)
// that small kernels write between launches -- at the start of a step, after each
// refinement decision, after each Krylov iteration -- and that no kernel changes while a
// launch reads it.  Every block of a launch therefore derives the same list of work items
// (the active slots' virtual blocks, in slot order) and takes items blockIdx.x,
// blockIdx.x + gridDim.x, ...: item g is block vb of the instance's own grid, so the
// instance computes exactly what it computes alone (same partition, same reduction order).
struct BSlot {
  int inst;  // instance of the batch (position in the masks)
  int vg;    // blocks of the instance's own launch
};
constexpr int kMaxSlots = 1024;  // slots of one batched launch

// Prefix sums of the active slots' block counts in shared memory `pre` (nslots + 1
// entries); returns the number of work items.  All threads of the block call it.
__device__ __forceinline__ int batch_prefix(const BSlot* S, int nslots, const int* mask, int* pre) {
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  for (int s = tid; s < nslots; s += nt) pre[s + 1] = mask[S[s].inst] ? S[s].vg : 0;
  __syncthreads();
  if (tid < 32) {
    // lane l sums slots [l c, (l + 1) c), a warp scan of the chunk sums, then the prefixes
    const int c = (nslots + 31) / 32, s0 = tid * c, s1 = min(nslots, s0 + c);
    int sum = 0;
    for (int s = s0; s < s1; ++s) sum += pre[s + 1];
    int inc = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, inc, off);
      if (tid >= off) inc += o;
    }
    int run = inc - sum;
    if (tid == 0) pre[0] = 0;
    for (int s = s0; s < s1; ++s) {
      run += pre[s + 1];
      pre[s + 1] = run;
    }
  }
  __syncthreads();
  return pre[nslots];
}
// slot of work item g: the last s with pre[s] <= g
__device__ __forceinline__ int batch_slot(const int* pre, int nslots, int g) {
  int lo = 0, hi = nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Work-item loop of a batched kernel (see BSlot): s is the slot, vb / vg the virtual block
// of the instance's own grid.
#define POLAR_BATCH_LOOP(...)                                          \
  __shared__ int pre_[kMaxSlots + 1];                                  \
  const int total_ = batch_prefix(S, nslots, mask, pre_);              \
  for (int g_ = blockIdx.x; g_ < total_; g_ += gridDim.x) {            \
    const int s = batch_slot(pre_, nslots, g_);                        \
    const int vb = g_ - pre_[s], vg = S[s].vg;                         \
    __VA_ARGS__;                                                       \
  }

enum {
  G_ALL = 0,     // every instance
  G_STEP = 1,    // instances running this step (not halted by an earlier failure)
  G_REFINE = 2,  // instances in the current refinement sweep
  G_32 = 3,      // ... whose sweep takes the FP32 inner solve (mixed path)
  G_64 = 4       // ... whose sweep takes an FP64 inner solve (FP64 path, mixed fallback)
};
// Step data of one instance for the batched control kernels (one thread per instance).
struct CtlArgs {
  const StepParams* sched;  // the instance's schedule
  const int* kstep;         // its step counter
  int* kstep_w;
  StepParams* sp;           // its current step's parameters
  StepOut* out;             // its per-step results
  KrylovScalars* ks;
  int inst;                 // position in the batch (and in its masks)
  int pad;
};

__device__ __forceinline__ bool gate_pass(int g, const KrylovScalars* ks, const StepParams* sp) {
  switch (g) {
    case G_STEP: return ks->step_on != 0;
    case G_REFINE: return ks->refine_on != 0;
    case G_32: return ks->refine_on && !ks->use64;
    case G_64: return ks->refine_on && (ks->use64 || !sp->mixed);
    default: return true;
  }
}

struct Reduce {
  double* part;        // partial sums, kMaxBlocks * 4
  KrylovScalars* ks;   // device scalars
};
constexpr int kMaxBlocks = 2048;

// Per-step parameters read by the kernels from device memory: [0] alpha, [1] beta.
using Params = const double*;

int grid_for(size_t work, int threads);


// ----------------------------------------------------------------- kernel arguments
// (lone launches pass them by value; batched launches read one per instance from device
// memory)
// ------------------------------------------------------------------ point loops
// Tiles of TK consecutive rings of one parity block x TJ consecutive angles; every
// warp reads TK consecutive entries of a radial line (coalesced).
struct Tiling {
  int TK, TJ;
  int tko, tke, tj;  // tiles along k (odd, even) and along j
  int ntiles;
};

__host__ __device__ inline Tiling make_tiling(const Shape& sh) {
  Tiling t;
  const int kmax = sh.no > sh.ne ? sh.no : sh.ne;
  t.TK = 32;
  while (t.TK < kmax && t.TK < 256) t.TK <<= 1;
  t.TJ = 256 / t.TK;
  t.tko = (sh.no + t.TK - 1) / t.TK;
  t.tke = (sh.ne + t.TK - 1) / t.TK;
  t.tj = (sh.n + t.TJ - 1) / t.TJ;
  t.ntiles = (t.tko + t.tke) * t.tj;
  return t;
}

enum { M_APPLY = 0, M_RESID64 = 1, M_DOTV = 2, M_DOTT = 3 };

template <typename T>
struct StArgs {
  LevelView<T> L;
  Params par;
  const T* x;
  const T* b;   // M_RESID64: right-hand side
  T* y;
  const T* d1;  // M_DOTV: rhat; M_DOTT: s
  Reduce red;
  Tiling t;
};

struct RhsArgs {
  LevelView<double> L;
  const StepParams* sp;
  const double* u;
  double* e;
  int nsrc;
  const double* vsrc[4];
  const double* bnd[4];
  Reduce red;
  Tiling t;
};

// Arguments of the vector kernels of the Krylov solves (one struct for all of them; each
// kernel reads the fields its comment names).  Lone launches pass it by value, batched
// launches hold one per instance in device memory.
template <typename T>
struct VecArgs {
  size_t nv;
  T* v0;
  T* v1;
  T* v2;
  T* v3;
  T* v4;
  T* v5;
  T* v6;
  T* v7;
  const T* diag;
  const double* sc;
  const StepParams* sp;
  Reduce red;
  CondHandle cond;
  double* w0;  // FP64 vectors of the refinement kernels
  double* w1;
  int flag;
};

struct RefreshLevel {
  Shape sh;
  const double* vol;
  const double* rs;
  const double* w;
  const double* e;
  const double* s;
  const double* nn;
  const double* o;
  double* sc;
  void* diag;
  double* diag64;  // FP64 copy of diag when T is float (level 0 only), else null
  double* dinv;    // level 0: 1 / diag in FP64 (both precisions), else null
  void* rsum;      // row sums alpha vol + beta rs when T is float (level 0 only), else null
  void* fl;
  void* fui;
  void* fcu;
  void* fq;
  void* fring;
  void* fz;
  double* ws;  // 2 nv doubles: forward values y and pivot reciprocals (FP64)
  int ring0;   // first CTA of this level in the refresh grid
};
constexpr int kMaxLevels = 20;
struct RefreshArgs {
  RefreshLevel lv[kMaxLevels];
  int nlev;
  const StepParams* sp;
  const double* stamp;  // null: refresh when sp->do_refresh; else refresh unless stamp
                        // holds this step's (alpha, beta) (factors already current)
};

constexpr int RF = 4;     // rings per CTA
constexpr int TF = 128;   // threads per ring

template <typename T>
struct RingArgs {
  LevelView<T> L;   // level being smoothed
  LevelView<T> C;   // next coarser level (RING_POST, even rings)
  const T* b;       // right-hand side of this level
  T* x;             // solution of this level (updated in place)
  const T* X;       // solution of the coarser level (RING_POST)
  Params par;
  const int* done;
  int parity;       // 1: odd rings, 0: even rings (+ origin)
  int mode;
};

template <typename T>
struct RestrictArgs {
  LevelView<T> L;
  LevelView<T> C;
  const T* x;
  T* B;
  Params par;
  const int* done;
};

template <typename T>
struct CoarsestArgs {
  LevelView<T> L;
  const T* b;
  T* x;
  Params par;
  const int* done;
  const StepParams* sp;  // refresh form (k_schur): the step's parameters
  const double* stamp;
};

// ----------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return the number of kernels launched.

// Stencil of the fine level.  Modes:
//   apply:   y = S x
//   resid:   y = b - S x
//   dot v:   y = S x, alpha_k = rho / (rhat . y)            (BiCGStab)
//   dot t:   y = S x, omega = (t . s) / (t . t)             (BiCGStab)
template <typename T>
int launch_apply(const LevelView<T>& L, Params p, const T* x, T* y, cudaStream_t st, Reduce red);
template <typename T>
int launch_apply_dot(const LevelView<T>& L, Params p, const T* x, T* y, const T* d1, int mode,
                     cudaStream_t st, Reduce red);

// FP64 residual with reductions (rmax, Jacobi-scaled smax, xmax): r = b - S x
int launch_resid64(const LevelView<double>& L, Params p, const double* x, const double* b,
                   double* r, cudaStream_t st, Reduce red);

// FP64 right-hand side of the theta-step in S form:
//   e = (V/dt) u - (1 - theta) (V L) u + sum_q cf[q] Vsrc[q] - e_{m,j} sum_q cg[q] bnd[q][j]
// (cg already carries the weights of both time levels).
int launch_rhs(const LevelView<double>& L, const StepParams* sp, const double* u, int nsrc,
               const double* const* vsrc, const double* const* bnd, double* e, cudaStream_t st,
               Reduce red);

// Per-step refresh of every level: diag, angular line factors, origin scalars and the
// coarsest-level Schur data.  Factors are formed in FP64 and stored in T.  With `stamp`
// (2 doubles) the refresh runs unless stamp holds the step's (alpha, beta), and records
// them afterwards (factors formed only on demand); without it, when sp->do_refresh.
template <typename T>
int launch_refresh(const LevelView<double>* L64, LevelView<T>* LT, int nlev,
                   const StepParams* sp, double* ws, cudaStream_t st, double* stamp = nullptr);

// Multigrid V(1,1) cycle pieces (polar_mg.cu).  mode 0 = pre-smoothing (the level's
// x starts from zero), 1 = post-smoothing (x of the odd rings is corrected on the fly
// with the coarser level's solution X); parity 1 = odd rings, 0 = even rings + origin.
enum { RING_PRE = 0, RING_POST = 1 };
// tile shape of a ring solve launch: RW lines per CTA, TW chunk threads per line, P angles
// per thread, CS CTAs per cluster along the angle, ST staged operand loads (two CTAs/SM)
struct RingShape {
  int RW, TW, P, CS, ST;
};
template <typename T>
int launch_ring(const LevelView<T>& L, const LevelView<T>& C, const T* b, T* x, const T* X,
                Params p, int parity, int mode, const int* done, cudaStream_t st,
                const RingShape* shape = nullptr);
template <typename T>
void ring_candidates(int nlines, int n, std::vector<RingShape>& out);
template <typename T>
RingShape ring_default(int nlines, int n);
// right-hand side of the coarser level from the odd rings' residual after pre-smoothing
template <typename T>
int launch_restrict(const LevelView<T>& L, const LevelView<T>& C, const T* x, T* B, Params p,
                    const int* done, cudaStream_t st);
// exact solve of the coarsest level (origin + one ring)
template <typename T>
int launch_coarsest(const LevelView<T>& L, const T* b, T* x, Params p, const int* done,
                    cudaStream_t st);


// ----------------------------------------------------------------- batched launchers
// Each launches `grid` blocks over the slots S[0, nslots) with per-slot arguments A (see
// BSlot); the active instances are those with mask[inst] != 0.
template <typename T>
int launch_stencil_b(int mode, const StArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                     int grid, int TK, cudaStream_t st);
int launch_rhs_b(const RhsArgs* A, const BSlot* S, int nslots, const int* mask, int grid, int TK,
                 cudaStream_t st);
enum { V_BICG_INIT, V_BICG_S, V_BICG_UPDATE, V_BICG_P, V_CG_RHO, V_CG_P, V_CG_UPDATE,
       V_SCALE_CAST, V_CORRECT, V_COPY };
template <typename T>
int launch_vec_b(int kind, const VecArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                 int grid, cudaStream_t st);
enum { C_SCHED_BEGIN, C_DECIDE, C_AFTER_INNER, C_SCHED_END, C_SCHED_NEXT };
// one thread per instance of A (count of them); the gate is read live (G_*)
int launch_ctl_b(int kind, const CtlArgs* A, int count, int gate, cudaStream_t st);
// mask[A[k].inst] = gate passes (and, with need_running, done == 0) for the count
// instances of A; `cond` (if any) = whether any passes
int launch_mask_b(const CtlArgs* A, int count, int gate, int need_running, int* mask,
                  CondHandle cond, cudaStream_t st);
template <typename T>
int launch_refresh_b(const RefreshArgs* A, const BSlot* S, int nslots, const int* mask, int grid,
                     cudaStream_t st);
template <typename T>
int launch_ring_b(const RingShape& s, const RingArgs<T>* A, const BSlot* S, int nslots,
                  const int* mask, int grid, cudaStream_t st);
template <typename T>
int launch_restrict_b(const RestrictArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                      int grid, cudaStream_t st);
// coarsest-level solve (schur = 0) or its per-step Schur data (schur = 1), one CTA per
// instance of the (P, TW) shape coarsest_shape gives for its n
template <typename T>
int launch_coarsest_b(int P, int TW, int schur, const CoarsestArgs<T>* A, const BSlot* S,
                      int nslots, const int* mask, int grid, cudaStream_t st);
template <typename T>
void coarsest_shape(int n, int* P, int* TW);
// stamps[s] = (alpha, beta) of sps[s] for the active slots
int launch_stamp_b(const BSlot* S, int nslots, const int* mask, double* const* stamps,
                   const StepParams* const* sps, cudaStream_t st);
// refresh arguments of one context's levels (as launch_refresh builds them); *nblocks:
// the refresh grid of that context
template <typename T>
RefreshArgs make_refresh_args(const LevelView<double>* L64, LevelView<T>* LT, int nlev,
                              const StepParams* sp, double* ws, double* stamp, int* nblocks);

// ---- BiCGStab vector kernels
template <typename T>
int launch_bicg_init(size_t nv, const T* r, T* rhat, T* p, T* v, T* x, const StepParams* sp,
                     CondHandle cond, cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_s(size_t nv, const T* r, const T* v, T* s, cudaStream_t st, Reduce red);
// ---- conjugate gradients (symmetric systems)
template <typename T>
int launch_cg_rho(size_t nv, const T* r, const T* z, cudaStream_t st, Reduce red);
template <typename T>
int launch_cg_p(size_t nv, T* p, const T* z, cudaStream_t st, Reduce red);
template <typename T>
int launch_cg_update(size_t nv, T* x, const T* p, T* r, const T* q, const T* diag,
                     const double* sc, CondHandle cond, cudaStream_t st, Reduce red);
int launch_choose_inner(CondHandle c32, CondHandle c64, cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_update(size_t nv, T* x, const T* phat, const T* shat, T* r, const T* s,
                       const T* t, const T* rhat, const T* diag, const double* sc,
                       cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_p(size_t nv, T* p, const T* r, const T* v, CondHandle cond, cudaStream_t st,
                  Reduce red);

// ---- device-side step control (graph mode; the host does the same in eager mode)
// reset the step state
int launch_step_begin(const StepParams* sp, cudaStream_t st, Reduce red);
// schedule-driven steps: load step *kstep of `sched` into `sp` and reset the step state
// (cond = 1), or record the step as skipped (cond = 0) after an earlier failure
int launch_sched_begin(const StepParams* sched, const int* kstep, StepParams* sp,
                       StepOut* out, CondHandle cond, cudaStream_t st, Reduce red);
// record the step's result; a failure halts the rest of the schedule
int launch_sched_end(const int* kstep, StepOut* out, cudaStream_t st, Reduce red);
// next step of the schedule
int launch_sched_next(int* kstep, cudaStream_t st);
// after an FP64 residual: converged / failed / continue; sets `cond` to continue
int launch_refine_decide(const StepParams* sp, CondHandle cond, cudaStream_t st, Reduce red);
// after an inner solve: count its iterations, fail on a non-finite value
int launch_after_inner(int tolerant, cudaStream_t st, Reduce red);
// U = X when the step converged
int launch_commit(size_t nv, double* U, const double* X, cudaStream_t st, Reduce red);

// ---- mixed-precision helpers
template <typename T>
int launch_scale_cast(size_t nv, const double* r, T* rs, cudaStream_t st, Reduce red);
template <typename T>
int launch_correct(size_t nv, double* x, const T* d, cudaStream_t st, Reduce red);
// copy of n doubles (skipped when the step failed)
int launch_copy(size_t n, const double* a, double* b, cudaStream_t st, Reduce red);
int launch_to_float(size_t n, const double* a, float* b, cudaStream_t st);
int launch_check_finite(size_t n, const double* a, cudaStream_t st, Reduce red);
// v = -mobility grad u at the radial ((m+1) n) and angular (m n) faces, u in the interface
// layout, r (m+2) and theta (n) the mesh, g (n) the values on r = 1
int launch_face_drift(int m, int n, const double* u, const double* r, const double* th,
                      const double* g, double mobility, double* vr, double* vt, cudaStream_t st);
// Device assembly of the conservative operator (polar_assemble.cu).  Coefficients in the
// caller's face layouts (any pointer may be null: D = d_const, no drift, b = b_const).
struct AsmIn {
  int m, n;
  const double* r;   // m + 2 radii
  const double* th;  // n angles
  const double* dr;  // (m+1) n radial-face D
  const double* dt;  // m n angular-face D
  double d_const;
  const double* vr;  // (m+1) n radial-face drift
  const double* vt;  // m n angular-face drift
  const double* b;   // N node reaction (interface order)
  double b_const;
};
// level 0: couplings w, e, s, nn and row sums rs of every ring node (split layout), the
// origin couplings o (n) and scalars sc[2] = sum_j o_j, sc[4] = rs0 (vol and sc[3] static)
int launch_assemble_level0(const AsmIn& in, const Shape& sh, const double* vol, double* w,
                           double* e, double* s, double* nn, double* rs, double* o, double* sc,
                           cudaStream_t st);
// one level of the radial hierarchy: the fine level's odd-ring weights ia, ib, then the
// coarse level's couplings, row sums, volumes, origin couplings and scalars
struct CoarsenLevel {
  Shape sh;
  double *w, *e, *s, *nn, *rs, *vol, *o, *ia, *ib, *sc;
};
int launch_coarsen(const CoarsenLevel& f, const CoarsenLevel& c, cudaStream_t st);

// Anderson acceleration of a fixed-point iteration on level-0 vectors (split layout; only
// the N unknowns are read or written).  kMaxAnderson columns at most.
constexpr int kMaxAnderson = 5;
struct AndersonCols {
  const double* v[kMaxAnderson + 1];
  int count;
};
// f = g - x; with `last`, also dF = f - f_last and dX = x - x_last
int launch_aa_columns(const Shape& sh, const double* g, const double* x, const double* f_last,
                      const double* x_last, double* f, double* dF, double* dX, bool last,
                      cudaStream_t st);
// per-block partial dot products of the columns c[0..k-1] with each other (a <= b, row
// by row) and with c[k]: k (k + 1) / 2 + k values per block, `blocks` blocks
int launch_aa_dots(const Shape& sh, const AndersonCols& c, double* partials, int blocks,
                   cudaStream_t st);
// x -= sum_a gamma_a (dX_a + dF_a), the columns in order
int launch_aa_update(const Shape& sh, const AndersonCols& dX, const AndersonCols& dF,
                     const double* gamma_host, double* x, cudaStream_t st);

// out[0] = max_k |a_k - b_k|, out[1] = max_k |a_k| over n doubles (out zeroed first; NaN
// counts as +inf)
int launch_max_change(size_t n, const double* a, const double* b, double* out, cudaStream_t st);

// interface layout (origin, then radial lines j = 0..n-1 of m values) <-> split layout;
// `scale` (nullable, split layout) multiplies on the way in, `div` divides on the way out
int launch_pack(const Shape& sh, const double* in, const double* scale, double* out,
                cudaStream_t st);
int launch_unpack(const Shape& sh, const double* in, const double* div, double* out,
                  cudaStream_t st);

}  // namespace polar
