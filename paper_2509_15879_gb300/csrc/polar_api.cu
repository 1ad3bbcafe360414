// C ABI of the polar theta-step library: argument checking, device buffers, the
// upload of the operator and its multigrid hierarchy (assembled on the host by
// polar_host.cpp), and the host orchestration of one implicit step (Eq. 2.5):
//   right-hand side (FP64) -> per-step refresh of the ring factors -> refinement loop
//   { FP64 residual -> scaled cast -> BiCGStab in the inner precision, preconditioned
//     by one multigrid V-cycle -> FP64 correction }.
// The system is solved in the form S = V/dt + theta V L (every row scaled by its
// control volume), which leaves the solution unchanged and keeps the matrix entries
// within a few orders of magnitude on graded meshes.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/polar.h"
#include "polar_fft.h"
#include "polar_host.h"
#include "polar_internal.h"

using namespace polar;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA,          \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

#define TRY(expr)                    \
  do {                               \
    int rc_ = (expr);                \
    if (rc_ != POLAR_OK) return rc_; \
  } while (0)

template <typename T>
struct KVecs {
  T *r, *rhat, *p, *v, *s, *t, *phat, *shat, *d;
};

// Device arrays of one multigrid level.
struct DevLevel {
  Shape sh;
  double *vol, *rs, *w, *e, *s, *nn, *o, *ia, *ib, *sc;
  float *w32, *e32, *s32, *nn32, *o32, *ia32, *ib32;
  // per-step refresh, FP64 (FP64 path; level 0 diag also for the mixed path)
  double *diag, *fl, *fui, *fcu, *fq, *fring, *fz;
  double* dinv;  // level 0: 1 / diag of the FP64 operator
  // per-step refresh, FP32 (mixed path)
  float *diag32, *fl32, *fui32, *fcu32, *fq32, *fring32, *fz32, *rsum32;
  // V-cycle right-hand side and solution (levels >= 1), in the inner precision
  void *b, *x;
  double *b64, *x64;  // the same in FP64 (b, x themselves in the FP64 path)
};

struct PendingTimer {
  int kind;
  cudaEvent_t a, b;
  double bytes, flops;
};
struct KernelStat {
  std::string name;
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double flops = 0.0;
};

}  // namespace

struct polar_ctx;
struct polar_batch;
// Electron-hole pair coupled to a Poisson potential (see polar_gummel_step).
struct polar_gummel {
  polar_ctx* phi = nullptr;
  polar_ctx* car[2] = {nullptr, nullptr};  // electrons, holes
  polar_batch* pair = nullptr;             // the carriers advanced as one batch
  polar_gummel_desc d{};
  double* save[2] = {nullptr, nullptr};    // carriers' states at the start of the step
  double* phi_prev = nullptr;              // previous iterate of the potential
  double* change = nullptr;                // max |phi - phi_prev|, max |phi|
  // per carrier: its D faces and reaction on the device, the drift faces
  double* dr[2] = {nullptr, nullptr};
  double* dt[2] = {nullptr, nullptr};
  double* b[2] = {nullptr, nullptr};
  double* vr[2] = {nullptr, nullptr};
  double* vt[2] = {nullptr, nullptr};
  // Anderson acceleration: last iterate and residual, the current residual, and the
  // difference columns (ring buffers of `depth` each), dot-product partials
  double *x_last = nullptr, *f_last = nullptr, *f_cur = nullptr;
  double* dX[kMaxAnderson] = {};
  double* dF[kMaxAnderson] = {};
  double* partials = nullptr;
  std::vector<double> partials_host;
};
constexpr int kAABlocks = 304;
struct polar_batch {
  std::vector<polar_ctx*> ctx;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  std::vector<int64_t> gens;   // context generations the graph was captured with
  void* arena = nullptr;       // argument tables and work lists of the batched launches
  size_t arena_bytes = 0;
  // groups of instances of similar size, each a parallel branch of the step graph, with
  // its kernels per step: fixed, per refinement sweep, per FP32 / FP64 Krylov iteration
  struct Group {
    std::vector<int> members;
    int64_t fixed = 0, sweep = 0, iter32 = 0, iter64 = 0;
  };
  std::vector<Group> groups;
  int64_t launches = 0;        // kernels launched by the batch's graphs
};

struct polar_ctx {
  int m = 0, n = 0;
  int scheme = 0, precision = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<double> r, theta;
  std::vector<void*> allocs;      // every device buffer of the context
  polar_alloc_fn alloc = nullptr; // caller's allocator (null: cudaMalloc / cudaFree)
  polar_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  size_t alloc_bytes = 0;         // bytes held in `allocs`
  std::vector<DevLevel> lv;
  std::vector<LevelView<double>> v64;
  std::vector<LevelView<float>> v32;
  int nsrc = 0;
  double* vsrc[4] = {nullptr, nullptr, nullptr, nullptr};
  double* bnd[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<double> bnd_host[4];  // host copies of the Dirichlet fields
  HostCoeffs hk;                    // the coefficients the levels were assembled from
  bool have_coeffs = false, have_state = false;
  double t = 0.0;
  double* U = nullptr;
  double* X = nullptr;
  double* e = nullptr;
  double* r64 = nullptr;
  double* io = nullptr;  // interface-layout staging (N doubles)
  double* ws = nullptr;  // refresh workspace
  StepParams* sp = nullptr;       // device parameters of the current step
  StepParams* sp_host = nullptr;  // pinned staging copy
  double cur_alpha = -1.0, cur_beta = -1.0;  // values the refresh was made for
  cudaStream_t cs = nullptr;      // stream the launchers enqueue on (st, or the capture stream)
  cudaStream_t cap = nullptr;     // private stream for graph capture
  cudaGraph_t graph = nullptr;    // one theta-step with device-side loops
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;          // gexec matches the current coefficients
  bool use_graph = true;
  int64_t graph_kernels_fixed = 0, graph_kernels_sweep = 0, graph_kernels_iter = 0;
  int64_t graph_kernels_iter64 = 0;  // mixed path: an FP64 Krylov iteration over the FP32 V-cycle
  bool symmetric = false;  // S is symmetric (no drift): CG instead of BiCGStab
  bool steady = false;     // the running advance solves the steady problem (alpha = 0)
  double* mesh_dev = nullptr;  // r (m+2), theta (n), boundary values (n): face fields
  // direct solve of separable operators (Fourier in theta, tridiagonal in r)
  bool separable = false;     // the current coefficients are separable
  bool direct_now = false;    // the current advance uses the direct inner solve
  FftPlan plan{};
  SepRings sep{};
  double *fx_r = nullptr, *fx_i = nullptr, *fcp = nullptr, *fzv = nullptr;
  int64_t generation = 0;         // bumped whenever a captured graph goes stale
  // ring-solve tile shapes per level, [mode * 2 + parity], for FP32 and FP64 ring solves
  // (autotuned on first use; a mixed context tunes both)
  std::vector<std::array<RingShape, 4>> tiles32, tiles64;
  bool tuned = false;
  double* stamp64 = nullptr;  // mixed path: (alpha, beta) its FP64 factors were formed for
  bool autotune = true;
  // device-side schedule of a polar_advance (graph mode)
  StepParams* sched = nullptr;
  StepOut* dout = nullptr;
  int* kstep = nullptr;
  int sched_cap = 0;
  StepParams* sched_host = nullptr;
  StepOut* out_host = nullptr;
  KVecs<double> kv64{};
  KVecs<float> kv32{};
  double* part = nullptr;
  KrylovScalars* ks = nullptr;
  KrylovScalars* ks_host = nullptr;
  int64_t launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<PendingTimer> pending;
  std::vector<KernelStat> kstats;

  Reduce red() const { return Reduce{part, ks}; }
  Params par() const { return reinterpret_cast<const double*>(sp); }
  size_t N() const { return (size_t)m * n + 1; }
  const Shape& sh0() const { return lv[0].sh; }
  size_t nv() const { return lv[0].sh.nv; }
  int nlev() const { return (int)lv.size(); }
};

namespace {

// One zeroed device buffer of the context, from the caller's allocator when one was given
// (zeroed on the context's stream, the stream the allocator hands the memory out for).
template <typename T>
int dalloc(polar_ctx* c, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  void* q = nullptr;
  if (c->alloc) {
    q = c->alloc(bytes, c->st, c->alloc_user);
    if (!q) return fail(POLAR_ENOMEM, "the caller's allocator returned NULL");
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      c->free_fn(q, c->st, c->alloc_user);
      return fail(POLAR_ENOMEM, "the caller's allocator returned memory not aligned to 256 bytes");
    }
  } else {
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(POLAR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  c->allocs.push_back(q);
  c->alloc_bytes += bytes;
  cudaError_t e = cudaMemsetAsync(q, 0, bytes, c->st);
  if (e != cudaSuccess) return fail(POLAR_ECUDA, cudaGetErrorString(e));
  *p = static_cast<T*>(q);
  return POLAR_OK;
}

int check_launch(polar_ctx* c, int n) {
  if (n < 0) {
    const cudaError_t e = cudaGetLastError();
    return fail(POLAR_ECUDA, std::string("kernel launch (cluster): ") + cudaGetErrorString(e));
  }
  c->launches += n;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(POLAR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return POLAR_OK;
}

#define LAUNCH(expr) TRY(check_launch(c, (expr)))

// Event timing of individual kernels: every launch of a named kernel class is
// bracketed by two events on the context's stream when timing is on; the pairs are
// resolved (stream synchronised) when more than kMaxPending accumulate or on query.
constexpr size_t kMaxPending = 4096;

int kind_index(polar_ctx* c, const char* name) {
  for (size_t k = 0; k < c->kstats.size(); ++k)
    if (c->kstats[k].name == name) return (int)k;
  c->kstats.push_back(KernelStat{name});
  return (int)c->kstats.size() - 1;
}

cudaEvent_t take_event(polar_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int resolve_timers(polar_ctx* c) {
  if (c->pending.empty()) return POLAR_OK;
  CUDA_TRY(cudaStreamSynchronize(c->st));
  for (const PendingTimer& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    KernelStat& k = c->kstats[p.kind];
    k.launches += 1;
    k.ms += ms;
    k.bytes += p.bytes;
    k.flops += p.flops;
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  c->pending.clear();
  return POLAR_OK;
}

int timed_begin(polar_ctx* c, cudaEvent_t* e) {
  *e = nullptr;
  if (!c->timing) return POLAR_OK;
  if (c->pending.size() >= kMaxPending) TRY(resolve_timers(c));
  *e = take_event(c);
  CUDA_TRY(cudaEventRecord(*e, c->st));
  return POLAR_OK;
}

int timed_end(polar_ctx* c, cudaEvent_t a, const char* name, double bytes, double flops) {
  if (!a) return POLAR_OK;
  cudaEvent_t b = take_event(c);
  CUDA_TRY(cudaEventRecord(b, c->st));
  c->pending.push_back(PendingTimer{kind_index(c, name), a, b, bytes, flops});
  return POLAR_OK;
}

// LAUNCH with event timing under a kernel-class name, the launch's algorithmic bytes and
// its arithmetic (flops per point as the kernel's source performs them, an FMA counting
// two, times the points it covers; 0 where not modelled).
#define TLAUNCHF(name, bytes, flops, expr)                             \
  do {                                                                 \
    cudaEvent_t ev_;                                                   \
    TRY(timed_begin(c, &ev_));                                         \
    LAUNCH(expr);                                                      \
    TRY(timed_end(c, ev_, name, (double)(bytes), (double)(flops)));    \
  } while (0)
#define TLAUNCH(name, bytes, expr) TLAUNCHF(name, bytes, 0.0, expr)

void release(polar_ctx* c) {
  for (const PendingTimer& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  c->pending.clear();
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  c->ev_free.clear();
  for (void* p : c->allocs) {
    if (c->free_fn) {
      c->free_fn(p, c->st, c->alloc_user);
    } else {
      cudaFree(p);
    }
  }
  c->allocs.clear();
  c->alloc_bytes = 0;
  if (c->ks_host) cudaFreeHost(c->ks_host);
  c->ks_host = nullptr;
  if (c->sp_host) cudaFreeHost(c->sp_host);
  c->sp_host = nullptr;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  if (c->cap) cudaStreamDestroy(c->cap);
  c->cap = nullptr;
  if (c->sched_host) cudaFreeHost(c->sched_host);
  if (c->out_host) cudaFreeHost(c->out_host);
  c->sched_host = nullptr;
  c->out_host = nullptr;
}

// Fetch caller data (host or device pointer) into a host vector.
int fetch(const double* p, size_t count, int memory, std::vector<double>& out) {
  out.resize(count);
  if (count == 0) return POLAR_OK;
  if (memory == POLAR_DEVICE) {
    CUDA_TRY(cudaMemcpy(out.data(), p, count * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), p, count * sizeof(double));
  }
  for (double v : out)
    if (!std::isfinite(v)) return fail(POLAR_ENONFINITE, "non-finite value in a coefficient array");
  return POLAR_OK;
}

// ---------------------------------------------------------------------------------
// device buffers

template <typename T>
int alloc_kvecs(polar_ctx* c, KVecs<T>& k) {
  T** all[] = {&k.r, &k.rhat, &k.p, &k.v, &k.s, &k.t, &k.phat, &k.shat, &k.d};
  for (T** p : all) TRY(dalloc(c, p, c->nv()));
  return POLAR_OK;
}

int alloc_levels(polar_ctx* c) {
  int m = c->m;
  for (;;) {
    DevLevel d{};
    d.sh = make_shape(m, c->n);
    c->lv.push_back(d);
    if (m <= 1) break;
    m /= 2;
  }
  const bool mixed = c->precision == POLAR_MIXED;
  size_t wsz = 0;
  for (int l = 0; l < c->nlev(); ++l) {
    DevLevel& d = c->lv[l];
    const size_t nv = d.sh.nv;
    const size_t nr = 2 * (size_t)d.sh.m;
    double** s64[] = {&d.vol, &d.rs, &d.w, &d.e, &d.s, &d.nn, &d.ia, &d.ib};
    for (double** p : s64) TRY(dalloc(c, p, nv));
    TRY(dalloc(c, &d.o, (size_t)c->n));
    TRY(dalloc(c, &d.sc, 8));
    if (l == 0) TRY(dalloc(c, &d.dinv, nv));
    // FP64 per-step factors and coarse vectors: the FP64 path's, and in the mixed path
    // those of its FP64 solve, which takes over a step whose FP32 refinement stalls
    TRY(dalloc(c, &d.diag, nv));
    double** f64[] = {&d.fl, &d.fui, &d.fcu, &d.fq};
    for (double** p : f64) TRY(dalloc(c, p, nv));
    TRY(dalloc(c, &d.fring, nr));
    TRY(dalloc(c, &d.fz, (size_t)c->n));
    if (l > 0) {
      TRY(dalloc(c, &d.b64, nv));
      TRY(dalloc(c, &d.x64, nv));
    }
    if (!mixed) {
      d.b = d.b64;
      d.x = d.x64;
    } else {
      float** s32[] = {&d.w32, &d.e32, &d.s32, &d.nn32, &d.ia32, &d.ib32};
      for (float** p : s32) TRY(dalloc(c, p, nv));
      TRY(dalloc(c, &d.o32, (size_t)c->n));
      float** f32[] = {&d.diag32, &d.fl32, &d.fui32, &d.fcu32, &d.fq32};
      for (float** p : f32) TRY(dalloc(c, p, nv));
      if (l == 0) TRY(dalloc(c, &d.rsum32, nv));
      TRY(dalloc(c, &d.fring32, nr));
      TRY(dalloc(c, &d.fz32, (size_t)c->n));
      if (l > 0) {
        float *b = nullptr, *x = nullptr;
        TRY(dalloc(c, &b, nv));
        TRY(dalloc(c, &x, nv));
        d.b = b;
        d.x = x;
      }
    }
    wsz += 2 * nv;  // refresh workspace: y and the pivot reciprocals
  }
  TRY(dalloc(c, &c->ws, wsz));
  c->v64.resize(c->nlev());
  c->v32.resize(c->nlev());
  for (int l = 0; l < c->nlev(); ++l) {
    DevLevel& d = c->lv[l];
    LevelView<double>& a = c->v64[l];
    a = LevelView<double>{};
    a.sh = d.sh;
    a.vol = d.vol;
    a.rs = d.rs;
    a.w = d.w;
    a.e = d.e;
    a.s = d.s;
    a.nn = d.nn;
    a.o = d.o;
    a.ia = d.ia;
    a.ib = d.ib;
    a.diag = d.diag;
    a.dinv = d.dinv;
    a.fl = d.fl;
    a.fui = d.fui;
    a.fcu = d.fcu;
    a.fq = d.fq;
    a.fring = d.fring;
    a.fz = d.fz;
    a.sc = d.sc;
    LevelView<float>& b = c->v32[l];
    b = LevelView<float>{};
    b.sh = d.sh;
    b.w = d.w32;
    b.e = d.e32;
    b.s = d.s32;
    b.nn = d.nn32;
    b.o = d.o32;
    b.ia = d.ia32;
    b.ib = d.ib32;
    b.diag = d.diag32;
    b.rsum = d.rsum32;
    b.fl = d.fl32;
    b.fui = d.fui32;
    b.fcu = d.fcu32;
    b.fq = d.fq32;
    b.fring = d.fring32;
    b.fz = d.fz32;
    b.sc = d.sc;
  }
  return POLAR_OK;
}

// host array (q = j m + i - 1, origin value separate) -> split layout of the level
std::vector<double> to_split(const Shape& sh, const std::vector<double>& a, double origin) {
  std::vector<double> out(sh.nv, 0.0);
  out[0] = origin;
  for (int j = 0; j < sh.n; ++j)
    for (int i = 1; i <= sh.m; ++i) out[sh.at(i, j)] = a[(size_t)j * sh.m + (i - 1)];
  return out;
}

int upload(double* dst, const std::vector<double>& h) {
  CUDA_TRY(cudaMemcpy(dst, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  return POLAR_OK;
}

int upload_level(polar_ctx* c, int l, const HLevel& H) {
  DevLevel& d = c->lv[l];
  const Shape& sh = d.sh;
  TRY(upload(d.vol, to_split(sh, H.vol, H.vol0)));
  TRY(upload(d.rs, to_split(sh, H.rs, H.rs0)));
  TRY(upload(d.w, to_split(sh, H.w, 0.0)));
  TRY(upload(d.e, to_split(sh, H.e, 0.0)));
  TRY(upload(d.s, to_split(sh, H.s, 0.0)));
  TRY(upload(d.nn, to_split(sh, H.nn, 0.0)));
  TRY(upload(d.ia, to_split(sh, H.ia, 0.0)));
  TRY(upload(d.ib, to_split(sh, H.ib, 0.0)));
  TRY(upload(d.o, H.o));
  double osum = 0.0;
  for (double v : H.o) osum += v;
  const double sc[8] = {0.0, 0.0, osum, H.vol0, H.rs0, 0.0, 0.0, 0.0};
  CUDA_TRY(cudaMemcpy(d.sc, sc, sizeof(sc), cudaMemcpyHostToDevice));
  if (c->precision == POLAR_MIXED) {
    const double* s64[] = {d.w, d.e, d.s, d.nn, d.ia, d.ib};
    float* s32[] = {d.w32, d.e32, d.s32, d.nn32, d.ia32, d.ib32};
    for (int a = 0; a < 6; ++a) LAUNCH(launch_to_float(sh.nv, s64[a], s32[a], c->st));
    LAUNCH(launch_to_float((size_t)c->n, d.o, d.o32, c->st));
  }
  return POLAR_OK;
}

// ---------------------------------------------------------------------------------
// solver

int read_scalars(polar_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->ks_host, c->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

template <typename T>
const std::vector<LevelView<T>>& views(const polar_ctx* c) {
  if constexpr (sizeof(T) == 8) {
    return c->v64;
  } else {
    return c->v32;
  }
}

// Per-step refresh: the matrix S = alpha V + beta V L changes with dt and theta.  The
// kernel reads alpha, beta and do_refresh from the step parameters.
// Kernel-class name for the per-kernel timing: ".f32" marks FP32 launches (a mixed
// context runs FP32 and FP64 versions of the same kernels).
template <typename T>
const char* tname(const char* base) {
  static thread_local std::string s;
  s = std::string(base) + (sizeof(T) == 4 ? ".f32" : "");
  return s.c_str();
}

// `stamp` (the mixed path's FP64 factors): formed on demand, once per (alpha, beta).
template <typename T>
int launch_refresh_all(polar_ctx* c, double* stamp = nullptr) {
  std::vector<LevelView<T>> vt = views<T>(c);
  double pts = 0.0;
  for (const DevLevel& d : c->lv) pts += (double)d.sh.m * d.sh.n;
  // reads 6 FP64 coefficient arrays, writes diag and 4 factor arrays
  // about 47 flops per point (diagonal, pivot matrices, the three recurrences)
  TLAUNCHF(stamp ? "refresh64" : "refresh", pts * (6.0 * 8 + 5.0 * sizeof(T)), 47.0 * pts,
          launch_refresh<T>(c->v64.data(), vt.data(), c->nlev(), c->sp, c->ws, c->cs, stamp));
  return POLAR_OK;
}

template <typename T>
std::vector<std::array<RingShape, 4>>& tiles_of(polar_ctx* c) {
  return sizeof(T) == 8 ? c->tiles64 : c->tiles32;
}

// tuned tile shape of a ring-solve launch (null: the launcher's default)
template <typename T>
const RingShape* tile(polar_ctx* c, int l, int mode, int parity) {
  const std::vector<std::array<RingShape, 4>>& t = tiles_of<T>(c);
  if (!c->tuned || l >= (int)t.size()) return nullptr;
  const RingShape& s = t[l][mode * 2 + parity];
  return s.P > 0 ? &s : nullptr;
}

// V-cycle vectors of level l >= 1 in precision T
template <typename T>
T* coarse_b(const polar_ctx* c, int l) {
  return static_cast<T*>(sizeof(T) == 8 ? static_cast<void*>(c->lv[l].b64) : c->lv[l].b);
}
template <typename T>
T* coarse_x(const polar_ctx* c, int l) {
  return static_cast<T*>(sizeof(T) == 8 ? static_cast<void*>(c->lv[l].x64) : c->lv[l].x);
}

// x = M^{-1} b: one V(1,1) cycle of the radial multigrid (polar_mg.cu), one kernel per
// half-sweep and level.
template <typename T>
int vcycle(polar_ctx* c, const T* b, T* x) {
  const std::vector<LevelView<T>>& L = views<T>(c);
  const int nl = c->nlev();
  // Driven from the host, iterations run in batches past convergence, and the V-cycle's
  // kernels test the solve's `done` flag.  In a captured graph the loop stops exactly at
  // convergence, so they skip that dependent load (a cycle that follows a breakdown only
  // writes scratch vectors that the next solve overwrites).
  const int* done = (c->cs == c->st) ? &c->ks->done : nullptr;
  const double B = sizeof(T);
  const Params par = c->par();
  auto bof = [&](int l) { return l == 0 ? b : static_cast<const T*>(coarse_b<T>(c, l)); };
  auto xof = [&](int l) { return l == 0 ? x : coarse_x<T>(c, l); };
  // kernel classes are timed per level group: the fine level, level 1, and the rest
  auto nm = [&](const char* base, int l) {
    static thread_local std::string s;
    s = std::string(base) + (l == 0 ? "@L0" : l == 1 ? "@L1" : "@L2+") +
        (sizeof(T) == 4 ? ".f32" : "");
    return s.c_str();
  };
  const int lc = nl - 1;
  for (int l = 0; l < lc; ++l) {
    const Shape& s = L[l].sh;
    const double po = (double)s.no * s.n, pe = (double)s.ne * s.n;
    // algorithmic words: odd line solve reads b and 4 factors, writes x (6 per point);
    // even: b, w, e, the odd neighbours, 4 factors, writes x (9); restriction reads
    // w, e, ia, ib of the odd rings and x of the even ones, writes the coarse rhs.
    // Flops per point: the line solve 13 (forward 3 + replay 2, 1/u y 1, backward 3 +
    // replay 2, Sherman-Morrison 2), the right-hand side 0 / 5 / 13 (b only / plain
    // neighbours / corrected odd neighbours); restriction 11 per coarse point
    TLAUNCHF(nm("ring_pre_odd", l), 6 * B * po, 13.0 * po,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, par, 1, RING_PRE, done, c->cs,
                           tile<T>(c, l, RING_PRE, 1)));
    TLAUNCHF(nm("ring_pre_even", l), 9 * B * pe, 18.0 * pe,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, par, 0, RING_PRE, done, c->cs,
                           tile<T>(c, l, RING_PRE, 0)));
    TLAUNCHF(nm("restrict", l), B * (4 * po + 2 * pe), 11.0 * L[l + 1].sh.m * s.n,
            launch_restrict<T>(L[l], L[l + 1], xof(l), coarse_b<T>(c, l + 1), par, done,
                               c->cs));
  }
  TLAUNCH(tname<T>("coarsest"), 8 * B * L[nl - 1].sh.n,
          launch_coarsest<T>(L[nl - 1], bof(nl - 1), xof(nl - 1), par, done, c->cs));
  for (int l = lc - 1; l >= 0; --l) {
    const Shape& s = L[l].sh;
    const double po = (double)s.no * s.n, pe = (double)s.ne * s.n;
    // even rings after the correction also read x, ia, ib of the odd rings and the
    // coarse solution (8 per even point + 3 per odd point + 1 per coarse point)
    TLAUNCHF(nm("ring_post_even", l), B * (8 * pe + 3 * po + pe), 26.0 * pe,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), coarse_x<T>(c, l + 1),
                           par, 0, RING_POST, done, c->cs, tile<T>(c, l, RING_POST, 0)));
    TLAUNCHF(nm("ring_post_odd", l), 9 * B * po, 18.0 * po,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, par, 1, RING_POST, done, c->cs,
                           tile<T>(c, l, RING_POST, 1)));
  }
  return POLAR_OK;
}

// ---- autotuner of the ring-solve tiles.  Every (level, mode, parity) launch of the
// V-cycle is timed with CUDA events for each candidate shape on the context's own data
// (after a refresh); the fastest is kept.  Results are shared between contexts through a
// cache keyed by precision, mode, parity and the power-of-two buckets of the line count
// and the ring length.
using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_lock;
std::map<TuneKey, RingShape> g_tune_cache;

// POLAR_TUNE_LOG=1 in the environment prints every tuned ring launch (shape and time)
bool tune_log() {
  static const bool on = [] {
    const char* v = getenv("POLAR_TUNE_LOG");
    return v && *v && *v != '0';
  }();
  return on;
}

int bucket(int v) {
  int b = 1;
  while (b < v) b <<= 1;
  return b;
}

template <typename T>
KVecs<T>& kvecs(polar_ctx* c);

template <typename T>
int tune_rings(polar_ctx* c) {
  const std::vector<LevelView<T>>& L = views<T>(c);
  const int nl = c->nlev();
  const int lc = nl - 1;
  tiles_of<T>(c).assign(nl, std::array<RingShape, 4>{});
  CUDA_TRY(cudaMemsetAsync(&c->ks->done, 0, sizeof(int), c->st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  std::vector<RingShape> cand;
  int rc = POLAR_OK;
  const int* done = &c->ks->done;
  for (int l = 0; l < lc && rc == POLAR_OK; ++l) {
    T* b = l == 0 ? kvecs<T>(c).p : coarse_b<T>(c, l);
    T* x = l == 0 ? kvecs<T>(c).phat : coarse_x<T>(c, l);
    const T* X = coarse_x<T>(c, l + 1);
    for (int mode = 0; mode < 2 && rc == POLAR_OK; ++mode)
      for (int parity = 0; parity < 2 && rc == POLAR_OK; ++parity) {
        const int lines = parity ? L[l].sh.no : L[l].sh.ne;
        if (lines == 0) continue;
        const TuneKey key{(int)sizeof(T), mode, parity, bucket(lines), bucket(L[l].sh.n)};
        {
          std::lock_guard<std::mutex> g(g_tune_lock);
          auto it = g_tune_cache.find(key);
          if (it != g_tune_cache.end()) {
            tiles_of<T>(c)[l][mode * 2 + parity] = it->second;
            continue;
          }
        }
        ring_candidates<T>(lines, L[l].sh.n, cand);
        RingShape best = ring_default<T>(lines, L[l].sh.n);
        float best_ms = 1e30f;
        for (const RingShape& s : cand) {
          auto go = [&]() {
            return launch_ring<T>(L[l], L[l + 1], b, x, mode ? X : nullptr, c->par(), parity, mode,
                                  done, c->st, &s);
          };
          if (go() < 0) {
            (void)cudaGetLastError();  // shape not launchable here: skip it
            continue;
          }
          cudaEventRecord(e0, c->st);
          for (int r = 0; r < 3; ++r) go();
          cudaEventRecord(e1, c->st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(POLAR_ECUDA, "autotuner: ring launch failed");
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) {
            best_ms = ms;
            best = s;
          }
        }
        tiles_of<T>(c)[l][mode * 2 + parity] = best;
        if (tune_log())
          fprintf(stderr, "polar tune: %s level %d lines %d n %d %s %s -> RW %d TW %d P %d CS %d "
                  "ST %d: %.2f us\n", sizeof(T) == 8 ? "fp64" : "fp32", l, lines, L[l].sh.n,
                  mode ? "post" : "pre", parity ? "odd" : "even", best.RW, best.TW, best.P,
                  best.CS, best.ST, 1e3 * best_ms / 3);
        std::lock_guard<std::mutex> g(g_tune_lock);
        g_tune_cache[key] = best;
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  return rc;
}

template <typename T>
KVecs<T>& kvecs(polar_ctx* c) {
  if constexpr (sizeof(T) == 8) {
    return c->kv64;
  } else {
    return c->kv32;
  }
}

// One BiCGStab iteration, right-preconditioned by one V-cycle per application; all
// scalars stay on the device.  `cond` (graph mode) receives "keep iterating".
template <typename T>
int bicg_iteration(polar_ctx* c, CondHandle cond) {
  KVecs<T>& k = kvecs<T>(c);
  const LevelView<T>& L0 = views<T>(c)[0];
  const Reduce red = c->red();
  const size_t nv = c->nv();
  const double B = sizeof(T), pts = (double)c->m * c->n;
  TRY(vcycle<T>(c, k.p, k.phat));
  // stencil with dot: reads x, diag, 4 couplings, d1; writes y (8 words per point);
  // 12 flops per point (the 5-point row 10, the dot 2)
  TLAUNCHF(tname<T>("stencil_dot"), 8 * B * pts, 12.0 * pts, launch_apply_dot<T>(L0, c->par(), k.phat, k.v, k.rhat, 0, c->cs, red));
  TLAUNCHF(tname<T>("bicg_s"), 3 * B * nv, 2.0 * pts, launch_bicg_s<T>(nv, k.r, k.v, k.s, c->cs, red));
  TRY(vcycle<T>(c, k.s, k.shat));
  TLAUNCHF(tname<T>("stencil_dot"), 8 * B * pts, 12.0 * pts, launch_apply_dot<T>(L0, c->par(), k.shat, k.t, k.s, 1, c->cs, red));
  TLAUNCHF(tname<T>("bicg_update"), 9 * B * nv, 9.0 * pts,
          launch_bicg_update<T>(nv, k.d, k.phat, k.shat, k.r, k.s, k.t, k.rhat, L0.diag,
                                L0.sc, c->cs, red));
  TLAUNCHF(tname<T>("bicg_p"), 4 * B * nv, 4.0 * pts, launch_bicg_p<T>(nv, k.p, k.r, k.v, cond, c->cs, red));
  return POLAR_OK;
}

// One preconditioned CG iteration (symmetric S): z = M r, rho = r.z, p = z + beta p,
// q = S p with alpha = rho / p.q, x += alpha p, r -= alpha q and the stopping test.  One
// V-cycle per iteration where BiCGStab takes two.
template <typename T>
int cg_iteration(polar_ctx* c, CondHandle cond) {
  KVecs<T>& k = kvecs<T>(c);
  const LevelView<T>& L0 = views<T>(c)[0];
  const Reduce red = c->red();
  const size_t nv = c->nv();
  const double B = sizeof(T), pts = (double)c->m * c->n;
  TRY(vcycle<T>(c, k.r, k.phat));
  TLAUNCHF(tname<T>("cg_rho"), 2 * B * nv, 2.0 * pts, launch_cg_rho<T>(nv, k.r, k.phat, c->cs, red));
  TLAUNCHF(tname<T>("cg_p"), 3 * B * nv, 2.0 * pts, launch_cg_p<T>(nv, k.p, k.phat, c->cs, red));
  // stencil with dot: reads p, diag, 4 couplings; writes q (7 words per point)
  TLAUNCHF(tname<T>("stencil_dot"), 7 * B * pts, 12.0 * pts, launch_apply_dot<T>(L0, c->par(), k.p, k.v, k.p, 0, c->cs, red));
  TLAUNCHF(tname<T>("cg_update"), 7 * B * nv, 5.0 * pts,
          launch_cg_update<T>(nv, k.d, k.p, k.r, k.v, L0.diag, L0.sc, cond, c->cs, red));
  return POLAR_OK;
}

// The inner Krylov iteration: CG when S is symmetric, BiCGStab otherwise.
template <typename T>
int krylov_iteration(polar_ctx* c, CondHandle cond) {
  return c->symmetric ? cg_iteration<T>(c, cond) : bicg_iteration<T>(c, cond);
}

template <typename T>
int bicg_begin(polar_ctx* c, CondHandle cond) {
  KVecs<T>& k = kvecs<T>(c);
  const size_t nv = c->nv();
  const Reduce red = c->red();
  TLAUNCH(tname<T>("scale_cast"), (8.0 + sizeof(T)) * nv, launch_scale_cast<T>(nv, c->r64, k.r, c->cs, red));
  TLAUNCH(tname<T>("bicg_init"), 5.0 * sizeof(T) * nv,
          launch_bicg_init<T>(nv, k.r, k.rhat, k.p, k.v, k.d, c->sp, cond, c->cs, red));
  return POLAR_OK;
}

int resid(polar_ctx* c) {
  const double pts = (double)c->m * c->n;
  // 12 flops per point: the 5-point row, the difference from e, the Jacobi scaling
  TLAUNCHF("resid64", 8.0 * 8 * pts, 12.0 * pts, launch_resid64(c->v64[0], c->par(), c->X, c->e, c->r64, c->cs, c->red()));
  return POLAR_OK;
}

template <typename T>
int correct(polar_ctx* c) {
  const size_t nv = c->nv();
  TLAUNCH(tname<T>("correct"), (16.0 + sizeof(T)) * nv, launch_correct<T>(nv, c->X, kvecs<T>(c).d, c->cs, c->red()));
  return POLAR_OK;
}

int rhs(polar_ctx* c) {
  const double* srcs[4] = {c->vsrc[0], c->vsrc[1], c->vsrc[2], c->vsrc[3]};
  const double* bnds[4] = {c->bnd[0], c->bnd[1], c->bnd[2], c->bnd[3]};
  // flops per point: the explicit half 12, the sources and boundary terms of both levels
  TLAUNCHF("rhs", (8.0 + c->nsrc) * 8 * c->m * c->n, (12.0 + 4.0 * c->nsrc) * c->m * c->n,
          launch_rhs(c->v64[0], c->sp, c->U, c->nsrc, srcs, bnds, c->e, c->cs, c->red()));
  return POLAR_OK;
}

// Direct inner solve of a separable operator: the FP64 residual scaled by its max norm
// (k_scale_cast), Fourier transform along theta, one tridiagonal solve per mode, inverse
// transform, then X += rmax d in FP64 (k_correct).
int direct_inner(polar_ctx* c) {
  const size_t nv = c->nv();
  const double pts = (double)c->m * c->n;
  TLAUNCH("scale_cast", 16.0 * nv, launch_scale_cast<double>(nv, c->r64, c->kv64.r, c->cs, c->red()));
  // ring values in and out (16 B), the mode coefficients through the three kernels (48 B)
  // and the tridiagonal factors (8 B) per point
  TLAUNCH("direct_solve", 72.0 * pts,
          launch_direct_solve(c->sh0(), c->plan, c->sep, c->par(), c->kv64.r, c->kv64.d,
                              c->fx_r, c->fx_i, c->fcp, c->fzv, c->ks, c->cs));
  return POLAR_OK;
}

// Eager step: the host drives the refinement and Krylov loops (used when per-kernel
// timing is on, and as the fallback when a graph cannot be built).
template <typename T>
int step_eager(polar_ctx* c, polar_step_stats& stats) {
  c->cs = c->st;
  LAUNCH(launch_step_begin(c->sp, c->cs, c->red()));  // step flags a graph run may have left set
  TRY(rhs(c));
  if (c->sp_host->do_refresh) TRY(launch_refresh_all<T>(c));
  CUDA_TRY(cudaMemcpyAsync(c->X, c->U, c->nv() * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  // the refinement decisions (converged, failed, switch of the mixed path to its FP64 solve)
  // are taken on the device by the kernels the step graph runs; the host only reads them
  for (;;) {
    TRY(resid(c));
    LAUNCH(launch_refine_decide(c->sp, 0, c->cs, c->red()));
    TRY(read_scalars(c));
    const KrylovScalars& h = *c->ks_host;
    stats.refinements = h.sweeps;
    stats.scaled_resid = h.scaled;
    stats.iters = h.iters_total;
    stats.fp64_iters = h.iters64;
    if (h.failed == POLAR_ENONFINITE) return fail(POLAR_ENONFINITE, "non-finite residual");
    if (h.failed)
      return fail(POLAR_ENOCONV, "refinement did not reach the tolerance (scaled residual " +
                                     std::to_string(h.scaled) + ")");
    if (h.converged) break;
    if (c->direct_now) {
      TRY(direct_inner(c));
      LAUNCH(launch_after_inner(0, c->cs, c->red()));
      TRY(correct<double>(c));
      continue;
    }
    const bool x64 = h.use64 && sizeof(T) == 4;
    if (x64) {
      TRY(launch_refresh_all<double>(c, c->stamp64));  // FP64 factors, once per (alpha, beta)
      TRY(bicg_begin<double>(c, 0));
    } else {
      TRY(bicg_begin<T>(c, 0));
    }
    int batch = 2;
    for (;;) {
      for (int it = 0; it < batch; ++it) {
        if (x64) {
          TRY(krylov_iteration<double>(c, 0));
        } else {
          TRY(krylov_iteration<T>(c, 0));
        }
      }
      TRY(read_scalars(c));
      if (c->ks_host->done != 0) break;
      batch = std::min(batch * 2, 8);
    }
    // as in the graph: iteration counts, a non-finite FP32 solve of the mixed path dropped
    // (the step moves to the FP64 solve), a non-finite FP64 solve failing the step
    LAUNCH(launch_after_inner(sizeof(T) == 4 && !x64, c->cs, c->red()));
    if (x64) {
      TRY(correct<double>(c));
    } else {
      TRY(correct<T>(c));
    }
  }
  std::swap(c->U, c->X);
  c->graph_ok = false;  // the graph was captured with the previous U and X
  c->generation += 1;
  return POLAR_OK;
}

// ---- graph mode: one theta-step as a CUDA graph whose refinement and Krylov loops are
// conditional WHILE nodes, so a step needs no host round trip until it has finished.

int capture_begin(polar_ctx* c, cudaGraph_t g, const cudaGraphNode_t* dep, size_t ndep) {
  CUDA_TRY(cudaStreamBeginCaptureToGraph(c->cap, g, dep, nullptr, ndep, cudaStreamCaptureModeThreadLocal));
  c->cs = c->cap;
  return POLAR_OK;
}

int capture_end(polar_ctx* c, std::vector<cudaGraphNode_t>* sinks) {
  if (sinks) {
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(c->cap, &status, nullptr, nullptr, &deps, nullptr, &nd));
    sinks->assign(deps, deps + nd);
  }
  cudaGraph_t out = nullptr;
  CUDA_TRY(cudaStreamEndCapture(c->cap, &out));
  c->cs = c->st;
  return POLAR_OK;
}

int add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
             cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
             cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  CUDA_TRY(cudaGraphAddNode(node, g, deps.data(), nullptr, deps.size(), &np));
  *body = np.conditional.phGraph_out[0];
  return POLAR_OK;
}

// Appends one inner solve to graph g after `deps`: scaled cast and BiCGStab set-up,
// WHILE (iterate) { iteration }, bookkeeping and correction of X; *sinks receives its
// last node and *iter_kernels the kernels of one iteration.  x64 selects the mixed path's
// FP64 Krylov solve over the FP32 V-cycle.
template <typename T>
int append_inner(polar_ctx* c, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                 bool x64, std::vector<cudaGraphNode_t>* sinks, int64_t* iter_kernels) {
  cudaGraphConditionalHandle hin;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&hin, g, 0, 0));
  TRY(capture_begin(c, g, deps.empty() ? nullptr : deps.data(), deps.size()));
  if (x64) {
    TRY(launch_refresh_all<double>(c, c->stamp64));  // FP64 factors, once per (alpha, beta)
    TRY(bicg_begin<double>(c, (CondHandle)hin));
  } else {
    TRY(bicg_begin<T>(c, (CondHandle)hin));
  }
  std::vector<cudaGraphNode_t> s1;
  TRY(capture_end(c, &s1));
  cudaGraphNode_t nin;
  cudaGraph_t bin;
  TRY(add_cond(g, s1, hin, cudaGraphCondTypeWhile, &nin, &bin));
  const int64_t a = c->launches;
  TRY(capture_begin(c, bin, nullptr, 0));
  if (x64) {
    TRY(krylov_iteration<double>(c, (CondHandle)hin));
  } else {
    TRY(krylov_iteration<T>(c, (CondHandle)hin));
  }
  TRY(capture_end(c, nullptr));
  *iter_kernels = c->launches - a;
  c->launches = a;
  TRY(capture_begin(c, g, &nin, 1));
  LAUNCH(launch_after_inner(sizeof(T) == 4 && !x64, c->cs, c->red()));
  if (x64) {
    TRY(correct<double>(c));
  } else {
    TRY(correct<T>(c));
  }
  TRY(capture_end(c, sinks));
  return POLAR_OK;
}

// Appends the direct inner solve (separable operators) to graph g: scaled cast, the
// transform / tridiagonal / inverse-transform kernels, bookkeeping and correction of X.
int append_direct(polar_ctx* c, cudaGraph_t g, std::vector<cudaGraphNode_t>* sinks) {
  TRY(capture_begin(c, g, nullptr, 0));
  TRY(direct_inner(c));
  LAUNCH(launch_after_inner(0, c->cs, c->red()));
  TRY(correct<double>(c));
  TRY(capture_end(c, sinks));
  return POLAR_OK;
}

// Appends one schedule-driven theta-step of this context to graph g (no dependencies on
// the graph's other nodes):
//   load step *kstep of the schedule -> IF (no earlier failure) {
//     right-hand side, refresh, X = U, residual, decide ->
//     WHILE (refine) { scaled cast, BiCGStab init -> WHILE (iterate) { iteration },
//                      correction, residual, decide } -> commit U = X, record result }
//   -> next step.
template <typename T>
int append_step(polar_ctx* c, cudaGraph_t g) {
  if (!c->cap) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  const int64_t l0 = c->launches;
  cudaGraphConditionalHandle hif, hout;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&hif, g, 0, 0));
  std::vector<cudaGraphNode_t> sinks;
  TRY(capture_begin(c, g, nullptr, 0));
  LAUNCH(launch_sched_begin(c->sched, c->kstep, c->sp, c->dout, (CondHandle)hif, c->cs, c->red()));
  TRY(capture_end(c, &sinks));
  cudaGraphNode_t nif, nout;
  cudaGraph_t bif, bout;
  TRY(add_cond(g, sinks, hif, cudaGraphCondTypeIf, &nif, &bif));
  CUDA_TRY(cudaGraphConditionalHandleCreate(&hout, bif, 0, 0));
  TRY(capture_begin(c, bif, nullptr, 0));
  TRY(rhs(c));
  TRY(launch_refresh_all<T>(c));
  LAUNCH(launch_copy(c->nv(), c->U, c->X, c->cs, c->red()));
  TRY(resid(c));
  LAUNCH(launch_refine_decide(c->sp, (CondHandle)hout, c->cs, c->red()));
  TRY(capture_end(c, &sinks));
  const int64_t l2 = c->launches;
  TRY(add_cond(bif, sinks, hout, cudaGraphCondTypeWhile, &nout, &bout));
  int64_t iter_k = 0, iter64_k = 0, fixed64 = 0;
  std::vector<cudaGraphNode_t> body;
  if (c->direct_now) {
    TRY(append_direct(c, bout, &body));
  } else if (sizeof(T) == 8) {
    TRY(append_inner<T>(c, bout, body, false, &body, &iter_k));
  } else {
    // mixed path: IF (FP32 refinement) { FP32 Krylov solve } then
    //             IF (stalled) { FP64 Krylov solve over the FP32 V-cycle }
    cudaGraphConditionalHandle h32, h64;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h32, bout, 0, 0));
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h64, bout, 0, 0));
    TRY(capture_begin(c, bout, nullptr, 0));
    LAUNCH(launch_choose_inner((CondHandle)h32, (CondHandle)h64, c->cs, c->red()));
    TRY(capture_end(c, &sinks));
    cudaGraphNode_t n32, n64;
    cudaGraph_t b32, b64;
    TRY(add_cond(bout, sinks, h32, cudaGraphCondTypeIf, &n32, &b32));
    std::vector<cudaGraphNode_t> none, tail;
    TRY(append_inner<T>(c, b32, none, false, &tail, &iter_k));
    TRY(add_cond(bout, std::vector<cudaGraphNode_t>{n32}, h64, cudaGraphCondTypeIf, &n64, &b64));
    const int64_t before64 = c->launches;
    TRY(append_inner<T>(c, b64, none, true, &tail, &iter64_k));
    fixed64 = c->launches - before64;
    body.assign(1, n64);
  }
  TRY(capture_begin(c, bout, body.data(), body.size()));
  TRY(resid(c));
  LAUNCH(launch_refine_decide(c->sp, (CondHandle)hout, c->cs, c->red()));
  TRY(capture_end(c, nullptr));
  const int64_t l3 = c->launches;  // (append_inner leaves the iteration kernels out)
  TRY(capture_begin(c, bif, &nout, 1));
  LAUNCH(launch_commit(c->nv(), c->U, c->X, c->cs, c->red()));
  LAUNCH(launch_sched_end(c->kstep, c->dout, c->cs, c->red()));
  TRY(capture_end(c, nullptr));
  TRY(capture_begin(c, g, &nif, 1));
  LAUNCH(launch_sched_next(c->kstep, c->cs));
  TRY(capture_end(c, nullptr));
  const int64_t l7 = c->launches;
  // kernels per executed step: fixed ones, per refinement sweep, per Krylov iteration
  // (a mixed sweep runs one of its two inner solves; counted as the FP32 one)
  c->graph_kernels_fixed = (l2 - l0) + (l7 - l3);
  c->graph_kernels_sweep = (l3 - l2) - fixed64;
  c->graph_kernels_iter = iter_k;
  c->graph_kernels_iter64 = iter64_k;
  c->launches = l0;  // captured launches run only when the graph is launched
  return POLAR_OK;
}

template <typename T>
int build_graph(polar_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  c->graph = g;
  TRY(append_step<T>(c, g));
  CUDA_TRY(cudaGraphInstantiate(&c->gexec, g, 0));
  c->graph_ok = true;
  return POLAR_OK;
}

// ends a capture left open by a failed graph build
void abandon_capture(polar_ctx* c) {
  cudaGraph_t junk = nullptr;
  cudaStreamCaptureStatus status;
  if (c->cap && cudaStreamIsCapturing(c->cap, &status) == cudaSuccess &&
      status != cudaStreamCaptureStatusNone)
    cudaStreamEndCapture(c->cap, &junk);
  if (junk) cudaGraphDestroy(junk);
  (void)cudaGetLastError();
  c->cs = c->st;
}

polar_solver_opts resolve_opts(const polar_solver_opts* o) {
  polar_solver_opts r;
  r.tol = 1e-14;
  r.max_iter = 500;
  r.max_refine = 12;
  r.inner_tol = 1e-5;
  r.method = POLAR_SOLVE_AUTO;
  r.reserved = 0;
  if (o) {
    if (o->tol > 0) r.tol = o->tol;
    if (o->max_iter > 0) r.max_iter = o->max_iter;
    if (o->max_refine > 0) r.max_refine = o->max_refine;
    if (o->inner_tol > 0) r.inner_tol = o->inner_tol;
    r.method = o->method;
  }
  return r;
}

// Picks the inner solve of the coming steps (the direct one for separable operators
// unless the caller asks for Krylov); a change invalidates the captured step graphs.
int choose_method(polar_ctx* c, const polar_solver_opts& o) {
  if (o.method != POLAR_SOLVE_AUTO && o.method != POLAR_SOLVE_KRYLOV &&
      o.method != POLAR_SOLVE_DIRECT)
    return fail(POLAR_EINVAL, "unknown solver method");
  if (o.method == POLAR_SOLVE_DIRECT && !c->separable)
    return fail(POLAR_EINVAL, "the direct solve needs a separable operator (uniform angles, "
                              "angle-independent coefficients)");
  const bool direct = c->separable && o.method != POLAR_SOLVE_KRYLOV;
  if (direct != c->direct_now) {
    c->direct_now = direct;
    c->graph_ok = false;
    c->generation += 1;
  }
  return POLAR_OK;
}

// Writes the step parameters to the device (the stream orders them before the step).
int set_step_params(polar_ctx* c, double alpha, double theta, const double* cf, const double* cg,
                    const polar_solver_opts& o) {
  StepParams& p = *c->sp_host;
  p = StepParams{};
  p.alpha = alpha;
  p.beta = theta;
  p.omt = 1.0 - theta;
  for (int q = 0; q < 4; ++q) {
    p.cf[q] = cf[q];
    p.cg[q] = cg[q];
  }
  p.tol = o.tol;
  p.inner_tol = (c->precision == POLAR_FP64) ? 0.0 : o.inner_tol;
  p.max_iter = o.max_iter;
  p.max_refine = o.max_refine;
  p.do_refresh = (alpha != c->cur_alpha || theta != c->cur_beta) ? 1 : 0;
  p.mixed = (c->precision == POLAR_MIXED && !c->direct_now) ? 1 : 0;
  CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_host, sizeof(StepParams), cudaMemcpyHostToDevice, c->st));
  c->cur_alpha = alpha;
  c->cur_beta = theta;
  return POLAR_OK;
}

// Step parameters of level k -> k+1 of a schedule (theta-step of Eq. 2.5 with the
// separable sources and Dirichlet data weighted at both levels).
int make_params(polar_ctx* c, double t0, double t1, double theta, const double* w_old,
                const double* w_new, const polar_solver_opts& o, double prev_alpha,
                double prev_beta, StepParams& p) {
  const double dt = t1 - t0;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(POLAR_EINVAL, "dt must be positive and finite");
  p = StepParams{};
  p.alpha = c->steady ? 0.0 : 1.0 / dt;  // steady solve: L U = f (no time derivative)
  p.beta = theta;
  p.omt = 1.0 - theta;
  for (int q = 0; q < c->nsrc; ++q) {
    if (!std::isfinite(w_old[q]) || !std::isfinite(w_new[q]))
      return fail(POLAR_ENONFINITE, "non-finite source weight");
    p.cf[q] = (1.0 - theta) * w_old[q] + theta * w_new[q];
    p.cg[q] = -((1.0 - theta) * w_old[q] + theta * w_new[q]);
  }
  p.tol = o.tol;
  p.inner_tol = (c->precision == POLAR_FP64) ? 0.0 : o.inner_tol;
  p.max_iter = o.max_iter;
  p.max_refine = o.max_refine;
  p.do_refresh = (p.alpha != prev_alpha || theta != prev_beta) ? 1 : 0;
  p.mixed = (c->precision == POLAR_MIXED && !c->direct_now) ? 1 : 0;
  return POLAR_OK;
}

int check_schedule_args(polar_ctx* c, int32_t nsteps, const double* t, double theta,
                        const double* w) {
  if (!c || !t) return fail(POLAR_EINVAL, "null argument");
  if (nsteps < 0) return fail(POLAR_EINVAL, "nsteps must be >= 0");
  if (c->nsrc > 0 && !w) return fail(POLAR_EINVAL, "weights required");
  if (!c->have_coeffs || !c->have_state) return fail(POLAR_ESTATE, "set_coeffs and set_state must come first");
  if (!(theta > 0.0 && theta <= 1.0)) return fail(POLAR_EINVAL, "theta must lie in (0, 1]");
  if (std::fabs(t[0] - c->t) > 1e-12 * std::max(1.0, std::fabs(c->t)))
    return fail(POLAR_EINVAL, "t[0] must equal the current time");
  for (int k = 0; k < nsteps; ++k)
    if (!(t[k + 1] > t[k]) || !std::isfinite(t[k + 1]))
      return fail(POLAR_EINVAL, "time levels must increase");
  return POLAR_OK;
}

// Uploads the schedule of an advance (graph mode) and resets the device step counter.
int load_schedule(polar_ctx* c, int32_t K, const double* t, double theta, const double* w,
                  const polar_solver_opts& o) {
  if (K > c->sched_cap) {
    const int cap = std::max(K, 2 * c->sched_cap);
    TRY(dalloc(c, &c->sched, (size_t)cap));
    TRY(dalloc(c, &c->dout, (size_t)cap));
    if (!c->kstep) TRY(dalloc(c, &c->kstep, 1));
    if (c->sched_host) cudaFreeHost(c->sched_host);
    if (c->out_host) cudaFreeHost(c->out_host);
    c->sched_host = nullptr;
    c->out_host = nullptr;
    CUDA_TRY(cudaMallocHost((void**)&c->sched_host, (size_t)cap * sizeof(StepParams)));
    CUDA_TRY(cudaMallocHost((void**)&c->out_host, (size_t)cap * sizeof(StepOut)));
    c->sched_cap = cap;
    // step graphs (this context's and any batch graph holding it) captured the old
    // schedule and result arrays: they must be captured again
    c->graph_ok = false;
    c->generation += 1;
  }
  const int Q = c->nsrc;
  double pa = c->cur_alpha, pb = c->cur_beta;
  for (int k = 0; k < K; ++k) {
    TRY(make_params(c, t[k], t[k + 1], theta, Q ? w + (size_t)k * Q : nullptr,
                    Q ? w + (size_t)(k + 1) * Q : nullptr, o, pa, pb, c->sched_host[k]));
    pa = c->sched_host[k].alpha;
    pb = theta;
  }
  CUDA_TRY(cudaMemcpyAsync(c->sched, c->sched_host, (size_t)K * sizeof(StepParams),
                           cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(cudaMemsetAsync(c->kstep, 0, sizeof(int), c->st));
  CUDA_TRY(cudaMemsetAsync(&c->ks->halt, 0, sizeof(int), c->st));
  return POLAR_OK;
}

// Reads the results of the K steps just run, fills stats, advances t to the last
// committed level and returns the first failure.
int finish_schedule(polar_ctx* c, int32_t K, const double* t, polar_step_stats* stats,
                    bool count_launches = true) {
  CUDA_TRY(cudaMemcpyAsync(c->out_host, c->dout, (size_t)K * sizeof(StepOut),
                           cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  int rc = POLAR_OK;
  int done = 0;
  for (int k = 0; k < K; ++k) {
    const StepOut& r = c->out_host[k];
    if (stats) {
      stats[k] = polar_step_stats{};
      stats[k].iters = r.iters;
      stats[k].refinements = r.sweeps;
      stats[k].status = r.status;
      stats[k].fp64_iters = r.iters64;
      stats[k].scaled_resid = r.scaled;
    }
    if (!count_launches) {
      if (r.status != POLAR_ESTATE) {
        c->cur_alpha = c->sched_host[k].alpha;
        c->cur_beta = c->sched_host[k].beta;
      }
    } else if (r.status != POLAR_ESTATE) {
      c->launches += 2 + c->graph_kernels_fixed + (int64_t)std::max(r.sweeps - 1, 0) * c->graph_kernels_sweep +
                     (int64_t)(r.iters - r.iters64) * c->graph_kernels_iter +
                     (int64_t)r.iters64 * c->graph_kernels_iter64;
      c->cur_alpha = c->sched_host[k].alpha;  // the refresh state follows every executed step
      c->cur_beta = c->sched_host[k].beta;
    } else {
      c->launches += 2;
    }
    if (rc == POLAR_OK && r.status != POLAR_OK) {
      rc = r.status;
      if (r.status == POLAR_ENONFINITE) fail(rc, "non-finite value in the solve of step " + std::to_string(k));
      else fail(rc, "step " + std::to_string(k) + ": refinement did not reach the tolerance (scaled residual " +
                        std::to_string(r.scaled) + ")");
    }
    if (r.status == POLAR_OK && rc == POLAR_OK) done = k + 1;
  }
  c->t = t[done];
  return rc;
}

// Host-driven steps (per-kernel timing on, or no graph): one step at a time.
int advance_eager(polar_ctx* c, int32_t K, const double* t, double theta, const double* w,
                  const polar_solver_opts& o, polar_step_stats* stats) {
  const int Q = c->nsrc;
  for (int k = 0; k < K; ++k) {
    polar_step_stats st{};
    StepParams& p = *c->sp_host;
    int rc = make_params(c, t[k], t[k + 1], theta, Q ? w + (size_t)k * Q : nullptr,
                         Q ? w + (size_t)(k + 1) * Q : nullptr, o, c->cur_alpha, c->cur_beta, p);
    if (rc == POLAR_OK) {
      CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_host, sizeof(StepParams), cudaMemcpyHostToDevice, c->st));
      c->cur_alpha = p.alpha;
      c->cur_beta = theta;
      rc = (c->precision == POLAR_FP64) ? step_eager<double>(c, st) : step_eager<float>(c, st);
    }
    st.status = rc;
    if (stats) stats[k] = st;
    if (rc != POLAR_OK) {
      if (stats)
        for (int q = k + 1; q < K; ++q) {
          stats[q] = polar_step_stats{};
          stats[q].status = POLAR_ESTATE;
        }
      return rc;
    }
    c->t = t[k + 1];  // the exact level, not an accumulated sum
  }
  return POLAR_OK;
}

// Refresh for the first step of a schedule, then tune the ring tiles on that data.
int prepare_tuning(polar_ctx* c, const double* t, double theta, const double* w,
                   const polar_solver_opts& o) {
  const int Q = c->nsrc;
  StepParams& p = *c->sp_host;
  TRY(make_params(c, t[0], t[1], theta, Q ? w : nullptr, Q ? w + Q : nullptr, o, -1.0, -1.0, p));
  CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_host, sizeof(StepParams), cudaMemcpyHostToDevice, c->st));
  if (c->precision == POLAR_FP64) {
    TRY(launch_refresh_all<double>(c));
    TRY(tune_rings<double>(c));
  } else {
    TRY(launch_refresh_all<float>(c));
    TRY(tune_rings<float>(c));
    // the FP64 ring solves of the mixed path's FP64 solve
    TRY(launch_refresh_all<double>(c, c->stamp64));
    TRY(tune_rings<double>(c));
  }
  c->tuned = true;
  c->cur_alpha = p.alpha;
  c->cur_beta = theta;
  c->graph_ok = false;  // captured launches must use the tuned shapes
  c->generation += 1;
  return POLAR_OK;
}

int advance(polar_ctx* c, int32_t K, const double* t, double theta, const double* w,
            const polar_solver_opts* opts, polar_step_stats* stats) {
  TRY(check_schedule_args(c, K, t, theta, w));
  CUDA_TRY(cudaSetDevice(c->device));
  c->cs = c->st;
  const polar_solver_opts o = resolve_opts(opts);
  TRY(choose_method(c, o));
  if (K == 0) return POLAR_OK;
  if (c->autotune && !c->tuned && !c->direct_now) TRY(prepare_tuning(c, t, theta, w, o));
  if (!c->use_graph || c->timing) return advance_eager(c, K, t, theta, w, o, stats);
  TRY(load_schedule(c, K, t, theta, w, o));
  if (!c->graph_ok) {
    const int rc = (c->precision == POLAR_FP64) ? build_graph<double>(c) : build_graph<float>(c);
    if (rc != POLAR_OK) {
      abandon_capture(c);
      c->use_graph = false;
      return advance_eager(c, K, t, theta, w, o, stats);
    }
  }
  for (int k = 0; k < K; ++k) CUDA_TRY(cudaGraphLaunch(c->gexec, c->st));
  return finish_schedule(c, K, t, stats);
}

// Whether V L (hence S = alpha V + beta V L) is symmetric: every coupling equals its mirror
// (radial faces, angular faces with the wrap, the origin's faces).  The conservative
// scheme without drift stores one conductance per face on both sides, so the test is exact.
bool is_symmetric(const HLevel& L) {
  const int m = L.m, n = L.n;
  for (int j = 0; j < n; ++j) {
    if (L.o[j] != L.w[L.q(1, j)]) return false;
    const int jm = (j == 0) ? n - 1 : j - 1;
    for (int i = 1; i <= m; ++i) {
      if (i > 1 && L.w[L.q(i, j)] != L.e[L.q(i - 1, j)]) return false;
      if (L.s[L.q(i, j)] != L.nn[L.q(i, jm)]) return false;
    }
  }
  return true;
}

// Separability of the fine level (the direct solve applies): every ring's coefficients
// (control volume, row sum, the four couplings) equal across the angles, the two angular
// couplings of a row equal, the origin's couplings equal -- to 1e-9 relative: uniform
// angles computed as 2 pi j / n already differ in their spacings by ~1e-12 relative at
// n = 8192, and the direct solve of the j = 0 coefficients is then a preconditioner whose
// FP64 refinement contracts by about kappa * 1e-9 per sweep.
constexpr double kSepTol = 1e-9;
bool is_separable(const HLevel& L) {
  const int m = L.m, n = L.n;
  auto ring_const = [&](const std::vector<double>& a, int i) {
    const double ref = a[L.q(i, 0)];
    double amax = 0.0;
    for (int j = 0; j < n; ++j) amax = std::max(amax, std::fabs(a[L.q(i, j)]));
    for (int j = 0; j < n; ++j)
      if (std::fabs(a[L.q(i, j)] - ref) > kSepTol * amax) return false;
    return true;
  };
  for (int i = 1; i <= m; ++i) {
    for (const std::vector<double>* a : {&L.vol, &L.rs, &L.w, &L.e, &L.s, &L.nn})
      if (!ring_const(*a, i)) return false;
    for (int j = 0; j < n; ++j) {
      const double sv = L.s[L.q(i, j)], nv = L.nn[L.q(i, j)];
      if (std::fabs(sv - nv) > kSepTol * std::max(std::fabs(sv), std::fabs(nv))) return false;
    }
  }
  double omax = 0.0;
  for (double v : L.o) omax = std::max(omax, std::fabs(v));
  for (double v : L.o)
    if (std::fabs(v - L.o[0]) > kSepTol * omax) return false;
  return true;
}

// Device data of the direct solve for a separable fine level: the rings' coefficients,
// the transform tables and the work arrays (allocated on first use).
int setup_direct(polar_ctx* c, const HLevel& H) {
  int M = 0, logM = 0, rw = 0;
  c->separable = is_separable(H) && fft_plan_sizes(c->n, &M, &logM, &rw);
  if (!c->separable) return POLAR_OK;
  const int m = c->m, n = c->n, nh = n / 2 + 1;
  FftPlan& P = c->plan;
  SepRings& R = c->sep;
  if (!c->fx_r) {
    double *twr, *twi, *chr, *chi, *bhr, *bhi, *lam, *vol, *rs, *w, *e, *sv;
    TRY(dalloc(c, &twr, (size_t)M / 2));
    TRY(dalloc(c, &twi, (size_t)M / 2));
    TRY(dalloc(c, &chr, (size_t)n));
    TRY(dalloc(c, &chi, (size_t)n));
    TRY(dalloc(c, &bhr, (size_t)M));
    TRY(dalloc(c, &bhi, (size_t)M));
    TRY(dalloc(c, &lam, (size_t)nh));
    double** ring[] = {&vol, &rs, &w, &e, &sv};
    for (double** p : ring) TRY(dalloc(c, p, (size_t)m));
    TRY(dalloc(c, &c->fx_r, (size_t)m * nh));
    TRY(dalloc(c, &c->fx_i, (size_t)m * nh));
    TRY(dalloc(c, &c->fcp, (size_t)m * nh));
    TRY(dalloc(c, &c->fzv, (size_t)m));
    P = FftPlan{n, nh, M, logM, rw, twr, twi, chr, chi, bhr, bhi, lam};
    R.vol = vol;
    R.rs = rs;
    R.w = w;
    R.e = e;
    R.s = sv;
    CUDA_TRY(cudaStreamSynchronize(c->st));  // zeroed before the uploads below
    std::vector<double> htwr, htwi, hchr, hchi, hlam;
    fft_host_tables(n, M, htwr, htwi, hchr, hchi, hlam);
    TRY(upload(twr, htwr));
    TRY(upload(twi, htwi));
    TRY(upload(chr, hchr));
    TRY(upload(chi, hchi));
    TRY(upload(lam, hlam));
    if (M != n) LAUNCH(launch_chirp_filter(P, bhr, bhi, c->st));
  }
  R.m = m;
  std::vector<double> a[5];
  for (int i = 1; i <= m; ++i) {
    const size_t q = H.q(i, 0);
    a[0].push_back(H.vol[q]);
    a[1].push_back(H.rs[q]);
    a[2].push_back(H.w[q]);
    a[3].push_back(H.e[q]);
    a[4].push_back(H.s[q]);
  }
  double* dst[5] = {const_cast<double*>(R.vol), const_cast<double*>(R.rs),
                    const_cast<double*>(R.w), const_cast<double*>(R.e),
                    const_cast<double*>(R.s)};
  for (int k = 0; k < 5; ++k) TRY(upload(dst[k], a[k]));
  R.vol0 = H.vol0;
  R.rs0 = H.rs0;
  R.o = H.o[0];
  R.osum = 0.0;
  for (double v : H.o) R.osum += v;
  return POLAR_OK;
}

// ---- batched execution: one launch per kernel class and phase for all instances.
//
// A batch step graph is built in two passes of the same code: the plan pass collects every
// launch's per-slot argument table and slot list in a host image; the image goes to the
// device in one copy; the capture pass records the launches, whose tables now sit at the
// same offsets of the device arena.  Every instance keeps its own grid partition (a slot's
// virtual blocks), so its arithmetic -- and its result -- is the same as when it runs alone.
// Active-instance masks, written between launches by k_mask_b at the points where instances
// start or stop (step start, refinement decisions, Krylov iterations), decide which slots a
// launch serves; WHILE nodes loop while any instance is still active.

// the masks of a batch step (one int per instance each)
enum { MK_STEP, MK_REF, MK_32, MK_64, MK_DIR, MK_IT32, MK_IT64, MK_COUNT };

struct BatchBuild {
  polar_batch* b = nullptr;
  bool plan = true;                  // plan pass (collect) or capture pass (launch)
  std::vector<unsigned char> image;  // arena image (plan pass)
  unsigned char* dev = nullptr;      // arena (capture pass)
  size_t off = 0;
  cudaStream_t cs = nullptr;         // capture stream
  int64_t launches = 0;              // kernels captured so far
  int sms = 152;                     // SMs of the device (grid sizes)
  int* mask[MK_COUNT] = {};

  // a table in the arena: appended in the plan pass, its device address in the capture pass
  template <class A>
  const A* put(const std::vector<A>& v) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += std::max<size_t>(v.size(), 1) * sizeof(A);
    if (plan) {
      image.resize(off);
      if (!v.empty()) std::memcpy(image.data() + at, v.data(), v.size() * sizeof(A));
      return nullptr;
    }
    return reinterpret_cast<const A*>(dev + at);
  }
  // launch helper: counts, checks, skips in the plan pass
  template <class F>
  int launch(F f) {
    if (plan) return POLAR_OK;
    const int k = f();
    if (k < 0) {
      const cudaError_t e = cudaGetLastError();
      return fail(POLAR_ECUDA, std::string("batched launch: ") + cudaGetErrorString(e));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(POLAR_ECUDA, std::string("batched launch: ") + cudaGetErrorString(e));
    launches += k;
    return POLAR_OK;
  }
  // grid of a launch with `items` work items: per_sm blocks per SM at most
  int grid(int64_t items, int per_sm) const {
    return (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * per_sm));
  }
};

// per-instance facts the planner groups by
struct BInst {
  polar_ctx* c;
  int idx;          // position in the batch (and in the masks)
  bool mixed;       // FP32 inner solves (and the FP64 fallback)
  bool direct;      // separable: the direct inner solve
};

int stencil_grid(const Shape& sh) {
  const Tiling t = make_tiling(sh);
  return t.ntiles > kMaxBlocks ? kMaxBlocks : t.ntiles;
}

template <typename T>
StArgs<T> st_args(const polar_ctx* c, const T* x, T* y, const T* d1, const T* b) {
  StArgs<T> a{};
  a.L = views<T>(c)[0];
  a.par = c->par();
  a.x = x;
  a.b = b;
  a.y = y;
  a.d1 = d1;
  a.red = c->red();
  a.t = make_tiling(a.L.sh);
  return a;
}

template <typename T>
VecArgs<T> vargs(const polar_ctx* c) {
  VecArgs<T> a{};
  a.nv = c->nv();
  a.red = c->red();
  a.sp = c->sp;
  return a;
}

int64_t slot_items(const std::vector<BSlot>& s) {
  int64_t t = 0;
  for (const BSlot& x : s) t += x.vg;
  return t;
}

// Stencil launches: instances grouped by their tiling's TK (the block shape).
template <typename T, class MakeArgs>
int batch_stencil(BatchBuild& B, int mode, const std::vector<const BInst*>& list, int mk,
                  MakeArgs make) {
  for (int TK = 32; TK <= 256; TK <<= 1) {
    std::vector<BSlot> slots;
    std::vector<StArgs<T>> args;
    for (const BInst* i : list)
      if (make_tiling(i->c->sh0()).TK == TK) {
        slots.push_back(BSlot{i->idx, stencil_grid(i->c->sh0())});
        args.push_back(make(i->c));
      }
    if (slots.empty()) continue;
    const StArgs<T>* A = B.put(args);
    const BSlot* S = B.put(slots);
    const int g = B.grid(slot_items(slots), 8);
    const int* M = B.mask[mk];
    TRY(B.launch([&] { return launch_stencil_b<T>(mode, A, S, (int)slots.size(), M, g, TK, B.cs); }));
  }
  return POLAR_OK;
}

// Vector-kernel launch over `list` (grid_for(nv) blocks each).
template <typename T, class MakeArgs>
int batch_vec(BatchBuild& B, int kind, const std::vector<const BInst*>& list, int mk,
              MakeArgs make) {
  if (list.empty()) return POLAR_OK;
  std::vector<VecArgs<T>> args;
  std::vector<BSlot> slots;
  for (const BInst* i : list) {
    args.push_back(make(i->c));
    slots.push_back(BSlot{i->idx, grid_for(i->c->nv(), 256)});
  }
  const VecArgs<T>* A = B.put(args);
  const BSlot* S = B.put(slots);
  const int g = B.grid(slot_items(slots), 8);
  const int* M = B.mask[mk];
  return B.launch([&] { return launch_vec_b<T>(kind, A, S, (int)slots.size(), M, g, B.cs); });
}

CtlArgs ctl_args(const BInst* i) {
  polar_ctx* c = i->c;
  CtlArgs a{};
  a.sched = c->sched;
  a.kstep = c->kstep;
  a.kstep_w = c->kstep;
  a.sp = c->sp;
  a.out = c->dout;
  a.ks = c->ks;
  a.inst = i->idx;
  return a;
}

int batch_ctl(BatchBuild& B, int kind, const std::vector<const BInst*>& list, int gate) {
  if (list.empty()) return POLAR_OK;
  std::vector<CtlArgs> args;
  for (const BInst* i : list) args.push_back(ctl_args(i));
  const CtlArgs* A = B.put(args);
  return B.launch([&] { return launch_ctl_b(kind, A, (int)args.size(), gate, B.cs); });
}

// mask `mk` of the instances of `list` (the others keep 0); cond (if any) = any active
int batch_mask(BatchBuild& B, const std::vector<const BInst*>& list, int gate, int need_running,
               int mk, CondHandle cond) {
  if (list.empty() && !cond) return POLAR_OK;
  std::vector<CtlArgs> args;
  for (const BInst* i : list) args.push_back(ctl_args(i));
  const CtlArgs* A = B.put(args);
  int* M = B.mask[mk];
  return B.launch([&] {
    return launch_mask_b(A, (int)args.size(), gate, need_running, M, cond, B.cs);
  });
}

// Inputs and outputs of one V-cycle per instance (level 0 vectors in precision T).
template <typename T>
struct VIO {
  const T* b;
  T* x;
};

// One batched V(1,1) cycle of every instance of `list`: down through the levels
// (pre-smoothing of odd then even rings, restriction), the coarsest solves, up again
// (post-smoothing of even then odd rings).  A phase serves the instances that have the
// level; ring launches are grouped by tile shape (the block and cluster shape of a
// launch).  Each instance checks its own `done` flag, as its lone cycle does.
template <typename T>
int batch_vcycle(BatchBuild& B, const std::vector<const BInst*>& list,
                 const std::vector<VIO<T>>& io, int mk) {
  int lmax = 0;
  for (const BInst* i : list) lmax = std::max(lmax, i->c->nlev() - 1);
  auto bof = [&](int k, int l) { return l == 0 ? io[k].b : static_cast<const T*>(coarse_b<T>(list[k]->c, l)); };
  auto xof = [&](int k, int l) { return l == 0 ? io[k].x : coarse_x<T>(list[k]->c, l); };
  auto ring_phase = [&](int l, int mode, int parity) -> int {
    // (shape -> instances) for this level, mode and parity
    std::vector<std::pair<RingShape, std::vector<int>>> groups;
    for (int k = 0; k < (int)list.size(); ++k) {
      polar_ctx* c = list[k]->c;
      if (l >= c->nlev() - 1) continue;
      const LevelView<T>& L = views<T>(c)[l];
      const int nl = parity ? L.sh.no : L.sh.ne;
      if (nl == 0) continue;
      const RingShape* t = tile<T>(c, l, mode, parity);
      const RingShape s = t ? *t : ring_default<T>(nl, L.sh.n);
      bool found = false;
      for (auto& g : groups)
        if (std::memcmp(&g.first, &s, sizeof(RingShape)) == 0) {
          g.second.push_back(k);
          found = true;
        }
      if (!found) groups.push_back({s, {k}});
    }
    for (auto& g : groups) {
      const RingShape& s = g.first;
      std::vector<RingArgs<T>> args;
      std::vector<BSlot> slots;
      for (int k : g.second) {
        polar_ctx* c = list[k]->c;
        const std::vector<LevelView<T>>& L = views<T>(c);
        RingArgs<T> a{};
        a.L = L[l];
        a.C = L[l + 1];
        a.b = bof(k, l);
        a.x = xof(k, l);
        a.X = mode == RING_POST ? coarse_x<T>(c, l + 1) : nullptr;
        a.par = c->par();
        a.done = &c->ks->done;
        a.parity = parity;
        a.mode = mode;
        const int nl = parity ? L[l].sh.no : L[l].sh.ne;
        slots.push_back(BSlot{list[k]->idx, (nl + s.RW - 1) / s.RW});
        args.push_back(a);
      }
      const RingArgs<T>* A = B.put(args);
      const BSlot* S = B.put(slots);
      // columns of CS CTAs (one work item each): a few CTAs per SM in all
      const int per = std::max(1, 2048 / (s.RW * s.TW));
      const int cols = (int)std::max<int64_t>(
          1, std::min<int64_t>(slot_items(slots), (int64_t)B.sms * per / s.CS));
      const int* M = B.mask[mk];
      TRY(B.launch([&] { return launch_ring_b<T>(s, A, S, (int)slots.size(), M, cols, B.cs); }));
    }
    return POLAR_OK;
  };
  for (int l = 0; l < lmax; ++l) {
    TRY(ring_phase(l, RING_PRE, 1));
    TRY(ring_phase(l, RING_PRE, 0));
    std::vector<BSlot> slots;
    std::vector<RestrictArgs<T>> args;
    for (int k = 0; k < (int)list.size(); ++k) {
      polar_ctx* c = list[k]->c;
      if (l >= c->nlev() - 1) continue;
      const std::vector<LevelView<T>>& L = views<T>(c);
      args.push_back(RestrictArgs<T>{L[l], L[l + 1], xof(k, l), coarse_b<T>(c, l + 1), c->par(),
                                     &c->ks->done});
      slots.push_back(BSlot{list[k]->idx, grid_for((size_t)L[l + 1].sh.m * L[l].sh.n, 256)});
    }
    if (!slots.empty()) {
      const RestrictArgs<T>* A = B.put(args);
      const BSlot* S = B.put(slots);
      const int g = B.grid(slot_items(slots), 8);
      const int* M = B.mask[mk];
      TRY(B.launch([&] { return launch_restrict_b<T>(A, S, (int)slots.size(), M, g, B.cs); }));
    }
  }
  // coarsest levels, grouped by their launch shape
  std::vector<std::pair<std::pair<int, int>, std::vector<int>>> cg;
  for (int k = 0; k < (int)list.size(); ++k) {
    const LevelView<T>& L = views<T>(list[k]->c).back();
    int P = 0, TW = 0;
    coarsest_shape<T>(L.sh.n, &P, &TW);
    bool found = false;
    for (auto& g : cg)
      if (g.first == std::make_pair(P, TW)) {
        g.second.push_back(k);
        found = true;
      }
    if (!found) cg.push_back({{P, TW}, {k}});
  }
  for (auto& g : cg) {
    std::vector<CoarsestArgs<T>> args;
    std::vector<BSlot> slots;
    for (int k : g.second) {
      polar_ctx* c = list[k]->c;
      const int lc = c->nlev() - 1;
      CoarsestArgs<T> a{};
      a.L = views<T>(c)[lc];
      a.b = bof(k, lc);
      a.x = xof(k, lc);
      a.par = c->par();
      a.done = &c->ks->done;
      slots.push_back(BSlot{list[k]->idx, 1});
      args.push_back(a);
    }
    const CoarsestArgs<T>* A = B.put(args);
    const BSlot* S = B.put(slots);
    const int P = g.first.first, TW = g.first.second;
    const int gr = B.grid(slot_items(slots), 2);
    const int* M = B.mask[mk];
    TRY(B.launch([&] { return launch_coarsest_b<T>(P, TW, 0, A, S, (int)slots.size(), M, gr, B.cs); }));
  }
  for (int l = lmax - 1; l >= 0; --l) {
    TRY(ring_phase(l, RING_POST, 0));
    TRY(ring_phase(l, RING_POST, 1));
  }
  return POLAR_OK;
}

// Per-step refresh of every instance of `list` in precision T (the refresh kernel checks
// each instance's do_refresh, or its stamp when `stamped`), then the coarsest levels'
// Schur data and, when stamped, the stamps.
template <typename T>
int batch_refresh(BatchBuild& B, const std::vector<const BInst*>& list, bool stamped, int mk) {
  if (list.empty()) return POLAR_OK;
  std::vector<RefreshArgs> args;
  std::vector<BSlot> slots;
  for (const BInst* i : list) {
    polar_ctx* c = i->c;
    std::vector<LevelView<T>> vt = views<T>(c);
    int nb = 0;
    args.push_back(make_refresh_args<T>(c->v64.data(), vt.data(), c->nlev(), c->sp, c->ws,
                                        stamped ? c->stamp64 : nullptr, &nb));
    slots.push_back(BSlot{i->idx, nb});
  }
  const RefreshArgs* A = B.put(args);
  const BSlot* S = B.put(slots);
  const int g = B.grid(slot_items(slots), 2);
  const int* M = B.mask[mk];
  TRY(B.launch([&] { return launch_refresh_b<T>(A, S, (int)slots.size(), M, g, B.cs); }));
  std::vector<std::pair<std::pair<int, int>, std::vector<const BInst*>>> cg;
  for (const BInst* i : list) {
    int P = 0, TW = 0;
    coarsest_shape<T>(views<T>(i->c).back().sh.n, &P, &TW);
    bool found = false;
    for (auto& g2 : cg)
      if (g2.first == std::make_pair(P, TW)) {
        g2.second.push_back(i);
        found = true;
      }
    if (!found) cg.push_back({{P, TW}, {i}});
  }
  for (auto& g2 : cg) {
    std::vector<CoarsestArgs<T>> sargs;
    std::vector<BSlot> ss;
    for (const BInst* i : g2.second) {
      polar_ctx* c = i->c;
      CoarsestArgs<T> a{};
      a.L = views<T>(c).back();
      a.sp = c->sp;
      a.stamp = stamped ? c->stamp64 : nullptr;
      ss.push_back(BSlot{i->idx, 1});
      sargs.push_back(a);
    }
    const CoarsestArgs<T>* A2 = B.put(sargs);
    const BSlot* S2 = B.put(ss);
    const int P = g2.first.first, TW = g2.first.second;
    const int gr = B.grid(slot_items(ss), 2);
    TRY(B.launch([&] { return launch_coarsest_b<T>(P, TW, 1, A2, S2, (int)ss.size(), M, gr, B.cs); }));
  }
  if (stamped) {
    std::vector<double*> stamps;
    std::vector<const StepParams*> sps;
    for (const BInst* i : list) {
      stamps.push_back(i->c->stamp64);
      sps.push_back(i->c->sp);
    }
    double* const* ST = B.put(stamps);
    const StepParams* const* SP = B.put(sps);
    TRY(B.launch([&] { return launch_stamp_b(S, (int)slots.size(), M, ST, SP, B.cs); }));
  }
  return POLAR_OK;
}

// One Krylov iteration of every instance of `list` in precision T: CG for the symmetric
// ones, BiCGStab for the others (each instance's kernels in its lone order).
template <typename T>
int batch_iteration(BatchBuild& B, const std::vector<const BInst*>& list, int mk) {
  std::vector<const BInst*> cgl, bil;
  for (const BInst* i : list) (i->c->symmetric ? cgl : bil).push_back(i);
  std::vector<VIO<T>> io;
  for (const BInst* i : list) {
    KVecs<T>& k = kvecs<T>(i->c);
    io.push_back(i->c->symmetric ? VIO<T>{k.r, k.phat} : VIO<T>{k.p, k.phat});
  }
  TRY(batch_vcycle<T>(B, list, io, mk));
  TRY(batch_vec<T>(B, V_CG_RHO, cgl, mk, [](polar_ctx* c) {
    VecArgs<T> a = vargs<T>(c);
    a.v0 = kvecs<T>(c).r;
    a.v1 = kvecs<T>(c).phat;
    return a;
  }));
  TRY(batch_vec<T>(B, V_CG_P, cgl, mk, [](polar_ctx* c) {
    VecArgs<T> a = vargs<T>(c);
    a.v0 = kvecs<T>(c).p;
    a.v1 = kvecs<T>(c).phat;
    return a;
  }));
  // q = S p (CG) and v = S phat (BiCGStab), both the stencil's DOTV mode
  TRY(batch_stencil<T>(B, M_DOTV, list, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    return c->symmetric ? st_args<T>(c, k.p, k.v, k.p, nullptr)
                        : st_args<T>(c, k.phat, k.v, k.rhat, nullptr);
  }));
  TRY(batch_vec<T>(B, V_CG_UPDATE, cgl, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    VecArgs<T> a = vargs<T>(c);
    a.v0 = k.d;
    a.v1 = k.p;
    a.v2 = k.r;
    a.v3 = k.v;
    a.diag = views<T>(c)[0].diag;
    a.sc = views<T>(c)[0].sc;
    return a;
  }));
  if (bil.empty()) return POLAR_OK;
  TRY(batch_vec<T>(B, V_BICG_S, bil, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    VecArgs<T> a = vargs<T>(c);
    a.v0 = k.r;
    a.v1 = k.v;
    a.v2 = k.s;
    return a;
  }));
  std::vector<VIO<T>> io2;
  for (const BInst* i : bil) io2.push_back(VIO<T>{kvecs<T>(i->c).s, kvecs<T>(i->c).shat});
  TRY(batch_vcycle<T>(B, bil, io2, mk));
  TRY(batch_stencil<T>(B, M_DOTT, bil, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    return st_args<T>(c, k.shat, k.t, k.s, nullptr);
  }));
  TRY(batch_vec<T>(B, V_BICG_UPDATE, bil, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    VecArgs<T> a = vargs<T>(c);
    a.v0 = k.d;
    a.v1 = k.phat;
    a.v2 = k.shat;
    a.v3 = k.r;
    a.v4 = k.s;
    a.v5 = k.t;
    a.v6 = k.rhat;
    a.diag = views<T>(c)[0].diag;
    a.sc = views<T>(c)[0].sc;
    return a;
  }));
  TRY(batch_vec<T>(B, V_BICG_P, bil, mk, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    VecArgs<T> a = vargs<T>(c);
    a.v0 = k.p;
    a.v1 = k.r;
    a.v2 = k.v;
    return a;
  }));
  return POLAR_OK;
}

// Batched direct solves (separable instances): scaled cast, transform / modes / inverse.
int batch_direct(BatchBuild& B, const std::vector<const BInst*>& list, int mk, int gate) {
  if (list.empty()) return POLAR_OK;
  TRY(batch_vec<double>(B, V_SCALE_CAST, list, mk, [](polar_ctx* c) {
    VecArgs<double> a = vargs<double>(c);
    a.v0 = c->kv64.r;
    a.w0 = c->r64;
    return a;
  }));
  std::vector<DirectArgs> args;
  std::vector<BSlot> sr, sm;
  std::vector<KrylovScalars*> ks;
  size_t smem = 0;
  for (const BInst* i : list) {
    polar_ctx* c = i->c;
    DirectArgs a{};
    a.sh = c->sh0();
    a.P = c->plan;
    a.R = c->sep;
    a.par = c->par();
    a.b = c->kv64.r;
    a.x = c->kv64.d;
    a.Xr = c->fx_r;
    a.Xi = c->fx_i;
    a.cp = c->fcp;
    a.z = c->fzv;
    const int rw = c->plan.rw;
    sr.push_back(BSlot{i->idx, (a.sh.no + rw - 1) / rw + (a.sh.ne + rw - 1) / rw});
    sm.push_back(BSlot{i->idx, (c->plan.nh + 127) / 128});
    ks.push_back(c->ks);
    smem = std::max(smem, dft_smem(c->plan));
    args.push_back(a);
  }
  const DirectArgs* A = B.put(args);
  const BSlot* Sr = B.put(sr);
  const BSlot* Sm = B.put(sm);
  KrylovScalars* const* KS = B.put(ks);
  const int gr = B.grid(slot_items(sr), 2), gm = B.grid(slot_items(sm), 8);
  const int* M = B.mask[mk];
  TRY(B.launch([&] {
    return launch_direct_b(A, Sr, Sm, (int)sr.size(), M, KS, gr, gm, smem, B.cs);
  }));
  TRY(batch_ctl(B, C_AFTER_INNER, list, gate));
  return batch_vec<double>(B, V_CORRECT, list, mk, [](polar_ctx* c) {
    VecArgs<double> a = vargs<double>(c);
    a.v0 = c->kv64.d;
    a.w0 = c->X;
    return a;
  });
}

// capture helpers of the batch (its own capture stream)
int bcap_begin(BatchBuild& B, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps) {
  if (B.plan) return POLAR_OK;
  CUDA_TRY(cudaStreamBeginCaptureToGraph(B.cs, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                         deps.size(), cudaStreamCaptureModeThreadLocal));
  return POLAR_OK;
}
int bcap_end(BatchBuild& B, std::vector<cudaGraphNode_t>* sinks) {
  if (B.plan) return POLAR_OK;
  if (sinks) {
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(B.cs, &status, nullptr, nullptr, &deps, nullptr, &nd));
    sinks->assign(deps, deps + nd);
  }
  cudaGraph_t out = nullptr;
  CUDA_TRY(cudaStreamEndCapture(B.cs, &out));
  return POLAR_OK;
}
int bcond(BatchBuild& B, cudaGraph_t g, CondHandle* h) {
  *h = 0;
  if (B.plan) return POLAR_OK;
  cudaGraphConditionalHandle c;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&c, g, 0, 0));
  *h = (CondHandle)c;
  return POLAR_OK;
}
int bwhile(BatchBuild& B, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, CondHandle h,
           cudaGraphNode_t* node, cudaGraph_t* body) {
  if (B.plan) {
    *node = nullptr;
    *body = nullptr;
    return POLAR_OK;
  }
  return add_cond(g, deps, (cudaGraphConditionalHandle)h, cudaGraphCondTypeWhile, node, body);
}

// One inner Krylov solve of the instances of `list` in precision T (gate: the branch, whose
// mask mk_branch is set), appended to graph g after `deps`: set-up, WHILE (any iterating)
// { iteration }, counts and correction of X.  *sinks receives the last node.
template <typename T>
int batch_inner(BatchBuild& B, cudaGraph_t g, std::vector<cudaGraphNode_t> deps,
                const std::vector<const BInst*>& list, int gate, int mk_branch, int mk_it,
                bool fp64_refresh, std::vector<cudaGraphNode_t>* sinks, int64_t* per_iter) {
  CondHandle hit = 0;
  TRY(bcond(B, g, &hit));
  TRY(bcap_begin(B, g, deps));
  if (fp64_refresh) {  // mixed instances entering their FP64 solve: FP64 factors on demand
    std::vector<const BInst*> mixed;
    for (const BInst* i : list)
      if (i->mixed) mixed.push_back(i);
    TRY(batch_refresh<double>(B, mixed, true, mk_branch));
  }
  TRY(batch_vec<T>(B, V_SCALE_CAST, list, mk_branch, [](polar_ctx* c) {
    VecArgs<T> a = vargs<T>(c);
    a.v0 = kvecs<T>(c).r;
    a.w0 = c->r64;
    return a;
  }));
  TRY(batch_vec<T>(B, V_BICG_INIT, list, mk_branch, [](polar_ctx* c) {
    KVecs<T>& k = kvecs<T>(c);
    VecArgs<T> a = vargs<T>(c);
    a.v0 = k.r;
    a.v1 = k.rhat;
    a.v2 = k.p;
    a.v3 = k.v;
    a.v4 = k.d;
    return a;
  }));
  TRY(batch_mask(B, list, gate, 1, mk_it, hit));
  std::vector<cudaGraphNode_t> s1;
  TRY(bcap_end(B, &s1));
  cudaGraphNode_t nit;
  cudaGraph_t bit;
  TRY(bwhile(B, g, s1, hit, &nit, &bit));
  const int64_t a0 = B.launches;
  TRY(bcap_begin(B, bit, {}));
  TRY(batch_iteration<T>(B, list, mk_it));
  TRY(batch_mask(B, list, gate, 1, mk_it, hit));
  TRY(bcap_end(B, nullptr));
  *per_iter = B.launches - a0;
  TRY(bcap_begin(B, g, std::vector<cudaGraphNode_t>{nit}));
  TRY(batch_ctl(B, C_AFTER_INNER, list, gate));
  TRY(batch_vec<T>(B, V_CORRECT, list, mk_branch, [](polar_ctx* c) {
    VecArgs<T> a = vargs<T>(c);
    a.v0 = kvecs<T>(c).d;
    a.w0 = c->X;
    return a;
  }));
  TRY(bcap_end(B, sinks));
  return POLAR_OK;
}

// The FP64 residual of the instances of `list` (r64 = e - S X with its max-norm reductions).
int batch_resid(BatchBuild& B, const std::vector<const BInst*>& list, int mk) {
  return batch_stencil<double>(B, M_RESID64, list, mk, [](polar_ctx* c) {
    return st_args<double>(c, c->X, c->r64, nullptr, c->e);
  });
}

// Masks after a refinement decision: the refining instances (and `cond` = any), then
// those of each inner-solve branch.
int batch_masks(BatchBuild& B, const std::vector<const BInst*>& all,
                const std::vector<const BInst*>& krylov32, const std::vector<const BInst*>& krylov64,
                const std::vector<const BInst*>& direct, CondHandle cond) {
  TRY(batch_mask(B, all, G_REFINE, 0, MK_REF, cond));
  TRY(batch_mask(B, krylov32, G_32, 0, MK_32, 0));
  TRY(batch_mask(B, krylov64, G_64, 0, MK_64, 0));
  return batch_mask(B, direct, G_64, 0, MK_DIR, 0);
}

// One theta-step of the instances of a group, appended to the step graph as a branch:
//   schedule step -> right-hand sides, refreshes, X = U, residuals, decisions ->
//   WHILE (any refining) { FP32 solves | FP64 solves | direct solves, residuals,
//                          decisions } -> commit, results, next step.
int batch_group_step(BatchBuild& B, cudaGraph_t g, const std::vector<const BInst*>& members,
                     polar_batch::Group* grp) {
  std::vector<const BInst*> all, krylov32, krylov64, direct, f64, f32;
  for (const BInst* i : members) {
    all.push_back(i);
    if (i->direct) {
      direct.push_back(i);
    } else {
      krylov64.push_back(i);           // FP64 instances and the mixed ones' FP64 solve
      if (i->mixed) krylov32.push_back(i);
    }
    (i->mixed ? f32 : f64).push_back(i);
  }
  CondHandle hre = 0;
  TRY(bcond(B, g, &hre));
  const int64_t l0 = B.launches;
  TRY(bcap_begin(B, g, {}));
  TRY(batch_ctl(B, C_SCHED_BEGIN, all, G_ALL));
  TRY(batch_mask(B, all, G_STEP, 0, MK_STEP, 0));
  for (int TK = 32; TK <= 256; TK <<= 1) {
    std::vector<BSlot> slots;
    std::vector<RhsArgs> args;
    for (const BInst* i : all) {
      polar_ctx* c = i->c;
      if (make_tiling(c->sh0()).TK != TK) continue;
      RhsArgs a{};
      a.L = c->v64[0];
      a.sp = c->sp;
      a.u = c->U;
      a.e = c->e;
      a.nsrc = c->nsrc;
      for (int q = 0; q < c->nsrc; ++q) {
        a.vsrc[q] = c->vsrc[q];
        a.bnd[q] = c->bnd[q];
      }
      a.red = c->red();
      a.t = make_tiling(c->sh0());
      args.push_back(a);
      slots.push_back(BSlot{i->idx, stencil_grid(c->sh0())});
    }
    if (slots.empty()) continue;
    const RhsArgs* A = B.put(args);
    const BSlot* S = B.put(slots);
    const int gr = B.grid(slot_items(slots), 8);
    const int* M = B.mask[MK_STEP];
    TRY(B.launch([&] { return launch_rhs_b(A, S, (int)slots.size(), M, gr, TK, B.cs); }));
  }
  TRY(batch_refresh<double>(B, f64, false, MK_STEP));
  TRY(batch_refresh<float>(B, f32, false, MK_STEP));
  TRY(batch_vec<double>(B, V_COPY, all, MK_STEP, [](polar_ctx* c) {
    VecArgs<double> a = vargs<double>(c);
    a.w0 = c->U;
    a.w1 = c->X;
    a.flag = 0;
    return a;
  }));
  TRY(batch_resid(B, all, MK_STEP));
  TRY(batch_ctl(B, C_DECIDE, all, G_STEP));
  TRY(batch_masks(B, all, krylov32, krylov64, direct, hre));
  std::vector<cudaGraphNode_t> sinks;
  TRY(bcap_end(B, &sinks));
  const int64_t l1 = B.launches;
  cudaGraphNode_t nre;
  cudaGraph_t bre;
  TRY(bwhile(B, g, sinks, hre, &nre, &bre));
  std::vector<cudaGraphNode_t> tail;
  int64_t it32 = 0, it64 = 0;
  if (!krylov32.empty())
    TRY(batch_inner<float>(B, bre, tail, krylov32, G_32, MK_32, MK_IT32, false, &tail, &it32));
  if (!krylov64.empty())
    TRY(batch_inner<double>(B, bre, tail, krylov64, G_64, MK_64, MK_IT64, !krylov32.empty(), &tail,
                            &it64));
  TRY(bcap_begin(B, bre, tail));
  TRY(batch_direct(B, direct, MK_DIR, G_64));
  TRY(batch_resid(B, all, MK_REF));
  TRY(batch_ctl(B, C_DECIDE, all, G_REFINE));
  TRY(batch_masks(B, all, krylov32, krylov64, direct, hre));
  TRY(bcap_end(B, nullptr));
  const int64_t l2 = B.launches;
  TRY(bcap_begin(B, g, std::vector<cudaGraphNode_t>{nre}));
  TRY(batch_vec<double>(B, V_COPY, all, MK_STEP, [](polar_ctx* c) {
    VecArgs<double> a = vargs<double>(c);
    a.w0 = c->X;
    a.w1 = c->U;
    a.flag = 1;  // commit only a converged step
    return a;
  }));
  TRY(batch_ctl(B, C_SCHED_END, all, G_STEP));
  TRY(batch_ctl(B, C_SCHED_NEXT, all, G_ALL));
  TRY(bcap_end(B, nullptr));
  const int64_t l3 = B.launches;
  grp->fixed = (l1 - l0) + (l3 - l2);
  grp->sweep = (l2 - l1) - it32 - it64;
  grp->iter32 = it32;
  grp->iter64 = it64;
  return POLAR_OK;
}

// One theta-step of every instance as one graph: the groups' steps are parallel branches
// (a group's latency-bound phases -- coarse levels, the last iterations of its slowest
// instance -- overlap the other groups' work).
int batch_step_graph(BatchBuild& B, cudaGraph_t g, const std::vector<BInst>& inst) {
  for (int k = 0; k < MK_COUNT; ++k)  // masks first: same arena offsets in both passes
    B.mask[k] = const_cast<int*>(B.put(std::vector<int>(inst.size(), 0)));
  for (polar_batch::Group& grp : B.b->groups) {
    std::vector<const BInst*> members;
    for (int i : grp.members) members.push_back(&inst[i]);
    TRY(batch_group_step(B, g, members, &grp));
  }
  return POLAR_OK;
}

// Groups of the batch: instances sorted by size, cut into up to kBatchGroups contiguous
// groups of about equal total points.
constexpr int kBatchGroups = 8;
void make_batch_groups(polar_batch* b) {
  const int count = (int)b->ctx.size();
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->ctx[x]->nv() < b->ctx[y]->nv(); });
  double total = 0;
  for (polar_ctx* c : b->ctx) total += (double)c->nv();
  const int G = std::min(kBatchGroups, count);
  b->groups.assign(1, polar_batch::Group{});
  double acc = 0;
  for (int i : order) {
    if (acc > total * (double)b->groups.size() / G && (int)b->groups.size() < G &&
        !b->groups.back().members.empty())
      b->groups.emplace_back();
    b->groups.back().members.push_back(i);
    acc += (double)b->ctx[i]->nv();
  }
}

// Assembles the fine level from c->hk, coarsens it, uploads every level and marks the
// per-step parts and the step graphs stale.
int reassemble(polar_ctx* c) {
  std::vector<HLevel> H(c->nlev());
  if (c->scheme == POLAR_SCHEME_CONSERVATIVE) {
    assemble_conservative(c->r, c->theta, c->hk, H[0]);
  } else {
    assemble_paper(c->r, c->theta, c->hk, H[0]);
  }
  c->symmetric = is_symmetric(H[0]);
  TRY(setup_direct(c, H[0]));
  for (int l = 0; l + 1 < c->nlev(); ++l) coarsen(H[l], H[l + 1]);
  for (int l = 0; l < c->nlev(); ++l) TRY(upload_level(c, l, H[l]));
  c->cur_alpha = c->cur_beta = -1.0;  // the per-step parts must be refreshed
  // new coefficients: the mixed path tries its FP32 solve again from the next step
  CUDA_TRY(cudaMemsetAsync(&c->ks->sticky64, 0, sizeof(int), c->st));
  if (c->stamp64) CUDA_TRY(cudaMemsetAsync(c->stamp64, 0, 2 * sizeof(double), c->st));
  c->graph_ok = false;
  c->generation += 1;
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

// The same from coefficients already on the device (conservative scheme): level 0 and
// the radial hierarchy assembled by kernels on the context's stream.  The operator is
// taken as non-separable (Krylov inner solve); `symmetric` says whether it has no drift.
int reassemble_device(polar_ctx* c, const AsmIn& in, bool symmetric) {
  auto lev = [&](int l) {
    DevLevel& d = c->lv[l];
    return CoarsenLevel{d.sh, d.w, d.e, d.s, d.nn, d.rs, d.vol, d.o, d.ia, d.ib, d.sc};
  };
  DevLevel& d0 = c->lv[0];
  LAUNCH(launch_assemble_level0(in, d0.sh, d0.vol, d0.w, d0.e, d0.s, d0.nn, d0.rs, d0.o, d0.sc,
                                c->st));
  for (int l = 0; l + 1 < c->nlev(); ++l) LAUNCH(launch_coarsen(lev(l), lev(l + 1), c->st));
  if (c->precision == POLAR_MIXED) {
    for (DevLevel& d : c->lv) {
      const double* s64[] = {d.w, d.e, d.s, d.nn, d.ia, d.ib};
      float* s32[] = {d.w32, d.e32, d.s32, d.nn32, d.ia32, d.ib32};
      for (int a = 0; a < 6; ++a) LAUNCH(launch_to_float(d.sh.nv, s64[a], s32[a], c->st));
      LAUNCH(launch_to_float((size_t)c->n, d.o, d.o32, c->st));
    }
  }
  // The arrays keep their addresses, so the captured graphs stay valid unless the solver's
  // structure changes (CG for a symmetric operator, BiCGStab otherwise; a separable
  // operator's direct solve is left through choose_method).  The next step refreshes the
  // factors: cur_alpha is reset, and so are the mixed path's FP64 stamp and countdown.
  if (symmetric != c->symmetric) {
    c->symmetric = symmetric;
    c->graph_ok = false;
    c->generation += 1;
  }
  c->separable = false;
  c->cur_alpha = c->cur_beta = -1.0;
  CUDA_TRY(cudaMemsetAsync(&c->ks->sticky64, 0, sizeof(int), c->st));
  if (c->stamp64) CUDA_TRY(cudaMemsetAsync(c->stamp64, 0, 2 * sizeof(double), c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

// Radii and angles of the mesh on the device (r, then theta, then n scratch values).
int ensure_mesh_dev(polar_ctx* c) {
  if (c->mesh_dev) return POLAR_OK;
  const int m = c->m, n = c->n;
  TRY(dalloc(c, &c->mesh_dev, (size_t)m + 2 + 2 * (size_t)n));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  std::vector<double> mesh(c->r);
  mesh.insert(mesh.end(), c->theta.begin(), c->theta.end());
  CUDA_TRY(cudaMemcpy(c->mesh_dev, mesh.data(), mesh.size() * sizeof(double),
                      cudaMemcpyHostToDevice));
  return POLAR_OK;
}

// (Re)builds the batch's step graph: plan pass, arena upload, capture pass.
int build_batch_graph(polar_batch* b) {
  CUDA_TRY(cudaStreamSynchronize(b->st));  // no launch of the old graph still reads the arena
  if (b->ex) cudaGraphExecDestroy(b->ex);
  if (b->g) cudaGraphDestroy(b->g);
  b->ex = nullptr;
  b->g = nullptr;
  if (!b->cap) CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  make_batch_groups(b);
  std::vector<BInst> inst;
  for (int i = 0; i < (int)b->ctx.size(); ++i) {
    polar_ctx* c = b->ctx[i];
    inst.push_back(BInst{c, i, c->precision == POLAR_MIXED && !c->direct_now, c->direct_now});
  }
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BatchBuild plan;
  plan.b = b;
  plan.plan = true;
  plan.sms = sms;
  TRY(batch_step_graph(plan, nullptr, inst));
  polar_ctx* c0 = b->ctx[0];
  if (plan.off > b->arena_bytes) {
    if (b->arena) {
      if (c0->free_fn) c0->free_fn(b->arena, c0->st, c0->alloc_user);
      else cudaFree(b->arena);
    }
    b->arena = nullptr;
    b->arena_bytes = 0;
    void* q = nullptr;
    if (c0->alloc) {
      q = c0->alloc(plan.off, c0->st, c0->alloc_user);
      if (!q) return fail(POLAR_ENOMEM, "the caller's allocator returned NULL (batch tables)");
    } else {
      CUDA_TRY(cudaMalloc(&q, plan.off));
    }
    b->arena = q;
    b->arena_bytes = plan.off;
  }
  CUDA_TRY(cudaMemcpy(b->arena, plan.image.data(), plan.off, cudaMemcpyHostToDevice));
  BatchBuild cap;
  cap.b = b;
  cap.plan = false;
  cap.dev = static_cast<unsigned char*>(b->arena);
  cap.cs = b->cap;
  cap.sms = sms;
  CUDA_TRY(cudaGraphCreate(&b->g, 0));
  const int rc = batch_step_graph(cap, b->g, inst);
  if (rc != POLAR_OK) {
    cudaGraph_t junk = nullptr;
    cudaStreamCaptureStatus status;
    if (cudaStreamIsCapturing(b->cap, &status) == cudaSuccess &&
        status != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(b->cap, &junk);
    if (junk) cudaGraphDestroy(junk);
    (void)cudaGetLastError();
    return rc;
  }
  if (cap.off != plan.off) return fail(POLAR_ECUDA, "batch plan and capture disagree");
  CUDA_TRY(cudaGraphInstantiate(&b->ex, b->g, 0));
  b->gens.resize(b->ctx.size());
  for (size_t i = 0; i < b->ctx.size(); ++i) b->gens[i] = b->ctx[i]->generation;
  return POLAR_OK;
}

}  // namespace

namespace polar {
// error reporting for the other translation units of the library (polar_last_error)
int report_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }
}  // namespace polar

// ======================================================================= C ABI
extern "C" {

const char* polar_last_error(void) { return g_err.c_str(); }

int polar_mesh_create(const polar_mesh_desc* d, polar_ctx** out) {
  if (!d || !out) return fail(POLAR_EINVAL, "null argument");
  *out = nullptr;
  const int m = d->nr, n = d->ntheta;
  if (m < 2 || n < 4) return fail(POLAR_EINVAL, "need nr >= 2 and ntheta >= 4");
  if (n > 16384) return fail(POLAR_EINVAL, "ntheta above 16384 is not supported");
  if (!d->r || !d->theta) return fail(POLAR_EINVAL, "r and theta are required");
  if (d->scheme != POLAR_SCHEME_CONSERVATIVE && d->scheme != POLAR_SCHEME_PAPER)
    return fail(POLAR_EINVAL, "unknown scheme");
  if (d->precision != POLAR_FP64 && d->precision != POLAR_MIXED)
    return fail(POLAR_EINVAL, "unknown precision");
  if ((d->alloc != nullptr) != (d->free != nullptr))
    return fail(POLAR_EINVAL, "alloc and free hooks go together");
  if ((size_t)m * (size_t)n > (size_t)1 << 31) return fail(POLAR_EINVAL, "mesh too large");
  if (d->r[0] != 0.0 || d->r[m + 1] != 1.0) return fail(POLAR_EINVAL, "r must run from 0 to 1");
  for (int i = 1; i <= m + 1; ++i)
    if (!(d->r[i] > d->r[i - 1]) || !std::isfinite(d->r[i]))
      return fail(POLAR_EINVAL, "r must be strictly increasing");
  for (int j = 0; j < n; ++j)
    if (!std::isfinite(d->theta[j])) return fail(POLAR_EINVAL, "theta must be finite");
  for (int j = 1; j < n; ++j)
    if (!(d->theta[j] > d->theta[j - 1])) return fail(POLAR_EINVAL, "theta must be strictly increasing");
  if (!(d->theta[n - 1] - d->theta[0] < 2.0 * M_PI))
    return fail(POLAR_EINVAL, "theta must span less than 2 pi");

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return fail(POLAR_ECUDA, "no CUDA device");
  }
  polar_ctx* c = new polar_ctx();
  c->m = m;
  c->n = n;
  c->scheme = d->scheme;
  c->precision = d->precision;
  c->st = static_cast<cudaStream_t>(d->stream);
  c->cs = c->st;
  c->alloc = d->alloc;
  c->free_fn = d->free;
  c->alloc_user = d->alloc_user;
  cudaGetDevice(&c->device);
  c->r.assign(d->r, d->r + m + 2);
  c->theta.assign(d->theta, d->theta + n);
  int rc = alloc_levels(c);
  auto chk = [&](int v) {
    if (rc == POLAR_OK) rc = v;
  };
  if (rc == POLAR_OK) {
    const size_t nv = c->nv();
    chk(dalloc(c, &c->U, nv));
    chk(dalloc(c, &c->X, nv));
    chk(dalloc(c, &c->e, nv));
    chk(dalloc(c, &c->r64, nv));
    chk(dalloc(c, &c->io, c->N()));
    chk(dalloc(c, &c->sp, 1));
    // FP64 Krylov vectors in both paths: the mixed path falls back to an FP64 Krylov
    // solve over its FP32 V-cycle when its FP32 refinement stalls
    chk(alloc_kvecs(c, c->kv64));
    if (c->precision == POLAR_MIXED) chk(alloc_kvecs(c, c->kv32));
    chk(dalloc(c, &c->part, (size_t)kMaxBlocks * 4));
    if (c->precision == POLAR_MIXED) chk(dalloc(c, &c->stamp64, 2));  // zero: no factors yet
    chk(dalloc(c, &c->ks, 1));
  }
  if (rc == POLAR_OK && cudaMallocHost((void**)&c->ks_host, sizeof(KrylovScalars)) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = fail(POLAR_ENOMEM, "cudaMallocHost failed");
  }
  if (rc == POLAR_OK && cudaMallocHost((void**)&c->sp_host, sizeof(StepParams)) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = fail(POLAR_ENOMEM, "cudaMallocHost failed");
  }
  if (rc == POLAR_OK && cudaStreamSynchronize(c->st) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = fail(POLAR_ECUDA, "stream synchronisation after the allocations failed");
  }
  if (rc != POLAR_OK) {
    cudaStreamSynchronize(c->st);
    release(c);
    delete c;
    return rc;
  }
  *out = c;
  return POLAR_OK;
}

int polar_mesh_destroy(polar_ctx* c) {
  if (!c) return POLAR_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  release(c);
  delete c;
  return POLAR_OK;
}

int polar_set_coeffs(polar_ctx* c, const polar_coeffs* k) {
  if (!c || !k) return fail(POLAR_EINVAL, "null argument");
  if (k->memory != POLAR_HOST && k->memory != POLAR_DEVICE) return fail(POLAR_EINVAL, "bad memory flag");
  if (k->nsrc < 0 || k->nsrc > 4) return fail(POLAR_EINVAL, "nsrc must lie in [0, 4]");
  for (int q = 0; q < k->nsrc; ++q)
    if (!k->src[q] || !k->bnd[q]) return fail(POLAR_EINVAL, "src[q] and bnd[q] are required");
  if (!std::isfinite(k->d_const) || !std::isfinite(k->b_const) || !std::isfinite(k->d0))
    return fail(POLAR_ENONFINITE, "non-finite scalar coefficient");
  if (c->scheme == POLAR_SCHEME_PAPER && (k->v_rface || k->v_tface))
    return fail(POLAR_EINVAL, "the PAPER scheme takes the drift as e_node");
  if (c->scheme == POLAR_SCHEME_CONSERVATIVE && k->e_node)
    return fail(POLAR_EINVAL, "e_node belongs to the PAPER scheme");
  CUDA_TRY(cudaSetDevice(c->device));
  const int m = c->m, n = c->n;
  const size_t N = c->N(), nf = (size_t)(m + 1) * n, nt = (size_t)m * n;
  HostCoeffs K;
  K.d_const = k->d_const;
  K.d0 = k->d0;
  if (k->d_rface) TRY(fetch(k->d_rface, nf, k->memory, K.dr));
  if (k->d_tface) TRY(fetch(k->d_tface, nt, k->memory, K.dt));
  if (k->v_rface) TRY(fetch(k->v_rface, nf, k->memory, K.vr));
  if (k->v_tface) TRY(fetch(k->v_tface, nt, k->memory, K.vt));
  if (k->e_node) TRY(fetch(k->e_node, N, k->memory, K.en));
  if (k->b) {
    TRY(fetch(k->b, N, k->memory, K.b));
  } else {
    K.b.assign(N, k->b_const);
  }
  std::vector<std::vector<double>> srcs(k->nsrc), bnds(k->nsrc);
  for (int q = 0; q < k->nsrc; ++q) {
    TRY(fetch(k->src[q], N, k->memory, srcs[q]));
    TRY(fetch(k->bnd[q], (size_t)n, k->memory, bnds[q]));
  }
  c->hk = std::move(K);
  TRY(reassemble(c));
  // sources in the split layout, scaled by the control volumes
  for (int q = 0; q < k->nsrc; ++q) {
    if (!c->vsrc[q]) {  // allocated on first use, reused by later set_coeffs calls
      TRY(dalloc(c, &c->vsrc[q], c->nv()));
      TRY(dalloc(c, &c->bnd[q], (size_t)n));
      CUDA_TRY(cudaStreamSynchronize(c->st));  // zeroed before the copies below
    }
    CUDA_TRY(cudaMemcpy(c->io, srcs[q].data(), N * sizeof(double), cudaMemcpyHostToDevice));
    LAUNCH(launch_pack(c->sh0(), c->io, c->lv[0].vol, c->vsrc[q], c->st));
    CUDA_TRY(cudaMemcpy(c->bnd[q], bnds[q].data(), n * sizeof(double), cudaMemcpyHostToDevice));
    c->bnd_host[q] = std::move(bnds[q]);
  }
  c->nsrc = k->nsrc;
  c->graph_ok = false;                // the step graph bakes in the source count
  CUDA_TRY(cudaStreamSynchronize(c->st));
  c->have_coeffs = true;
  return POLAR_OK;
}

int polar_set_state(polar_ctx* c, const double* u, double t, int32_t memory) {
  if (!c || !u) return fail(POLAR_EINVAL, "null argument");
  if (memory != POLAR_HOST && memory != POLAR_DEVICE) return fail(POLAR_EINVAL, "bad memory flag");
  if (!std::isfinite(t)) return fail(POLAR_ENONFINITE, "non-finite time");
  CUDA_TRY(cudaSetDevice(c->device));
  const size_t N = c->N();
  CUDA_TRY(cudaMemcpyAsync(c->io, u, N * sizeof(double),
                           memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->st));
  c->ks_host->done = 0;
  CUDA_TRY(cudaMemsetAsync(&c->ks->done, 0, sizeof(int), c->st));
  LAUNCH(launch_check_finite(N, c->io, c->st, c->red()));
  TRY(read_scalars(c));
  if (c->ks_host->done == 3) return fail(POLAR_ENONFINITE, "non-finite value in the state");
  LAUNCH(launch_pack(c->sh0(), c->io, nullptr, c->U, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  c->t = t;
  c->have_state = true;
  return POLAR_OK;
}

int polar_get_state(polar_ctx* c, double* u, double* t, int32_t memory) {
  if (!c) return fail(POLAR_EINVAL, "null argument");
  if (!c->have_state) return fail(POLAR_ESTATE, "no state set");
  if (memory != POLAR_HOST && memory != POLAR_DEVICE) return fail(POLAR_EINVAL, "bad memory flag");
  CUDA_TRY(cudaSetDevice(c->device));
  if (u) {
    LAUNCH(launch_unpack(c->sh0(), c->U, nullptr, c->io, c->st));
    CUDA_TRY(cudaMemcpyAsync(u, c->io, c->N() * sizeof(double),
                             memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->st));
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  if (t) *t = c->t;
  return POLAR_OK;
}

int polar_step(polar_ctx* c, double dt, double theta, const double* w_old, const double* w_new,
               const polar_solver_opts* opts, polar_step_stats* stats) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(POLAR_EINVAL, "dt must be positive and finite");
  if (c->nsrc > 0 && (!w_old || !w_new)) return fail(POLAR_EINVAL, "source weights required");
  const double t[2] = {c->t, c->t + dt};
  double w[8];
  for (int q = 0; q < c->nsrc; ++q) {
    w[q] = w_old[q];
    w[c->nsrc + q] = w_new[q];
  }
  return advance(c, 1, t, theta, c->nsrc ? w : nullptr, opts, stats);
}

int polar_advance(polar_ctx* c, int32_t nsteps, const double* t, double theta, const double* w,
                  const polar_solver_opts* opts, polar_step_stats* stats) {
  return advance(c, nsteps, t, theta, w, opts, stats);
}

int polar_solve_steady(polar_ctx* c, const double* w, const polar_solver_opts* opts,
                       polar_step_stats* stats) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  if (c->nsrc > 0 && !w) return fail(POLAR_EINVAL, "source weights required");
  // one step of the theta-machinery with alpha = 0 and theta = 1: (V L) U = V f + Dirichlet
  // terms, started from the current state; the time stays where it is
  const double t0 = c->t;
  const double t[2] = {t0, t0 + 1.0};
  double ww[8];
  for (int q = 0; q < c->nsrc; ++q) ww[q] = ww[c->nsrc + q] = w[q];
  c->steady = true;
  const int rc = advance(c, 1, t, 1.0, c->nsrc ? ww : nullptr, opts, stats);
  c->steady = false;
  c->t = t0;
  return rc;
}

int polar_face_drift(polar_ctx* c, double mobility, const double* g, double* v_rface,
                     double* v_tface, int32_t memory) {
  if (!c || !g || !v_rface || !v_tface) return fail(POLAR_EINVAL, "null argument");
  if (!c->have_state) return fail(POLAR_ESTATE, "no state set");
  if (memory != POLAR_HOST && memory != POLAR_DEVICE) return fail(POLAR_EINVAL, "bad memory flag");
  if (!std::isfinite(mobility)) return fail(POLAR_EINVAL, "non-finite mobility");
  CUDA_TRY(cudaSetDevice(c->device));
  const int m = c->m, n = c->n;
  TRY(ensure_mesh_dev(c));
  double* gdev = c->mesh_dev + m + 2 + n;
  CUDA_TRY(cudaMemcpyAsync(gdev, g, n * sizeof(double),
                           memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->st));
  const size_t nr = (size_t)(m + 1) * n, nt = (size_t)m * n;
  // the faces are written to the Krylov work vectors first (they hold nv >= (m+1) n doubles)
  double* vr = memory == POLAR_DEVICE ? v_rface : c->kv64.r;
  double* vt = memory == POLAR_DEVICE ? v_tface : c->kv64.s;
  LAUNCH(launch_unpack(c->sh0(), c->U, nullptr, c->io, c->st));
  LAUNCH(launch_face_drift(m, n, c->io, c->mesh_dev, c->mesh_dev + m + 2, gdev, mobility, vr, vt,
                           c->st));
  if (memory == POLAR_HOST) {
    CUDA_TRY(cudaMemcpyAsync(v_rface, vr, nr * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(cudaMemcpyAsync(v_tface, vt, nt * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

// Anderson step of the Gummel map (the potential's state g = G(x), x in phi_prev): the
// new difference columns, gamma from the normal equations by Cholesky (the oldest column
// dropped while a pivot is not above 1e-13 of the largest diagonal entry), then the
// extrapolated potential written over the state.
static int anderson_update(polar_gummel* G, int* cols, int& ncols, bool& have_last) {
  polar_ctx* c = G->phi;
  const Shape sh = c->sh0();
  const size_t nv = c->nv();
  const int depth = G->d.depth;
  int slot = 0;
  if (have_last) {
    if (ncols < depth) {
      slot = ncols;
      cols[ncols++] = slot;
    } else {
      slot = cols[0];
      for (int a = 0; a + 1 < ncols; ++a) cols[a] = cols[a + 1];
      cols[ncols - 1] = slot;
    }
  }
  LAUNCH(launch_aa_columns(sh, c->U, G->phi_prev, G->f_last, G->x_last, G->f_cur, G->dF[slot],
                           G->dX[slot], have_last, c->st));
  CUDA_TRY(cudaMemcpyAsync(G->x_last, G->phi_prev, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                           c->st));
  std::swap(G->f_last, G->f_cur);  // f_last now holds this residual
  have_last = true;
  for (int first = 0; first < ncols; ++first) {
    const int k = ncols - first;
    AndersonCols dc{};
    for (int a = 0; a < k; ++a) dc.v[a] = G->dF[cols[first + a]];
    dc.v[k] = G->f_last;
    for (int a = k + 1; a <= kMaxAnderson; ++a) dc.v[a] = G->f_last;
    dc.count = k + 1;
    const int nd = k * (k + 1) / 2 + k;
    LAUNCH(launch_aa_dots(sh, dc, G->partials, kAABlocks, c->st));
    G->partials_host.resize((size_t)kAABlocks * nd);
    CUDA_TRY(cudaMemcpyAsync(G->partials_host.data(), G->partials,
                             G->partials_host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
    std::vector<double> dots(nd, 0.0);
    for (int b = 0; b < kAABlocks; ++b)
      for (int q = 0; q < nd; ++q) dots[q] += G->partials_host[(size_t)b * nd + q];
    // Gram matrix (upper triangle row by row) and right-hand side, in the kernel's order
    std::vector<double> A((size_t)k * k), rhs(k);
    int q = 0;
    for (int a = 0; a < k; ++a) {
      for (int b = a; b < k; ++b) A[(size_t)a * k + b] = A[(size_t)b * k + a] = dots[q++];
      rhs[a] = dots[q++];
    }
    double top = 0.0;
    for (int a = 0; a < k; ++a) top = std::max(top, A[(size_t)a * k + a]);
    std::vector<double> L((size_t)k * k, 0.0);
    bool ok = true;
    for (int i = 0; i < k && ok; ++i)
      for (int j = 0; j <= i; ++j) {
        double acc = A[(size_t)i * k + j];
        for (int p = 0; p < j; ++p) acc -= L[(size_t)i * k + p] * L[(size_t)j * k + p];
        if (i == j) {
          if (!(acc > 1e-13 * top)) {
            ok = false;
            break;
          }
          L[(size_t)i * k + i] = std::sqrt(acc);
        } else {
          L[(size_t)i * k + j] = acc / L[(size_t)j * k + j];
        }
      }
    if (!ok) continue;  // drop the oldest column
    std::vector<double> y(k), gam(k);
    for (int i = 0; i < k; ++i) {
      double acc = rhs[i];
      for (int p = 0; p < i; ++p) acc -= L[(size_t)i * k + p] * y[p];
      y[i] = acc / L[(size_t)i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double acc = y[i];
      for (int p = i + 1; p < k; ++p) acc -= L[(size_t)p * k + i] * gam[p];
      gam[i] = acc / L[(size_t)i * k + i];
    }
    AndersonCols cx{}, cf{};
    for (int a = 0; a < k; ++a) {
      cx.v[a] = G->dX[cols[first + a]];
      cf.v[a] = G->dF[cols[first + a]];
    }
    cx.count = cf.count = k;
    LAUNCH(launch_aa_update(sh, cx, cf, gam.data(), c->U, c->st));
    break;
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

int polar_gummel_create(polar_ctx* phi, polar_ctx* electrons, polar_ctx* holes,
                        const polar_gummel_desc* d, polar_gummel** out) {
  if (!phi || !electrons || !holes || !d || !out) return fail(POLAR_EINVAL, "null argument");
  *out = nullptr;
  if (phi == electrons || phi == holes || electrons == holes)
    return fail(POLAR_EINVAL, "the potential and the two carriers need three contexts");
  polar_ctx* cs[3] = {phi, electrons, holes};
  for (polar_ctx* c : cs) {
    if (c->m != phi->m || c->n != phi->n || c->r != phi->r || c->theta != phi->theta ||
        c->device != phi->device)
      return fail(POLAR_EINVAL, "the three contexts must share one mesh and device");
    if (c->scheme != POLAR_SCHEME_CONSERVATIVE)
      return fail(POLAR_EINVAL, "the coupled system runs on the conservative scheme");
    if (!c->have_coeffs) return fail(POLAR_ESTATE, "set the coefficients of all three contexts first");
  }
  if (d->src_electrons < 0 || d->src_electrons >= phi->nsrc || d->src_holes < 0 ||
      d->src_holes >= phi->nsrc || d->src_electrons == d->src_holes)
    return fail(POLAR_EINVAL, "the carrier source slots must be two distinct sources of the potential");
  if (!std::isfinite(d->mobility[0]) || !std::isfinite(d->mobility[1]) || !(d->tol > 0) ||
      d->max_iter < 1 || d->depth < 0 || d->depth > kMaxAnderson)
    return fail(POLAR_EINVAL, "bad mobility, tol, max_iter or depth");
  CUDA_TRY(cudaSetDevice(phi->device));
  polar_gummel* G = new polar_gummel();
  G->phi = phi;
  G->car[0] = electrons;
  G->car[1] = holes;
  G->d = *d;
  const size_t nv = phi->nv();
  int rc = POLAR_OK;
  if (rc == POLAR_OK) rc = dalloc(phi, &G->save[0], nv);
  if (rc == POLAR_OK) rc = dalloc(phi, &G->save[1], nv);
  if (rc == POLAR_OK) rc = dalloc(phi, &G->phi_prev, nv);
  if (rc == POLAR_OK) rc = dalloc(phi, &G->change, 2);
  if (rc == POLAR_OK && d->depth > 0) {
    rc = dalloc(phi, &G->x_last, nv);
    if (rc == POLAR_OK) rc = dalloc(phi, &G->f_last, nv);
    if (rc == POLAR_OK) rc = dalloc(phi, &G->f_cur, nv);
    for (int a = 0; a < d->depth && rc == POLAR_OK; ++a) {
      rc = dalloc(phi, &G->dX[a], nv);
      if (rc == POLAR_OK) rc = dalloc(phi, &G->dF[a], nv);
    }
    if (rc == POLAR_OK) rc = dalloc(phi, &G->partials, (size_t)kAABlocks * 20);
  }
  if (rc == POLAR_OK) rc = ensure_mesh_dev(phi);
  const size_t nf = (size_t)(phi->m + 1) * phi->n, nt = (size_t)phi->m * phi->n;
  for (int k = 0; k < 2 && rc == POLAR_OK; ++k) {
    polar_ctx* c = G->car[k];
    const HostCoeffs& K = c->hk;
    rc = dalloc(c, &G->vr[k], nf);
    if (rc == POLAR_OK) rc = dalloc(c, &G->vt[k], nt);
    if (rc == POLAR_OK && !K.dr.empty()) rc = dalloc(c, &G->dr[k], nf);
    if (rc == POLAR_OK && !K.dt.empty()) rc = dalloc(c, &G->dt[k], nt);
    if (rc == POLAR_OK && !K.b.empty()) rc = dalloc(c, &G->b[k], K.b.size());
    if (rc == POLAR_OK) {
      cudaError_t e = cudaStreamSynchronize(c->st);  // zeroed before the copies
      if (e == cudaSuccess && G->dr[k])
        e = cudaMemcpy(G->dr[k], K.dr.data(), nf * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && G->dt[k])
        e = cudaMemcpy(G->dt[k], K.dt.data(), nt * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && G->b[k])
        e = cudaMemcpy(G->b[k], K.b.data(), K.b.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) rc = fail(POLAR_ECUDA, cudaGetErrorString(e));
    }
  }
  if (rc == POLAR_OK) rc = polar_batch_create(G->car, 2, electrons->st, &G->pair);
  if (rc != POLAR_OK) {
    delete G;  // the buffers stay with the potential's context until it is destroyed
    return rc;
  }
  *out = G;
  return POLAR_OK;
}

int polar_gummel_destroy(polar_gummel* G) {
  if (!G) return POLAR_OK;
  polar_batch_destroy(G->pair);
  delete G;
  return POLAR_OK;
}

int polar_gummel_step(polar_gummel* G, const double* t, double theta, const double* const* w,
                      const double* w_phi, const polar_solver_opts* opts,
                      polar_gummel_stats* stats) {
  if (!G || !t) return fail(POLAR_EINVAL, "null argument");
  polar_ctx* phi = G->phi;
  polar_ctx* const* car = G->car;
  if (phi->nsrc > 0 && !w_phi) return fail(POLAR_EINVAL, "the potential's source weights are required");
  for (int k = 0; k < 2; ++k)
    if (car[k]->nsrc > 0 && (!w || !w[k])) return fail(POLAR_EINVAL, "carrier source weights required");
  if (!phi->have_state || !car[0]->have_state || !car[1]->have_state)
    return fail(POLAR_ESTATE, "set the states of all three contexts first");
  if (!(t[1] > t[0]) || !std::isfinite(t[1])) return fail(POLAR_EINVAL, "need t[1] > t[0]");
  CUDA_TRY(cudaSetDevice(phi->device));
  polar_ctx* c = phi;  // the context the launch checks report on
  const int m = phi->m, n = phi->n;
  const size_t nv = phi->nv(), nf = (size_t)(m + 1) * n, nt = (size_t)m * n;
  if (stats) *stats = polar_gummel_stats{};
  for (int k = 0; k < 2; ++k) {
    CUDA_TRY(cudaMemcpyAsync(G->save[k], car[k]->U, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                             car[k]->st));
    CUDA_TRY(cudaStreamSynchronize(car[k]->st));
  }
  // potential on r = 1: the weighted Dirichlet fields of the potential's context
  std::vector<double> g(n, 0.0);
  for (int q = 0; q < phi->nsrc; ++q)
    for (int j = 0; j < n; ++j) g[j] += w_phi[q] * phi->bnd_host[q][j];
  double* gdev = phi->mesh_dev + m + 2 + n;
  CUDA_TRY(cudaMemcpy(gdev, g.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  const int src_slot[2] = {G->d.src_electrons, G->d.src_holes};
  double change = 0.0;
  int it = 0;
  bool converged = false;
  int cols[kMaxAnderson];  // Anderson difference columns in use, oldest first
  int ncols = 0;
  bool have_last = false;
  for (it = 0; it < G->d.max_iter; ++it) {
    // the carrier densities as the potential's sources (split layout times volumes)
    for (int k = 0; k < 2; ++k) {
      LAUNCH(launch_unpack(car[k]->sh0(), car[k]->U, nullptr, phi->io, phi->st));
      LAUNCH(launch_pack(phi->sh0(), phi->io, phi->lv[0].vol, phi->vsrc[src_slot[k]], phi->st));
    }
    CUDA_TRY(cudaStreamSynchronize(phi->st));
    polar_step_stats ps{};
    TRY(polar_solve_steady(phi, w_phi, opts, &ps));
    if (stats) stats->phi = ps;
    if (it > 0) {
      LAUNCH(launch_max_change(nv, phi->U, G->phi_prev, G->change, phi->st));
      double h[2];
      CUDA_TRY(cudaMemcpyAsync(h, G->change, sizeof(h), cudaMemcpyDeviceToHost, phi->st));
      CUDA_TRY(cudaStreamSynchronize(phi->st));
      change = h[1] > 0 ? h[0] / h[1] : h[0];
      if (change <= G->d.tol) {
        converged = true;
        ++it;
        break;
      }
      if (G->d.depth > 0) TRY(anderson_update(G, cols, ncols, have_last));
    }
    CUDA_TRY(cudaMemcpyAsync(G->phi_prev, phi->U, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                             phi->st));
    // drift of each carrier from the potential (face kernel), the carriers' operators and
    // hierarchies re-assembled with it on the device
    LAUNCH(launch_unpack(phi->sh0(), phi->U, nullptr, phi->io, phi->st));
    for (int k = 0; k < 2; ++k)
      LAUNCH(launch_face_drift(m, n, phi->io, phi->mesh_dev, phi->mesh_dev + m + 2, gdev,
                               G->d.mobility[k], G->vr[k], G->vt[k], phi->st));
    CUDA_TRY(cudaStreamSynchronize(phi->st));
    for (int k = 0; k < 2; ++k) {
      const HostCoeffs& K = car[k]->hk;
      const AsmIn in{m, n, phi->mesh_dev, phi->mesh_dev + m + 2, G->dr[k], G->dt[k], K.d_const,
                     G->vr[k], G->vt[k], G->b[k], 0.0};
      TRY(reassemble_device(car[k], in, G->d.mobility[k] == 0.0));
      CUDA_TRY(cudaMemcpyAsync(car[k]->U, G->save[k], nv * sizeof(double), cudaMemcpyDeviceToDevice,
                               car[k]->st));
      CUDA_TRY(cudaStreamSynchronize(car[k]->st));
      car[k]->t = t[0];
    }
    // both carriers one theta-step from the start of the step, as one batch
    const double* ts[2] = {t, t};
    const double th[2] = {theta, theta};
    const double* ws[2] = {w ? w[0] : nullptr, w ? w[1] : nullptr};
    polar_step_stats cst[2] = {};
    TRY(polar_batch_advance(G->pair, 1, ts, th, ws, opts, cst));
    if (stats) {
      stats->carrier[0] = cst[0];
      stats->carrier[1] = cst[1];
    }
  }
  if (stats) {
    stats->iters = it;
    stats->change = change;
    stats->status = converged ? POLAR_OK : POLAR_ENOCONV;
  }
  if (!converged) return fail(POLAR_ENOCONV, "Gummel iteration did not reach tol");
  return POLAR_OK;
}

int polar_batch_create(polar_ctx* const* ctxs, int32_t count, void* stream, polar_batch** out) {
  if (!ctxs || !out || count <= 0) return fail(POLAR_EINVAL, "need count > 0 contexts");
  if (count > kMaxSlots) return fail(POLAR_EINVAL, "at most 1024 contexts in a batch");
  *out = nullptr;
  int dev = -1;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return fail(POLAR_EINVAL, "null context in the batch");
    if (dev >= 0 && ctxs[i]->device != dev) return fail(POLAR_EINVAL, "all contexts must share one device");
    dev = ctxs[i]->device;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return fail(POLAR_EINVAL, "a context appears twice in the batch");
  }
  polar_batch* b = new polar_batch();
  b->ctx.assign(ctxs, ctxs + count);
  b->st = static_cast<cudaStream_t>(stream);
  *out = b;
  return POLAR_OK;
}

int polar_batch_destroy(polar_batch* b) {
  if (!b) return POLAR_OK;
  if (!b->ctx.empty()) cudaSetDevice(b->ctx[0]->device);
  cudaStreamSynchronize(b->st);
  if (b->ex) cudaGraphExecDestroy(b->ex);
  if (b->g) cudaGraphDestroy(b->g);
  if (b->arena) {
    polar_ctx* c0 = b->ctx[0];
    if (c0->free_fn) c0->free_fn(b->arena, c0->st, c0->alloc_user);
    else cudaFree(b->arena);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return POLAR_OK;
}

int64_t polar_batch_kernel_launches(const polar_batch* b) { return b ? b->launches : 0; }

int polar_batch_advance(polar_batch* b, int32_t nsteps, const double* const* t, const double* theta,
                        const double* const* w, const polar_solver_opts* opts,
                        polar_step_stats* stats) {
  if (!b || !t || !theta) return fail(POLAR_EINVAL, "null argument");
  const int count = (int)b->ctx.size();
  const polar_solver_opts o = resolve_opts(opts);
  CUDA_TRY(cudaSetDevice(b->ctx[0]->device));
  for (int i = 0; i < count; ++i) {
    polar_ctx* c = b->ctx[i];
    TRY(check_schedule_args(c, nsteps, t[i], theta[i], w ? w[i] : nullptr));
    if (!c->use_graph) return fail(POLAR_ESTATE, "a context of the batch cannot run as a graph");
    TRY(choose_method(c, o));
  }
  if (nsteps == 0) return POLAR_OK;
  for (int i = 0; i < count; ++i) {
    polar_ctx* c = b->ctx[i];
    c->cs = c->st;
    if (c->autotune && !c->tuned && !c->direct_now)
      TRY(prepare_tuning(c, t[i], theta[i], w ? w[i] : nullptr, o));
    TRY(load_schedule(c, nsteps, t[i], theta[i], w ? w[i] : nullptr, o));
    CUDA_TRY(cudaStreamSynchronize(c->st));  // uploads land before the batch graph runs
  }
  bool stale = !b->ex || (int)b->gens.size() != count;
  for (int i = 0; !stale && i < count; ++i) stale = b->gens[i] != b->ctx[i]->generation;
  if (stale) TRY(build_batch_graph(b));
  // one graph launch advances every instance by one step: each kernel class runs once per
  // phase over all instances
  for (int k = 0; k < nsteps; ++k) CUDA_TRY(cudaGraphLaunch(b->ex, b->st));
  CUDA_TRY(cudaStreamSynchronize(b->st));
  int rc = POLAR_OK;
  for (int i = 0; i < count; ++i) {
    const int r = finish_schedule(b->ctx[i], nsteps, t[i], stats ? stats + (size_t)i * nsteps : nullptr,
                                  false);
    if (rc == POLAR_OK && r != POLAR_OK) rc = r;
  }
  // kernels launched: per step the fixed ones, then every loop runs as long as its slowest
  // instance
  for (int k = 0; k < nsteps; ++k)
    for (const polar_batch::Group& grp : b->groups) {
      int sweeps = 0, it32 = 0, it64 = 0;
      for (int i : grp.members) {
        const polar_ctx* c = b->ctx[i];
        const StepOut& r = c->out_host[k];
        if (r.status == POLAR_ESTATE) continue;
        sweeps = std::max(sweeps, r.sweeps - 1);
        const int i64 = c->precision == POLAR_MIXED ? r.iters64 : r.iters;
        it64 = std::max(it64, i64);
        it32 = std::max(it32, r.iters - i64);
      }
      b->launches += grp.fixed + (int64_t)sweeps * grp.sweep + (int64_t)it32 * grp.iter32 +
                     (int64_t)it64 * grp.iter64;
    }
  return rc;
}

int polar_apply_operator(polar_ctx* c, double alpha, double beta, const double* x, double* y,
                         int32_t memory) {
  if (!c || !x || !y) return fail(POLAR_EINVAL, "null argument");
  if (!c->have_coeffs) return fail(POLAR_ESTATE, "set_coeffs must come first");
  if (memory != POLAR_HOST && memory != POLAR_DEVICE) return fail(POLAR_EINVAL, "bad memory flag");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(POLAR_EINVAL, "non-finite alpha/beta");
  CUDA_TRY(cudaSetDevice(c->device));
  const size_t N = c->N();
  const cudaMemcpyKind in = memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind outk = memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // S = alpha V + beta V L on the FP64 fine level (diag from a refresh), y = S x / V
  c->cs = c->st;
  const double zero[4] = {0, 0, 0, 0};
  TRY(set_step_params(c, alpha, beta, zero, zero, resolve_opts(nullptr)));
  if (c->sp_host->do_refresh) {
    if (c->precision == POLAR_FP64) {
      TRY(launch_refresh_all<double>(c));
    } else {
      TRY(launch_refresh_all<float>(c));
    }
  }
  CUDA_TRY(cudaMemcpyAsync(c->io, x, N * sizeof(double), in, c->st));
  LAUNCH(launch_pack(c->sh0(), c->io, nullptr, c->r64, c->st));
  LAUNCH(launch_apply<double>(c->v64[0], c->par(), c->r64, c->e, c->st, c->red()));
  LAUNCH(launch_unpack(c->sh0(), c->e, c->lv[0].vol, c->io, c->st));
  CUDA_TRY(cudaMemcpyAsync(y, c->io, N * sizeof(double), outk, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

int64_t polar_kernel_launches(const polar_ctx* c) { return c ? c->launches : 0; }

int polar_is_separable(const polar_ctx* c) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  if (!c->have_coeffs) return fail(POLAR_ESTATE, "set_coeffs must come first");
  return c->separable ? 1 : 0;
}

int polar_timing_enable(polar_ctx* c, int32_t on) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  TRY(resolve_timers(c));
  c->kstats.clear();
  c->timing = on != 0;
  return POLAR_OK;
}

int polar_timing_flops(polar_ctx* c, int32_t index, double* flops) {
  if (!c || !flops) return fail(POLAR_EINVAL, "null argument");
  CUDA_TRY(cudaSetDevice(c->device));
  TRY(resolve_timers(c));
  if (index < 0 || index >= (int32_t)c->kstats.size()) return fail(POLAR_EINVAL, "no such kernel class");
  *flops = c->kstats[index].flops;
  return POLAR_OK;
}

int polar_timing_query(polar_ctx* c, int32_t index, char* name, size_t name_len,
                       int64_t* launches, double* total_ms, double* bytes) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  TRY(resolve_timers(c));
  if (index < 0 || index >= (int32_t)c->kstats.size()) return fail(POLAR_EINVAL, "no such kernel class");
  const KernelStat& k = c->kstats[index];
  if (name && name_len > 0) {
    std::strncpy(name, k.name.c_str(), name_len - 1);
    name[name_len - 1] = '\0';
  }
  if (launches) *launches = k.launches;
  if (total_ms) *total_ms = k.ms;
  if (bytes) *bytes = k.bytes;
  return POLAR_OK;
}

}  // extern "C"
