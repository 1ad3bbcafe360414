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
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polar.h"
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
  // per-step refresh, FP32 (mixed path)
  float *diag32, *fl32, *fui32, *fcu32, *fq32, *fring32, *fz32;
  // V-cycle right-hand side and solution (levels >= 1), in the inner precision
  void *b, *x;
};

struct PendingTimer {
  int kind;
  cudaEvent_t a, b;
  double bytes;
};
struct KernelStat {
  std::string name;
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

}  // namespace

struct polar_ctx {
  int m = 0, n = 0;
  int scheme = 0, precision = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<double> r, theta;
  std::vector<void*> allocs;
  std::vector<DevLevel> lv;
  std::vector<LevelView<double>> v64;
  std::vector<LevelView<float>> v32;
  int nsrc = 0;
  double* vsrc[4] = {nullptr, nullptr, nullptr, nullptr};
  double* bnd[4] = {nullptr, nullptr, nullptr, nullptr};
  bool have_coeffs = false, have_state = false;
  double t = 0.0;
  double* U = nullptr;
  double* X = nullptr;
  double* e = nullptr;
  double* r64 = nullptr;
  double* io = nullptr;  // interface-layout staging (N doubles)
  double* ws = nullptr;  // refresh workspace
  double* par = nullptr; // device [alpha, beta]
  double* par_host = nullptr;
  double cur_alpha = -1.0, cur_beta = -1.0;  // values the refresh was made for
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
  size_t N() const { return (size_t)m * n + 1; }
  const Shape& sh0() const { return lv[0].sh; }
  size_t nv() const { return lv[0].sh.nv; }
  int nlev() const { return (int)lv.size(); }
};

namespace {

template <typename T>
int dalloc(polar_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(POLAR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  e = cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(POLAR_ECUDA, cudaGetErrorString(e));
  *p = static_cast<T*>(q);
  return POLAR_OK;
}

int check_launch(polar_ctx* c, int n) {
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

int timed_end(polar_ctx* c, cudaEvent_t a, const char* name, double bytes) {
  if (!a) return POLAR_OK;
  cudaEvent_t b = take_event(c);
  CUDA_TRY(cudaEventRecord(b, c->st));
  c->pending.push_back(PendingTimer{kind_index(c, name), a, b, bytes});
  return POLAR_OK;
}

// LAUNCH with event timing under a kernel-class name and the launch's algorithmic bytes.
#define TLAUNCH(name, bytes, expr)                 \
  do {                                             \
    cudaEvent_t ev_;                               \
    TRY(timed_begin(c, &ev_));                     \
    LAUNCH(expr);                                  \
    TRY(timed_end(c, ev_, name, (double)(bytes))); \
  } while (0)

void release(polar_ctx* c) {
  for (const PendingTimer& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  c->pending.clear();
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  c->ev_free.clear();
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->ks_host) cudaFreeHost(c->ks_host);
  c->ks_host = nullptr;
  if (c->par_host) cudaFreeHost(c->par_host);
  c->par_host = nullptr;
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
    if (!mixed || l == 0) TRY(dalloc(c, &d.diag, nv));
    if (!mixed) {
      double** f64[] = {&d.fl, &d.fui, &d.fcu, &d.fq};
      for (double** p : f64) TRY(dalloc(c, p, nv));
      TRY(dalloc(c, &d.fring, nr));
      TRY(dalloc(c, &d.fz, (size_t)c->n));
      if (l > 0) {
        double *b = nullptr, *x = nullptr;
        TRY(dalloc(c, &b, nv));
        TRY(dalloc(c, &x, nv));
        d.b = b;
        d.x = x;
      }
    } else {
      float** s32[] = {&d.w32, &d.e32, &d.s32, &d.nn32, &d.ia32, &d.ib32};
      for (float** p : s32) TRY(dalloc(c, p, nv));
      TRY(dalloc(c, &d.o32, (size_t)c->n));
      float** f32[] = {&d.diag32, &d.fl32, &d.fui32, &d.fcu32, &d.fq32};
      for (float** p : f32) TRY(dalloc(c, p, nv));
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
    wsz += 3 * nv;
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

// Per-step refresh: the matrix S = alpha V + beta V L changes with dt and theta.
template <typename T>
int refresh(polar_ctx* c, double alpha, double beta) {
  if (alpha == c->cur_alpha && beta == c->cur_beta) return POLAR_OK;
  c->par_host[0] = alpha;
  c->par_host[1] = beta;
  CUDA_TRY(cudaMemcpyAsync(c->par, c->par_host, 2 * sizeof(double), cudaMemcpyHostToDevice, c->st));
  std::vector<LevelView<T>> vt = views<T>(c);
  double pts = 0.0;
  for (const DevLevel& d : c->lv) pts += (double)d.sh.m * d.sh.n;
  // reads 6 FP64 coefficient arrays, writes diag and 4 factor arrays
  TLAUNCH("refresh", pts * (6.0 * 8 + 5.0 * sizeof(T)),
          launch_refresh<T>(c->v64.data(), vt.data(), c->nlev(), c->par, c->ws, c->st));
  // the host copy of the parameters must not change before the copy above ran
  CUDA_TRY(cudaStreamSynchronize(c->st));
  c->cur_alpha = alpha;
  c->cur_beta = beta;
  return POLAR_OK;
}

// x = M^{-1} b: one V(1,1) cycle of the radial multigrid (polar_mg.cu).
template <typename T>
int vcycle(polar_ctx* c, const T* b, T* x) {
  const std::vector<LevelView<T>>& L = views<T>(c);
  const int nl = c->nlev();
  const int* done = &c->ks->done;
  const double B = sizeof(T);
  auto bof = [&](int l) { return l == 0 ? b : static_cast<const T*>(c->lv[l].b); };
  auto xof = [&](int l) { return l == 0 ? x : static_cast<T*>(c->lv[l].x); };
  for (int l = 0; l + 1 < nl; ++l) {
    const Shape& s = L[l].sh;
    const double po = (double)s.no * s.n, pe = (double)s.ne * s.n;
    // algorithmic words: odd line solve reads b and 4 factors, writes x (6 per point);
    // even: b, w, e, the odd neighbours, 4 factors, writes x (9); restriction reads
    // w, e, ia, ib of the odd rings and x of the even ones, writes the coarse rhs
    TLAUNCH("ring_pre_odd", 6 * B * po,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, c->par, 1, RING_PRE, done, c->st));
    TLAUNCH("ring_pre_even", 9 * B * pe,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, c->par, 0, RING_PRE, done, c->st));
    TLAUNCH("restrict", B * (4 * po + 2 * pe),
            launch_restrict<T>(L[l], L[l + 1], xof(l), static_cast<T*>(c->lv[l + 1].b), c->par, done,
                               c->st));
  }
  TLAUNCH("coarsest", 8 * B * L[nl - 1].sh.n,
          launch_coarsest<T>(L[nl - 1], bof(nl - 1), xof(nl - 1), c->par, done, c->st));
  for (int l = nl - 2; l >= 0; --l) {
    const Shape& s = L[l].sh;
    const double po = (double)s.no * s.n, pe = (double)s.ne * s.n;
    // even rings after the correction also read x, ia, ib of the odd rings and the
    // coarse solution (8 per even point + 3 per odd point + 1 per coarse point)
    TLAUNCH("ring_post_even", B * (8 * pe + 3 * po + pe),
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), static_cast<const T*>(c->lv[l + 1].x),
                           c->par, 0, RING_POST, done, c->st));
    TLAUNCH("ring_post_odd", 9 * B * po,
            launch_ring<T>(L[l], L[l + 1], bof(l), xof(l), nullptr, c->par, 1, RING_POST, done, c->st));
  }
  return POLAR_OK;
}

// Inner BiCGStab solve S d = r (r holds the scaled right-hand side), right-preconditioned
// by one V-cycle per application; all scalars stay on the device.
template <typename T>
int inner_solve(polar_ctx* c, KVecs<T>& k, double rel_tol, int max_iter, int* iters) {
  const LevelView<T>& L0 = views<T>(c)[0];
  const Reduce red = c->red();
  const size_t nv = c->nv();
  const double B = sizeof(T), pts = (double)c->m * c->n;
  TLAUNCH("bicg_init", 5 * B * nv,
          launch_bicg_init<T>(nv, k.r, k.rhat, k.p, k.v, k.d, true, rel_tol, max_iter, c->st, red));
  int batch = 2;
  for (;;) {
    for (int it = 0; it < batch; ++it) {
      TRY(vcycle<T>(c, k.p, k.phat));
      // stencil with dot: reads x, diag, 4 couplings, d1; writes y (8 words per point)
      TLAUNCH("stencil_dot", 8 * B * pts,
              launch_apply_dot<T>(L0, c->par, k.phat, k.v, k.rhat, 0, c->st, red));
      TLAUNCH("bicg_s", 3 * B * nv, launch_bicg_s<T>(nv, k.r, k.v, k.s, c->st, red));
      TRY(vcycle<T>(c, k.s, k.shat));
      TLAUNCH("stencil_dot", 8 * B * pts, launch_apply_dot<T>(L0, c->par, k.shat, k.t, k.s, 1, c->st, red));
      TLAUNCH("bicg_update", 8 * B * nv,
              launch_bicg_update<T>(nv, k.d, k.phat, k.shat, k.r, k.s, k.t, k.rhat, c->st, red));
      TLAUNCH("bicg_p", 4 * B * nv, launch_bicg_p<T>(nv, k.p, k.r, k.v, c->st, red));
    }
    TRY(read_scalars(c));
    if (c->ks_host->done != 0) break;
    batch = std::min(batch * 2, 8);
  }
  *iters = c->ks_host->iters;
  return POLAR_OK;
}

template <typename T>
int solve_step(polar_ctx* c, const polar_solver_opts& o, polar_step_stats& stats) {
  KVecs<T>* k;
  if constexpr (sizeof(T) == 8) {
    k = &c->kv64;
  } else {
    k = &c->kv32;
  }
  const size_t nv = c->nv();
  CUDA_TRY(cudaMemcpyAsync(c->X, c->U, nv * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  const Reduce red = c->red();
  const double inner_tol = (sizeof(T) == 8) ? std::min(o.inner_tol, 1e-12) : o.inner_tol;
  const double pts = (double)c->m * c->n;
  stats.iters = 0;
  stats.refinements = 0;
  for (int sweep = 0;; ++sweep) {
    TLAUNCH("resid64", 8.0 * 8 * pts, launch_resid64(c->v64[0], c->par, c->X, c->e, c->r64, c->st, red));
    TRY(read_scalars(c));
    stats.refinements += 1;
    const double xmax = std::max(c->ks_host->xmax, 1e-300);
    const double scaled = c->ks_host->smax / xmax;
    stats.scaled_resid = scaled;
    if (!std::isfinite(scaled) || !std::isfinite(c->ks_host->rmax))
      return fail(POLAR_ENONFINITE, "non-finite residual");
    if (scaled <= o.tol) break;
    if (sweep >= o.max_refine)
      return fail(POLAR_ENOCONV, "refinement did not reach the tolerance (scaled residual " +
                                     std::to_string(scaled) + ")");
    TLAUNCH("scale_cast", (8.0 + sizeof(T)) * nv, launch_scale_cast<T>(nv, c->r64, k->r, c->st, red));
    int it = 0;
    TRY(inner_solve<T>(c, *k, inner_tol, o.max_iter, &it));
    stats.iters += it;
    if (c->ks_host->done == 3) return fail(POLAR_ENONFINITE, "non-finite value in the Krylov solve");
    TLAUNCH("correct", (16.0 + sizeof(T)) * nv, launch_correct<T>(nv, c->X, k->d, c->st, red));
  }
  std::swap(c->U, c->X);
  return POLAR_OK;
}

polar_solver_opts resolve_opts(const polar_solver_opts* o) {
  polar_solver_opts r;
  r.tol = 1e-14;
  r.max_iter = 500;
  r.max_refine = 12;
  r.inner_tol = 1e-5;
  if (o) {
    if (o->tol > 0) r.tol = o->tol;
    if (o->max_iter > 0) r.max_iter = o->max_iter;
    if (o->max_refine > 0) r.max_refine = o->max_refine;
    if (o->inner_tol > 0) r.inner_tol = o->inner_tol;
  }
  return r;
}

int do_step(polar_ctx* c, double dt, double theta, const double* w_old, const double* w_new,
            const polar_solver_opts* opts, polar_step_stats* stats) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  if (!c->have_coeffs || !c->have_state) return fail(POLAR_ESTATE, "set_coeffs and set_state must come first");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(POLAR_EINVAL, "dt must be positive and finite");
  if (!(theta > 0.0 && theta <= 1.0)) return fail(POLAR_EINVAL, "theta must lie in (0, 1]");
  if (c->nsrc > 0 && (!w_old || !w_new)) return fail(POLAR_EINVAL, "source weights required");
  double cf[4] = {0, 0, 0, 0}, cg[4] = {0, 0, 0, 0};
  for (int q = 0; q < c->nsrc; ++q) {
    if (!std::isfinite(w_old[q]) || !std::isfinite(w_new[q]))
      return fail(POLAR_ENONFINITE, "non-finite source weight");
    cf[q] = (1.0 - theta) * w_old[q] + theta * w_new[q];
    cg[q] = -((1.0 - theta) * w_old[q] + theta * w_new[q]);
  }
  polar_solver_opts o = resolve_opts(opts);
  polar_step_stats st{};
  CUDA_TRY(cudaSetDevice(c->device));
  const double alpha = 1.0 / dt;
  // e = V U/dt - (1-theta) (V L U + e_m g_old) + (1-theta) V f_old + theta (V f_new - e_m g_new)
  const double* srcs[4] = {c->vsrc[0], c->vsrc[1], c->vsrc[2], c->vsrc[3]};
  const double* bnds[4] = {c->bnd[0], c->bnd[1], c->bnd[2], c->bnd[3]};
  TLAUNCH("rhs", (8.0 + c->nsrc) * 8 * c->m * c->n,
          launch_rhs(c->v64[0], alpha, 1.0 - theta, c->U, c->nsrc, srcs, bnds, cf, cg, c->e, c->st,
                     c->red()));
  int rc = (c->precision == POLAR_FP64) ? refresh<double>(c, alpha, theta)
                                        : refresh<float>(c, alpha, theta);
  if (rc == POLAR_OK)
    rc = (c->precision == POLAR_FP64) ? solve_step<double>(c, o, st) : solve_step<float>(c, o, st);
  st.status = rc;
  if (stats) *stats = st;
  if (rc != POLAR_OK) return rc;
  c->t += dt;
  return POLAR_OK;
}

}  // namespace

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
    chk(dalloc(c, &c->par, 2));
    if (c->precision == POLAR_FP64) {
      chk(alloc_kvecs(c, c->kv64));
    } else {
      chk(alloc_kvecs(c, c->kv32));
    }
    chk(dalloc(c, &c->part, (size_t)kMaxBlocks * 4));
    chk(dalloc(c, &c->ks, 1));
  }
  if (rc == POLAR_OK && cudaMallocHost((void**)&c->ks_host, sizeof(KrylovScalars)) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = fail(POLAR_ENOMEM, "cudaMallocHost failed");
  }
  if (rc == POLAR_OK && cudaMallocHost((void**)&c->par_host, 2 * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    rc = fail(POLAR_ENOMEM, "cudaMallocHost failed");
  }
  if (rc != POLAR_OK) {
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
  // fine level and its radial hierarchy
  std::vector<HLevel> H(c->nlev());
  if (c->scheme == POLAR_SCHEME_CONSERVATIVE) {
    assemble_conservative(c->r, c->theta, K, H[0]);
  } else {
    assemble_paper(c->r, c->theta, K, H[0]);
  }
  for (int l = 0; l + 1 < c->nlev(); ++l) coarsen(H[l], H[l + 1]);
  for (int l = 0; l < c->nlev(); ++l) TRY(upload_level(c, l, H[l]));
  // sources in the split layout, scaled by the control volumes
  for (int q = 0; q < k->nsrc; ++q) {
    if (!c->vsrc[q]) {  // allocated on first use, reused by later set_coeffs calls
      TRY(dalloc(c, &c->vsrc[q], c->nv()));
      TRY(dalloc(c, &c->bnd[q], (size_t)n));
    }
    CUDA_TRY(cudaMemcpy(c->io, srcs[q].data(), N * sizeof(double), cudaMemcpyHostToDevice));
    LAUNCH(launch_pack(c->sh0(), c->io, c->lv[0].vol, c->vsrc[q], c->st));
    CUDA_TRY(cudaMemcpy(c->bnd[q], bnds[q].data(), n * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->nsrc = k->nsrc;
  c->cur_alpha = c->cur_beta = -1.0;  // the per-step parts must be refreshed
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
  return do_step(c, dt, theta, w_old, w_new, opts, stats);
}

int polar_advance(polar_ctx* c, int32_t nsteps, const double* t, double theta, const double* w,
                  const polar_solver_opts* opts, polar_step_stats* stats) {
  if (!c || !t) return fail(POLAR_EINVAL, "null argument");
  if (nsteps < 0) return fail(POLAR_EINVAL, "nsteps must be >= 0");
  if (c->nsrc > 0 && !w) return fail(POLAR_EINVAL, "weights required");
  if (!c->have_coeffs || !c->have_state) return fail(POLAR_ESTATE, "set_coeffs and set_state must come first");
  if (std::fabs(t[0] - c->t) > 1e-12 * std::max(1.0, std::fabs(c->t)))
    return fail(POLAR_EINVAL, "t[0] must equal the current time");
  for (int k = 0; k < nsteps; ++k)
    if (!(t[k + 1] > t[k])) return fail(POLAR_EINVAL, "time levels must increase");
  const int Q = c->nsrc;
  for (int k = 0; k < nsteps; ++k) {
    polar_step_stats s{};
    const double tk = c->t;
    int rc = do_step(c, t[k + 1] - t[k], theta, Q ? w + (size_t)k * Q : nullptr,
                     Q ? w + (size_t)(k + 1) * Q : nullptr, opts, &s);
    if (rc == POLAR_OK) c->t = t[k + 1];  // the exact level, not an accumulated sum
    else c->t = tk;
    if (stats) stats[k] = s;
    if (rc != POLAR_OK) {
      if (stats)
        for (int q = k + 1; q < nsteps; ++q) {
          stats[q] = polar_step_stats{};
          stats[q].status = POLAR_ESTATE;
        }
      return rc;
    }
  }
  return POLAR_OK;
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
  if (c->precision == POLAR_FP64) {
    TRY(refresh<double>(c, alpha, beta));
  } else {
    TRY(refresh<float>(c, alpha, beta));
  }
  CUDA_TRY(cudaMemcpyAsync(c->io, x, N * sizeof(double), in, c->st));
  LAUNCH(launch_pack(c->sh0(), c->io, nullptr, c->r64, c->st));
  LAUNCH(launch_apply<double>(c->v64[0], c->par, c->r64, c->e, c->st, c->red()));
  LAUNCH(launch_unpack(c->sh0(), c->e, c->lv[0].vol, c->io, c->st));
  CUDA_TRY(cudaMemcpyAsync(y, c->io, N * sizeof(double), outk, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

int64_t polar_kernel_launches(const polar_ctx* c) { return c ? c->launches : 0; }

int polar_timing_enable(polar_ctx* c, int32_t on) {
  if (!c) return fail(POLAR_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  TRY(resolve_timers(c));
  c->kstats.clear();
  c->timing = on != 0;
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
