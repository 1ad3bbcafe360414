// C ABI of the polar theta-step library: argument checking, device buffers, the
// assembly of the 5-point operator from the caller's coefficients (Sections 3.2.1,
// 3.2.2), and the host orchestration of one implicit step (Eq. 2.5):
//   right-hand side (FP64) -> line factors -> refinement loop
//   { FP64 residual -> scaled cast -> BiCGStab with the alternating line
//     preconditioner in the inner precision -> FP64 correction }.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polar.h"
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

template <typename T>
struct KVecs {
  T *r, *rhat, *p, *v, *s, *t, *phat, *shat, *d, *w, *tmp;
};

template <typename T>
struct OpBuf {
  T *R, *W, *E, *S, *N, *o;
  OpView<T> view(int m, int n, int ld) const { return OpView<T>{m, n, ld, R, W, E, S, N, o}; }
};

}  // namespace

struct polar_ctx {
  int m = 0, n = 0, ld = 0;
  size_t nv = 0;
  int scheme = 0, precision = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<double> r, theta;
  std::vector<void*> allocs;
  OpBuf<double> op64{};
  OpBuf<float> op32{};
  double C0 = 0.0;  // diagonal of the origin row of L (host copy)
  int nsrc = 0;
  double* src[4] = {nullptr, nullptr, nullptr, nullptr};
  double* bnd[4] = {nullptr, nullptr, nullptr, nullptr};
  bool have_coeffs = false, have_state = false;
  double t = 0.0;
  double* U = nullptr;
  double* X = nullptr;
  double* e = nullptr;
  double* r64 = nullptr;
  double* io = nullptr;  // interface-layout staging (N doubles)
  KVecs<double> kv64{};
  KVecs<float> kv32{};
  LineFactors<double> f64{};
  LineFactors<float> f32{};
  double* part = nullptr;
  KrylovScalars* ks = nullptr;
  KrylovScalars* ks_host = nullptr;
  int64_t launches = 0;

  Reduce red() const { return Reduce{part, ks}; }
  size_t N() const { return (size_t)m * n + 1; }
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

#define TRY(expr)               \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != POLAR_OK) return rc_; \
  } while (0)

template <typename T>
int alloc_kvecs(polar_ctx* c, KVecs<T>& k) {
  T** all[] = {&k.r, &k.rhat, &k.p, &k.v, &k.s, &k.t, &k.phat, &k.shat, &k.d, &k.w, &k.tmp};
  for (T** p : all) TRY(dalloc(c, p, c->nv));
  return POLAR_OK;
}

template <typename T>
int alloc_factors(polar_ctx* c, LineFactors<T>& f) {
  T** all[] = {&f.rl, &f.rui, &f.rcu, &f.al, &f.aui, &f.acu, &f.aq};
  for (T** p : all) TRY(dalloc(c, p, c->nv));
  TRY(dalloc(c, &f.avf, (size_t)c->m));
  TRY(dalloc(c, &f.ainv, (size_t)c->m));
  TRY(dalloc(c, &f.ws, 2 * c->nv));
  return POLAR_OK;
}

template <typename T>
int alloc_op(polar_ctx* c, OpBuf<T>& o) {
  T** all[] = {&o.R, &o.W, &o.E, &o.S, &o.N};
  for (T** p : all) TRY(dalloc(c, p, c->nv));
  TRY(dalloc(c, &o.o, (size_t)c->n));
  return POLAR_OK;
}

int check_launch(polar_ctx* c, int n) {
  c->launches += n;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(POLAR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return POLAR_OK;
}

#define LAUNCH(expr) TRY(check_launch(c, (expr)))

void release(polar_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->ks_host) cudaFreeHost(c->ks_host);
  c->ks_host = nullptr;
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

// ---------------------------------------------------------------------------------------
// Mesh metrics (Sections 2.1 and 3.1): h_i = r_i - r_{i-1}; r_{i+1/2} midpoints;
// mu_j = theta_j - theta_{j-1} with mu_0 = mu_n the wrap-around step; cell widths
// k_i = (h_i + h_{i+1})/2 and w_j = (mu_j + mu_{j+1})/2; control volumes
// V_ij = r_i k_i w_j and V_0 = pi h_1^2 / 4 (the disk of radius h_1/2, Section 3.2.2).
struct Metrics {
  int m, n;
  std::vector<double> h, rh, mu, w, k;
  Metrics(const std::vector<double>& r, const std::vector<double>& th) {
    m = (int)r.size() - 2;
    n = (int)th.size();
    h.assign(m + 2, 0.0);
    for (int i = 1; i <= m + 1; ++i) h[i] = r[i] - r[i - 1];
    rh.assign(m + 1, 0.0);
    for (int i = 0; i <= m; ++i) rh[i] = 0.5 * (r[i] + r[i + 1]);
    mu.assign(n + 1, 0.0);
    for (int j = 1; j < n; ++j) mu[j] = th[j] - th[j - 1];
    mu[n] = 2.0 * M_PI + th[0] - th[n - 1];
    mu[0] = mu[n];
    w.assign(n, 0.0);
    for (int j = 0; j < n; ++j) w[j] = 0.5 * (mu[j] + mu[j + 1]);
    k.assign(m + 1, 0.0);
    for (int i = 1; i <= m; ++i) k[i] = 0.5 * (h[i] + h[i + 1]);
  }
};

// Rows of L in difference form (see polar_internal.h): R = row sum, W/E/S/N the
// off-diagonal couplings, o the origin row's couplings to ring 1, C0 its diagonal.
struct HostOp {
  std::vector<double> R, W, E, S, N, o;
  double C0 = 0.0;
};

// CONSERVATIVE operator: for every face, outward flux = length * ((D/spacing + v+) U_in
// - (D/spacing + v-) U_out); the row of a cell is the sum of its outward fluxes divided
// by its control volume, plus b U.  Radial face (i+1/2, j): length w_j r_{i+1/2},
// spacing h_{i+1}.  Angular face (i, j+1/2): length k_i, spacing r_i mu_{j+1}.
void build_conservative(const polar_ctx* c, const Metrics& g, const std::vector<double>& dr,
                        const std::vector<double>& dt, const std::vector<double>& vr,
                        const std::vector<double>& vt, const std::vector<double>& b, double d_const,
                        HostOp& L) {
  const int m = c->m, n = c->n, ld = c->ld;
  const std::vector<double>& r = c->r;
  auto at = [&](int i, int j) { return (size_t)kOfs + (size_t)j * ld + (i - 1); };
  auto V = [&](int i, int j) { return r[i] * g.k[i] * g.w[j]; };
  const double V0 = M_PI * g.h[1] * g.h[1] / 4.0;
  // A face contributes cin/V (diagonal) and -cout/V (coupling) to the row of its inner
  // cell, so (cin - cout)/V = len v/V to that row sum; likewise -len v/V to the outer one.
  double C0 = 0.0, R0 = 0.0;
  for (int j = 0; j < n; ++j) {
    // radial faces i = 0..m
    for (int i = 0; i <= m; ++i) {
      const double D = dr.empty() ? d_const : dr[(size_t)j * (m + 1) + i];
      const double v = vr.empty() ? 0.0 : vr[(size_t)j * (m + 1) + i];
      const double len = g.w[j] * g.rh[i];
      const double cond = D / g.h[i + 1];
      const double cin = len * (cond + std::max(v, 0.0));
      const double cout = len * (cond + std::max(-v, 0.0));
      if (i == 0) {
        C0 += cin / V0;
        R0 += len * v / V0;
        L.o[j] = -cout / V0;
      } else {
        const double Vi = V(i, j);
        L.R[at(i, j)] += len * v / Vi;
        L.E[at(i, j)] = -cout / Vi;  // i = m: coupling to the Dirichlet value
      }
      if (i < m) {
        const double Vo = V(i + 1, j);
        L.R[at(i + 1, j)] -= len * v / Vo;
        L.W[at(i + 1, j)] = -cin / Vo;  // i = 0: ring 1's coupling to the origin
      }
    }
    // angular faces (i, j+1/2), i = 1..m
    const int jp = (j + 1) % n;
    for (int i = 1; i <= m; ++i) {
      const double D = dt.empty() ? d_const : dt[(size_t)j * m + (i - 1)];
      const double v = vt.empty() ? 0.0 : vt[(size_t)j * m + (i - 1)];
      const double len = g.k[i];
      const double cond = D / (r[i] * g.mu[j + 1]);
      const double cin = len * (cond + std::max(v, 0.0));
      const double cout = len * (cond + std::max(-v, 0.0));
      const double Vl = V(i, j), Vr = V(i, jp);
      L.R[at(i, j)] += len * v / Vl;
      L.N[at(i, j)] = -cout / Vl;
      L.R[at(i, jp)] -= len * v / Vr;
      L.S[at(i, jp)] = -cin / Vr;
    }
  }
  // reaction
  for (int j = 0; j < n; ++j)
    for (int i = 1; i <= m; ++i) L.R[at(i, j)] += b[1 + (size_t)j * m + (i - 1)];
  L.R[0] = R0 + b[0];
  L.C0 = C0 + b[0];
}

// PAPER operator: the printed ring rows of Section 3.2.1 (scalar E at nodes, forward
// differences) and the printed origin row of Section 3.2.2, plus b U.
void build_paper(const polar_ctx* c, const Metrics& g, const std::vector<double>& dr,
                 const std::vector<double>& dt, const std::vector<double>& en,
                 const std::vector<double>& b, double d_const, double d0, HostOp& L) {
  const int m = c->m, n = c->n, ld = c->ld;
  const std::vector<double>& r = c->r;
  auto at = [&](int i, int j) { return (size_t)kOfs + (size_t)j * ld + (i - 1); };
  for (int j = 0; j < n; ++j) {
    const int jm = (j + n - 1) % n;
    const double muj = g.mu[j], muj1 = g.mu[j + 1];
    for (int i = 1; i <= m; ++i) {
      const size_t q = 1 + (size_t)j * m + (i - 1);
      const double Dm = dr.empty() ? d_const : dr[(size_t)j * (m + 1) + i - 1];
      const double Dp = dr.empty() ? d_const : dr[(size_t)j * (m + 1) + i];
      const double Dn = dt.empty() ? d_const : dt[(size_t)j * m + i - 1];
      const double Ds = dt.empty() ? d_const : dt[(size_t)jm * m + i - 1];
      const double E = en.empty() ? 0.0 : en[q];
      const double hi = g.h[i], hi1 = g.h[i + 1], ri = r[i];
      const double rm = g.rh[i - 1], rp = g.rh[i];
      const double west = -2.0 * rm * Dm / (ri * hi * (hi + hi1));
      const double east = -(2.0 * rp * Dp / (ri * hi1 * (hi + hi1)) + E / hi1);
      const double south = -2.0 * Ds / (ri * ri * muj * (muj + muj1));
      const double north = -(2.0 * Dn / (ri * ri * muj1 * (muj + muj1)) + E / (ri * muj1));
      // The printed diagonal is the sum of the diffusion and drift coefficients above
      // plus b, so the row sum of the printed row is b exactly.
      L.R[at(i, j)] = b[q];
      L.W[at(i, j)] = west;
      L.E[at(i, j)] = east;
      L.S[at(i, j)] = south;
      L.N[at(i, j)] = north;
    }
  }
  const double h1 = g.h[1];
  const double E0 = en.empty() ? 0.0 : en[0];
  L.C0 = 4.0 * d0 / (h1 * h1) + E0 / h1 + b[0];
  for (int j = 0; j < n; ++j) L.o[j] = -(4.0 * d0 / (n * h1 * h1) - E0 / (n * h1));
  L.R[0] = b[0] + 2.0 * E0 / h1;  // C0 + sum_j o_j
}

template <typename T>
int precond(polar_ctx* c, const OpView<T>& op, const LineFactors<T>& f, KVecs<T>& k, T alpha,
            T beta, const T* y, T* z) {
  const int* done = &c->ks->done;
  LAUNCH(launch_radial_solve<T>(op, f, y, z, c->st, done));
  LAUNCH(launch_resid<T>(op, alpha, beta, z, y, k.w, c->st, c->red()));
  LAUNCH(launch_angular_solve<T>(op, f, k.w, z, z, k.tmp, c->st, done));
  return POLAR_OK;
}

int read_scalars(polar_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->ks_host, c->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

// Inner BiCGStab solve A d = r (r already holds the scaled right-hand side).
template <typename T>
int inner_solve(polar_ctx* c, const OpView<T>& op, const LineFactors<T>& f, KVecs<T>& k,
                double alpha, double beta, double rel_tol, int max_iter, int* iters) {
  const T a = (T)alpha, b = (T)beta;
  const Reduce red = c->red();
  LAUNCH(launch_bicg_init<T>(c->nv, k.r, k.rhat, k.p, k.v, k.d, true, rel_tol, max_iter, c->st, red));
  int batch = 2;
  for (;;) {
    for (int it = 0; it < batch; ++it) {
      TRY(precond<T>(c, op, f, k, a, b, k.p, k.phat));
      LAUNCH(launch_apply_dot<T>(op, a, b, k.phat, k.v, k.rhat, 0, c->st, red));
      LAUNCH(launch_bicg_s<T>(c->nv, k.r, k.v, k.s, c->st, red));
      TRY(precond<T>(c, op, f, k, a, b, k.s, k.shat));
      LAUNCH(launch_apply_dot<T>(op, a, b, k.shat, k.t, k.s, 1, c->st, red));
      LAUNCH(launch_bicg_update<T>(c->nv, k.d, k.phat, k.shat, k.r, k.s, k.t, k.rhat, c->st, red));
      LAUNCH(launch_bicg_p<T>(c->nv, k.p, k.r, k.v, c->st, red));
    }
    TRY(read_scalars(c));
    if (c->ks_host->done != 0) break;
    batch = std::min(batch * 2, 16);
  }
  *iters = c->ks_host->iters;
  return POLAR_OK;
}

template <typename T>
int solve_step(polar_ctx* c, double dt, double theta, const polar_solver_opts& o,
               polar_step_stats& stats) {
  const double alpha = 1.0 / dt, beta = theta;
  const OpView<double> op64 = c->op64.view(c->m, c->n, c->ld);
  OpView<T> opT;
  LineFactors<T>* f;
  KVecs<T>* k;
  if constexpr (sizeof(T) == 8) {
    opT = op64;
    f = &c->f64;
    k = &c->kv64;
  } else {
    opT = c->op32.view(c->m, c->n, c->ld);
    f = &c->f32;
    k = &c->kv32;
  }
  LAUNCH(launch_factor<T>(op64, alpha, beta, *f, c->st));
  f->diag0 = (T)(alpha + beta * c->C0);
  CUDA_TRY(cudaMemcpyAsync(c->X, c->U, c->nv * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  const Reduce red = c->red();
  const double inner_tol = (sizeof(T) == 8) ? std::min(o.inner_tol, 1e-12) : o.inner_tol;
  stats.iters = 0;
  stats.refinements = 0;
  for (int sweep = 0;; ++sweep) {
    LAUNCH(launch_resid64(op64, alpha, beta, c->X, c->e, c->r64, c->C0, c->st, red));
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
    LAUNCH(launch_scale_cast<T>(c->nv, c->r64, k->r, c->st, red));
    int it = 0;
    TRY(inner_solve<T>(c, opT, *f, *k, alpha, beta, inner_tol, o.max_iter, &it));
    stats.iters += it;
    if (c->ks_host->done == 3) return fail(POLAR_ENONFINITE, "non-finite value in the Krylov solve");
    LAUNCH(launch_correct<T>(c->nv, c->X, k->d, c->st, red));
  }
  std::swap(c->U, c->X);
  return POLAR_OK;
}

polar_solver_opts resolve_opts(const polar_solver_opts* o) {
  polar_solver_opts r;
  r.tol = 1e-14;
  r.max_iter = 4000;
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
  // e = U/dt - (1-theta) (L U + E_m g_old) + (1-theta) f_old + theta (f_new - E_m g_new)
  const OpView<double> op64 = c->op64.view(c->m, c->n, c->ld);
  const double* srcs[4] = {c->src[0], c->src[1], c->src[2], c->src[3]};
  const double* bnds[4] = {c->bnd[0], c->bnd[1], c->bnd[2], c->bnd[3]};
  LAUNCH(launch_rhs(op64, 1.0 / dt, -(1.0 - theta), c->U, c->nsrc, srcs, bnds, cf, cg, c->e, c->st,
                    c->red()));
  int rc = (c->precision == POLAR_FP64) ? solve_step<double>(c, dt, theta, o, st)
                                        : solve_step<float>(c, dt, theta, o, st);
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
  c->ld = (m + 3) & ~3;
  c->nv = (size_t)kOfs + (size_t)n * c->ld;
  c->scheme = d->scheme;
  c->precision = d->precision;
  c->st = static_cast<cudaStream_t>(d->stream);
  cudaGetDevice(&c->device);
  c->r.assign(d->r, d->r + m + 2);
  c->theta.assign(d->theta, d->theta + n);
  int rc = POLAR_OK;
  auto chk = [&](int v) {
    if (rc == POLAR_OK) rc = v;
  };
  chk(alloc_op(c, c->op64));
  if (c->precision == POLAR_MIXED) chk(alloc_op(c, c->op32));
  chk(dalloc(c, &c->U, c->nv));
  chk(dalloc(c, &c->X, c->nv));
  chk(dalloc(c, &c->e, c->nv));
  chk(dalloc(c, &c->r64, c->nv));
  chk(dalloc(c, &c->io, c->N()));
  if (c->precision == POLAR_FP64) {
    chk(alloc_kvecs(c, c->kv64));
    chk(alloc_factors(c, c->f64));
  } else {
    chk(alloc_kvecs(c, c->kv32));
    chk(alloc_factors(c, c->f32));
  }
  chk(dalloc(c, &c->part, (size_t)kMaxBlocks * 4));
  chk(dalloc(c, &c->ks, 1));
  if (rc == POLAR_OK && cudaMallocHost((void**)&c->ks_host, sizeof(KrylovScalars)) != cudaSuccess) {
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
  std::vector<double> dr, dt, vr, vt, en, b;
  if (k->d_rface) TRY(fetch(k->d_rface, nf, k->memory, dr));
  if (k->d_tface) TRY(fetch(k->d_tface, nt, k->memory, dt));
  if (k->v_rface) TRY(fetch(k->v_rface, nf, k->memory, vr));
  if (k->v_tface) TRY(fetch(k->v_tface, nt, k->memory, vt));
  if (k->e_node) TRY(fetch(k->e_node, N, k->memory, en));
  if (k->b) {
    TRY(fetch(k->b, N, k->memory, b));
  } else {
    b.assign(N, k->b_const);
  }
  std::vector<std::vector<double>> srcs(k->nsrc), bnds(k->nsrc);
  for (int q = 0; q < k->nsrc; ++q) {
    TRY(fetch(k->src[q], N, k->memory, srcs[q]));
    TRY(fetch(k->bnd[q], (size_t)n, k->memory, bnds[q]));
  }
  Metrics g(c->r, c->theta);
  HostOp L;
  L.R.assign(c->nv, 0.0);
  L.W.assign(c->nv, 0.0);
  L.E.assign(c->nv, 0.0);
  L.S.assign(c->nv, 0.0);
  L.N.assign(c->nv, 0.0);
  L.o.assign(n, 0.0);
  if (c->scheme == POLAR_SCHEME_CONSERVATIVE) {
    build_conservative(c, g, dr, dt, vr, vt, b, k->d_const, L);
  } else {
    build_paper(c, g, dr, dt, en, b, k->d_const, k->d0, L);
  }
  c->C0 = L.C0;
  const size_t bytes = c->nv * sizeof(double);
  CUDA_TRY(cudaMemcpy(c->op64.R, L.R.data(), bytes, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->op64.W, L.W.data(), bytes, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->op64.E, L.E.data(), bytes, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->op64.S, L.S.data(), bytes, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->op64.N, L.N.data(), bytes, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->op64.o, L.o.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  if (c->precision == POLAR_MIXED) {
    const double* s64[] = {c->op64.R, c->op64.W, c->op64.E, c->op64.S, c->op64.N};
    float* s32[] = {c->op32.R, c->op32.W, c->op32.E, c->op32.S, c->op32.N};
    for (int a = 0; a < 5; ++a) LAUNCH(launch_to_float(c->nv, s64[a], s32[a], c->st));
    LAUNCH(launch_to_float((size_t)n, c->op64.o, c->op32.o, c->st));
  }
  // sources in the padded layout
  for (int q = 0; q < k->nsrc; ++q) {
    if (!c->src[q]) {  // allocated on first use, reused by later set_coeffs calls
      TRY(dalloc(c, &c->src[q], c->nv));
      TRY(dalloc(c, &c->bnd[q], (size_t)n));
    }
    CUDA_TRY(cudaMemcpy(c->io, srcs[q].data(), N * sizeof(double), cudaMemcpyHostToDevice));
    LAUNCH(launch_pack(m, n, c->ld, c->io, c->src[q], c->st));
    CUDA_TRY(cudaMemcpy(c->bnd[q], bnds[q].data(), n * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->nsrc = k->nsrc;
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
  LAUNCH(launch_pack(c->m, c->n, c->ld, c->io, c->U, c->st));
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
    LAUNCH(launch_unpack(c->m, c->n, c->ld, c->U, c->io, c->st));
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
  CUDA_TRY(cudaSetDevice(c->device));
  const size_t N = c->N();
  const cudaMemcpyKind in = memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind outk = memory == POLAR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(c->io, x, N * sizeof(double), in, c->st));
  LAUNCH(launch_pack(c->m, c->n, c->ld, c->io, c->r64, c->st));
  LAUNCH(launch_apply<double>(c->op64.view(c->m, c->n, c->ld), alpha, beta, c->r64, c->e, c->st,
                              c->red()));
  LAUNCH(launch_unpack(c->m, c->n, c->ld, c->e, c->io, c->st));
  CUDA_TRY(cudaMemcpyAsync(y, c->io, N * sizeof(double), outk, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return POLAR_OK;
}

int64_t polar_kernel_launches(const polar_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
