// CUDA kernels of the implicit theta-step on the polar mesh (sm_103a): the 5-point
// operator with its origin row, the right-hand side, the BiCGStab vector updates and
// the mixed-precision helpers.  The multigrid preconditioner is in polar_mg.cu.
//
// Every kernel here streams its vectors once (HBM-bound; on GB300 the FP64 ones are
// close to the FP64 issue limit as well): nothing is a dense contraction, so no
// tensor-core path exists.  Reductions are deterministic: every block reduces its
// elements in a fixed order, writes one partial per block, and the last block to
// arrive (atomic counter + fences) sums the partials in block order and finishes the
// scalar recurrences of the Krylov solver on the device.
#include "polar_internal.h"

#include <algorithm>
#include <cmath>

namespace polar {

#define FULLMASK 0xffffffffu

int grid_for(size_t work, int threads) {
  size_t b = (work + (size_t)threads - 1) / (size_t)threads;
  if (b > (size_t)kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

// ------------------------------------------------------------------ reductions
// Slots [0, kmax) are sums, slots [kmax, K) are maxima of non-negative values.
template <int K, int KMAX>
__device__ __forceinline__ void warp_reduce(double (&v)[K]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double o = __shfl_down_sync(FULLMASK, v[k], off);
      v[k] = (k < KMAX) ? v[k] + o : fmax(v[k], o);
    }
  }
}

// Block-wide reduction; the result is valid in thread 0.  Fixed order: deterministic.
template <int K, int KMAX>
__device__ void block_reduce(double (&v)[K]) {
  __shared__ double sh[K][32];
  const int nt = blockDim.x * blockDim.y;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
  warp_reduce<K, KMAX>(v);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (lane < nw) ? sh[k][lane] : ((k < KMAX) ? 0.0 : 0.0);
    warp_reduce<K, KMAX>(v);
  }
  __syncthreads();
}

// Publishes this block's partials (thread 0 holds them) and reports whether this
// block is the last one of the grid to arrive.
template <int K>
__device__ bool publish_and_arrive(const double (&v)[K], double* part, unsigned int* counter,
                                   int bid, int nb) {
  __shared__ unsigned int s_last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[k * kMaxBlocks + bid] = v[k];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned int)nb - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Called by every thread of the last block: totals in block order (result in thread 0).
template <int K, int KMAX>
__device__ void grid_totals(const double* part, double (&tot)[K], int nb) {
  const int nt = blockDim.x * blockDim.y;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = 0.0;
  for (int b = tid; b < nb; b += nt) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double p = __ldcg(part + k * kMaxBlocks + b);
      tot[k] = (k < KMAX) ? tot[k] + p : fmax(tot[k], p);
    }
  }
  block_reduce<K, KMAX>(tot);
}

__device__ __forceinline__ double absfin(double v) { return isfinite(v) ? fabs(v) : INFINITY; }

// |v| as the bit pattern of a non-negative double, NaN mapped to +inf.  Non-negative
// doubles order like their bit patterns, so running maxima are integer maxima: no FP64
// instruction per point (GB300's FP64 pipe is the scarce unit of the FP64 kernels).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  const unsigned long long u =
      static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
  return u > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : u;
}
__device__ __forceinline__ double bits_to_double(unsigned long long u) {
  return __longlong_as_double(static_cast<long long>(u));
}

// Calls f(i, j, idx, west, east, south, north) for every point of this thread; west and
// east are indices of the radial neighbours (west = 0 is the origin for ring 1, east =
// SIZE_MAX marks the Dirichlet ring), south/north the periodic angular neighbours.
template <typename F>
__device__ __forceinline__ void for_points(const Shape& sh, const Tiling& t, int vb, int vg, F f) {
  const int n = sh.n, m = sh.m;
  for (int tile = vb; tile < t.ntiles; tile += vg) {
    const int tj = tile % t.tj;
    const int tk = tile / t.tj;
    const bool odd = tk < t.tko;
    const int k = (odd ? tk : tk - t.tko) * t.TK + threadIdx.x;
    const int j = tj * t.TJ + threadIdx.y;
    if (j >= n || k >= (odd ? sh.no : sh.ne)) continue;
    const int i = odd ? 2 * k + 1 : 2 * k + 2;
    size_t idx, west, east, south, north;
    const int jm = (j == 0) ? n - 1 : j - 1, jp = (j == n - 1) ? 0 : j + 1;
    if (odd) {
      idx = sh.odd0 + (size_t)j * sh.ldo + k;
      south = sh.odd0 + (size_t)jm * sh.ldo + k;
      north = sh.odd0 + (size_t)jp * sh.ldo + k;
      west = (k == 0) ? 0 : sh.even0 + (size_t)j * sh.lde + (k - 1);
      east = (i < m) ? sh.even0 + (size_t)j * sh.lde + k : (size_t)-1;
    } else {
      idx = sh.even0 + (size_t)j * sh.lde + k;
      south = sh.even0 + (size_t)jm * sh.lde + k;
      north = sh.even0 + (size_t)jp * sh.lde + k;
      west = sh.odd0 + (size_t)j * sh.ldo + k;
      east = (i < m) ? sh.odd0 + (size_t)j * sh.ldo + (k + 1) : (size_t)-1;
    }
    f(i, j, idx, west, east, south, north);
  }
}

// ------------------------------------------------------------------ stencil
template <int MODE>
struct Slots {
  static constexpr int K = (MODE == M_RESID64) ? 4 : (MODE == M_DOTV) ? 2 : (MODE == M_DOTT) ? 3 : 1;
  static constexpr int KMAX = (MODE == M_RESID64) ? 1 : K;
};

// y = S x in the direct form diag x + beta (w xW + e xE + s xS + nn xN) (Section 3.2.1
// rows scaled by the control volumes); slot 0 collects sum_j o_j x_{1,j} for the
// origin row (Section 3.2.2) in FP64, which the last block finishes.  The dot products
// of the Krylov modes accumulate per thread in T (FP32 in the mixed path's inner
// solves) and in FP64 across threads and blocks; the residual's maxima are kept as
// integer maxima of bit patterns, its Jacobi scaling multiplies by 1 / diag.
template <typename T, int MODE>
__device__ __forceinline__ void stencil_body(const StArgs<T>& a, int vb, int vg) {
  if (MODE >= M_DOTV && a.red.ks->done) return;
  constexpr int K = Slots<MODE>::K, KMAX = Slots<MODE>::KMAX;
  const T beta = (T)a.par[1];
  const LevelView<T>& L = a.L;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  T dot1 = T(0), dot2 = T(0);
  unsigned long long rbits = 0, sbits = 0, xbits = 0;
  const T* __restrict__ x = a.x;
  const T x0 = x[0];
  for_points(L.sh, a.t, vb, vg, [&](int i, int j, size_t idx, size_t west, size_t east,
                                    size_t south, size_t north) {
    const T xc = x[idx];
    const T xw = (west == 0) ? x0 : x[west];
    const T xe = (east == (size_t)-1) ? T(0) : x[east];
    T val;
    if (sizeof(T) == 8) {
      // FP64: direct form diag x + beta (w xW + e xE + s xS + nn xN)
      T off = L.w[idx] * xw;
      off = fma(L.e[idx], xe, off);
      off = fma(L.s[idx], x[south], off);
      off = fma(L.nn[idx], x[north], off);
      val = fma(beta, off, L.diag[idx] * xc);
      if (i == 1) acc[0] = fma((double)L.o[j], (double)xc, acc[0]);
    } else {
      // FP32: difference form rsum x + beta (w (xW - x) + ...): near the origin the angular
      // couplings exceed the row sum by many orders of magnitude, and differences of
      // neighbouring values lose no digits where the direct form would cancel
      T off = L.w[idx] * (xw - xc);
      off = fma(L.e[idx], xe - xc, off);
      off = fma(L.s[idx], x[south] - xc, off);
      off = fma(L.nn[idx], x[north] - xc, off);
      val = fma(beta, off, L.rsum[idx] * xc);
      if (i == 1) acc[0] = fma((double)L.o[j], (double)xc - (double)x0, acc[0]);
    }
    if (MODE == M_RESID64) {
      val = a.b[idx] - val;
      const unsigned long long ar = abs_bits((double)val);
      rbits = ar > rbits ? ar : rbits;
      // |r| / diag (diag > 0: S is an M-matrix with a positive diagonal)
      const unsigned long long sr = abs_bits(bits_to_double(ar) * L.dinv[idx]);
      sbits = sr > sbits ? sr : sbits;
      const unsigned long long ax = abs_bits((double)xc);
      xbits = ax > xbits ? ax : xbits;
    }
    if (MODE == M_DOTV) dot1 = fma(a.d1[idx], val, dot1);
    if (MODE == M_DOTT) {
      dot1 = fma(val, a.d1[idx], dot1);
      dot2 = fma(val, val, dot2);
    }
    a.y[idx] = val;
  });
  if (MODE == M_RESID64) {
    acc[1] = bits_to_double(rbits);
    acc[2] = bits_to_double(sbits);
    acc[3] = bits_to_double(xbits);
  }
  if (MODE == M_DOTV) acc[1] = (double)dot1;
  if (MODE == M_DOTT) {
    acc[1] = (double)dot1;
    acc[2] = (double)dot2;
  }
  block_reduce<K, KMAX>(acc);
  if (!publish_and_arrive<K>(acc, a.red.part, &a.red.ks->counter, vb, vg)) return;

  // ---- last block: origin row and the scalar epilogue
  double tot[K];
  grid_totals<K, KMAX>(a.red.part, tot, vg);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid != 0) return;
  KrylovScalars* ks = a.red.ks;
  const double d0 = L.sc[0];
  const double x0d = (double)x0;
  double y0 = (sizeof(T) == 8) ? fma((double)beta, tot[0], d0 * x0d)
                                : fma((double)beta, tot[0], L.sc[5] * x0d);
  if (MODE == M_RESID64) y0 = (double)a.b[0] - y0;
  const T y0t = (T)y0;
  a.y[0] = y0t;
  if (MODE == M_RESID64) {
    const double ar = absfin(y0);
    ks->rmax = fmax(tot[1], ar);
    ks->smax = fmax(tot[2], ar / fabs(d0));
    ks->xmax = fmax(tot[3], absfin(x0d));
  }
  if (MODE == M_DOTV) {
    const double dot = tot[1] + (double)a.d1[0] * (double)y0t;
    if (!isfinite(dot)) {
      ks->done = 3;
    } else if (dot == 0.0) {
      ks->done = 2;
    } else {
      ks->alpha = ks->rho / dot;
    }
  }
  if (MODE == M_DOTT) {
    const double ts = tot[1] + (double)y0t * (double)a.d1[0];
    const double tt = tot[2] + (double)y0t * (double)y0t;
    if (!isfinite(ts) || !isfinite(tt)) ks->done = 3;
    ks->omega = (tt > 0.0) ? ts / tt : 0.0;
  }
  ks->counter = 0;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_stencil(StArgs<T> a) {
  stencil_body<T, MODE>(a, blockIdx.x, gridDim.x);
}
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_stencil_b(const StArgs<T>* A, const BSlot* S, int nslots,
                                                   const int* mask) {
  POLAR_BATCH_LOOP({
    const StArgs<T> a = A[s];
    stencil_body<T, MODE>(a, vb, vg);
  })
}

template <typename T, int MODE>
static int stencil_launch(StArgs<T>& a, cudaStream_t st) {
  a.t = make_tiling(a.L.sh);
  const int grid = a.t.ntiles > kMaxBlocks ? kMaxBlocks : a.t.ntiles;
  k_stencil<T, MODE><<<grid, dim3(a.t.TK, a.t.TJ), 0, st>>>(a);
  return 1;
}

template <typename T>
int launch_apply(const LevelView<T>& L, Params p, const T* x, T* y, cudaStream_t st, Reduce red) {
  StArgs<T> a{};
  a.L = L;
  a.par = p;
  a.x = x;
  a.y = y;
  a.red = red;
  return stencil_launch<T, M_APPLY>(a, st);
}

template <typename T>
int launch_apply_dot(const LevelView<T>& L, Params p, const T* x, T* y, const T* d1, int mode,
                     cudaStream_t st, Reduce red) {
  StArgs<T> a{};
  a.L = L;
  a.par = p;
  a.x = x;
  a.y = y;
  a.d1 = d1;
  a.red = red;
  if (mode == 0) return stencil_launch<T, M_DOTV>(a, st);
  return stencil_launch<T, M_DOTT>(a, st);
}

int launch_resid64(const LevelView<double>& L, Params p, const double* x, const double* b,
                   double* r, cudaStream_t st, Reduce red) {
  StArgs<double> a{};
  a.L = L;
  a.par = p;
  a.x = x;
  a.b = b;
  a.y = r;
  a.red = red;
  return stencil_launch<double, M_RESID64>(a, st);
}

// ------------------------------------------------------------------ right-hand side

// e = alpha V u - (1 - theta) (V L) u + sum_q cf_q V src_q + e_{m,j} g_j, the explicit
// half of Eq. (2.5) with the sources of both levels and the Dirichlet data of both
// levels (g_j = sum_q cg_q bnd_q[j], Eq. 2.9) moved to the right-hand side.
__device__ __forceinline__ void rhs_body(const RhsArgs& a, int vb, int vg) {
  const LevelView<double>& L = a.L;
  const double alpha = a.sp->alpha, omt = a.sp->omt;
  double cf[4], cg[4];
  for (int q = 0; q < 4; ++q) {
    cf[q] = a.sp->cf[q];
    cg[q] = a.sp->cg[q];
  }
  double acc[1] = {0.0};
  const double* __restrict__ u = a.u;
  const double u0 = u[0];
  for_points(L.sh, a.t, vb, vg, [&](int i, int j, size_t idx, size_t west, size_t east,
                                    size_t south, size_t north) {
    const double uc = u[idx];
    const double uw = (west == 0) ? u0 : u[west];
    const double ue = (east == (size_t)-1) ? 0.0 : u[east];
    const double w = L.w[idx], e = L.e[idx], s = L.s[idx], nn = L.nn[idx];
    const double rsd = L.rs[idx] - w - e - s - nn;
    double Lu = rsd * uc;
    Lu = fma(w, uw, Lu);
    Lu = fma(e, ue, Lu);
    Lu = fma(s, u[south], Lu);
    Lu = fma(nn, u[north], Lu);
    double val = fma(-omt, Lu, alpha * L.vol[idx] * uc);
    for (int q = 0; q < a.nsrc; ++q) val = fma(cf[q], a.vsrc[q][idx], val);
    if (i == L.sh.m) {
      double g = 0.0;
      for (int q = 0; q < a.nsrc; ++q) g = fma(cg[q], a.bnd[q][j], g);
      val = fma(e, g, val);
    }
    if (i == 1) acc[0] = fma(L.o[j], uc, acc[0]);
    a.e[idx] = val;
  });
  block_reduce<1, 1>(acc);
  if (!publish_and_arrive<1>(acc, a.red.part, &a.red.ks->counter, vb, vg)) return;
  double tot[1];
  grid_totals<1, 1>(a.red.part, tot, vg);
  if (threadIdx.x + blockDim.x * threadIdx.y != 0) return;
  const double vol0 = L.sc[3], rs0 = L.sc[4], osum = L.sc[2];
  const double Lu0 = fma(rs0 - osum, u0, tot[0]);
  double e0 = fma(-omt, Lu0, alpha * vol0 * u0);
  for (int q = 0; q < a.nsrc; ++q) e0 = fma(cf[q], a.vsrc[q][0], e0);
  a.e[0] = e0;
  a.red.ks->counter = 0;
}

__global__ void __launch_bounds__(256) k_rhs(RhsArgs a) { rhs_body(a, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(256) k_rhs_b(const RhsArgs* A, const BSlot* S, int nslots,
                                               const int* mask) {
  POLAR_BATCH_LOOP({
    const RhsArgs a = A[s];
    rhs_body(a, vb, vg);
  })
}

int launch_rhs(const LevelView<double>& L, const StepParams* sp, const double* u, int nsrc,
               const double* const* vsrc, const double* const* bnd, double* e, cudaStream_t st,
               Reduce red) {
  RhsArgs a{};
  a.L = L;
  a.sp = sp;
  a.u = u;
  a.e = e;
  a.nsrc = nsrc;
  for (int q = 0; q < nsrc; ++q) {
    a.vsrc[q] = vsrc[q];
    a.bnd[q] = bnd[q];
  }
  a.red = red;
  a.t = make_tiling(L.sh);
  const int grid = a.t.ntiles > kMaxBlocks ? kMaxBlocks : a.t.ntiles;
  k_rhs<<<grid, dim3(a.t.TK, a.t.TJ), 0, st>>>(a);
  return 1;
}

// ------------------------------------------------------------------ BiCGStab vectors
constexpr int kVT = 256;

__device__ __forceinline__ void set_cond(CondHandle cond, bool value) {
  if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, value ? 1u : 0u);
}


// Batched wrapper of a vector-kernel body: block w.vb of instance w.inst's own grid.
#define POLAR_VEC_BATCHED(NAME, BODY)                                                   \
  template <typename T>                                                                \
  __global__ void __launch_bounds__(kVT) NAME(const VecArgs<T>* A, const BSlot* S,     \
                                              int nslots, const int* mask) {           \
    POLAR_BATCH_LOOP({                                                                 \
      const VecArgs<T> a = A[s];                                                       \
      BODY<T>(a, vb, vg);                                                              \
    })                                                                                 \
  }                                                                                    \
  template <typename T>                                                                \
  __global__ void __launch_bounds__(kVT) NAME##_lone(VecArgs<T> a) {                   \
    BODY<T>(a, blockIdx.x, gridDim.x);                                                 \
  }

// init: r = v0 -> rhat v1, p v2, v v3 = 0, x v4 = 0; the solve's scalars and threshold
template <typename T>
__device__ __forceinline__ void bicg_init_body(const VecArgs<T>& a, int vb, int vg) {
  const StepParams* sp = a.sp;
  const Reduce red = a.red;
  const size_t nv = a.nv;
  const T* r = a.v0;
  T *rhat = a.v1, *p = a.v2, *v = a.v3, *x = a.v4;
  const double rel_tol = sp->inner_tol;
  const int max_iter = sp->max_iter;
  double acc[1];
  T s = T(0);  // per thread in T, across threads in FP64
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)vg * kVT) {
    const T rv = r[k];
    rhat[k] = rv;
    p[k] = rv;
    v[k] = T(0);
    x[k] = T(0);
    s = fma(rv, rv, s);
  }
  acc[0] = (double)s;
  block_reduce<1, 1>(acc);
  if (!publish_and_arrive<1>(acc, red.part, &red.ks->counter, vb, vg)) return;
  double tot[1];
  grid_totals<1, 1>(red.part, tot, vg);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  ks->rr0 = tot[0];
  ks->rr = tot[0];
  ks->rho = tot[0];
  ks->tol2 = rel_tol * rel_tol * tot[0];
  // The inner residual is r / rmax with r the FP64 residual, so its Jacobi-scaled max
  // norm starts at smax / rmax.  The solve stops once that norm has fallen by the
  // larger of the requested reduction and what the outer test still needs (a tenth of
  // tol max|x| after the correction): the max norm, like the outer test, so that a few
  // rows cannot hide behind a small 2-norm of many.
  const double need = (ks->smax > 0.0) ? 0.1 * sp->tol * ks->xmax / ks->smax : 1.0;
  ks->sm_tol = fmax(rel_tol, need) * (ks->rmax > 0.0 ? ks->smax / ks->rmax : 0.0);
  ks->sm = INFINITY;
  ks->sm_best = INFINITY;
  ks->sm_best_it = 0;
  ks->alpha = 1.0;
  ks->omega = 1.0;
  ks->beta = 0.0;
  ks->iters = 0;
  ks->max_iter = max_iter;
  ks->done = !isfinite(tot[0]) ? 3 : (tot[0] == 0.0 ? 1 : 0);
  ks->counter = 0;
  set_cond(a.cond, ks->done == 0);
}
POLAR_VEC_BATCHED(k_bicg_init, bicg_init_body)

// s v2 = r v0 - alpha v v1
template <typename T>
__device__ __forceinline__ void bicg_s_body(const VecArgs<T>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  if (ks->done) return;
  const T alpha = (T)ks->alpha;
  const T *r = a.v0, *v = a.v1;
  T* s = a.v2;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    s[k] = fma(-alpha, v[k], r[k]);
}
POLAR_VEC_BATCHED(k_bicg_s, bicg_s_body)

// |r| / d in FP32 (a stopping test needs no more), in FP64 when d is outside the FP32
// range; padding entries have d = 0
template <typename T>
__device__ __forceinline__ float scaled_abs(T r, T d) {
  if (!(d > T(0))) return 0.f;
  const float df = (float)d;
  if (df >= 1e-30f && df <= 1e30f) return fabsf((float)r) / df;
  return (float)fmin(fabs((double)r) / (double)d, 3.0e38);
}

// FP32 inner solves: true once the Jacobi-scaled residual `sm` has not halved for
// kStallIters iterations (the FP32 operator cannot resolve what is left).
template <typename T>
__device__ __forceinline__ bool fp32_stalled(KrylovScalars* ks, double sm) {
  if (sizeof(T) != 4) return false;
  if (sm < 0.5 * ks->sm_best) {
    ks->sm_best = sm;
    ks->sm_best_it = ks->iters;
    return false;
  }
  return ks->iters - ks->sm_best_it >= kStallIters;
}

// x v0 += alpha phat v1 + omega shat v2;  r v3 = s v4 - omega t v5;  rho = rhat v6 . r,
// rr = r . r and the stopping test on max |r_i| / diag_i
template <typename T>
__device__ __forceinline__ void bicg_update_body(const VecArgs<T>& a, int vb, int vg) {
  const Reduce red = a.red;
  if (red.ks->done) return;
  const T alpha = (T)red.ks->alpha, omega = (T)red.ks->omega;
  const T d0 = (T)a.sc[0];  // the origin's diagonal lives in the level scalars
  T* x = a.v0;
  const T *phat = a.v1, *shat = a.v2;
  T* r = a.v3;
  const T *s = a.v4, *t = a.v5, *rhat = a.v6, *diag = a.diag;
  T s1 = T(0), s2 = T(0);  // per thread in T, across threads in FP64
  float sm = 0.f;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT) {
    x[k] = fma(omega, shat[k], fma(alpha, phat[k], x[k]));
    const T rn = fma(-omega, t[k], s[k]);
    r[k] = rn;
    s1 = fma(rhat[k], rn, s1);
    s2 = fma(rn, rn, s2);
    sm = fmaxf(sm, scaled_abs<T>(rn, k == 0 ? d0 : diag[k]));
  }
  double acc[3] = {(double)s1, (double)s2, isfinite(sm) ? (double)sm : INFINITY};
  block_reduce<3, 2>(acc);
  if (!publish_and_arrive<3>(acc, red.part, &red.ks->counter, vb, vg)) return;
  double tot[3];
  grid_totals<3, 2>(red.part, tot, vg);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  const double rho_new = tot[0], rr = tot[1];
  ks->rr = rr;
  ks->sm = tot[2];
  ks->iters += 1;
  if (!isfinite(rr) || !isfinite(rho_new)) {
    ks->done = 3;
  } else if (tot[2] <= ks->sm_tol) {
    ks->done = 1;
  } else if (ks->iters >= ks->max_iter || fp32_stalled<T>(ks, tot[2])) {
    ks->done = 4;
  } else if (ks->omega == 0.0 || rho_new == 0.0 || ks->rho == 0.0) {
    ks->done = 2;
  } else {
    ks->beta = (rho_new / ks->rho) * (ks->alpha / ks->omega);
    ks->rho = rho_new;
  }
  ks->counter = 0;
}
POLAR_VEC_BATCHED(k_bicg_update, bicg_update_body)

// p v0 = r v1 + beta (p - omega v v2); "keep iterating" to the graph's WHILE node
template <typename T>
__device__ __forceinline__ void bicg_p_body(const VecArgs<T>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  const bool running = ks->done == 0;
  if (vb == 0 && threadIdx.x == 0) set_cond(a.cond, running);
  if (!running) return;
  const T beta = (T)ks->beta, omega = (T)ks->omega;
  T* p = a.v0;
  const T *r = a.v1, *v = a.v2;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    p[k] = fma(beta, fma(-omega, v[k], p[k]), r[k]);
}
POLAR_VEC_BATCHED(k_bicg_p, bicg_p_body)

template <typename T>
VecArgs<T> vec_args(size_t nv, Reduce red) {
  VecArgs<T> a{};
  a.nv = nv;
  a.red = red;
  return a;
}

template <typename T>
int launch_bicg_init(size_t nv, const T* r, T* rhat, T* p, T* v, T* x, const StepParams* sp,
                     CondHandle cond, cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = const_cast<T*>(r);
  a.v1 = rhat;
  a.v2 = p;
  a.v3 = v;
  a.v4 = x;
  a.sp = sp;
  a.cond = cond;
  k_bicg_init_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}
template <typename T>
int launch_bicg_s(size_t nv, const T* r, const T* v, T* s, cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = const_cast<T*>(r);
  a.v1 = const_cast<T*>(v);
  a.v2 = s;
  k_bicg_s_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}
template <typename T>
int launch_bicg_update(size_t nv, T* x, const T* phat, const T* shat, T* r, const T* s,
                       const T* t, const T* rhat, const T* diag, const double* sc,
                       cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = x;
  a.v1 = const_cast<T*>(phat);
  a.v2 = const_cast<T*>(shat);
  a.v3 = r;
  a.v4 = const_cast<T*>(s);
  a.v5 = const_cast<T*>(t);
  a.v6 = const_cast<T*>(rhat);
  a.diag = diag;
  a.sc = sc;
  k_bicg_update_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}
template <typename T>
int launch_bicg_p(size_t nv, T* p, const T* r, const T* v, CondHandle cond, cudaStream_t st,
                  Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = p;
  a.v1 = const_cast<T*>(r);
  a.v2 = const_cast<T*>(v);
  a.cond = cond;
  k_bicg_p_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}

// ------------------------------------------------------------------ conjugate gradients
// Preconditioned CG for symmetric systems (no drift: S = alpha V + beta V L is symmetric
// positive definite and the V(1,1) cycle with its zebra smoother in mirrored order is a
// symmetric preconditioner).  One iteration: z = M r (V-cycle), rho = r.z and
// beta = rho / rho_prev (k_cg_rho), p = z + beta p (k_cg_p), q = S p with
// alpha = rho / p.q (the stencil's DOTV mode with d1 = p), then x += alpha p,
// r -= alpha q and the stopping test (k_cg_update).  Set-up is k_bicg_init (x = 0, the
// stopping threshold; its p = r is scaled by beta = 0 in the first iteration).

// rho = r v0 . z v1
template <typename T>
__device__ __forceinline__ void cg_rho_body(const VecArgs<T>& a, int vb, int vg) {
  const Reduce red = a.red;
  if (red.ks->done) return;
  const T *r = a.v0, *z = a.v1;
  T s = T(0);  // per thread in T, across threads in FP64
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    s = fma(r[k], z[k], s);
  double acc[1] = {(double)s};
  block_reduce<1, 1>(acc);
  if (!publish_and_arrive<1>(acc, red.part, &red.ks->counter, vb, vg)) return;
  double tot[1];
  grid_totals<1, 1>(red.part, tot, vg);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  const double rho = tot[0];
  if (!isfinite(rho)) {
    ks->done = 3;
  } else if (rho == 0.0) {
    ks->done = 2;
  } else {
    ks->beta = (ks->iters == 0) ? 0.0 : rho / ks->rho;
    ks->rho = rho;
  }
  ks->counter = 0;
}
POLAR_VEC_BATCHED(k_cg_rho, cg_rho_body)

// p v0 = z v1 + beta p
template <typename T>
__device__ __forceinline__ void cg_p_body(const VecArgs<T>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  if (ks->done) return;
  const T beta = (T)ks->beta;
  T* p = a.v0;
  const T* z = a.v1;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    p[k] = fma(beta, p[k], z[k]);
}
POLAR_VEC_BATCHED(k_cg_p, cg_p_body)

// x v0 += alpha p v1;  r v2 -= alpha q v3;  stopping test on max |r_i| / diag_i
template <typename T>
__device__ __forceinline__ void cg_update_body(const VecArgs<T>& a, int vb, int vg) {
  const Reduce red = a.red;
  if (red.ks->done) {
    if (vb == 0 && threadIdx.x == 0) set_cond(a.cond, false);
    return;
  }
  const T alpha = (T)red.ks->alpha;
  const T d0 = (T)a.sc[0];
  T* x = a.v0;
  const T* p = a.v1;
  T* r = a.v2;
  const T *q = a.v3, *diag = a.diag;
  float sm = 0.f;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT) {
    x[k] = fma(alpha, p[k], x[k]);
    const T rn = fma(-alpha, q[k], r[k]);
    r[k] = rn;
    sm = fmaxf(sm, scaled_abs<T>(rn, k == 0 ? d0 : diag[k]));
  }
  double acc[1] = {isfinite(sm) ? (double)sm : INFINITY};
  block_reduce<1, 0>(acc);
  if (!publish_and_arrive<1>(acc, red.part, &red.ks->counter, vb, vg)) return;
  double tot[1];
  grid_totals<1, 0>(red.part, tot, vg);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  ks->sm = tot[0];
  ks->iters += 1;
  if (!isfinite(tot[0])) {
    ks->done = 3;
  } else if (tot[0] <= ks->sm_tol) {
    ks->done = 1;
  } else if (ks->iters >= ks->max_iter || fp32_stalled<T>(ks, tot[0])) {
    ks->done = 4;
  }
  ks->counter = 0;
  set_cond(a.cond, ks->done == 0);
}
POLAR_VEC_BATCHED(k_cg_update, cg_update_body)

template <typename T>
int launch_cg_rho(size_t nv, const T* r, const T* z, cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = const_cast<T*>(r);
  a.v1 = const_cast<T*>(z);
  k_cg_rho_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}
template <typename T>
int launch_cg_p(size_t nv, T* p, const T* z, cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = p;
  a.v1 = const_cast<T*>(z);
  k_cg_p_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}
template <typename T>
int launch_cg_update(size_t nv, T* x, const T* p, T* r, const T* q, const T* diag,
                     const double* sc, CondHandle cond, cudaStream_t st, Reduce red) {
  VecArgs<T> a = vec_args<T>(nv, red);
  a.v0 = x;
  a.v1 = const_cast<T*>(p);
  a.v2 = r;
  a.v3 = const_cast<T*>(q);
  a.diag = diag;
  a.sc = sc;
  a.cond = cond;
  k_cg_update_lone<T><<<grid_for(nv, kVT), kVT, 0, st>>>(a);
  return 1;
}

// ------------------------------------------------------------------ step control
// The mixed path starts a step with the FP64 solve while the sticky countdown of an
// earlier switch runs.
__device__ __forceinline__ void start_step(const StepParams& p, KrylovScalars* ks) {
  ks->use64 = (p.mixed && ks->sticky64 > 0) ? 1 : 0;
  if (ks->use64) ks->sticky64 -= 1;
}

__global__ void k_step_begin(const StepParams* sp, KrylovScalars* ks) {
  ks->step_on = 1;
  ks->failed = 0;
  start_step(*sp, ks);
  ks->inner_done = 0;
  ks->prev_scaled = INFINITY;
  ks->iters64 = 0;
  ks->sweeps = 0;
  ks->iters_total = 0;
  ks->converged = 0;
  ks->scaled = 0.0;
  ks->done = 0;
  ks->counter = 0;
}
int launch_step_begin(const StepParams* sp, cudaStream_t st, Reduce red) {
  k_step_begin<<<1, 1, 0, st>>>(sp, red.ks);
  return 1;
}

__device__ __forceinline__ void sched_begin_body(const StepParams* sched, const int* kstep,
                                                 StepParams* sp, StepOut* out, CondHandle cond,
                                                 KrylovScalars* ks) {
  const int k = *kstep;
  if (ks->halt) {
    out[k] = StepOut{0, 0, -7, 0, 0.0};  // POLAR_ESTATE: not run
    ks->step_on = 0;
    ks->refine_on = 0;
    set_cond(cond, false);
    return;
  }
  ks->step_on = 1;
  *sp = sched[k];
  ks->failed = 0;
  start_step(sched[k], ks);
  ks->inner_done = 0;
  ks->prev_scaled = INFINITY;
  ks->iters64 = 0;
  ks->sweeps = 0;
  ks->iters_total = 0;
  ks->converged = 0;
  ks->scaled = 0.0;
  ks->done = 0;
  ks->counter = 0;
  set_cond(cond, true);
}
__global__ void k_sched_begin(const StepParams* sched, const int* kstep, StepParams* sp,
                              StepOut* out, CondHandle cond, KrylovScalars* ks) {
  sched_begin_body(sched, kstep, sp, out, cond, ks);
}
int launch_sched_begin(const StepParams* sched, const int* kstep, StepParams* sp, StepOut* out,
                       CondHandle cond, cudaStream_t st, Reduce red) {
  k_sched_begin<<<1, 1, 0, st>>>(sched, kstep, sp, out, cond, red.ks);
  return 1;
}

__global__ void k_sched_end(const int* kstep, StepOut* out, KrylovScalars* ks) {
  out[*kstep] = StepOut{ks->iters_total, ks->sweeps, ks->failed, ks->iters64, ks->scaled};
  if (ks->failed) ks->halt = 1;
}
int launch_sched_end(const int* kstep, StepOut* out, cudaStream_t st, Reduce red) {
  k_sched_end<<<1, 1, 0, st>>>(kstep, out, red.ks);
  return 1;
}

__global__ void k_sched_next(int* kstep) { *kstep += 1; }
int launch_sched_next(int* kstep, cudaStream_t st) {
  k_sched_next<<<1, 1, 0, st>>>(kstep);
  return 1;
}

// After the FP64 residual (rmax, smax, xmax): the step has converged when the
// Jacobi-scaled residual is within the tolerance; it fails after max_refine corrections
// or on a non-finite residual.
__device__ __forceinline__ void refine_decide_body(const StepParams* sp, CondHandle cond,
                                                   KrylovScalars* ks) {
  bool more = false;
  if (ks->failed == 0) {
    ks->sweeps += 1;
    const double scaled = ks->smax / fmax(ks->xmax, 1e-300);
    ks->scaled = scaled;
    if (!isfinite(scaled) || !isfinite(ks->rmax)) {
      ks->failed = -5;  // POLAR_ENONFINITE
    } else if (scaled <= sp->tol) {
      ks->converged = 1;
    } else if (ks->sweeps > sp->max_refine) {
      ks->failed = -4;  // POLAR_ENOCONV
    } else {
      more = true;
      // a correction that gained less than a factor 10, or an inner solve that broke
      // down or ran out of iterations, switches the step to the FP64 Krylov solve
      if (ks->sweeps > 1 && (scaled > 0.1 * ks->prev_scaled || ks->inner_done >= 2) &&
          !ks->use64) {
        ks->use64 = 1;
        if (sp->mixed) ks->sticky64 = kStickySteps;
      }
    }
    ks->prev_scaled = scaled;
  }
  ks->refine_on = more ? 1 : 0;
  set_cond(cond, more);
}
__global__ void k_refine_decide(const StepParams* sp, CondHandle cond, KrylovScalars* ks) {
  refine_decide_body(sp, cond, ks);
}

// Selects the inner solve of the next refinement sweep (mixed path).
__global__ void k_choose_inner(CondHandle c32, CondHandle c64, const KrylovScalars* ks) {
  set_cond(c32, ks->use64 == 0);
  set_cond(c64, ks->use64 != 0);
}
int launch_choose_inner(CondHandle c32, CondHandle c64, cudaStream_t st, Reduce red) {
  k_choose_inner<<<1, 1, 0, st>>>(c32, c64, red.ks);
  return 1;
}
int launch_refine_decide(const StepParams* sp, CondHandle cond, cudaStream_t st, Reduce red) {
  k_refine_decide<<<1, 1, 0, st>>>(sp, cond, red.ks);
  return 1;
}

// tolerant: the solve was the mixed path's FP32 one, whose non-finite end (FP32 overflow
// on a near-singular ring) only discards its correction and moves the step to the FP64
// Krylov solve; a non-finite FP64 solve fails the step.
__global__ void k_after_inner(KrylovScalars* ks, int tolerant) {
  ks->iters_total += ks->iters;
  if (ks->use64) ks->iters64 += ks->iters;
  ks->inner_done = ks->done;
  if (ks->done == 3 && !tolerant && ks->failed == 0) ks->failed = -5;  // POLAR_ENONFINITE
}
int launch_after_inner(int tolerant, cudaStream_t st, Reduce red) {
  k_after_inner<<<1, 1, 0, st>>>(red.ks, tolerant);
  return 1;
}

__global__ void __launch_bounds__(kVT) k_copy_if(size_t n, const double* a, double* b,
                                                 const KrylovScalars* ks, int need_converged) {
  if (ks->failed) return;
  if (need_converged && !ks->converged) return;
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < n; k += (size_t)gridDim.x * kVT)
    b[k] = a[k];
}
int launch_commit(size_t nv, double* U, const double* X, cudaStream_t st, Reduce red) {
  k_copy_if<<<grid_for(nv, kVT), kVT, 0, st>>>(nv, X, U, red.ks, 1);
  return 1;
}
int launch_copy(size_t n, const double* a, double* b, cudaStream_t st, Reduce red) {
  k_copy_if<<<grid_for(n, kVT), kVT, 0, st>>>(n, a, b, red.ks, 0);
  return 1;
}

// ------------------------------------------------------------------ refinement helpers
template <typename T>
__global__ void __launch_bounds__(kVT) k_scale_cast(size_t nv, const double* r, T* rs,
                                                    const KrylovScalars* ks) {
  const double inv = ks->rmax > 0.0 ? 1.0 / ks->rmax : 0.0;
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT)
    rs[k] = (T)(r[k] * inv);
}
template <typename T>
__global__ void __launch_bounds__(kVT) k_correct(size_t nv, double* x, const T* d,
                                                 const KrylovScalars* ks) {
  if (ks->failed || ks->inner_done == 3) return;  // no non-finite correction reaches x
  const double s = ks->rmax;
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT)
    x[k] = fma(s, (double)d[k], x[k]);
}
template <typename T>
int launch_scale_cast(size_t nv, const double* r, T* rs, cudaStream_t st, Reduce red) {
  k_scale_cast<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, r, rs, red.ks);
  return 1;
}
template <typename T>
int launch_correct(size_t nv, double* x, const T* d, cudaStream_t st, Reduce red) {
  k_correct<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, x, d, red.ks);
  return 1;
}

__global__ void k_to_float(size_t n, const double* a, float* b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}
int launch_to_float(size_t n, const double* a, float* b, cudaStream_t st) {
  k_to_float<<<grid_for(n, kVT), kVT, 0, st>>>(n, a, b);
  return 1;
}

__global__ void k_check_finite(size_t n, const double* a, KrylovScalars* ks) {
  bool bad = false;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[k]);
  if (bad) ks->done = 3;
}
int launch_check_finite(size_t n, const double* a, cudaStream_t st, Reduce red) {
  k_check_finite<<<grid_for(n, kVT), kVT, 0, st>>>(n, a, red.ks);
  return 1;
}

// ------------------------------------------------------------------ batched step control
// One block (one thread) per instance; CtlArgs[i] holds instance i's step data.
__global__ void k_sched_begin_b(const CtlArgs* A) {
  const CtlArgs a = A[blockIdx.x];
  sched_begin_body(a.sched, a.kstep, a.sp, a.out, 0, a.ks);
}
__global__ void k_refine_decide_b(const CtlArgs* A, int gate) {
  const CtlArgs a = A[blockIdx.x];
  if (!gate_pass(gate, a.ks, a.sp)) return;
  refine_decide_body(a.sp, 0, a.ks);
}
__global__ void k_after_inner_b(const CtlArgs* A, int gate) {
  const CtlArgs a = A[blockIdx.x];
  if (!gate_pass(gate, a.ks, a.sp)) return;
  KrylovScalars* ks = a.ks;
  ks->iters_total += ks->iters;
  if (ks->use64) ks->iters64 += ks->iters;
  ks->inner_done = ks->done;
  if (ks->done == 3 && gate != G_32 && ks->failed == 0) ks->failed = -5;  // POLAR_ENONFINITE
}
__global__ void k_sched_end_b(const CtlArgs* A, int gate) {
  const CtlArgs a = A[blockIdx.x];
  if (!gate_pass(gate, a.ks, a.sp)) return;
  KrylovScalars* ks = a.ks;
  a.out[*a.kstep] = StepOut{ks->iters_total, ks->sweeps, ks->failed, ks->iters64, ks->scaled};
  if (ks->failed) ks->halt = 1;
}
__global__ void k_sched_next_b(const CtlArgs* A) { *A[blockIdx.x].kstep_w += 1; }
// Active-instance mask of a list (one thread block): mask[A[k].inst] = the gate passes
// (and, with need_running, the instance's Krylov solve still runs); `cond` = any passes.
__global__ void k_mask_b(const CtlArgs* A, int count, int gate, int need_running, int* mask,
                         CondHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const CtlArgs& a = A[i];
    const int on = gate_pass(gate, a.ks, a.sp) && (!need_running || a.ks->done == 0);
    mask[a.inst] = on;
    if (on) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) set_cond(cond, any != 0);
}

// vector helpers: w0 -> w1 copies (flag: only when the step converged), the scaled cast
// w0 -> v0 and the FP64 correction w0 += rmax v0
__device__ __forceinline__ void copy_if_body(const VecArgs<double>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  if (ks->failed) return;
  if (a.flag && !ks->converged) return;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    a.w1[k] = a.w0[k];
}
template <typename T>
__device__ __forceinline__ void copy_if_body_t(const VecArgs<T>& a, int vb, int vg) {
  copy_if_body(a, vb, vg);
}
template <typename T>
__device__ __forceinline__ void scale_cast_body(const VecArgs<T>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  const double inv = ks->rmax > 0.0 ? 1.0 / ks->rmax : 0.0;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    a.v0[k] = (T)(a.w0[k] * inv);
}
template <typename T>
__device__ __forceinline__ void correct_body(const VecArgs<T>& a, int vb, int vg) {
  const KrylovScalars* ks = a.red.ks;
  if (ks->failed || ks->inner_done == 3) return;  // no non-finite correction reaches x
  const double s = ks->rmax;
  for (size_t k = vb * (size_t)kVT + threadIdx.x; k < a.nv; k += (size_t)vg * kVT)
    a.w0[k] = fma(s, (double)a.v0[k], a.w0[k]);
}
POLAR_VEC_BATCHED(k_copy_b, copy_if_body_t)
POLAR_VEC_BATCHED(k_scale_cast_b, scale_cast_body)
POLAR_VEC_BATCHED(k_correct_b, correct_body)

// ------------------------------------------------------------------ face fields
// v = -mobility grad u at the faces of the scheme (u in the interface layout): radial face
// (i+1/2, j), i = 0..m, at j (m+1) + i:  -mobility (u_{i+1,j} - u_{i,j}) / h_{i+1} with
// u_{0,j} the origin and u_{m+1,j} = g_j;  angular face (i, j+1/2), i = 1..m, at j m + i - 1:
// -mobility (u_{i,j+1} - u_{i,j}) / (r_i mu_{j+1}), mu_n = 2 pi + theta_0 - theta_{n-1}.
__global__ void k_face_drift(int m, int n, const double* u, const double* r, const double* th,
                             const double* g, double mobility, double* vr, double* vt) {
  const size_t nr = (size_t)(m + 1) * n, nt = (size_t)m * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nr + nt;
       q += (size_t)gridDim.x * blockDim.x) {
    if (q < nr) {
      const int j = (int)(q / (m + 1)), i = (int)(q - (size_t)j * (m + 1));
      const double uin = (i == 0) ? u[0] : u[1 + (size_t)j * m + (i - 1)];
      const double uout = (i == m) ? g[j] : u[1 + (size_t)j * m + i];
      vr[q] = -mobility * (uout - uin) / (r[i + 1] - r[i]);
    } else {
      const size_t t = q - nr;
      const int j = (int)(t / m), i = (int)(t - (size_t)j * m) + 1;
      const int jn = (j + 1 < n) ? j + 1 : 0;
      const double mu = (j + 1 < n) ? th[j + 1] - th[j] : 6.283185307179586 + th[0] - th[n - 1];
      const double ua = u[1 + (size_t)j * m + (i - 1)], ub = u[1 + (size_t)jn * m + (i - 1)];
      vt[t] = -mobility * (ub - ua) / (r[i] * mu);
    }
  }
}
int launch_face_drift(int m, int n, const double* u, const double* r, const double* th,
                      const double* g, double mobility, double* vr, double* vt, cudaStream_t st) {
  const size_t work = (size_t)(2 * m + 1) * n;
  k_face_drift<<<grid_for(work, kVT), kVT, 0, st>>>(m, n, u, r, th, g, mobility, vr, vt);
  return 1;
}

__global__ void k_max_change(size_t n, const double* a, const double* b,
                             unsigned long long* out) {
  unsigned long long d = 0, x = 0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    d = max(d, abs_bits(a[k] - b[k]));
    x = max(x, abs_bits(a[k]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
    x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, d);
    atomicMax(out + 1, x);
  }
}
int launch_max_change(size_t n, const double* a, const double* b, double* out, cudaStream_t st) {
  if (cudaMemsetAsync(out, 0, 2 * sizeof(double), st) != cudaSuccess) return -1;
  k_max_change<<<grid_for(n, kVT), kVT, 0, st>>>(n, a, b, reinterpret_cast<unsigned long long*>(out));
  return 1;
}

// ------------------------------------------------------------------ Anderson acceleration
// split index of unknown q (0: the origin, 1 + j m + (i - 1): node (i, j))
__device__ __forceinline__ size_t split_of(const Shape& sh, size_t q) {
  if (q == 0) return 0;
  const size_t jj = (q - 1) / sh.m;
  return sh.at((int)(q - 1 - jj * sh.m) + 1, (int)jj);
}

__global__ void k_aa_columns(Shape sh, const double* g, const double* x, const double* f_last,
                             const double* x_last, double* f, double* dF, double* dX, int last) {
  const size_t N = (size_t)sh.m * sh.n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    const size_t p = split_of(sh, q);
    const double fv = g[p] - x[p];
    f[p] = fv;
    if (last) {
      dF[p] = fv - f_last[p];
      dX[p] = x[p] - x_last[p];
    }
  }
}
int launch_aa_columns(const Shape& sh, const double* g, const double* x, const double* f_last,
                      const double* x_last, double* f, double* dF, double* dX, bool last,
                      cudaStream_t st) {
  k_aa_columns<<<grid_for((size_t)sh.m * sh.n + 1, kVT), kVT, 0, st>>>(sh, g, x, f_last, x_last,
                                                                       f, dF, dX, last ? 1 : 0);
  return 1;
}

constexpr int kAAMaxDots = kMaxAnderson * (kMaxAnderson + 1) / 2 + kMaxAnderson;
__global__ void __launch_bounds__(256) k_aa_dots(Shape sh, AndersonCols c, double* partials) {
  const int k = c.count - 1, nd = k * (k + 1) / 2 + k;
  double acc[kAAMaxDots];
#pragma unroll
  for (int d = 0; d < kAAMaxDots; ++d) acc[d] = 0.0;
  const size_t N = (size_t)sh.m * sh.n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    const size_t p = split_of(sh, q);
    double v[kMaxAnderson + 1];
#pragma unroll
    for (int a = 0; a <= kMaxAnderson; ++a) v[a] = a <= k ? c.v[a][p] : 0.0;
    int d = 0;
#pragma unroll
    for (int a = 0; a < kMaxAnderson; ++a)
#pragma unroll
      for (int b = 0; b <= kMaxAnderson; ++b) {
        // pairs (a, b) with a <= b < k, then (a, k): the columns against the right-hand side
        const bool pair = a < k && ((b >= a && b < k) || b == kMaxAnderson);
        if (pair) {
          const double w = (b == kMaxAnderson) ? v[k] : v[b];
          acc[d] = fma(v[a], w, acc[d]);
          ++d;
        }
      }
  }
  __shared__ double red[8][kAAMaxDots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < nd; ++d) {
    double s = acc[d];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][d] = s;
  }
  __syncthreads();
  if (threadIdx.x < nd) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    partials[(size_t)blockIdx.x * nd + threadIdx.x] = s;
  }
}
int launch_aa_dots(const Shape& sh, const AndersonCols& c, double* partials, int blocks,
                   cudaStream_t st) {
  k_aa_dots<<<blocks, 256, 0, st>>>(sh, c, partials);
  return 1;
}

struct AAGamma {
  double g[kMaxAnderson];
};
__global__ void k_aa_update(Shape sh, AndersonCols dX, AndersonCols dF, AAGamma gm, double* x) {
  const size_t N = (size_t)sh.m * sh.n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    const size_t p = split_of(sh, q);
    double v = x[p];
    for (int a = 0; a < dX.count; ++a) v -= gm.g[a] * (dX.v[a][p] + dF.v[a][p]);
    x[p] = v;
  }
}
int launch_aa_update(const Shape& sh, const AndersonCols& dX, const AndersonCols& dF,
                     const double* gamma_host, double* x, cudaStream_t st) {
  AAGamma gm{};
  for (int a = 0; a < dX.count; ++a) gm.g[a] = gamma_host[a];
  k_aa_update<<<grid_for((size_t)sh.m * sh.n + 1, kVT), kVT, 0, st>>>(sh, dX, dF, gm, x);
  return 1;
}

// ------------------------------------------------------------------ layout conversion
// interface index q = 1 + j m + (i - 1) <-> split index sh.at(i, j); q = 0 is the origin
__global__ void k_pack(Shape sh, const double* in, const double* scale, double* out) {
  const size_t N = (size_t)sh.m * sh.n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    size_t p = 0;
    if (q > 0) {
      const size_t jj = (q - 1) / sh.m;
      const int ii = (int)(q - 1 - jj * sh.m) + 1;
      p = sh.at(ii, (int)jj);
    }
    out[p] = scale ? in[q] * scale[p] : in[q];
  }
}
__global__ void k_unpack(Shape sh, const double* in, const double* div, double* out) {
  const size_t N = (size_t)sh.m * sh.n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    size_t p = 0;
    if (q > 0) {
      const size_t jj = (q - 1) / sh.m;
      const int ii = (int)(q - 1 - jj * sh.m) + 1;
      p = sh.at(ii, (int)jj);
    }
    out[q] = div ? in[p] / div[p] : in[p];
  }
}
int launch_pack(const Shape& sh, const double* in, const double* scale, double* out,
                cudaStream_t st) {
  k_pack<<<grid_for((size_t)sh.m * sh.n + 1, kVT), kVT, 0, st>>>(sh, in, scale, out);
  return 1;
}
int launch_unpack(const Shape& sh, const double* in, const double* div, double* out,
                  cudaStream_t st) {
  k_unpack<<<grid_for((size_t)sh.m * sh.n + 1, kVT), kVT, 0, st>>>(sh, in, div, out);
  return 1;
}


// ------------------------------------------------------------------ batched launchers
template <typename T>
int launch_stencil_b(int mode, const StArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                     int grid, int TK, cudaStream_t st) {
  if (nslots <= 0) return 0;
  const dim3 block(TK, 256 / TK);
  switch (mode) {
    case M_APPLY: k_stencil_b<T, M_APPLY><<<grid, block, 0, st>>>(A, S, nslots, mask); break;
    case M_DOTV: k_stencil_b<T, M_DOTV><<<grid, block, 0, st>>>(A, S, nslots, mask); break;
    case M_DOTT: k_stencil_b<T, M_DOTT><<<grid, block, 0, st>>>(A, S, nslots, mask); break;
    default:
      if constexpr (sizeof(T) == 8) {
        k_stencil_b<T, M_RESID64><<<grid, block, 0, st>>>(A, S, nslots, mask);
      } else {
        return -1;
      }
  }
  return 1;
}
int launch_rhs_b(const RhsArgs* A, const BSlot* S, int nslots, const int* mask, int grid, int TK,
                 cudaStream_t st) {
  if (nslots <= 0) return 0;
  k_rhs_b<<<grid, dim3(TK, 256 / TK), 0, st>>>(A, S, nslots, mask);
  return 1;
}
template <typename T>
int launch_vec_b(int kind, const VecArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                 int grid, cudaStream_t st) {
  if (nslots <= 0) return 0;
  switch (kind) {
    case V_BICG_INIT: k_bicg_init<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_BICG_S: k_bicg_s<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_BICG_UPDATE: k_bicg_update<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_BICG_P: k_bicg_p<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_CG_RHO: k_cg_rho<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_CG_P: k_cg_p<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_CG_UPDATE: k_cg_update<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_SCALE_CAST: k_scale_cast_b<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    case V_CORRECT: k_correct_b<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask); break;
    default:
      if constexpr (sizeof(T) == 8) {
        k_copy_b<T><<<grid, kVT, 0, st>>>(A, S, nslots, mask);
      } else {
        return -1;
      }
  }
  return 1;
}
int launch_ctl_b(int kind, const CtlArgs* A, int count, int gate, cudaStream_t st) {
  if (count <= 0) return 0;
  switch (kind) {
    case C_SCHED_BEGIN: k_sched_begin_b<<<count, 1, 0, st>>>(A); break;
    case C_DECIDE: k_refine_decide_b<<<count, 1, 0, st>>>(A, gate); break;
    case C_AFTER_INNER: k_after_inner_b<<<count, 1, 0, st>>>(A, gate); break;
    case C_SCHED_END: k_sched_end_b<<<count, 1, 0, st>>>(A, gate); break;
    default: k_sched_next_b<<<count, 1, 0, st>>>(A); break;
  }
  return 1;
}
int launch_mask_b(const CtlArgs* A, int count, int gate, int need_running, int* mask,
                  CondHandle cond, cudaStream_t st) {
  k_mask_b<<<1, 256, 0, st>>>(A, count, gate, need_running, mask, cond);
  return 1;
}

// ------------------------------------------------------------------ instantiations
#define POLAR_INST(T)                                                                          \
  template int launch_apply<T>(const LevelView<T>&, Params, const T*, T*, cudaStream_t,        \
                               Reduce);                                                        \
  template int launch_apply_dot<T>(const LevelView<T>&, Params, const T*, T*, const T*, int,   \
                                   cudaStream_t, Reduce);                                      \
  template int launch_bicg_init<T>(size_t, const T*, T*, T*, T*, T*, const StepParams*,        \
                                   CondHandle, cudaStream_t, Reduce);                          \
  template int launch_bicg_s<T>(size_t, const T*, const T*, T*, cudaStream_t, Reduce);         \
  template int launch_bicg_update<T>(size_t, T*, const T*, const T*, T*, const T*, const T*,   \
                                     const T*, const T*, const double*, cudaStream_t, Reduce); \
  template int launch_bicg_p<T>(size_t, T*, const T*, const T*, CondHandle, cudaStream_t,      \
                                Reduce);                                                       \
  template int launch_cg_rho<T>(size_t, const T*, const T*, cudaStream_t, Reduce);            \
  template int launch_cg_p<T>(size_t, T*, const T*, cudaStream_t, Reduce);                      \
  template int launch_cg_update<T>(size_t, T*, const T*, T*, const T*, const T*, const double*, \
                                   CondHandle, cudaStream_t, Reduce);                          \
  template int launch_scale_cast<T>(size_t, const double*, T*, cudaStream_t, Reduce);          \
  template int launch_correct<T>(size_t, double*, const T*, cudaStream_t, Reduce);          \
  template int launch_stencil_b<T>(int, const StArgs<T>*, const BSlot*, int, const int*, int, \
                                   int, cudaStream_t);                                      \
  template int launch_vec_b<T>(int, const VecArgs<T>*, const BSlot*, int, const int*, int,    \
                               cudaStream_t);

POLAR_INST(float)
POLAR_INST(double)

}  // namespace polar
