// CUDA kernels of the implicit theta-step on the polar mesh (sm_103a).
//
// Every kernel is bandwidth- or FP64-issue-bound: nothing here is a dense contraction,
// so no tensor-core path exists.  Reductions are deterministic: every block reduces
// its elements in a fixed order, writes one partial per block, and the last block to
// arrive (atomic counter + fences) sums the partials in block order and finishes the
// scalar recurrences of the Krylov solver on the device.
#include "polar_internal.h"

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
    for (int k = 0; k < K; ++k) v[k] = (lane < nw) ? sh[k][lane] : 0.0;
    warp_reduce<K, KMAX>(v);
  }
  __syncthreads();
}

// Publishes this block's partials (thread 0 holds them) and reports whether this
// block is the last one of the grid to arrive.
template <int K>
__device__ bool publish_and_arrive(const double (&v)[K], double* part, unsigned int* counter) {
  __shared__ unsigned int s_last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int bid = blockIdx.x + gridDim.x * blockIdx.y;
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[k * kMaxBlocks + bid] = v[k];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x * gridDim.y - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Called by every thread of the last block: totals in block order (result in thread 0).
template <int K, int KMAX>
__device__ void grid_totals(const double* part, double (&tot)[K]) {
  const int nb = gridDim.x * gridDim.y;
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

// ------------------------------------------------------------------ stencil
// One kernel body for every use of the 5-point operator; MODE selects the epilogue.
enum { M_APPLY = 0, M_RESID = 1, M_RHS = 2, M_RESID64 = 3, M_DOTV = 4, M_DOTT = 5 };

template <typename T>
struct StArgs {
  OpView<T> op;
  T alpha, beta;
  const T* x;
  const T* b;   // M_RESID / M_RESID64: right-hand side
  T* y;
  const T* d1;  // M_DOTV: rhat; M_DOTT: s
  int nsrc;
  const double* src[4];
  const double* bnd[4];
  double cf[4], cg[4];
  Reduce red;
  int nic, njg;  // tiles: nic chunks along i  x  njg groups of lines
  double c0;     // diagonal of the origin row of L
};

// Slots: [0] origin coupling sum_j o_j x_{1,j}; then mode-specific sums; maxima last.
template <int MODE>
struct Slots {
  static constexpr int K = (MODE == M_RESID64) ? 4 : (MODE == M_DOTV) ? 2 : (MODE == M_DOTT) ? 3 : 1;
  static constexpr int KMAX = (MODE == M_RESID64) ? 1 : K;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_stencil(StArgs<T> a) {
  if ((MODE >= M_DOTV || MODE == M_RESID) && a.red.ks->done) return;
  constexpr int K = Slots<MODE>::K, KMAX = Slots<MODE>::KMAX;
  const int m = a.op.m, n = a.op.n, ld = a.op.ld;
  const int TI = blockDim.x, TJ = blockDim.y;
  const int ntiles = a.nic * a.njg;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  T accT1 = T(0), accT2 = T(0);
  const T alpha = a.alpha, beta = a.beta;
  const T x0 = a.x[0];

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int jg = tile / a.nic, ic = tile - jg * a.nic;
    const int i = ic * TI + threadIdx.x + 1;
    const int j = jg * TJ + threadIdx.y;
    if (i > m || j >= n) continue;
    const size_t idx = kOfs + (size_t)j * ld + (i - 1);
    const ptrdiff_t ds = (j == 0) ? (ptrdiff_t)(n - 1) * ld : -(ptrdiff_t)ld;
    const ptrdiff_t dn = (j == n - 1) ? -(ptrdiff_t)(n - 1) * ld : (ptrdiff_t)ld;
    const T xc = a.x[idx];
    const T xw = (i == 1) ? x0 : a.x[idx - 1];
    const T xs = a.x[idx + ds];
    const T xn = a.x[idx + dn];
    T xe = (i == m) ? T(0) : a.x[idx + 1];
    if (MODE == M_RHS && i == m) {  // Dirichlet value on r = 1 (Eq. 2.9)
      double g = 0.0;
      for (int q = 0; q < a.nsrc; ++q) g = fma(a.cg[q], a.bnd[q][j], g);
      xe = (T)g;
    }
    const T cW = a.op.W[idx], cE = a.op.E[idx], cS = a.op.S[idx], cN = a.op.N[idx];
    T Lx = a.op.R[idx] * xc;
    Lx = fma(cW, xw - xc, Lx);
    Lx = fma(cE, xe - xc, Lx);
    Lx = fma(cS, xs - xc, Lx);
    Lx = fma(cN, xn - xc, Lx);
    T val = fma(beta, Lx, alpha * xc);
    if (i == 1) acc[0] = fma((double)a.op.o[j], (double)xc - (double)x0, acc[0]);
    if (MODE == M_RESID || MODE == M_RESID64) val = a.b[idx] - val;
    if (MODE == M_RHS) {
      double s = (double)val;
      for (int q = 0; q < a.nsrc; ++q) s = fma(a.cf[q], a.src[q][idx], s);
      val = (T)s;
    }
    if (MODE == M_RESID64) {
      const double cdiag = (double)a.op.R[idx] - (double)cW - (double)cE - (double)cS - (double)cN;
      const double dg = fabs((double)alpha + (double)beta * cdiag);
      const double ar = absfin((double)val);
      acc[1] = fmax(acc[1], ar);
      acc[2] = fmax(acc[2], ar / dg);
      acc[3] = fmax(acc[3], absfin((double)xc));
    }
    if (MODE == M_DOTV) accT1 = fma(a.d1[idx], val, accT1);
    if (MODE == M_DOTT) {
      accT1 = fma(val, a.d1[idx], accT1);
      accT2 = fma(val, val, accT2);
    }
    a.y[idx] = val;
  }
  if (MODE == M_DOTV) acc[1] = (double)accT1;
  if (MODE == M_DOTT) {
    acc[1] = (double)accT1;
    acc[2] = (double)accT2;
  }
  block_reduce<K, KMAX>(acc);
  if (!publish_and_arrive<K>(acc, a.red.part, &a.red.ks->counter)) return;

  // ---- last block: origin row (Section 3.2.2) and the scalar epilogue
  double tot[K];
  grid_totals<K, KMAX>(a.red.part, tot);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid != 0) return;
  KrylovScalars* ks = a.red.ks;
  const double x0d = (double)x0;
  const double L0 = fma((double)a.op.R[0], x0d, tot[0]);
  double y0 = fma((double)beta, L0, (double)alpha * x0d);
  if (MODE == M_RESID || MODE == M_RESID64) y0 = (double)a.b[0] - y0;
  if (MODE == M_RHS)
    for (int q = 0; q < a.nsrc; ++q) y0 = fma(a.cf[q], a.src[q][0], y0);
  const T y0t = (T)y0;
  a.y[0] = y0t;
  if (MODE == M_RESID64) {
    const double dg = fabs((double)alpha + (double)beta * a.c0);
    const double ar = absfin(y0);
    ks->rmax = fmax(tot[1], ar);
    ks->smax = fmax(tot[2], ar / dg);
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

template <typename T>
static void stencil_shape(const OpView<T>& op, dim3& blk, int& nic, int& njg) {
  int TI = 32;
  while (TI < op.m && TI < 256) TI <<= 1;
  const int TJ = 256 / TI;
  blk = dim3(TI, TJ);
  nic = (op.m + TI - 1) / TI;
  njg = (op.n + TJ - 1) / TJ;
}

template <typename T, int MODE>
static int stencil_launch(StArgs<T>& a, cudaStream_t st) {
  dim3 blk;
  stencil_shape(a.op, blk, a.nic, a.njg);
  size_t tiles = (size_t)a.nic * a.njg;
  int grid = tiles > (size_t)kMaxBlocks ? kMaxBlocks : (int)tiles;
  k_stencil<T, MODE><<<grid, blk, 0, st>>>(a);
  return 1;
}

template <typename T>
static StArgs<T> st_args(const OpView<T>& op, T alpha, T beta, const T* x, T* y, Reduce red) {
  StArgs<T> a{};
  a.op = op;
  a.alpha = alpha;
  a.beta = beta;
  a.x = x;
  a.y = y;
  a.red = red;
  return a;
}

template <typename T>
int launch_apply(const OpView<T>& op, T alpha, T beta, const T* x, T* y, cudaStream_t st,
                 Reduce red) {
  StArgs<T> a = st_args(op, alpha, beta, x, y, red);
  return stencil_launch<T, M_APPLY>(a, st);
}

template <typename T>
int launch_resid(const OpView<T>& op, T alpha, T beta, const T* x, const T* b, T* y,
                 cudaStream_t st, Reduce red) {
  StArgs<T> a = st_args(op, alpha, beta, x, y, red);
  a.b = b;
  return stencil_launch<T, M_RESID>(a, st);
}

int launch_rhs(const OpView<double>& op, double alpha, double beta, const double* x,
               int nsrc, const double* const* src, const double* const* bnd,
               const double* cf, const double* cg, double* e, cudaStream_t st, Reduce red) {
  StArgs<double> a = st_args(op, alpha, beta, x, e, red);
  a.nsrc = nsrc;
  for (int q = 0; q < nsrc; ++q) {
    a.src[q] = src[q];
    a.bnd[q] = bnd[q];
    a.cf[q] = cf[q];
    a.cg[q] = cg[q];
  }
  return stencil_launch<double, M_RHS>(a, st);
}

int launch_resid64(const OpView<double>& op, double alpha, double beta, const double* x,
                   const double* e, double* r, double c0, cudaStream_t st, Reduce red) {
  StArgs<double> a = st_args(op, alpha, beta, x, r, red);
  a.b = e;
  a.c0 = c0;
  return stencil_launch<double, M_RESID64>(a, st);
}

template <typename T>
int launch_apply_dot(const OpView<T>& op, T alpha, T beta, const T* x, T* y, const T* d1,
                     int mode, cudaStream_t st, Reduce red) {
  StArgs<T> a = st_args(op, alpha, beta, x, y, red);
  a.d1 = d1;
  if (mode == 0) return stencil_launch<T, M_DOTV>(a, st);
  return stencil_launch<T, M_DOTT>(a, st);
}

// ------------------------------------------------------------------ line factors
// LU factors (Doolittle, no pivoting: the line blocks of an M-matrix are diagonally
// dominant) of every radial line block, one thread per line.
__device__ __forceinline__ double diag_of(const OpView<double>& op, size_t idx) {
  return op.R[idx] - op.W[idx] - op.E[idx] - op.S[idx] - op.N[idx];
}

template <typename T>
__global__ void k_factor_radial(OpView<double> op, double alpha, double beta, T* rl, T* rui,
                                T* rcu) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= op.n) return;
  const int m = op.m;
  const size_t base = kOfs + (size_t)j * op.ld;
  double uprev = 1.0, cprev = 0.0;
  for (int k = 0; k < m; ++k) {
    const double a = (k > 0) ? beta * op.W[base + k] : 0.0;
    const double b = alpha + beta * diag_of(op, base + k);
    const double c = (k < m - 1) ? beta * op.E[base + k] : 0.0;
    const double l = (k > 0) ? a / uprev : 0.0;
    const double u = b - l * cprev;
    const double ui = 1.0 / u;
    rl[base + k] = (T)l;
    rui[base + k] = (T)ui;
    rcu[base + k] = (T)(c * ui);
    uprev = u;
    cprev = c;
  }
}

// Periodic angular line of ring i: A = A' + u v^T with gamma = -b_0,
// u = (gamma, 0, .., 0, c_{n-1}), v = (1, 0, .., 0, a_0 / gamma) (Sherman-Morrison);
// LU factors of the tridiagonal A', q = A'^{-1} u, vf = a_0 / gamma, inv1vq = 1/(1 + v.q).
template <typename T>
__global__ void k_factor_angular(OpView<double> op, double alpha, double beta, T* al, T* aui,
                                 T* acu, T* aq, T* avf, T* ainv, double* ws) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (i > op.m) return;
  const int n = op.n;
  const size_t ld = op.ld;
  const size_t col = kOfs + (size_t)(i - 1);
  const double a0 = beta * op.S[col];
  const double b0 = alpha + beta * diag_of(op, col);
  const double cn1 = beta * op.N[col + (size_t)(n - 1) * ld];
  const double gamma = -b0;
  const double vf = a0 / gamma;
  double uprev = 1.0, cprev = 0.0, yq = 0.0;
  // ws[idx] keeps the FP64 forward values of q and ws[idx + ld n] the FP64 pivot
  // reciprocals, so that q and 1 + v.q are formed in FP64 whatever T is.
  for (int j = 0; j < n; ++j) {
    const size_t idx = col + (size_t)j * ld;
    const double a = (j > 0) ? beta * op.S[idx] : 0.0;
    double b = alpha + beta * diag_of(op, idx);
    if (j == 0) b -= gamma;
    if (j == n - 1) b -= cn1 * vf;
    const double c = (j < n - 1) ? beta * op.N[idx] : 0.0;
    const double l = (j > 0) ? a / uprev : 0.0;
    const double u = b - l * cprev;
    const double ui = 1.0 / u;
    al[idx] = (T)l;
    aui[idx] = (T)ui;
    acu[idx] = (T)(c * ui);
    const double ur = (j == 0) ? gamma : ((j == n - 1) ? cn1 : 0.0);
    yq = ur - l * yq;
    ws[idx] = yq;
    ws[idx + op.ld * (size_t)n] = ui;  // second half: FP64 pivot reciprocal
    uprev = u;
    cprev = c;
  }
  // backward pass for q in FP64: q_j = ui_j y_j - (c_j ui_j) q_{j+1}
  double qnext = 0.0, q0 = 0.0, qn1 = 0.0;
  for (int j = n - 1; j >= 0; --j) {
    const size_t idx = col + (size_t)j * ld;
    const double ui = ws[idx + op.ld * (size_t)n];
    const double c = (j < n - 1) ? beta * op.N[idx] : 0.0;
    const double q = ui * (ws[idx] - c * qnext);
    aq[idx] = (T)q;
    if (j == n - 1) qn1 = q;
    if (j == 0) q0 = q;
    qnext = q;
  }
  avf[i - 1] = (T)vf;
  ainv[i - 1] = (T)(1.0 / (1.0 + q0 + vf * qn1));
}

template <typename T>
int launch_factor(const OpView<double>& op, double alpha, double beta, LineFactors<T>& f,
                  cudaStream_t st) {
  k_factor_radial<T><<<(op.n + 63) / 64, 64, 0, st>>>(op, alpha, beta, f.rl, f.rui, f.rcu);
  k_factor_angular<T><<<(op.m + 63) / 64, 64, 0, st>>>(op, alpha, beta, f.al, f.aui, f.acu, f.aq,
                                                      f.avf, f.ainv, f.ws);
  return 2;
}

// ------------------------------------------------------------------ line solves
// The forward and backward substitutions are first-order affine recurrences; each
// thread composes the maps of its chunk, a block scan of the composed maps gives every
// chunk its incoming value, and the chunk is replayed.  Composition: a map is (A, B),
// x -> A x + B; the scan forms  R_p = M_p o R_{p-1}.
template <typename T>
__device__ void scan_affine(T A, T B, T* sA, T* sB, int r, int pos, int RW, int TW) {
  sA[pos * RW + r] = A;
  sB[pos * RW + r] = B;
  __syncthreads();
  for (int off = 1; off < TW; off <<= 1) {
    const T a = sA[pos * RW + r], b = sB[pos * RW + r];
    T ao = T(1), bo = T(0);
    const bool has = pos >= off;
    if (has) {
      ao = sA[(pos - off) * RW + r];
      bo = sB[(pos - off) * RW + r];
    }
    __syncthreads();
    if (has) {
      sA[pos * RW + r] = a * ao;
      sB[pos * RW + r] = fma(a, bo, b);
    }
    __syncthreads();
  }
}

constexpr int kRT = 128;  // threads per radial line

__host__ __device__ inline int spad(int k) { return k + (k >> 5); }

template <typename T>
__global__ void __launch_bounds__(kRT) k_radial_solve(int m, int ld, const T* __restrict__ rl,
                                                      const T* __restrict__ rui,
                                                      const T* __restrict__ rcu,
                                                      const T* __restrict__ rhs, T* __restrict__ out,
                                                      T diag0, const int* done) {
  if (done && *done) return;
  extern __shared__ unsigned char smraw[];
  T* s = reinterpret_cast<T*>(smraw);
  T* sA = s + spad(m) + 1;
  T* sB = sA + kRT;
  const int j = blockIdx.x, t = threadIdx.x;
  const size_t base = kOfs + (size_t)j * ld;
  for (int k = t; k < m; k += kRT) s[spad(k)] = rhs[base + k];
  if (j == 0 && t == 0) out[0] = rhs[0] / diag0;
  __syncthreads();
  const int P = (m + kRT - 1) / kRT;
  const int k0 = min(m, t * P), k1 = min(m, k0 + P);
  T A = T(1), B = T(0);
  for (int k = k0; k < k1; ++k) {
    const T l = rl[base + k];
    B = s[spad(k)] - l * B;
    A = -l * A;
  }
  scan_affine(A, B, sA, sB, 0, t, 1, kRT);
  T prev = (t > 0) ? sB[t - 1] : T(0);
  for (int k = k0; k < k1; ++k) {
    const T y = s[spad(k)] - rl[base + k] * prev;
    s[spad(k)] = y;
    prev = y;
  }
  __syncthreads();
  A = T(1);
  B = T(0);
  for (int k = k1 - 1; k >= k0; --k) {
    const T ui = rui[base + k], cu = rcu[base + k];
    B = ui * s[spad(k)] - cu * B;
    A = -cu * A;
  }
  const int pos = kRT - 1 - t;
  scan_affine(A, B, sA, sB, 0, pos, 1, kRT);
  T next = (pos > 0) ? sB[pos - 1] : T(0);
  for (int k = k1 - 1; k >= k0; --k) {
    const T x = rui[base + k] * s[spad(k)] - rcu[base + k] * next;
    s[spad(k)] = x;
    next = x;
  }
  __syncthreads();
  for (int k = t; k < m; k += kRT) out[base + k] = s[spad(k)];
}

template <typename T>
int launch_radial_solve(const OpView<T>& op, const LineFactors<T>& f, const T* rhs, T* out,
                        cudaStream_t st, const int* done) {
  const size_t smem = sizeof(T) * ((size_t)spad(op.m) + 1 + 2 * kRT);
  static bool attr_set = false;  // one opt-in per instantiation for lines beyond 48 KB
  if (!attr_set) {
    cudaFuncSetAttribute(k_radial_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set = true;
  }
  k_radial_solve<T><<<op.n, kRT, smem, st>>>(op.m, op.ld, f.rl, f.rui, f.rcu, rhs, out, f.diag0,
                                            done);
  return 1;
}

// Angular solve: block = RW rings (threadIdx.x, adjacent in memory) x TW chunks of
// the angular line (threadIdx.y).
template <typename T>
__global__ void __launch_bounds__(256) k_angular_solve(int m, int n, int ld, const T* __restrict__ al,
                                                       const T* __restrict__ aui,
                                                       const T* __restrict__ acu,
                                                       const T* __restrict__ aq,
                                                       const T* __restrict__ avf,
                                                       const T* __restrict__ ainv, const T* rhs,
                                                       const T* base, T* out, T* tmp, T diag0,
                                                       const int* done) {
  if (done && *done) return;
  extern __shared__ unsigned char smraw[];
  const int RW = blockDim.x, TW = blockDim.y;
  T* sA = reinterpret_cast<T*>(smraw);
  T* sB = sA + RW * TW;
  T* sx0 = sB + RW * TW;
  T* sxn = sx0 + RW;
  const int r = threadIdx.x, c = threadIdx.y;
  const int i = blockIdx.x * RW + r + 1;
  const bool valid = i <= m;
  const int P = (n + TW - 1) / TW;
  const int j0 = min(n, c * P), j1 = min(n, j0 + P);
  const size_t col = kOfs + (size_t)(i - 1);
  if (blockIdx.x == 0 && r == 0 && c == 0) out[0] = (base ? base[0] : T(0)) + rhs[0] / diag0;
  T A = T(1), B = T(0);
  if (valid) {
    for (int j = j0; j < j1; ++j) {
      const size_t idx = col + (size_t)j * ld;
      const T l = al[idx];
      B = rhs[idx] - l * B;
      A = -l * A;
    }
  }
  scan_affine(A, B, sA, sB, r, c, RW, TW);
  T prev = (c > 0) ? sB[(c - 1) * RW + r] : T(0);
  if (valid) {
    for (int j = j0; j < j1; ++j) {
      const size_t idx = col + (size_t)j * ld;
      const T y = rhs[idx] - al[idx] * prev;
      tmp[idx] = y;
      prev = y;
    }
  }
  __syncthreads();
  A = T(1);
  B = T(0);
  if (valid) {
    for (int j = j1 - 1; j >= j0; --j) {
      const size_t idx = col + (size_t)j * ld;
      const T cu = acu[idx];
      B = aui[idx] * tmp[idx] - cu * B;
      A = -cu * A;
    }
  }
  const int pos = TW - 1 - c;
  scan_affine(A, B, sA, sB, r, pos, RW, TW);
  T next = (pos > 0) ? sB[(pos - 1) * RW + r] : T(0);
  if (valid) {
    for (int j = j1 - 1; j >= j0; --j) {
      const size_t idx = col + (size_t)j * ld;
      const T x = aui[idx] * tmp[idx] - acu[idx] * next;
      tmp[idx] = x;
      next = x;
      if (j == 0) sx0[r] = x;
      if (j == n - 1) sxn[r] = x;
    }
  }
  __syncthreads();
  if (valid) {
    const T sigma = (sx0[r] + avf[i - 1] * sxn[r]) * ainv[i - 1];
    for (int j = j0; j < j1; ++j) {
      const size_t idx = col + (size_t)j * ld;
      const T v = tmp[idx] - sigma * aq[idx];
      out[idx] = base ? base[idx] + v : v;
    }
  }
}

template <typename T>
int launch_angular_solve(const OpView<T>& op, const LineFactors<T>& f, const T* rhs,
                         const T* base, T* out, T* tmp, cudaStream_t st, const int* done) {
  int RW = 32;
  while (RW > 4 && (op.m + RW - 1) / RW < 2 * 152) RW >>= 1;
  int TW = 256 / RW;
  while (TW > 1 && (op.n + TW - 1) / TW < 2) TW >>= 1;
  const size_t smem = sizeof(T) * (2 * (size_t)RW * TW + 2 * RW);
  const int grid = (op.m + RW - 1) / RW;
  k_angular_solve<T><<<grid, dim3(RW, TW), smem, st>>>(op.m, op.n, op.ld, f.al, f.aui, f.acu,
                                                       f.aq, f.avf, f.ainv, rhs, base, out, tmp,
                                                       f.diag0, done);
  return 1;
}

// ------------------------------------------------------------------ BiCGStab vectors
constexpr int kVT = 256;

template <typename T>
__global__ void __launch_bounds__(kVT) k_bicg_init(size_t nv, const T* r, T* rhat, T* p, T* v,
                                                   T* x, int zero_x, double rel_tol,
                                                   int max_iter, Reduce red) {
  double acc[1];
  T s = T(0);
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT) {
    const T rv = r[k];
    rhat[k] = rv;
    p[k] = rv;
    v[k] = T(0);
    if (zero_x) x[k] = T(0);
    s = fma(rv, rv, s);
  }
  acc[0] = (double)s;
  block_reduce<1, 1>(acc);
  if (!publish_and_arrive<1>(acc, red.part, &red.ks->counter)) return;
  double tot[1];
  grid_totals<1, 1>(red.part, tot);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  ks->rr0 = tot[0];
  ks->rr = tot[0];
  ks->rho = tot[0];
  ks->tol2 = rel_tol * rel_tol * tot[0];
  ks->alpha = 1.0;
  ks->omega = 1.0;
  ks->beta = 0.0;
  ks->iters = 0;
  ks->max_iter = max_iter;
  ks->done = !isfinite(tot[0]) ? 3 : (tot[0] == 0.0 ? 1 : 0);
  ks->counter = 0;
}

template <typename T>
__global__ void __launch_bounds__(kVT) k_bicg_s(size_t nv, const T* r, const T* v, T* s,
                                                KrylovScalars* ks) {
  if (ks->done) return;
  const T alpha = (T)ks->alpha;
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT)
    s[k] = r[k] - alpha * v[k];
}

template <typename T>
__global__ void __launch_bounds__(kVT) k_bicg_update(size_t nv, T* x, const T* phat,
                                                     const T* shat, T* r, const T* s,
                                                     const T* t, const T* rhat, Reduce red) {
  if (red.ks->done) return;
  const T alpha = (T)red.ks->alpha, omega = (T)red.ks->omega;
  T s1 = T(0), s2 = T(0);
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT) {
    x[k] = fma(omega, shat[k], fma(alpha, phat[k], x[k]));
    const T rn = s[k] - omega * t[k];
    r[k] = rn;
    s1 = fma(rhat[k], rn, s1);
    s2 = fma(rn, rn, s2);
  }
  double acc[2] = {(double)s1, (double)s2};
  block_reduce<2, 2>(acc);
  if (!publish_and_arrive<2>(acc, red.part, &red.ks->counter)) return;
  double tot[2];
  grid_totals<2, 2>(red.part, tot);
  if (threadIdx.x != 0) return;
  KrylovScalars* ks = red.ks;
  const double rho_new = tot[0], rr = tot[1];
  ks->rr = rr;
  ks->iters += 1;
  if (!isfinite(rr) || !isfinite(rho_new)) {
    ks->done = 3;
  } else if (rr <= ks->tol2) {
    ks->done = 1;
  } else if (ks->iters >= ks->max_iter) {
    ks->done = 4;
  } else if (ks->omega == 0.0 || rho_new == 0.0 || ks->rho == 0.0) {
    ks->done = 2;
  } else {
    ks->beta = (rho_new / ks->rho) * (ks->alpha / ks->omega);
    ks->rho = rho_new;
  }
  ks->counter = 0;
}

template <typename T>
__global__ void __launch_bounds__(kVT) k_bicg_p(size_t nv, T* p, const T* r, const T* v,
                                                KrylovScalars* ks) {
  if (ks->done) return;
  const T beta = (T)ks->beta, omega = (T)ks->omega;
  for (size_t k = blockIdx.x * (size_t)kVT + threadIdx.x; k < nv; k += (size_t)gridDim.x * kVT)
    p[k] = fma(beta, p[k] - omega * v[k], r[k]);
}

template <typename T>
int launch_bicg_init(size_t nv, const T* r, T* rhat, T* p, T* v, T* x, bool zero_x,
                     double rel_tol, int max_iter, cudaStream_t st, Reduce red) {
  k_bicg_init<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, r, rhat, p, v, x, zero_x ? 1 : 0, rel_tol,
                                                    max_iter, red);
  return 1;
}
template <typename T>
int launch_bicg_s(size_t nv, const T* r, const T* v, T* s, cudaStream_t st, Reduce red) {
  k_bicg_s<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, r, v, s, red.ks);
  return 1;
}
template <typename T>
int launch_bicg_update(size_t nv, T* x, const T* phat, const T* shat, T* r, const T* s,
                       const T* t, const T* rhat, cudaStream_t st, Reduce red) {
  k_bicg_update<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, x, phat, shat, r, s, t, rhat, red);
  return 1;
}
template <typename T>
int launch_bicg_p(size_t nv, T* p, const T* r, const T* v, cudaStream_t st, Reduce red) {
  k_bicg_p<T><<<grid_for(nv, kVT), kVT, 0, st>>>(nv, p, r, v, red.ks);
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

// ------------------------------------------------------------------ layout conversion
__global__ void k_pack(int m, int n, int ld, const double* in, double* out) {
  const size_t N = (size_t)m * n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    if (q == 0) {
      out[0] = in[0];
    } else {
      const size_t jj = (q - 1) / m, ii = (q - 1) - jj * m;
      out[kOfs + jj * ld + ii] = in[q];
    }
  }
}
__global__ void k_unpack(int m, int n, int ld, const double* in, double* out) {
  const size_t N = (size_t)m * n + 1;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N;
       q += (size_t)gridDim.x * blockDim.x) {
    if (q == 0) {
      out[0] = in[0];
    } else {
      const size_t jj = (q - 1) / m, ii = (q - 1) - jj * m;
      out[q] = in[kOfs + jj * ld + ii];
    }
  }
}
int launch_pack(int m, int n, int ld, const double* in, double* out, cudaStream_t st) {
  k_pack<<<grid_for((size_t)m * n + 1, kVT), kVT, 0, st>>>(m, n, ld, in, out);
  return 1;
}
int launch_unpack(int m, int n, int ld, const double* in, double* out, cudaStream_t st) {
  k_unpack<<<grid_for((size_t)m * n + 1, kVT), kVT, 0, st>>>(m, n, ld, in, out);
  return 1;
}

// ------------------------------------------------------------------ instantiations
#define POLAR_INST(T)                                                                          \
  template int launch_apply<T>(const OpView<T>&, T, T, const T*, T*, cudaStream_t, Reduce);    \
  template int launch_resid<T>(const OpView<T>&, T, T, const T*, const T*, T*, cudaStream_t,   \
                               Reduce);                                                        \
  template int launch_apply_dot<T>(const OpView<T>&, T, T, const T*, T*, const T*, int,        \
                                   cudaStream_t, Reduce);                                      \
  template int launch_factor<T>(const OpView<double>&, double, double, LineFactors<T>&,        \
                                cudaStream_t);                                                 \
  template int launch_radial_solve<T>(const OpView<T>&, const LineFactors<T>&, const T*, T*,   \
                                      cudaStream_t, const int*);                               \
  template int launch_angular_solve<T>(const OpView<T>&, const LineFactors<T>&, const T*,      \
                                       const T*, T*, T*, cudaStream_t, const int*);            \
  template int launch_bicg_init<T>(size_t, const T*, T*, T*, T*, T*, bool, double, int,        \
                                   cudaStream_t, Reduce);                                      \
  template int launch_bicg_s<T>(size_t, const T*, const T*, T*, cudaStream_t, Reduce);         \
  template int launch_bicg_update<T>(size_t, T*, const T*, const T*, T*, const T*, const T*,   \
                                     const T*, cudaStream_t, Reduce);                          \
  template int launch_bicg_p<T>(size_t, T*, const T*, const T*, cudaStream_t, Reduce);         \
  template int launch_scale_cast<T>(size_t, const double*, T*, cudaStream_t, Reduce);          \
  template int launch_correct<T>(size_t, double*, const T*, cudaStream_t, Reduce);

POLAR_INST(float)
POLAR_INST(double)

}  // namespace polar
