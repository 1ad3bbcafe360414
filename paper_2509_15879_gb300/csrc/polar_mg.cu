// Multigrid preconditioner of the theta-step system S x = b (sm_103a).
//
// Levels coarsen the radial direction only (rings 2, 4, 6, ... of a level form the
// next coarser one); the angular direction keeps all n angles.  The smoother relaxes
// whole rings at once: every ring is a periodic tridiagonal system in the angle
// (Eqs. 2.6-2.7), solved exactly with LU factors and a Sherman-Morrison correction for
// the periodic corner entries, odd rings first, then the origin and the even rings
// (zebra order).  Because the radial couplings of the coarse levels are the Schur
// complements of the odd rings (cyclic reduction of every radial line, see
// polar_api.cu), this combination converges independently of the strong angular
// coupling near the origin and of the radial grading toward r = 0 and r = 1.
//
// Kernels:
//   k_refresh         per step: diag, ring factors, origin scalars of every level
//   k_ring<.., mode>  one zebra half-sweep of one level (all rings of one parity)
//   k_restrict        residual of the odd rings -> right-hand side of the coarser level
//   k_coarsest        exact solve of the coarsest level (origin + one ring)
// A V(1,1) cycle on L levels launches 5 (L - 1) + 1 kernels.
//
// The ring solve: the n angles of a ring are split into TW chunks of P consecutive
// angles (one thread each, values in registers).  The forward and backward
// substitutions are first-order affine recurrences; each thread composes the maps of
// its chunk, a block scan of the composed maps gives every chunk its incoming value,
// and the chunk is replayed.  Rings longer than one CTA can hold are split over the
// CTAs of a thread-block cluster, which exchange their segment maps and the ring's end
// values through distributed shared memory.
#include <cooperative_groups.h>

#include <algorithm>

#include <vector>

#include "polar_internal.h"

namespace cg = cooperative_groups;

namespace polar {

// ---------------------------------------------------------------------------------
// per-step refresh


// Whether a refresh has work: the step's do_refresh flag, or, for factors kept beside the
// step's own (the mixed path's FP64 factors, formed only when its FP64 solve runs), the
// stamp of the (alpha, beta) they were last formed for.
__device__ __forceinline__ bool refresh_due(const StepParams* sp, const double* stamp) {
  if (!stamp) return sp->do_refresh != 0;
  return !(stamp[0] == sp->alpha && stamp[1] == sp->beta);
}

// Ring i of a level is the periodic tridiagonal system
//   a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j  (indices mod n) with
//   a_j = beta s_ij,  b_j = alpha vol_ij + beta (rs - w - e - s - nn)_ij,  c_j = beta nn_ij.
// Sherman-Morrison: with gamma = -b_0, u = (gamma, 0, .., 0, c_{n-1}),
// v = (1, 0, .., 0, a_0 / gamma), the system is (T' + u v^T) x = d where T' is the
// non-periodic tridiagonal part with b'_0 = b_0 - gamma and
// b'_{n-1} = b_{n-1} - c_{n-1} a_0 / gamma.  Stored: Doolittle factors of T'
// (l_j = a_j / u_{j-1}, ui_j = 1 / u_j, cu_j = c_j / u_j), q = T'^{-1} u and, per ring,
// vf = a_0 / gamma and 1 / (1 + v.q).
//
// A CTA factors RF rings of one parity block (threadIdx.x; consecutive rings are
// adjacent in memory) with TF threads per ring (threadIdx.y), each owning a chunk of
// consecutive angles.  Every recurrence along the ring is turned into a scan over the
// chunks:
//   pivots  u_j = b'_j - a_j c_{j-1} / u_{j-1} is the projective action of the 2 x 2
//           matrices [[b'_j, -a_j c_{j-1}], [1, 0]] on (u_{j-1}, 1): each chunk composes
//           its matrices (rescaled by powers of two), an exclusive scan gives every chunk
//           its incoming pivot, and the chunk replays the recurrence from it;
//   y = L^{-1} u forward and q = U^{-1} y backward are affine recurrences, scanned the
//           same way (the backward one with the chunk order reversed).
// All arithmetic is FP64; only the stored factors take the inner precision T.

struct M2 {  // [[a, b], [c, d]]
  double a, b, c, d;
};
struct A2 {  // x -> a x + b
  double a, b;
};
__device__ __forceinline__ M2 comb(const M2& first, const M2& then) {  // then * first
  return M2{fma(then.a, first.a, then.b * first.c), fma(then.a, first.b, then.b * first.d),
            fma(then.c, first.a, then.d * first.c), fma(then.c, first.b, then.d * first.d)};
}
__device__ __forceinline__ A2 comb(const A2& first, const A2& then) {  // then o first
  return A2{then.a * first.a, fma(then.a, first.b, then.b)};
}
__device__ __forceinline__ M2 shfl_up(const M2& v, int off) {
  return M2{__shfl_up_sync(0xffffffffu, v.a, off), __shfl_up_sync(0xffffffffu, v.b, off),
            __shfl_up_sync(0xffffffffu, v.c, off), __shfl_up_sync(0xffffffffu, v.d, off)};
}
__device__ __forceinline__ A2 shfl_up(const A2& v, int off) {
  return A2{__shfl_up_sync(0xffffffffu, v.a, off), __shfl_up_sync(0xffffffffu, v.b, off)};
}
// rescales a matrix by a power of two (exact) so that its largest entry is in [1, 2)
__device__ __forceinline__ M2 renorm(const M2& m) {
  const double mx = fmax(fmax(fabs(m.a), fabs(m.b)), fmax(fabs(m.c), fabs(m.d)));
  if (!(mx > 0.0) || !isfinite(mx)) return m;
  const int e = ilogb(mx);
  return M2{ldexp(m.a, -e), ldexp(m.b, -e), ldexp(m.c, -e), ldexp(m.d, -e)};
}

// composition inside the scans: the matrix products are rescaled after every step (their
// entries hold different powers of the coupling, and unscaled products over a long ring
// underflow); the affine maps only shrink
__device__ __forceinline__ M2 scan_comb(const M2& first, const M2& then) {
  return renorm(comb(first, then));
}
__device__ __forceinline__ A2 scan_comb(const A2& first, const A2& then) {
  return comb(first, then);
}

// Exclusive scan over the TF chunks of each ring of the CTA (thread (r, c), linear index
// r + RF c): returns the composition of the maps of chunks 0..c-1 (identity for c = 0).
template <typename V>
__device__ V chunk_excl_scan(V v, const V& ident, V* sw) {
  const int tid = threadIdx.x + RF * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const int per = 32 / RF, pos = lane / RF, r = threadIdx.x;
  V inc = v;
#pragma unroll
  for (int off = 1; off < per; off <<= 1) {
    const V o = shfl_up(inc, off * RF);
    if (pos >= off) inc = scan_comb(o, inc);
  }
  V exc = shfl_up(inc, RF);
  if (pos == 0) exc = ident;
  if (pos == per - 1) sw[warp * RF + r] = inc;
  __syncthreads();
  V pre = ident;
  for (int w = 0; w < warp; ++w) pre = scan_comb(pre, sw[w * RF + r]);
  __syncthreads();
  return scan_comb(pre, exc);
}

template <typename T>
__device__ __forceinline__ void refresh_body(const RefreshArgs& A, int vb) {
  __shared__ M2 sm2[(RF * TF / 32) * RF];
  __shared__ A2 sa2[(RF * TF / 32) * RF];
  __shared__ double qend[2][RF];
  if (!refresh_due(A.sp, A.stamp)) return;
  // which level, parity block and group of RF rings this CTA takes
  int l = 0;
  while (l + 1 < A.nlev && vb >= A.lv[l + 1].ring0) ++l;
  const RefreshLevel& L = A.lv[l];
  const Shape sh = L.sh;
  int g = vb - L.ring0;
  const int godd = (sh.no + RF - 1) / RF;
  const int parity = g < godd ? 1 : 0;
  if (!parity) g -= godd;
  const int nlines = parity ? sh.no : sh.ne;
  const int r = threadIdx.x, cidx = threadIdx.y;
  const int k = g * RF + r;
  const bool valid = k < nlines;
  const int i = parity ? 2 * (valid ? k : 0) + 1 : 2 * (valid ? k : 0) + 2;
  const int local = parity ? k : sh.no + k;  // ring slot: odd rings, then even rings
  const int n = sh.n;
  const size_t ld = parity ? sh.ldo : sh.lde;
  const size_t q0 = sh.at(i, 0);
  const double alpha = A.sp->alpha, beta = A.sp->beta;
  T* diag = static_cast<T*>(L.diag);
  T* fl = static_cast<T*>(L.fl);
  T* fui = static_cast<T*>(L.fui);
  T* fcu = static_cast<T*>(L.fcu);
  T* fq = static_cast<T*>(L.fq);
  double* wy = L.ws;
  double* wu = L.ws + sh.nv;
  const int P = (n + TF - 1) / TF;
  auto bdiag = [&](size_t q) {
    return alpha * L.vol[q] + beta * (L.rs[q] - L.w[q] - L.e[q] - L.s[q] - L.nn[q]);
  };
  // Diagonal the ring is factored with.  FP64 factors: the ring's own.  FP32 factors (the
  // mixed path's smoother): where the upwinded drift diverges, a ring's diagonal can fall
  // to or below the sum of its two angular couplings (no longer diagonally dominant), and
  // an FP32 solve of that ring -- then the whole V-cycle -- goes wild; such a diagonal is
  // raised to (1 + 1e-7) times the couplings.  The operator itself is untouched: only the
  // smoother's rings are shifted, and diagonally dominant rings keep their own diagonal.
  auto bfac = [&](size_t q) {
    const double bd = bdiag(q);
    if (sizeof(T) == 8) return bd;
    const double off = beta * (fabs(L.s[q]) + fabs(L.nn[q]));
    return bd > off ? bd : (1.0 + 1e-7) * off;
  };
  // corner terms of the periodic system
  const double b0 = valid ? bfac(q0) : 1.0;
  const double gamma = -b0;
  const double a0 = valid ? beta * L.s[q0] : 0.0;
  const double cn1 = valid ? beta * L.nn[q0 + (size_t)(n - 1) * ld] : 0.0;
  const double vf = a0 / gamma;
  auto bmod = [&](int j, double bd) {
    double bb = bd;
    if (j == 0) bb -= gamma;
    if (j == n - 1) bb -= cn1 * vf;
    return bb;
  };
  auto cc = [&](int j) {  // c_j (0 past the end of the non-periodic part)
    return (j >= 0 && j < n - 1) ? beta * L.nn[q0 + (size_t)j * ld] : 0.0;
  };

  // ---- pivots: compose this chunk's matrices, scan, replay
  const int j0 = valid ? min(n, cidx * P) : n, j1 = valid ? min(n, j0 + P) : n;
  M2 m{1.0, 0.0, 0.0, 1.0};
  {
    double cprev = cc(j0 - 1);
    for (int j = j0; j < j1; ++j) {
      const size_t q = q0 + (size_t)j * ld;
      const double a = (j > 0) ? beta * L.s[q] : 0.0;
      const M2 mj{bmod(j, bfac(q)), -a * cprev, 1.0, 0.0};
      m = comb(m, mj);
      if (((j - j0) & 3) == 3) m = renorm(m);
      cprev = cc(j);
    }
    m = renorm(m);
  }
  const M2 pm = chunk_excl_scan(m, M2{1.0, 0.0, 0.0, 1.0}, sm2);
  // incoming state (u_{j0-1}, 1) ~ pm (1, 0)^T; chunk 0 starts from (1, 0): ui = 0
  double uiprev = (pm.a != 0.0) ? pm.c / pm.a : 0.0;
  double cprev = cc(j0 - 1);
  A2 fy{1.0, 0.0};
  for (int j = j0; j < j1; ++j) {
    const size_t q = q0 + (size_t)j * ld;
    const double bd = bdiag(q);
    diag[q] = (T)bd;
    if (L.diag64) L.diag64[q] = bd;
    if (L.dinv) L.dinv[q] = 1.0 / bd;
    if (L.rsum) static_cast<T*>(L.rsum)[q] = (T)(alpha * L.vol[q] + beta * L.rs[q]);
    const double a = (j > 0) ? beta * L.s[q] : 0.0;
    const double c = cc(j);
    const double lj = a * uiprev;
    const double ui = 1.0 / (bmod(j, bfac(q)) - lj * cprev);
    fl[q] = (T)lj;
    fui[q] = (T)ui;
    fcu[q] = (T)(c * ui);
    wu[q] = ui;
    // y_j = ur_j - l_j y_{j-1}, ur = (gamma, 0, .., 0, c_{n-1})
    const double ur = (j == 0) ? gamma : ((j == n - 1) ? cn1 : 0.0);
    fy = comb(fy, A2{-lj, ur});
    uiprev = ui;
    cprev = c;
  }
  // ---- y = L^{-1} u
  const A2 py = chunk_excl_scan(fy, A2{1.0, 0.0}, sa2);
  {
    double y = py.b;  // y_{j0-1} (y_{-1} = 0)
    for (int j = j0; j < j1; ++j) {
      const size_t q = q0 + (size_t)j * ld;
      const double lj = (j > 0) ? beta * L.s[q] * wu[q - ld] : 0.0;
      const double ur = (j == 0) ? gamma : ((j == n - 1) ? cn1 : 0.0);
      y = fma(-lj, y, ur);
      wy[q] = y;
    }
  }
  __syncthreads();
  // ---- q = U^{-1} y, chunks taken in reverse order (thread c owns chunk TF - 1 - c)
  const int rc = TF - 1 - cidx;
  const int k0 = valid ? min(n, rc * P) : n, k1 = valid ? min(n, k0 + P) : n;
  A2 fq2{1.0, 0.0};
  for (int j = k1 - 1; j >= k0; --j) {
    const size_t q = q0 + (size_t)j * ld;
    const double ui = wu[q];
    fq2 = comb(fq2, A2{-cc(j) * ui, ui * wy[q]});
  }
  const A2 pq = chunk_excl_scan(fq2, A2{1.0, 0.0}, sa2);
  {
    double qn = pq.b;  // q_{k1} (q_n = 0)
    for (int j = k1 - 1; j >= k0; --j) {
      const size_t q = q0 + (size_t)j * ld;
      const double ui = wu[q];
      qn = fma(-cc(j) * ui, qn, ui * wy[q]);
      fq[q] = (T)qn;
      if (j == 0) qend[0][r] = qn;
      if (j == n - 1) qend[1][r] = qn;
    }
  }
  __syncthreads();
  if (valid && cidx == 0) {
    T* fring = static_cast<T*>(L.fring);
    fring[2 * local] = (T)vf;
    fring[2 * local + 1] = (T)(1.0 / (1.0 + qend[0][r] + vf * qend[1][r]));
    if (i == 1) {
      // origin scalars of this level: diag0 = alpha vol0 + beta (rs0 - sum_j o_j)
      const double d0 = alpha * L.sc[3] + beta * (L.sc[4] - L.sc[2]);
      L.sc[0] = d0;
      L.sc[5] = alpha * L.sc[3] + beta * L.sc[4];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RF * TF) k_refresh(RefreshArgs A) {
  refresh_body<T>(A, blockIdx.x);
}

// Copies an instance's argument struct into shared memory (once per CTA): the batched
// launches of the large-argument kernels read their fields from there.
template <typename A>
__device__ __forceinline__ void stage_args(A& dst, const A& src) {
  static_assert(sizeof(A) % sizeof(int) == 0, "argument structs are whole words");
  const int nt = blockDim.x * blockDim.y;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  int* d = reinterpret_cast<int*>(&dst);
  const int* s = reinterpret_cast<const int*>(&src);
  for (int k = tid; k < (int)(sizeof(A) / sizeof(int)); k += nt) d[k] = s[k];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(RF * TF) k_refresh_b(const RefreshArgs* AA, const BSlot* S,
                                                     int nslots, const int* mask) {
  __shared__ RefreshArgs sA;
  POLAR_BATCH_LOOP({
    stage_args(sA, AA[s]);
    refresh_body<T>(sA, vb);
    __syncthreads();  // sA is restaged for the next item
  })
}

template <typename T>
static int launch_schur(const LevelView<T>& L, const StepParams* sp, const double* stamp,
                        cudaStream_t st);

// after a stamped refresh: record the (alpha, beta) the factors now hold
__global__ void k_stamp(const StepParams* sp, double* stamp) {
  stamp[0] = sp->alpha;
  stamp[1] = sp->beta;
}
// batched: one thread per instance (w.inst), stamp array given per instance
__global__ void k_stamp_b(const BSlot* S, int nslots, const int* mask, double* const* stamps,
                          const StepParams* const* sps) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
    if (!mask[S[s].inst]) continue;
    stamps[s][0] = sps[s]->alpha;
    stamps[s][1] = sps[s]->beta;
  }
}

template <typename T>
RefreshArgs make_refresh_args(const LevelView<double>* L64, LevelView<T>* LT, int nlev,
                              const StepParams* sp, double* ws, double* stamp, int* nblocks) {
  RefreshArgs A{};
  A.nlev = nlev;
  A.sp = sp;
  A.stamp = stamp;
  int rings = 0;
  size_t wofs = 0;
  for (int l = 0; l < nlev; ++l) {
    RefreshLevel& r = A.lv[l];
    const LevelView<double>& d = L64[l];
    r.sh = d.sh;
    r.vol = d.vol;
    r.rs = d.rs;
    r.w = d.w;
    r.e = d.e;
    r.s = d.s;
    r.nn = d.nn;
    r.o = d.o;
    r.sc = LT[l].sc;
    r.diag = LT[l].diag;
    r.diag64 = (sizeof(T) == 4 && l == 0) ? L64[0].diag : nullptr;
    r.dinv = (l == 0) ? L64[0].dinv : nullptr;
    r.rsum = (sizeof(T) == 4 && l == 0) ? (void*)LT[0].rsum : nullptr;
    r.fl = LT[l].fl;
    r.fui = LT[l].fui;
    r.fcu = LT[l].fcu;
    r.fq = LT[l].fq;
    r.fring = LT[l].fring;
    r.fz = LT[l].fz;
    r.ws = ws + wofs;
    wofs += 2 * d.sh.nv;
    r.ring0 = rings;  // first CTA of this level (groups of RF rings, odd block first)
    rings += (d.sh.no + RF - 1) / RF + (d.sh.ne + RF - 1) / RF;
  }
  *nblocks = rings;
  return A;
}

template <typename T>
int launch_refresh(const LevelView<double>* L64, LevelView<T>* LT, int nlev,
                   const StepParams* sp, double* ws, cudaStream_t st, double* stamp) {
  int rings = 0;
  const RefreshArgs A = make_refresh_args<T>(L64, LT, nlev, sp, ws, stamp, &rings);
  k_refresh<T><<<rings, dim3(RF, TF), 0, st>>>(A);
  int k = 1 + launch_schur<T>(LT[nlev - 1], sp, stamp, st);
  if (stamp) {
    k_stamp<<<1, 1, 0, st>>>(sp, stamp);
    ++k;
  }
  return k;
}

// Slot of the level scalars holding the coarsest level's Schur denominator: one per
// precision, since a mixed context forms FP32 and FP64 factors of the same levels.
template <typename T>
constexpr int kSchurSlot = sizeof(T) == 8 ? 6 : 1;

// ---------------------------------------------------------------------------------
// ring solves


// A radial position of a level, addressed along the angle: entry j at base + j * ld.
struct Line {
  size_t base;
  int ld;
  __device__ __forceinline__ size_t at(int j) const { return base + (size_t)j * ld; }
};

__device__ __forceinline__ Line line_of(const Shape& sh, int i) {
  return Line{sh.at(i, 0), (i & 1) ? sh.ldo : sh.lde};
}

// Coarse ring I of the next level: the origin for I = 0 (stride 0), a zero ring beyond
// the last one (weight 0, reads the origin slot harmlessly).
template <typename T>
struct CoarseRef {
  Line ln;
  T mul;       // 1, or 0 for the zero ring
  __device__ __forceinline__ T get(const T* X, int j) const {
    // a select, not a product: no FP64 instruction (the ring kernels are bound by them)
    return mul != T(0) ? X[ln.at(j)] : T(0);
  }
};
template <typename T>
__device__ __forceinline__ CoarseRef<T> coarse_ref(const Shape& C, int I) {
  if (I == 0) return CoarseRef<T>{Line{0, 0}, T(1)};
  if (I > C.m) return CoarseRef<T>{Line{0, 0}, T(0)};
  return CoarseRef<T>{line_of(C, I), T(1)};
}

// Odd ring q of the level with its coarse correction x_q + ia X_k + ib X_{k+1}
// (q = 2k + 1: its coarse neighbours are coarse rings k and k + 1).
template <typename T>
struct OddRef {
  Line ln;
  CoarseRef<T> lo, hi;
};
template <typename T>
__device__ __forceinline__ OddRef<T> odd_ref(const Shape& F, const Shape& C, int q) {
  const int k = q >> 1;
  return OddRef<T>{line_of(F, q), coarse_ref<T>(C, k), coarse_ref<T>(C, k + 1)};
}
template <typename T>
__device__ __forceinline__ T corrected(const OddRef<T>& o, const T* x, const T* ia, const T* ib,
                                       const T* X, int j) {
  const size_t p = o.ln.at(j);
  const T xl = o.lo.get(X, j);
  const T xh = o.hi.get(X, j);
  return fma(ia[p], xl, fma(ib[p], xh, x[p]));
}

// right-hand side of the angular line of ring i:
//   d_j = b_ij - beta (w_ij x_{i-1,j} + e_ij x_{i+1,j})
// with the neighbours as the sweep sees them (zero in the first half-sweep, corrected
// odd rings in the first post-smoothing half-sweep); x_{0,j} is the origin and
// x_{m+1,j} = 0.
template <typename T>
struct RingRhs {
  const T* b;
  const T* w;
  const T* e;
  const T* x;
  const T* ia;
  const T* ib;
  const T* X;
  Line own, wl, el;        // own line, west / east neighbour lines (wl.ld = 0: origin)
  OddRef<T> wo, eo;        // corrected odd neighbours (kind 2)
  T beta, emul;            // emul = 0 on the last ring (Dirichlet neighbour)
  int kind;                // 0: b only, 1: plain neighbours, 2: corrected odd neighbours
  __device__ __forceinline__ T operator()(int j) const {
    const size_t p = own.at(j);
    const T bv = b[p];
    if (kind == 0) return bv;
    T xw, xe;
    const bool east = emul != T(0);  // the last ring's east neighbour is the zero ring
    if (kind == 1) {
      xw = x[wl.at(j)];
      xe = east ? x[el.at(j)] : T(0);
    } else {
      xw = corrected(wo, x, ia, ib, X, j);
      xe = east ? corrected(eo, x, ia, ib, X, j) : T(0);
    }
    return bv - beta * fma(w[p], xw, e[p] * xe);
  }
};

template <typename T>
__device__ __forceinline__ RingRhs<T> make_ring_rhs(const RingArgs<T>& a, T beta, int i) {
  const Shape& sh = a.L.sh;
  RingRhs<T> r{};
  r.b = a.b;
  r.w = a.L.w;
  r.e = a.L.e;
  r.x = a.x;
  r.ia = a.L.ia;
  r.ib = a.L.ib;
  r.X = a.X;
  r.beta = beta;
  r.own = line_of(sh, i);
  const bool last = i >= sh.m;
  r.emul = last ? T(0) : T(1);
  r.wl = (i == 1) ? Line{0, 0} : line_of(sh, i - 1);
  r.el = last ? Line{0, 0} : line_of(sh, i + 1);
  if (a.mode == RING_PRE && a.parity == 1) {
    r.kind = 0;
  } else if (a.mode == RING_POST && a.parity == 0) {
    r.kind = 2;
    r.wo = odd_ref<T>(sh, a.C.sh, i - 1);
    r.eo = last ? odd_ref<T>(sh, a.C.sh, i - 1) : odd_ref<T>(sh, a.C.sh, i + 1);
  } else {
    r.kind = 1;
  }
  return r;
}

// Inclusive scan of affine maps x -> A x + B over the TW chunks of each line of the CTA
// (thread (r, c), linear index r + RW c, so a warp holds 32 / RW consecutive chunks of
// each of its RW lines).  Warp shuffles combine the chunks of a warp; the warp totals go
// through shared memory once.  Returns, for this thread, the composed map of the chunks
// before it (exclusive prefix) in (Ae, Be); `rev` scans from the last chunk down.
template <typename T>
__device__ __forceinline__ void chunk_scan(T A, T B, bool rev, T* sWA, T* sWB, T& Ae, T& Be,
                                           T& At, T& Bt) {
  const int RW = blockDim.x;
  const int tid = threadIdx.x + RW * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (RW * blockDim.y) >> 5;
  const int per = 32 / RW;              // chunks of one line inside a warp
  const int pos = lane / RW;            // position of this chunk inside the warp
  const int r = threadIdx.x;
  // warp-level inclusive scan (forward: from low positions, reverse: from high)
  T a = A, b = B;
  for (int off = 1; off < per; off <<= 1) {
    const T ao = rev ? __shfl_down_sync(0xffffffffu, a, off * RW) : __shfl_up_sync(0xffffffffu, a, off * RW);
    const T bo = rev ? __shfl_down_sync(0xffffffffu, b, off * RW) : __shfl_up_sync(0xffffffffu, b, off * RW);
    const bool has = rev ? (pos + off < per) : (pos >= off);
    if (has) {
      b = fma(a, bo, b);
      a = a * ao;
    }
  }
  // warp-local exclusive map: the inclusive map of the neighbouring position
  T ea = rev ? __shfl_down_sync(0xffffffffu, a, RW) : __shfl_up_sync(0xffffffffu, a, RW);
  T eb = rev ? __shfl_down_sync(0xffffffffu, b, RW) : __shfl_up_sync(0xffffffffu, b, RW);
  const bool first = rev ? (pos == per - 1) : (pos == 0);
  if (first) {
    ea = T(1);
    eb = T(0);
  }
  // warp totals (held by the last position of the scan direction)
  const bool last = rev ? (pos == 0) : (pos == per - 1);
  if (last) {
    sWA[warp * RW + r] = a;
    sWB[warp * RW + r] = b;
  }
  __syncthreads();
  // prefix of the warps before this one in the scan direction
  T pa = T(1), pb = T(0);
  if (!rev) {
    for (int w = 0; w < warp; ++w) {
      const T wa = sWA[w * RW + r], wb = sWB[w * RW + r];
      pb = fma(wa, pb, wb);
      pa = wa * pa;
    }
  } else {
    for (int w = nwarps - 1; w > warp; --w) {
      const T wa = sWA[w * RW + r], wb = sWB[w * RW + r];
      pb = fma(wa, pb, wb);
      pa = wa * pa;
    }
  }
  // exclusive = warp-local exclusive o (prefix of earlier warps)
  Ae = ea * pa;
  Be = fma(ea, pb, eb);
  // total of the CTA for this line
  At = T(1);
  Bt = T(0);
  for (int w = 0; w < nwarps; ++w) {
    const int ww = rev ? nwarps - 1 - w : w;
    const T wa = sWA[ww * RW + r], wb = sWB[ww * RW + r];
    Bt = fma(wa, Bt, wb);
    At = wa * At;
  }
  __syncthreads();  // the buffers are reused by the next scan
}

// Solves the periodic lines of one CTA (RW lines x TW chunks of P) or one cluster.
// Rhs(j) gives d_j of this thread's line; Out(j, x) stores the solution.  The chunk's
// right-hand side and LU factors are loaded once into registers (all loads in flight
// together); the Sherman-Morrison vector is read at the end.
// STAGED: the operands arrive in three groups -- right-hand side and l before the forward
// scan, 1/u and c/u after it, q at the end -- so that fewer registers are live and two
// CTAs share an SM (the kernel variant launched with two CTAs per SM), letting one CTA's
// scans overlap another's loads.  Unstaged: every operand is loaded up front.
template <typename T, int P, bool STAGED = false, typename Rhs, typename Fac, typename Out>
__device__ void solve_lines(int n, bool valid, Rhs rhs, Fac fac, T vf, T inv, Out out) {
  extern __shared__ unsigned char smraw[];
  const int RW = blockDim.x, TW = blockDim.y;
  const int r = threadIdx.x, c = threadIdx.y;
  const int nwarps = (RW * TW) >> 5;
  T* sWA = reinterpret_cast<T*>(smraw);
  T* sWB = sWA + nwarps * RW;
  T* segA = sWB + nwarps * RW;  // this CTA's segment map, per line
  T* segB = segA + RW;
  T* ends = segB + RW;          // [0, RW): x_0 of the line, [RW, 2 RW): x_{n-1}
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int gc = crank * TW + c;
  const int j0 = gc * P;
  // the Sherman-Morrison vector is loaded with the rest when registers allow (short
  // chunks), so that the final correction waits on no memory access
  constexpr bool kPrefetchQ = !STAGED && (P * sizeof(T) <= 32);
  // 1/u and c/u arrive after the forward scan in the staged variant and for long chunks
  // (P values of more than 64 bytes), whose four up-front operand arrays would not fit in
  // the 128 registers a 512-thread CTA allows; fu then shares the registers of fl (dead
  // after the forward replay)
  constexpr bool kLate = STAGED || (P * sizeof(T) > 64);
  T v[P], fl[P], fu_[kLate ? 1 : P], fc[P], fqv[kPrefetchQ ? P : 1];
  T* fu = kLate ? fl : fu_;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int j = j0 + p;
    const bool in = valid && j < n;
    v[p] = in ? rhs(j) : T(0);
    fl[p] = in ? fac.l(j) : T(0);
    if constexpr (!kLate) {
      fu_[p] = in ? fac.ui(j) : T(0);
      fc[p] = in ? fac.cu(j) : T(0);
    }
    if constexpr (kPrefetchQ) fqv[p] = in ? fac.q(j) : T(0);
  }
  // forward substitution y_j = d_j - l_j y_{j-1}  (padding: l = 0, d = 0 -> identity-like)
  T A = T(1), B = T(0);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    if (valid && j0 + p < n) {
      B = fma(-fl[p], B, v[p]);
      A = -fl[p] * A;
    }
  }
  T Ae, Be, At, Bt;
  chunk_scan(A, B, false, sWA, sWB, Ae, Be, At, Bt);
  T yin = T(0);
  if (CS > 1) {
    if (c == 0) {
      segA[r] = At;
      segB[r] = Bt;
    }
    cl.sync();
    for (int q = 0; q < crank; ++q) {
      const T* ra = cl.map_shared_rank(segA, q);
      const T* rb = cl.map_shared_rank(segB, q);
      yin = fma(ra[r], yin, rb[r]);
    }
    cl.sync();
  }
  T prev = fma(Ae, yin, Be);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    if (valid && j0 + p < n) {
      prev = fma(-fl[p], prev, v[p]);
      v[p] = prev;
    }
  }
  if constexpr (kLate) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int j = j0 + p;
      const bool in = valid && j < n;
      fu[p] = in ? fac.ui(j) : T(0);
      fc[p] = in ? fac.cu(j) : T(0);
    }
  }
  // backward substitution x_j = ui_j y_j - cu_j x_{j+1}: ui_j y_j formed once, in v
#pragma unroll
  for (int p = 0; p < P; ++p) v[p] *= fu[p];
  A = T(1);
  B = T(0);
#pragma unroll
  for (int p = P - 1; p >= 0; --p) {
    if (valid && j0 + p < n) {
      B = fma(-fc[p], B, v[p]);
      A = -fc[p] * A;
    }
  }
  chunk_scan(A, B, true, sWA, sWB, Ae, Be, At, Bt);
  T xin = T(0);
  if (CS > 1) {
    if (c == 0) {
      segA[r] = At;
      segB[r] = Bt;
    }
    cl.sync();
    for (int q = CS - 1; q > crank; --q) {
      const T* ra = cl.map_shared_rank(segA, q);
      const T* rb = cl.map_shared_rank(segB, q);
      xin = fma(ra[r], xin, rb[r]);
    }
  }
  T next = fma(Ae, xin, Be);
#pragma unroll
  for (int p = P - 1; p >= 0; --p) {
    if (valid && j0 + p < n) {
      next = fma(-fc[p], next, v[p]);
      v[p] = next;
    }
  }
  // Sherman-Morrison: x -= q (x_0 + vf x_{n-1}) / (1 + v.q)
  if (j0 == 0) ends[r] = v[0];
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (j0 + p == n - 1) ends[RW + r] = v[p];
  T x0v, xl;
  if (CS > 1) {
    cl.sync();
    const int owner = ((n - 1) / P) / TW;
    x0v = cl.map_shared_rank(ends, 0)[r];
    xl = cl.map_shared_rank(ends, owner)[RW + r];
  } else {
    __syncthreads();
    x0v = ends[r];
    xl = ends[RW + r];
  }
  const T sigma = fma(vf, xl, x0v) * inv;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int j = j0 + p;
    if (valid && j < n) {
      T qj;
      if constexpr (kPrefetchQ) {
        qj = fqv[p];
      } else {
        qj = fac.q(j);
      }
      out(j, fma(-sigma, qj, v[p]));
    }
  }
  if (CS > 1) cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T>
struct RingFac {
  const T* fl;
  const T* fui;
  const T* fcu;
  const T* fq;
  Line ln;
  __device__ __forceinline__ T l(int j) const { return fl[ln.at(j)]; }
  __device__ __forceinline__ T ui(int j) const { return fui[ln.at(j)]; }
  __device__ __forceinline__ T cu(int j) const { return fcu[ln.at(j)]; }
  __device__ __forceinline__ T q(int j) const { return fq[ln.at(j)]; }
};

// Origin relaxation: x_0 = (b_0 - beta sum_j o_j x_{1,j}) / diag0, x_1 from x (PRE) or
// after the coarse correction (POST).  Run by one CTA.
template <typename T>
__device__ void relax_origin(const RingArgs<T>& a, T beta) {
  __shared__ double red[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nt = blockDim.x * blockDim.y;
  double s = 0.0;
  const OddRef<T> r1 = odd_ref<T>(a.L.sh, a.C.sh, 1);
  for (int j = tid; j < a.L.sh.n; j += nt) {
    const T x1 = (a.mode == RING_PRE) ? a.x[r1.ln.at(j)] : corrected(r1, a.x, a.L.ia, a.L.ib, a.X, j);
    s = fma((double)a.L.o[j], (double)x1, s);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) tot += red[w];
    a.x[0] = (T)(((double)a.b[0] - (double)beta * tot) / a.L.sc[0]);
  }
}

// One zebra half-sweep over the lines [kbase, kbase + RW) of the parity (all threads of
// the CTA call it together).
template <typename T, int P, bool STAGED>
__device__ void ring_body(const RingArgs<T>& a, T beta, int kbase) {
  const Shape& sh = a.L.sh;
  const int nl = a.parity ? sh.no : sh.ne;
  const int k = kbase + threadIdx.x;
  const bool valid = k < nl;
  const int i = a.parity ? 2 * k + 1 : 2 * k + 2;
  const int ringslot = a.parity ? k : sh.no + k;
  T vf = T(0), inv = T(0);
  if (valid) {
    vf = a.L.fring[2 * ringslot];
    inv = a.L.fring[2 * ringslot + 1];
  }
  const Line own = line_of(sh, valid ? i : 1);
  RingFac<T> fac{a.L.fl, a.L.fui, a.L.fcu, a.L.fq, own};
  const RingRhs<T> rhs = make_ring_rhs(a, beta, valid ? i : 1);
  T* x = a.x;
  solve_lines<T, P, STAGED>(sh.n, valid, rhs, fac, vf, inv,
                            [&](int j, T v) { x[own.at(j)] = v; });
}

template <typename T, int P>
__global__ void __launch_bounds__(512) k_ring(RingArgs<T> a) {
  if (a.done && *a.done) return;
  const T beta = (T)a.par[1];
  ring_body<T, P, false>(a, beta, blockIdx.x * blockDim.x);
  // the origin is relaxed with the even rings; ring 1 (odd) is not written here
  if (a.parity == 0 && blockIdx.x == 0 && blockIdx.y == 0) relax_origin(a, beta);
}

// the same half-sweep with staged operand loads, two 512-thread CTAs per SM
template <typename T, int P>
__global__ void __launch_bounds__(512, 2) k_ring_staged(RingArgs<T> a) {
  if (a.done && *a.done) return;
  const T beta = (T)a.par[1];
  ring_body<T, P, true>(a, beta, blockIdx.x * blockDim.x);
  if (a.parity == 0 && blockIdx.x == 0 && blockIdx.y == 0) relax_origin(a, beta);
}

// Batched half-sweeps: CTA column blockIdx.x works on the RW lines from w.aux of instance
// w.inst (w.vb: its line group, 0 relaxes the origin with the even rings).  The gate and
// the instance's `done` flag are read before the cluster's first barrier; every CTA of a
// cluster reads the same work item, so a cluster returns as a whole.
template <typename T, int P, bool STAGED>
__device__ __forceinline__ void ring_batched(const RingArgs<T>* A, const BSlot* S, int nslots,
                                             const int* mask) {
  // every CTA of a cluster (one column, same blockIdx.x) takes the same work items
  __shared__ RingArgs<T> sa;
  POLAR_BATCH_LOOP({
    stage_args(sa, A[s]);
    if (!(sa.done && *sa.done)) {
      const T beta = (T)sa.par[1];
      ring_body<T, P, STAGED>(sa, beta, vb * (int)blockDim.x);
      if (sa.parity == 0 && vb == 0 && blockIdx.y == 0) relax_origin(sa, beta);
    }
    __syncthreads();  // sa is restaged for the next item
  })
}
template <typename T, int P>
__global__ void __launch_bounds__(512) k_ring_b(const RingArgs<T>* A, const BSlot* S, int nslots,
                                                const int* mask) {
  ring_batched<T, P, false>(A, S, nslots, mask);
}
template <typename T, int P>
__global__ void __launch_bounds__(512, 2) k_ring_staged_b(const RingArgs<T>* A, const BSlot* S,
                                                         int nslots, const int* mask) {
  ring_batched<T, P, true>(A, S, nslots, mask);
}

// residual of the odd rings after the pre-smoothing sweep, restricted to the coarser
// level: B_I = ib_{2I-1} r_{2I-1} + ia_{2I+1} r_{2I+1} and B_0 = sum_j ia_{1,j} r_{1,j}
// (the even rings and the origin have zero residual after their relaxation; an odd
// ring's residual is what its even neighbours changed: r_q = -beta (w x_{q-1} + e x_{q+1})).

template <typename T>
__device__ __forceinline__ T odd_resid(const LevelView<T>& L, const T* x, T beta, int q, int j) {
  const size_t p = L.sh.at(q, j);
  const T xw = (q == 1) ? x[0] : x[L.sh.at(q - 1, j)];
  const T xe = (q < L.sh.m) ? x[L.sh.at(q + 1, j)] : T(0);
  return -beta * fma(L.w[p], xw, L.e[p] * xe);
}

// threads [tid0, tid0 + nthreads) of the grid-stride loop; `origin` also forms B_0
// (one CTA, every thread of it)
template <typename T>
__device__ void restrict_body(const RestrictArgs<T>& a, T beta, size_t tid0, size_t nthreads,
                              bool origin) {
  const Shape& sh = a.L.sh;
  const int mc = a.C.sh.m, n = sh.n;
  const size_t total = (size_t)mc * n;
  for (size_t t = tid0; t < total; t += nthreads) {
    const int j = (int)(t / mc);
    const int I = (int)(t - (size_t)j * mc) + 1;
    const int qlo = 2 * I - 1, qhi = 2 * I + 1;
    T v = a.L.ib[sh.at(qlo, j)] * odd_resid(a.L, a.x, beta, qlo, j);
    if (qhi <= sh.m) v = fma(a.L.ia[sh.at(qhi, j)], odd_resid(a.L, a.x, beta, qhi, j), v);
    a.B[a.C.sh.at(I, j)] = v;
  }
  if (origin) {
    __shared__ double red[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nt = blockDim.x * blockDim.y;
    double s = 0.0;
    for (int j = tid; j < n; j += nt)
      s = fma((double)a.L.ia[sh.at(1, j)], (double)odd_resid(a.L, a.x, beta, 1, j), s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) tot += red[w];
      a.B[0] = (T)tot;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict(RestrictArgs<T> a) {
  if (a.done && *a.done) return;
  const T beta = (T)a.par[1];
  restrict_body(a, beta, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                (size_t)gridDim.x * blockDim.x, blockIdx.x == 0);
}
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_b(const RestrictArgs<T>* A, const BSlot* S,
                                                    int nslots, const int* mask) {
  POLAR_BATCH_LOOP({
    const RestrictArgs<T> a = A[s];
    if (!(a.done && *a.done)) {
      const T beta = (T)a.par[1];
      restrict_body(a, beta, vb * (size_t)blockDim.x + threadIdx.x, (size_t)vg * blockDim.x,
                    vb == 0);
    }
    __syncthreads();  // the origin part's shared reduction buffer is reused
  })
}

// coarsest level (origin + ring 1): y = T_1^{-1} b_1, x_0 = (b_0 - beta o.y) / denom,
// x_1 = y - z x_0 with z = T_1^{-1} (beta w_1) from the refresh.  One CTA (any RW: only
// line 0 is solved).
template <typename T, int P>
__device__ void coarsest_body(const LevelView<T>& L, const T* b, T* x, T beta) {
  const Shape& sh = L.sh;
  const Line own = line_of(sh, 1);
  RingFac<T> fac{L.fl, L.fui, L.fcu, L.fq, own};
  solve_lines<T, P>(
      sh.n, threadIdx.x == 0, [&](int j) { return b[own.at(j)]; }, fac, L.fring[0], L.fring[1],
      [&](int j, T v) { x[own.at(j)] = v; });
  __syncthreads();
  __shared__ double red[32];
  __shared__ T x0s;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nt = blockDim.x * blockDim.y;
  double s = 0.0;
  for (int j = tid; j < sh.n; j += nt) s = fma((double)L.o[j], (double)x[own.at(j)], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) tot += red[w];
    const T x0 = (T)(((double)b[0] - (double)beta * tot) / L.sc[kSchurSlot<T>]);
    x[0] = x0;
    x0s = x0;
  }
  __syncthreads();
  const T x0 = x0s;
  for (int j = tid; j < sh.n; j += nt) {
    const size_t p = own.at(j);
    x[p] = fma(-L.fz[j], x0, x[p]);
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(512) k_coarsest(LevelView<T> L, const T* b, T* x, Params par,
                                                   const int* done) {
  if (done && *done) return;
  coarsest_body<T, P>(L, b, x, (T)par[1]);
}
// batched: one CTA per instance (w.inst), its coarsest level, right-hand side and solution
template <typename T, int P>
__global__ void __launch_bounds__(512) k_coarsest_b(const CoarsestArgs<T>* A, const BSlot* S,
                                                    int nslots, const int* mask) {
  __shared__ CoarsestArgs<T> sa;
  POLAR_BATCH_LOOP({
    stage_args(sa, A[s]);
    if (!(sa.done && *sa.done)) coarsest_body<T, P>(sa.L, sa.b, sa.x, (T)sa.par[1]);
    __syncthreads();
  })
}

// Schur data of the coarsest level (after k_refresh): z = T_1^{-1} (beta w_1) by a ring
// solve, and the origin row's denominator diag0 - beta sum_j o_j z_j.
template <typename T, int P>
__device__ __forceinline__ void schur_body(const LevelView<T>& L, const StepParams* sp,
                                           const double* stamp) {
  if (!refresh_due(sp, stamp)) return;
  const T beta = (T)sp->beta;
  const Shape& sh = L.sh;
  const Line own = line_of(sh, 1);
  RingFac<T> fac{L.fl, L.fui, L.fcu, L.fq, own};
  T* fz = L.fz;
  const T* w = L.w;
  solve_lines<T, P>(
      sh.n, threadIdx.x == 0, [&](int j) { return beta * w[own.at(j)]; }, fac, L.fring[0],
      L.fring[1], [&](int j, T v) { fz[j] = v; });
  __syncthreads();
  __shared__ double red[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nt = blockDim.x * blockDim.y;
  double s = 0.0;
  for (int j = tid; j < sh.n; j += nt) s = fma((double)L.o[j], (double)fz[j], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int k = 0; k < (nt + 31) / 32; ++k) tot += red[k];
    L.sc[kSchurSlot<T>] = L.sc[0] - sp->beta * tot;
  }
}
template <typename T, int P>
__global__ void __launch_bounds__(512) k_schur(LevelView<T> L, const StepParams* sp,
                                               const double* stamp) {
  schur_body<T, P>(L, sp, stamp);
}
template <typename T, int P>
__global__ void __launch_bounds__(512) k_schur_b(const CoarsestArgs<T>* A, const BSlot* S,
                                                 int nslots, const int* mask) {
  __shared__ CoarsestArgs<T> sa;
  POLAR_BATCH_LOOP({
    stage_args(sa, A[s]);
    schur_body<T, P>(sa.L, sa.sp, sa.stamp);
    __syncthreads();
  })
}

// ---------------------------------------------------------------------------------
// launch configuration of the ring solves

constexpr int kRingThreads = 512;
constexpr int kMaxCluster = 16;

// RW lines per CTA (a full 32-byte sector of each line per row of angles), TW chunks
// of P angles, at most kRingThreads threads.  A CTA covers 512 / RW * P angles; longer
// rings are split over a cluster of CS CTAs (up to 16: 16384 angles in FP64 with
// P = 16, in FP32 with P = 32).
template <typename T>
static RingShape ring_shape(int nlines, int n) {
  RingShape s{};
  s.RW = (sizeof(T) == 8) ? 4 : 8;
  while (s.RW > 1 && s.RW > nlines) s.RW >>= 1;
  const int maxTW = kRingThreads / s.RW;
  const int maxP = (sizeof(T) == 8) ? 16 : 32;
  s.P = 8;
  while (s.P < maxP && (n + s.P - 1) / s.P > maxTW) s.P <<= 1;
  const int chunks = (n + s.P - 1) / s.P;
  s.TW = 1;
  while (s.TW < chunks) s.TW <<= 1;
  if (s.TW > maxTW) s.TW = maxTW;
  while (s.RW * s.TW < 32) s.TW <<= 1;  // whole warps (the scans shuffle across lanes)
  s.CS = (n + s.TW * s.P - 1) / (s.TW * s.P);
  s.ST = 0;
  return s;
}

template <typename T>
static size_t ring_smem(const RingShape& s) {
  const size_t warps = ((size_t)s.RW * s.TW + 31) / 32;
  return sizeof(T) * (2 * warps * s.RW + 4 * (size_t)s.RW);
}

template <typename T, int P>
static int launch_ring_p(const RingArgs<T>& a, const RingShape& s, int nl, cudaStream_t st) {
  const int grid = (nl + s.RW - 1) / s.RW;
  void (*kern)(RingArgs<T>) = s.ST ? k_ring_staged<T, P> : k_ring<T, P>;
  if (s.CS == 1) {
    kern<<<grid, dim3(s.RW, s.TW), ring_smem<T>(s), st>>>(a);
    return 1;
  }
  // a ring spread over the CS CTAs of a cluster (grid.y), which exchange segment maps
  // and end values through distributed shared memory
  if (s.CS > kMaxCluster) return -1;
  static bool allowed = false;
  if (!allowed && s.CS > 8) {
    cudaFuncSetAttribute(k_ring<T, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_ring_staged<T, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    allowed = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, s.CS, 1);
  cfg.blockDim = dim3(s.RW, s.TW, 1);
  cfg.dynamicSmemBytes = ring_smem<T>(s);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = s.CS;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a) == cudaSuccess ? 1 : -1;
}

// Candidate tile shapes of the ring solve for the autotuner: RW lines per CTA, P angles
// per thread, CS CTAs per cluster (TW follows), within the register and cluster limits.
template <typename T>
void ring_candidates(int nlines, int n, std::vector<RingShape>& out) {
  out.clear();
  const int maxP = (sizeof(T) == 8) ? 16 : 32;
  for (int RW = 1; RW <= 8; RW <<= 1) {
    if (RW > 1 && RW / 2 >= nlines) break;
    for (int P = 4; P <= maxP; P <<= 1) {
      for (int CS = 1; CS <= kMaxCluster; CS <<= 1) {
        RingShape s{RW, 1, P, CS, 0};
        const int chunks = (n + P * CS - 1) / (P * CS);
        while (s.TW < chunks) s.TW <<= 1;
        while (s.RW * s.TW < 32) s.TW <<= 1;
        if (s.RW * s.TW > kRingThreads) continue;
        if ((CS - 1) * s.TW * P >= n) continue;  // every CTA of the cluster holds angles
        out.push_back(s);
        // staged loads where a full-size CTA would otherwise hold one CTA per SM and the
        // three live operand arrays fit the two-CTA register budget
        if (s.RW * s.TW == kRingThreads && P >= 8 && P * sizeof(T) <= 64) {
          s.ST = 1;
          out.push_back(s);
        }
      }
    }
  }
}

template <typename T>
RingShape ring_default(int nlines, int n) {
  return ring_shape<T>(nlines, n);
}

template <typename T>
int launch_ring(const LevelView<T>& L, const LevelView<T>& C, const T* b, T* x, const T* X,
                Params p, int parity, int mode, const int* done, cudaStream_t st,
                const RingShape* shape) {
  RingArgs<T> a{};
  a.L = L;
  a.C = C;
  a.b = b;
  a.x = x;
  a.X = X;
  a.par = p;
  a.done = done;
  a.parity = parity;
  a.mode = mode;
  const int nl = parity ? L.sh.no : L.sh.ne;
  if (nl == 0) return 0;
  const RingShape s = shape ? *shape : ring_shape<T>(nl, L.sh.n);
  switch (s.P) {
    case 4: return launch_ring_p<T, 4>(a, s, nl, st);
    case 8: return launch_ring_p<T, 8>(a, s, nl, st);
    case 16: return launch_ring_p<T, 16>(a, s, nl, st);
    default: return launch_ring_p<T, 32>(a, s, nl, st);
  }
}

template <typename T>
int launch_restrict(const LevelView<T>& L, const LevelView<T>& C, const T* x, T* B, Params p,
                    const int* done, cudaStream_t st) {
  RestrictArgs<T> r{L, C, x, B, p, done};
  const size_t work = (size_t)C.sh.m * L.sh.n;
  k_restrict<T><<<grid_for(work, 256), 256, 0, st>>>(r);
  return 1;
}

template <typename T>
int launch_coarsest(const LevelView<T>& L, const T* b, T* x, Params p, const int* done,
                    cudaStream_t st) {
  RingShape s{};
  s.RW = 1;
  s.P = 8;
  while (s.P < 32 && (L.sh.n + s.P - 1) / s.P > kRingThreads) s.P <<= 1;
  s.TW = 32;
  while (s.TW < (L.sh.n + s.P - 1) / s.P) s.TW <<= 1;
  const size_t smem = ring_smem<T>(s);
  switch (s.P) {
    case 8: k_coarsest<T, 8><<<1, dim3(1, s.TW), smem, st>>>(L, b, x, p, done); break;
    case 16: k_coarsest<T, 16><<<1, dim3(1, s.TW), smem, st>>>(L, b, x, p, done); break;
    default: k_coarsest<T, 32><<<1, dim3(1, s.TW), smem, st>>>(L, b, x, p, done); break;
  }
  return 1;
}

template <typename T>
static int launch_schur(const LevelView<T>& L, const StepParams* sp, const double* stamp,
                        cudaStream_t st) {
  RingShape s{};
  s.RW = 1;
  s.P = 8;
  while (s.P < 32 && (L.sh.n + s.P - 1) / s.P > kRingThreads) s.P <<= 1;
  s.TW = 32;
  while (s.TW < (L.sh.n + s.P - 1) / s.P) s.TW <<= 1;
  const size_t smem = ring_smem<T>(s);
  switch (s.P) {
    case 8: k_schur<T, 8><<<1, dim3(1, s.TW), smem, st>>>(L, sp, stamp); break;
    case 16: k_schur<T, 16><<<1, dim3(1, s.TW), smem, st>>>(L, sp, stamp); break;
    default: k_schur<T, 32><<<1, dim3(1, s.TW), smem, st>>>(L, sp, stamp); break;
  }
  return 1;
}


// ---------------------------------------------------------------------------------
// batched launchers

template <typename T>
int launch_refresh_b(const RefreshArgs* A, const BSlot* S, int nslots, const int* mask, int grid,
                     cudaStream_t st) {
  if (nslots <= 0) return 0;
  k_refresh_b<T><<<grid, dim3(RF, TF), 0, st>>>(A, S, nslots, mask);
  return 1;
}

template <typename T, int P>
static int launch_ring_bp(const RingShape& s, const RingArgs<T>* A, const BSlot* S, int nslots,
                          const int* mask, int grid, cudaStream_t st) {
  void (*kern)(const RingArgs<T>*, const BSlot*, int, const int*) =
      s.ST ? k_ring_staged_b<T, P> : k_ring_b<T, P>;
  if (s.CS == 1) {
    kern<<<grid, dim3(s.RW, s.TW), ring_smem<T>(s), st>>>(A, S, nslots, mask);
    return 1;
  }
  if (s.CS > kMaxCluster) return -1;
  static bool allowed = false;
  if (!allowed && s.CS > 8) {
    cudaFuncSetAttribute(k_ring_b<T, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_ring_staged_b<T, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    allowed = true;
  }
  // grid columns are clusters of CS CTAs along y, each column taking the same work items
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, s.CS, 1);
  cfg.blockDim = dim3(s.RW, s.TW, 1);
  cfg.dynamicSmemBytes = ring_smem<T>(s);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = s.CS;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, A, S, nslots, mask) == cudaSuccess ? 1 : -1;
}

template <typename T>
int launch_ring_b(const RingShape& s, const RingArgs<T>* A, const BSlot* S, int nslots,
                  const int* mask, int grid, cudaStream_t st) {
  if (nslots <= 0) return 0;
  switch (s.P) {
    case 4: return launch_ring_bp<T, 4>(s, A, S, nslots, mask, grid, st);
    case 8: return launch_ring_bp<T, 8>(s, A, S, nslots, mask, grid, st);
    case 16: return launch_ring_bp<T, 16>(s, A, S, nslots, mask, grid, st);
    default: return launch_ring_bp<T, 32>(s, A, S, nslots, mask, grid, st);
  }
}

template <typename T>
int launch_restrict_b(const RestrictArgs<T>* A, const BSlot* S, int nslots, const int* mask,
                      int grid, cudaStream_t st) {
  if (nslots <= 0) return 0;
  k_restrict_b<T><<<grid, 256, 0, st>>>(A, S, nslots, mask);
  return 1;
}

template <typename T>
void coarsest_shape(int n, int* P, int* TW) {
  int p = 8;
  while (p < 32 && (n + p - 1) / p > kRingThreads) p <<= 1;
  int tw = 32;
  while (tw < (n + p - 1) / p) tw <<= 1;
  *P = p;
  *TW = tw;
}

template <typename T>
int launch_coarsest_b(int P, int TW, int schur, const CoarsestArgs<T>* A, const BSlot* S,
                      int nslots, const int* mask, int grid, cudaStream_t st) {
  if (nslots <= 0) return 0;
  RingShape s{};
  s.RW = 1;
  s.TW = TW;
  s.P = P;
  const size_t smem = ring_smem<T>(s);
  const dim3 block(1, TW);
  switch (P) {
    case 8:
      if (schur) k_schur_b<T, 8><<<grid, block, smem, st>>>(A, S, nslots, mask);
      else k_coarsest_b<T, 8><<<grid, block, smem, st>>>(A, S, nslots, mask);
      break;
    case 16:
      if (schur) k_schur_b<T, 16><<<grid, block, smem, st>>>(A, S, nslots, mask);
      else k_coarsest_b<T, 16><<<grid, block, smem, st>>>(A, S, nslots, mask);
      break;
    default:
      if (schur) k_schur_b<T, 32><<<grid, block, smem, st>>>(A, S, nslots, mask);
      else k_coarsest_b<T, 32><<<grid, block, smem, st>>>(A, S, nslots, mask);
      break;
  }
  return 1;
}

int launch_stamp_b(const BSlot* S, int nslots, const int* mask, double* const* stamps,
                   const StepParams* const* sps, cudaStream_t st) {
  if (nslots <= 0) return 0;
  k_stamp_b<<<(nslots + 127) / 128, 128, 0, st>>>(S, nslots, mask, stamps, sps);
  return 1;
}

// The ring kernels use dynamic shared memory only for the scan buffers
// (2 RW TW + 4 RW words): at most 16.1 KB, below the default 48 KB limit.

#define POLAR_MG_INST(T)                                                                      \
  template int launch_refresh<T>(const LevelView<double>*, LevelView<T>*, int,                \
                                 const StepParams*, double*, cudaStream_t, double*);          \
  template int launch_ring<T>(const LevelView<T>&, const LevelView<T>&, const T*, T*,          \
                              const T*, Params, int, int, const int*, cudaStream_t,           \
                              const RingShape*);                                              \
  template void ring_candidates<T>(int, int, std::vector<RingShape>&);                        \
  template RingShape ring_default<T>(int, int);                                               \
  template int launch_restrict<T>(const LevelView<T>&, const LevelView<T>&, const T*, T*,      \
                                  Params, const int*, cudaStream_t);                          \
  template int launch_coarsest<T>(const LevelView<T>&, const T*, T*, Params, const int*,       \
                                  cudaStream_t);                                              \
  template RefreshArgs make_refresh_args<T>(const LevelView<double>*, LevelView<T>*, int,     \
                                            const StepParams*, double*, double*, int*);       \
  template int launch_refresh_b<T>(const RefreshArgs*, const BSlot*, int, const int*, int,    \
                                   cudaStream_t);                                             \
  template int launch_ring_b<T>(const RingShape&, const RingArgs<T>*, const BSlot*, int,       \
                                const int*, int, cudaStream_t);                               \
  template int launch_restrict_b<T>(const RestrictArgs<T>*, const BSlot*, int, const int*,     \
                                    int, cudaStream_t);                                       \
  template void coarsest_shape<T>(int, int*, int*);                                           \
  template int launch_coarsest_b<T>(int, int, int, const CoarsestArgs<T>*, const BSlot*, int,  \
                                    const int*, int, cudaStream_t);

POLAR_MG_INST(float)
POLAR_MG_INST(double)

}  // namespace polar
