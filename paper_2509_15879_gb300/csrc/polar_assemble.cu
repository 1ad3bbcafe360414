// Device assembly of the conservative operator (Section 3.2.1 ring rows, Section 3.2.2
// origin row, upwinded drift) and of its radial hierarchy, for coefficients that change
// between steps: the drift of the electron-hole pair follows the potential at every
// Gummel iteration.  The formulas, and the order in which each row's terms are summed,
// are those of the host assembly (polar_host.cpp); products and sums use unfused
// intrinsics so that no FMA contraction changes their rounding.
#include "polar_internal.h"

namespace polar {

namespace {

constexpr double kTwoPi = 6.283185307179586;

// mesh metrics of Sections 2.1 / 3.1 (the host's Metrics, one value at a time)
__device__ __forceinline__ double h_of(const double* r, int i) { return __dsub_rn(r[i], r[i - 1]); }
__device__ __forceinline__ double rh_of(const double* r, int i) {
  return __dmul_rn(0.5, __dadd_rn(r[i], r[i + 1]));
}
__device__ __forceinline__ double mu_of(const double* th, int n, int j) {  // j = 0..n
  if (j == 0 || j == n) return __dsub_rn(__dadd_rn(kTwoPi, th[0]), th[n - 1]);
  return __dsub_rn(th[j], th[j - 1]);
}
__device__ __forceinline__ double wcell(const double* th, int n, int j) {
  return __dmul_rn(0.5, __dadd_rn(mu_of(th, n, j), mu_of(th, n, j + 1)));
}
__device__ __forceinline__ double kcell(const double* r, int i) {
  return __dmul_rn(0.5, __dadd_rn(h_of(r, i), h_of(r, i + 1)));
}

// flux coefficients of a face: len (cond + v+) and len (cond + v-)
__device__ __forceinline__ double cin_of(double len, double cond, double v) {
  return __dmul_rn(len, __dadd_rn(cond, fmax(v, 0.0)));
}
__device__ __forceinline__ double cout_of(double len, double cond, double v) {
  return __dmul_rn(len, __dadd_rn(cond, fmax(-v, 0.0)));
}

struct AsmArgs {
  AsmIn in;
  Shape sh;
  const double* vol;  // level 0 control volumes (split layout, static)
  double *w, *e, *s, *nn, *rs, *o, *sc;
};

__device__ __forceinline__ double dr_at(const AsmIn& a, int j, int i) {
  return a.dr ? a.dr[(size_t)j * (a.m + 1) + i] : a.d_const;
}
__device__ __forceinline__ double dt_at(const AsmIn& a, int j, int i) {
  return a.dt ? a.dt[(size_t)j * a.m + (i - 1)] : a.d_const;
}
__device__ __forceinline__ double vr_at(const AsmIn& a, int j, int i) {
  return a.vr ? a.vr[(size_t)j * (a.m + 1) + i] : 0.0;
}
__device__ __forceinline__ double vt_at(const AsmIn& a, int j, int i) {
  return a.vt ? a.vt[(size_t)j * a.m + (i - 1)] : 0.0;
}
__device__ __forceinline__ double b_at(const AsmIn& a, size_t iface) {
  return a.b ? a.b[iface] : a.b_const;
}

// Ring rows: the couplings of node (i, j) from its four faces and its row sum, summed in
// the order the host's face loops add them (the south face first, except on angle 0,
// whose south face is the last one the host visits).
__global__ void k_assemble_rings(AsmArgs A) {
  const AsmIn& a = A.in;
  const int m = a.m, n = a.n;
  const size_t total = (size_t)m * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / m), i = (int)(t - (size_t)j * m) + 1;
    const int jm = (j + n - 1) % n;
    const double wj = wcell(a.th, n, j);
    // radial faces i - 1/2 (west) and i + 1/2 (east)
    const double len_w = __dmul_rn(wj, rh_of(a.r, i - 1));
    const double vw = vr_at(a, j, i - 1);
    const double cin_w = cin_of(len_w, dr_at(a, j, i - 1) / h_of(a.r, i), vw);
    const double len_e = __dmul_rn(wj, rh_of(a.r, i));
    const double ve = vr_at(a, j, i);
    const double cout_e = cout_of(len_e, dr_at(a, j, i) / h_of(a.r, i + 1), ve);
    // angular faces j + 1/2 (north) and j - 1/2 (south)
    const double lt = kcell(a.r, i);
    const double vn = vt_at(a, j, i);
    const double cout_n = cout_of(lt, dt_at(a, j, i) / __dmul_rn(a.r[i], mu_of(a.th, n, j + 1)), vn);
    const double vs = vt_at(a, jm, i);
    const double cin_s = cin_of(lt, dt_at(a, jm, i) / __dmul_rn(a.r[i], mu_of(a.th, n, jm + 1)), vs);
    const double fs = __dmul_rn(lt, vs), fw = __dmul_rn(len_w, vw), fe = __dmul_rn(len_e, ve),
                 fn = __dmul_rn(lt, vn);
    double rs;
    if (j > 0) {
      rs = __dadd_rn(__dadd_rn(__dsub_rn(__dsub_rn(0.0, fs), fw), fe), fn);
    } else {
      rs = __dsub_rn(__dadd_rn(__dadd_rn(__dsub_rn(0.0, fw), fe), fn), fs);
    }
    const size_t p = A.sh.at(i, j);
    rs = __dadd_rn(rs, __dmul_rn(A.vol[p], b_at(a, 1 + t)));
    A.w[p] = -cin_w;
    A.e[p] = -cout_e;
    A.nn[p] = -cout_n;
    A.s[p] = -cin_s;
    A.rs[p] = rs;
  }
}

// Origin row (one block): o_j = -cout of radial face 1/2 at angle j; rs0 and sum_j o_j
// summed in angle order by one thread.
__global__ void k_assemble_origin(AsmArgs A) {
  const AsmIn& a = A.in;
  const int n = a.n;
  const double h1 = h_of(a.r, 1), rh0 = rh_of(a.r, 0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double len = __dmul_rn(wcell(a.th, n, j), rh0);
    A.o[j] = -cout_of(len, dr_at(a, j, 0) / h1, vr_at(a, j, 0));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rs0 = 0.0, osum = 0.0;
    for (int j = 0; j < n; ++j) {
      const double len = __dmul_rn(wcell(a.th, n, j), rh0);
      rs0 = __dadd_rn(rs0, __dmul_rn(len, vr_at(a, j, 0)));
    }
    const double vol0 = A.sc[3];
    rs0 = __dadd_rn(rs0, __dmul_rn(vol0, b_at(a, 0)));
    for (int j = 0; j < n; ++j) osum = __dadd_rn(osum, A.o[j]);
    A.rs[0] = rs0;
    A.sc[2] = osum;
    A.sc[4] = rs0;
  }
}

struct CoarsenArgs {
  Shape f, c;
  double *fw, *fe, *fs, *fnn, *frs, *fvol, *fo, *fia, *fib, *fsc;
  double *cw, *ce, *cs, *cnn, *crs, *cvol, *co, *csc;
};

// interpolation weights of the odd fine rings from their own radial rows
__global__ void k_coarsen_weights(CoarsenArgs A) {
  const int n = A.f.n, no = A.f.no;
  const size_t total = (size_t)no * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / no), k = 2 * (int)(t - (size_t)j * no) + 1;
    const size_t q = A.f.at(k, j);
    const double den = __dadd_rn(A.fw[q], A.fe[q]);
    if (den != 0.0) {
      A.fia[q] = A.fw[q] / den;
      A.fib[q] = A.fe[q] / den;
    } else {
      A.fia[q] = A.fib[q] = 0.5;
    }
  }
}

// coarse ring I = fine ring 2I: Schur-complement radial couplings, restricted angular
// couplings, row sums and volumes; the coarse origin couplings
__global__ void k_coarsen_rings(CoarsenArgs A) {
  const int n = A.f.n, m = A.f.m, mc = A.c.m;
  const size_t total = (size_t)mc * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / mc), I = (int)(t - (size_t)j * mc) + 1;
    const int k = 2 * I;
    const size_t qk = A.f.at(k, j), qlo = A.f.at(k - 1, j), qc = A.c.at(I, j);
    const bool hi = k + 1 <= m;
    const size_t qhi = hi ? A.f.at(k + 1, j) : 0;
    A.cw[qc] = __dmul_rn(A.fw[qk], A.fia[qlo]);
    A.ce[qc] = hi ? __dmul_rn(A.fe[qk], A.fib[qhi]) : A.fe[qk];
    const double bl = A.fib[qlo], ah = hi ? A.fia[qhi] : 0.0;
    auto lump = [&](const double* a) {
      return __dadd_rn(__dadd_rn(a[qk], __dmul_rn(bl, a[qlo])), hi ? __dmul_rn(ah, a[qhi]) : 0.0);
    };
    A.cs[qc] = lump(A.fs);
    A.cnn[qc] = lump(A.fnn);
    A.crs[qc] = lump(A.frs);
    A.cvol[qc] = lump(A.fvol);
  }
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < (size_t)n;
       j += (size_t)gridDim.x * blockDim.x)
    A.co[j] = __dmul_rn(A.fo[j], A.fib[A.f.at(1, (int)j)]);
}

// coarse origin scalars, summed over the angles in order by one thread
__global__ void k_coarsen_origin(CoarsenArgs A) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = A.f.n;
  double vol0 = A.fsc[3], rs0 = A.fsc[4], osum = 0.0;
  for (int j = 0; j < n; ++j) {
    const size_t q1 = A.f.at(1, j);
    vol0 = __dadd_rn(vol0, __dmul_rn(A.fia[q1], A.fvol[q1]));
  }
  for (int j = 0; j < n; ++j) {
    const size_t q1 = A.f.at(1, j);
    rs0 = __dadd_rn(rs0, __dmul_rn(A.fia[q1], A.frs[q1]));
  }
  for (int j = 0; j < n; ++j) osum = __dadd_rn(osum, A.co[j]);
  A.cvol[0] = vol0;
  A.crs[0] = rs0;
  A.csc[2] = osum;
  A.csc[3] = vol0;
  A.csc[4] = rs0;
}

}  // namespace

int launch_assemble_level0(const AsmIn& in, const Shape& sh, const double* vol, double* w,
                           double* e, double* s, double* nn, double* rs, double* o, double* sc,
                           cudaStream_t st) {
  AsmArgs A{in, sh, vol, w, e, s, nn, rs, o, sc};
  k_assemble_rings<<<grid_for((size_t)in.m * in.n, 256), 256, 0, st>>>(A);
  k_assemble_origin<<<1, 256, 0, st>>>(A);
  return 2;
}

int launch_coarsen(const CoarsenLevel& f, const CoarsenLevel& c, cudaStream_t st) {
  CoarsenArgs A{f.sh, c.sh, f.w, f.e, f.s, f.nn, f.rs, f.vol, f.o, f.ia, f.ib, f.sc,
                c.w, c.e, c.s, c.nn, c.rs, c.vol, c.o, c.sc};
  k_coarsen_weights<<<grid_for((size_t)f.sh.no * f.sh.n, 256), 256, 0, st>>>(A);
  k_coarsen_rings<<<grid_for((size_t)c.sh.m * c.sh.n, 256), 256, 0, st>>>(A);
  k_coarsen_origin<<<1, 32, 0, st>>>(A);
  return 3;
}

}  // namespace polar
