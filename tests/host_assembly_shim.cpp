// Test harness (CPU): exposes the library's host-side operator assembly, polar_host.cpp,
// through a plain C function so that the CPU tests can compare its rows with the FP64
// oracle's sparse matrix without a GPU.  Not part of the library.
#include <cstring>
#include <vector>

#include "polar_host.h"

namespace {
std::vector<double> take(const double* p, size_t count) {
  return p ? std::vector<double>(p, p + count) : std::vector<double>();
}
void put(const std::vector<double>& v, double* out) {
  std::memcpy(out, v.data(), v.size() * sizeof(double));
}
}  // namespace

// scheme 0: conservative, 1: paper.  Face arrays as at the C ABI (NULL: constant / absent).
// Outputs: vol, rs, w, e, s, nn (m*n each, q = j*m + i-1), o (n), scal = {vol0, rs0}.
extern "C" int assemble_level0(int scheme, int m, int n, const double* r, const double* th,
                               const double* dr, const double* dt, const double* vr,
                               const double* vt, const double* en, const double* b,
                               double d_const, double d0, double* vol, double* rs, double* w,
                               double* e, double* s, double* nn, double* o, double* scal) {
  polar::HostCoeffs K;
  const size_t N = (size_t)m * n + 1, nf = (size_t)(m + 1) * n, nt = (size_t)m * n;
  K.dr = take(dr, nf);
  K.dt = take(dt, nt);
  K.vr = take(vr, nf);
  K.vt = take(vt, nt);
  K.en = take(en, N);
  K.b = take(b, N);
  K.d_const = d_const;
  K.d0 = d0;
  const std::vector<double> rv(r, r + m + 2), tv(th, th + n);
  polar::HLevel L;
  if (scheme == 0) {
    polar::assemble_conservative(rv, tv, K, L);
  } else {
    polar::assemble_paper(rv, tv, K, L);
  }
  put(L.vol, vol);
  put(L.rs, rs);
  put(L.w, w);
  put(L.e, e);
  put(L.s, s);
  put(L.nn, nn);
  put(L.o, o);
  scal[0] = L.vol0;
  scal[1] = L.rs0;
  return 0;
}

// The same assembly followed by one radial coarsening: outputs the next coarser level
// (mc = m / 2 rings: vol, rs, w, e, s, nn, o, scal) and the fine odd rings' interpolation
// weights ia, ib (m*n, zero on even rings).
extern "C" int coarsen_level0(int scheme, int m, int n, const double* r, const double* th,
                              const double* dr, const double* dt, const double* vr,
                              const double* vt, const double* en, const double* b,
                              double d_const, double d0, double* vol, double* rs, double* w,
                              double* e, double* s, double* nn, double* o, double* scal,
                              double* ia, double* ib) {
  polar::HostCoeffs K;
  const size_t N = (size_t)m * n + 1, nf = (size_t)(m + 1) * n, nt = (size_t)m * n;
  K.dr = take(dr, nf);
  K.dt = take(dt, nt);
  K.vr = take(vr, nf);
  K.vt = take(vt, nt);
  K.en = take(en, N);
  K.b = take(b, N);
  K.d_const = d_const;
  K.d0 = d0;
  const std::vector<double> rv(r, r + m + 2), tv(th, th + n);
  polar::HLevel L, Lc;
  if (scheme == 0) {
    polar::assemble_conservative(rv, tv, K, L);
  } else {
    polar::assemble_paper(rv, tv, K, L);
  }
  polar::coarsen(L, Lc);
  put(Lc.vol, vol);
  put(Lc.rs, rs);
  put(Lc.w, w);
  put(Lc.e, e);
  put(Lc.s, s);
  put(Lc.nn, nn);
  put(Lc.o, o);
  scal[0] = Lc.vol0;
  scal[1] = Lc.rs0;
  put(L.ia, ia);
  put(L.ib, ib);
  return 0;
}
