// Host-side set-up of the theta-step operator: assembly from the caller's coefficients
// (Sections 2.1, 3.1, 3.2.1, 3.2.2) and the radial multigrid hierarchy.
#include "polar_host.h"

#include <algorithm>
#include <cmath>

namespace polar {

void HLevel::resize(int m_, int n_) {
  m = m_;
  n = n_;
  const size_t N = (size_t)m * n;
  for (std::vector<double>* v : {&vol, &rs, &w, &e, &s, &nn, &ia, &ib}) v->assign(N, 0.0);
  o.assign(n, 0.0);
  vol0 = rs0 = 0.0;
}

namespace {

// Mesh metrics (Sections 2.1 and 3.1): h_i = r_i - r_{i-1}; r_{i+1/2} midpoints;
// mu_j = theta_j - theta_{j-1} with mu_0 = mu_n the wrap-around step; cell widths
// k_i = (h_i + h_{i+1})/2 and w_j = (mu_j + mu_{j+1})/2.
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

double node_b(const HostCoeffs& k, size_t idx) { return k.b.empty() ? 0.0 : k.b[idx]; }

}  // namespace

void control_volumes(const std::vector<double>& r, const std::vector<double>& th, HLevel& L) {
  Metrics g(r, th);
  for (int j = 0; j < g.n; ++j)
    for (int i = 1; i <= g.m; ++i) L.vol[L.q(i, j)] = r[i] * g.k[i] * g.w[j];
  L.vol0 = M_PI * g.h[1] * g.h[1] / 4.0;
}

// Every face carries the flux  len * ((D / spacing + v+) U_in - (D / spacing + v-) U_out)
// out of its inner cell and into its outer cell.  Radial face (i+1/2, j): length
// w_j r_{i+1/2}, spacing h_{i+1}; angular face (i, j+1/2): length k_i, spacing
// r_i mu_{j+1}.  A row of V L is the sum of its cell's outward fluxes plus V b U; in
// difference form a face adds -cout to the inner cell's coupling, -cin to the outer
// cell's, and +len v / -len v to their row sums.
void assemble_conservative(const std::vector<double>& r, const std::vector<double>& th,
                           const HostCoeffs& K, HLevel& L) {
  Metrics g(r, th);
  const int m = g.m, n = g.n;
  L.resize(m, n);
  control_volumes(r, th, L);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i <= m; ++i) {  // radial faces
      const size_t f = (size_t)j * (m + 1) + i;
      const double D = K.dr.empty() ? K.d_const : K.dr[f];
      const double v = K.vr.empty() ? 0.0 : K.vr[f];
      const double len = g.w[j] * g.rh[i];
      const double cond = D / g.h[i + 1];
      const double cin = len * (cond + std::max(v, 0.0));
      const double cout = len * (cond + std::max(-v, 0.0));
      if (i == 0) {
        L.o[j] = -cout;
        L.rs0 += len * v;
      } else {
        L.e[L.q(i, j)] = -cout;  // i = m: coupling to the Dirichlet value
        L.rs[L.q(i, j)] += len * v;
      }
      if (i < m) {
        L.w[L.q(i + 1, j)] = -cin;  // i = 0: ring 1's coupling to the origin
        L.rs[L.q(i + 1, j)] -= len * v;
      }
    }
    const int jp = (j + 1) % n;
    for (int i = 1; i <= m; ++i) {  // angular faces
      const size_t f = (size_t)j * m + (i - 1);
      const double D = K.dt.empty() ? K.d_const : K.dt[f];
      const double v = K.vt.empty() ? 0.0 : K.vt[f];
      const double len = g.k[i];
      const double cond = D / (r[i] * g.mu[j + 1]);
      const double cin = len * (cond + std::max(v, 0.0));
      const double cout = len * (cond + std::max(-v, 0.0));
      L.nn[L.q(i, j)] = -cout;
      L.rs[L.q(i, j)] += len * v;
      L.s[L.q(i, jp)] = -cin;
      L.rs[L.q(i, jp)] -= len * v;
    }
  }
  for (int j = 0; j < n; ++j)
    for (int i = 1; i <= m; ++i) {
      const size_t q = L.q(i, j);
      L.rs[q] += L.vol[q] * node_b(K, 1 + q);
    }
  L.rs0 += L.vol0 * node_b(K, 0);
}

// Printed ring rows of Section 3.2.1 (scalar E at nodes, forward differences) and the
// printed origin row of Section 3.2.2, plus b U; every row times its control volume.
// The printed diagonal is the sum of the printed off-diagonal magnitudes plus b, so the
// row sum of L is b.
void assemble_paper(const std::vector<double>& r, const std::vector<double>& th,
                    const HostCoeffs& K, HLevel& L) {
  Metrics g(r, th);
  const int m = g.m, n = g.n;
  L.resize(m, n);
  control_volumes(r, th, L);
  for (int j = 0; j < n; ++j) {
    const int jm = (j + n - 1) % n;
    const double muj = g.mu[j], muj1 = g.mu[j + 1];
    for (int i = 1; i <= m; ++i) {
      const size_t q = L.q(i, j);
      const double Dm = K.dr.empty() ? K.d_const : K.dr[(size_t)j * (m + 1) + i - 1];
      const double Dp = K.dr.empty() ? K.d_const : K.dr[(size_t)j * (m + 1) + i];
      const double Dn = K.dt.empty() ? K.d_const : K.dt[(size_t)j * m + i - 1];
      const double Ds = K.dt.empty() ? K.d_const : K.dt[(size_t)jm * m + i - 1];
      const double E = K.en.empty() ? 0.0 : K.en[1 + q];
      const double hi = g.h[i], hi1 = g.h[i + 1], ri = r[i];
      const double rm = g.rh[i - 1], rp = g.rh[i];
      const double V = L.vol[q];
      L.w[q] = V * -2.0 * rm * Dm / (ri * hi * (hi + hi1));
      L.e[q] = V * -(2.0 * rp * Dp / (ri * hi1 * (hi + hi1)) + E / hi1);
      L.s[q] = V * -2.0 * Ds / (ri * ri * muj * (muj + muj1));
      L.nn[q] = V * -(2.0 * Dn / (ri * ri * muj1 * (muj + muj1)) + E / (ri * muj1));
      L.rs[q] = V * node_b(K, 1 + q);
    }
  }
  const double h1 = g.h[1];
  const double E0 = K.en.empty() ? 0.0 : K.en[0];
  const double V0 = L.vol0;
  for (int j = 0; j < n; ++j) L.o[j] = V0 * -(4.0 * K.d0 / (n * h1 * h1) - E0 / (n * h1));
  // diagonal 4 d0 / h1^2 + E0 / h1 + b0 = rs0 - sum_j o_j
  L.rs0 = V0 * (node_b(K, 0) + 2.0 * E0 / h1);
}

// Galerkin coarsening in r.  Coarse ring I is fine ring 2I.  An odd fine ring k is
// interpolated from its even neighbours with the weights of its own radial row,
//   x_k = ia_k x_{k-1} + ib_k x_{k+1},  ia = w_k / (w_k + e_k),  ib = e_k / (w_k + e_k)
// (x_0 the origin, x_{m+1} = 0), so the coarse radial couplings are the Schur
// complements of the odd rings (cyclic reduction of each radial line):
//   w^c_I = w_{2I} ia_{2I-1},   e^c_I = e_{2I} ib_{2I+1}   (e_{2I} itself if 2I = m).
// Angular couplings, row sums and volumes are summed with the restriction weights
// (the transpose of the interpolation) onto the coarse ring of their row.
void coarsen(HLevel& f, HLevel& c) {
  const int m = f.m, n = f.n, mc = m / 2;
  c.resize(mc, n);
  for (int j = 0; j < n; ++j)
    for (int k = 1; k <= m; k += 2) {
      const size_t q = f.q(k, j);
      const double den = f.w[q] + f.e[q];
      if (den != 0.0) {
        f.ia[q] = f.w[q] / den;
        f.ib[q] = f.e[q] / den;
      } else {
        f.ia[q] = f.ib[q] = 0.5;
      }
    }
  for (int j = 0; j < n; ++j) {
    for (int I = 1; I <= mc; ++I) {
      const int k = 2 * I;
      const size_t qk = f.q(k, j), qlo = f.q(k - 1, j);
      const size_t qc = c.q(I, j);
      const bool hi = k + 1 <= m;
      const size_t qhi = hi ? f.q(k + 1, j) : 0;
      c.w[qc] = f.w[qk] * f.ia[qlo];
      c.e[qc] = hi ? f.e[qk] * f.ib[qhi] : f.e[qk];
      const double bl = f.ib[qlo], ah = hi ? f.ia[qhi] : 0.0;
      auto lump = [&](const std::vector<double>& a) {
        return a[qk] + bl * a[qlo] + (hi ? ah * a[qhi] : 0.0);
      };
      c.s[qc] = lump(f.s);
      c.nn[qc] = lump(f.nn);
      c.rs[qc] = lump(f.rs);
      c.vol[qc] = lump(f.vol);
    }
    const size_t q1 = f.q(1, j);
    c.o[j] = f.o[j] * f.ib[q1];
  }
  c.vol0 = f.vol0;
  c.rs0 = f.rs0;
  for (int j = 0; j < n; ++j) {
    const size_t q1 = f.q(1, j);
    c.vol0 += f.ia[q1] * f.vol[q1];
    c.rs0 += f.ia[q1] * f.rs[q1];
  }
}

}  // namespace polar
