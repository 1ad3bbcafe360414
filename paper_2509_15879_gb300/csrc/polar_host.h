// Host-side set-up of the theta-step operator (polar_host.cpp): the discrete operator
// of Sections 3.2.1/3.2.2 assembled from the caller's coefficients, scaled by the control
// volumes, and its radial multigrid hierarchy.  Runs once per polar_set_coeffs.
#pragma once
#include <vector>

namespace polar {

// One level of V L (control volume times the row of L) in difference form, arrays
// indexed q = j m + (i - 1) (ring i = 1..m, angle j = 0..n-1):
//   (V L x)_ij = rs x_ij + w (x_{i-1,j} - x_ij) + e (x_{i+1,j} - x_ij)
//              + s (x_{i,j-1} - x_ij) + nn (x_{i,j+1} - x_ij)
//   (V L x)_0  = rs0 x_0 + sum_j o_j (x_{1,j} - x_0)
// with x_{0,j} the origin and x_{m+1,j} the Dirichlet ring (its coupling is e at i = m).
struct HLevel {
  int m = 0, n = 0;
  std::vector<double> vol, rs, w, e, s, nn;
  std::vector<double> ia, ib;  // odd rings: interpolation weights from the coarser level
  std::vector<double> o;       // n
  double vol0 = 0.0, rs0 = 0.0;
  void resize(int m_, int n_);
  size_t q(int i, int j) const { return (size_t)j * m + (size_t)(i - 1); }
};

struct HostCoeffs {
  std::vector<double> dr, dt, vr, vt, en, b;  // empty = constant / absent
  double d_const = 1.0, d0 = 1.0;
};

// CONSERVATIVE scheme: shared face fluxes (diffusion + first-order upwinded drift).
void assemble_conservative(const std::vector<double>& r, const std::vector<double>& th,
                           const HostCoeffs& k, HLevel& L);
// PAPER scheme: the printed ring rows of Section 3.2.1 and origin row of Section 3.2.2.
void assemble_paper(const std::vector<double>& r, const std::vector<double>& th,
                    const HostCoeffs& k, HLevel& L);
// Control volumes V_ij = r_i k_i w_j and V_0 = pi h_1^2 / 4.
void control_volumes(const std::vector<double>& r, const std::vector<double>& th, HLevel& L);

// Next coarser level (rings 2, 4, ... of f); fills f.ia / f.ib.
void coarsen(HLevel& f, HLevel& c);

}  // namespace polar
