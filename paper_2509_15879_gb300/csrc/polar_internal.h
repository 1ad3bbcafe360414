// Internal declarations shared by the host orchestration (polar_api.cu) and the
// kernels (polar_kernels.cu).  Nothing here is part of the C ABI.
//
// Device vector layout ("padded layout"): element 0 is the origin, elements 1..3 are
// zero padding, and radial line j (angle theta_j) occupies [kOfs + j*ld, kOfs + j*ld + m)
// with ld = m rounded up to a multiple of 4, so every line starts on a 32-byte
// boundary for FP64 and a 16-byte boundary for FP32.  Entries [m, ld) of every line
// are kept at zero by every kernel that writes a vector.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace polar {

constexpr int kOfs = 4;

// The discrete operator L of one instance, as 5-point rows (Section 3.2.1) kept in
// difference form: with the diagonal C = R - W - E - S - N,
//   (L x)_{i,j} = R x_{i,j} + W (x_{i-1,j} - x_{i,j}) + E (x_{i+1,j} - x_{i,j})
//               + S (x_{i,j-1} - x_{i,j}) + N (x_{i,j+1} - x_{i,j}),
// with x_{0,j} = x_0 (the origin, Eq. 2.8), periodic j (Eqs. 2.6-2.7), and x_{m+1,j}
// the Dirichlet value (Eq. 2.9; zero in the homogeneous operator).  R is the row sum
// (b plus the drift divergence), so smooth vectors lose no digits to the cancellation
// of the huge angular couplings near the origin, also in FP32.
// Origin row (Section 3.2.2): (L x)_0 = R[0] x_0 + sum_j o[j] (x_{1,j} - x_0).
template <typename T>
struct OpView {
  int m, n, ld;
  const T* R;
  const T* W;
  const T* E;
  const T* S;
  const T* N;
  const T* o;  // n coefficients of the origin row
};

// LU factors of the line blocks of A = alpha I + beta L (per time step).
// Radial line j (rows i = 1..m, tridiagonal, origin and boundary couplings dropped):
//   forward  y_k = d_k - l_k y_{k-1};  backward  x_k = ui_k y_k - cu_k x_{k+1}.
// Angular line i (rows j = 0..n-1, periodic): the same factors of the tridiagonal
// part A' after the Sherman-Morrison splitting A = A' + u v^T, plus q = A'^{-1} u and
// per ring vf = v_{n-1} and inv1vq = 1 / (1 + v.q).
template <typename T>
struct LineFactors {
  T* rl;
  T* rui;
  T* rcu;
  T* al;
  T* aui;
  T* acu;
  T* aq;
  T* avf;     // m
  T* ainv;    // m
  double* ws; // 2 nv doubles: FP64 forward values of q and FP64 pivots (factor kernel only)
  T diag0;    // A_00, the origin block of the preconditioner
};

// Scalars of one Krylov solve, kept on the device so that no iteration needs the host.
struct KrylovScalars {
  double rho, alpha, omega, beta;
  double rr0, rr, tol2;
  double dot[4];
  int done;        // 0 running, 1 converged, 2 breakdown, 3 non-finite
  int iters;
  int max_iter;
  int pad0;
  // refinement (FP64) reductions
  double rmax;     // max |r_i|
  double smax;     // max |r_i| / A_ii
  double xmax;     // max |x_i|
  unsigned int counter;
  unsigned int pad1;
};

struct Reduce {
  double* part;        // partial sums, kMaxBlocks * 4
  KrylovScalars* ks;   // device scalars
};
constexpr int kMaxBlocks = 2048;

int grid_for(size_t work, int threads);

// ----------------------------------------------------------------- kernel launchers
// All launchers enqueue on `st` and return the number of kernels launched.

// y = alpha x + beta L x (+ optional terms; see polar_kernels.cu for each mode)
template <typename T>
int launch_apply(const OpView<T>& op, T alpha, T beta, const T* x, T* y, cudaStream_t st,
                 Reduce red);

// y = b - (alpha x + beta L x)
template <typename T>
int launch_resid(const OpView<T>& op, T alpha, T beta, const T* x, const T* b, T* y,
                 cudaStream_t st, Reduce red);

// FP64 right-hand side of the theta-step:
// e = alpha x + beta L_g x + sum_q cf[q] src[q], where L_g takes x_{m+1,j} =
// sum_q cg[q] bnd[q][j] as the Dirichlet value
int launch_rhs(const OpView<double>& op, double alpha, double beta, const double* x,
               int nsrc, const double* const* src, const double* const* bnd,
               const double* cf, const double* cg, double* e, cudaStream_t st, Reduce red);

// FP64 residual of the implicit system with reductions into red.ks:
// r = e - (alpha x + beta L x); rmax, smax (Jacobi-scaled), xmax.
// c0 is the diagonal of the origin row of L.
int launch_resid64(const OpView<double>& op, double alpha, double beta, const double* x,
                   const double* e, double* r, double c0, cudaStream_t st, Reduce red);

// factors in precision T, computed in FP64 from the FP64 operator
template <typename T>
int launch_factor(const OpView<double>& op, double alpha, double beta, LineFactors<T>& f,
                  cudaStream_t st);

// out = M_r^{-1} rhs (radial lines + origin block)
template <typename T>
int launch_radial_solve(const OpView<T>& op, const LineFactors<T>& f, const T* rhs, T* out,
                        cudaStream_t st, const int* done);
// out = base + M_a^{-1} rhs (angular periodic lines + origin block); tmp is scratch
template <typename T>
int launch_angular_solve(const OpView<T>& op, const LineFactors<T>& f, const T* rhs,
                         const T* base, T* out, T* tmp, cudaStream_t st, const int* done);

// ---- Krylov (BiCGStab) kernels; see polar_kernels.cu
template <typename T>
int launch_bicg_init(size_t nv, const T* r, T* rhat, T* p, T* v, T* x, bool zero_x,
                     double rel_tol, int max_iter, cudaStream_t st, Reduce red);
template <typename T>
int launch_apply_dot(const OpView<T>& op, T alpha, T beta, const T* x, T* y, const T* d1,
                     int mode, cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_s(size_t nv, const T* r, const T* v, T* s, cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_update(size_t nv, T* x, const T* phat, const T* shat, T* r, const T* s,
                       const T* t, const T* rhat, cudaStream_t st, Reduce red);
template <typename T>
int launch_bicg_p(size_t nv, T* p, const T* r, const T* v, cudaStream_t st, Reduce red);

// ---- mixed-precision helpers
// rs = r * (1 / ks->rmax) in precision T
template <typename T>
int launch_scale_cast(size_t nv, const double* r, T* rs, cudaStream_t st, Reduce red);
// x += ks->rmax * d
template <typename T>
int launch_correct(size_t nv, double* x, const T* d, cudaStream_t st, Reduce red);
// float copy of a double array
int launch_to_float(size_t n, const double* a, float* b, cudaStream_t st);
// nonfinite check of n doubles: sets ks->done = 3 if any is NaN/Inf
int launch_check_finite(size_t n, const double* a, cudaStream_t st, Reduce red);

// interface layout <-> padded layout
int launch_pack(int m, int n, int ld, const double* in, double* out, cudaStream_t st);
int launch_unpack(int m, int n, int ld, const double* in, double* out, cudaStream_t st);

}  // namespace polar
