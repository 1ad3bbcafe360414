// Direct (Fourier in theta, tridiagonal in r) solve of separable theta-step systems:
// declarations shared by polar_fft.cu and the host orchestration in polar_api.cu.
#pragma once
#include <cstddef>
#include <vector>

#include "polar_internal.h"

namespace polar {

constexpr int kFftMaxM = 8192;                 // longest transform held in shared memory
constexpr size_t kFftSmemCap = 128 * 1024;     // shared memory of one transform CTA

// Transform of length n along every ring: M = n (power of two) or the Bluestein length
// M >= 2n - 1; rw rings per CTA.  Device tables: twiddles exp(-2 pi i k / M), k < M/2;
// chirp exp(-i pi k^2 / n), k < n (Bluestein only); transform of the chirp filter (M
// values, Bluestein only); lam_p = cos(2 pi p / n), p < nh = n/2 + 1.
struct FftPlan {
  int n, nh, M, logM, rw;
  const double *twr, *twi, *chr, *chi, *bhr, *bhi, *lam;
};

// Angle-independent coefficients of the fine level in the difference form of V L
// (ring i at index i - 1, m each), the origin's uniform coupling o and sum n o.
struct SepRings {
  int m;
  const double *vol, *rs, *w, *e, *s;
  double vol0, rs0, o, osum;
};

// Arguments of one instance's direct solve (batched launches).
struct DirectArgs {
  Shape sh;
  FftPlan P;
  SepRings R;
  Params par;
  const double* b;  // right-hand side (split layout)
  double* x;        // solution
  double *Xr, *Xi, *cp, *z;
};

// shared memory of one transform CTA of plan P
size_t dft_smem(const FftPlan& P);
// Sizes of the transform for n angles; false when n is too long for shared memory.
bool fft_plan_sizes(int n, int* M, int* logM, int* rw);
// Host tables of the plan (FP64 cos / sin of exact arguments).
void fft_host_tables(int n, int M, std::vector<double>& twr, std::vector<double>& twi,
                     std::vector<double>& chr, std::vector<double>& chi,
                     std::vector<double>& lam);
// Bhat = FFT_M(chirp filter), once per mesh (Bluestein plans only).
int launch_chirp_filter(const FftPlan& P, double* bhr, double* bhi, cudaStream_t st);
// Batched direct solves over `nslots` slots (see BSlot): Srings gives each slot's ring-group
// count, Smodes its mode-block count (128 modes each); ks[s] the slot's solver scalars;
// smem: the largest transform's shared memory.
int launch_direct_b(const DirectArgs* A, const BSlot* Srings, const BSlot* Smodes, int nslots,
                    const int* mask, KrylovScalars* const* ks, int grid_rings, int grid_modes,
                    size_t smem, cudaStream_t st);
// x = S^{-1} b for the separable S = alpha V + beta V L (split layout, FP64).  Work
// arrays: Xr, Xi, cp of m * nh doubles, z of m.  Sets ks->iters = 0, ks->done = 1.
int launch_direct_solve(const Shape& sh, const FftPlan& P, const SepRings& R, Params par,
                        const double* b, double* x, double* Xr, double* Xi, double* cp,
                        double* z, KrylovScalars* ks, cudaStream_t st);

}  // namespace polar
