// Direct solve of the theta-step system for separable operators (sm_103a): uniform
// angles and ring coefficients that do not depend on the angle (Section 2.1, the
// Swarztrauber-Sweet structure of the origin row).  Then every ring row reads
//   diag_i x_ij + beta (w_i x_{i-1,j} + e_i x_{i+1,j} + s_i (x_{i,j-1} + x_{i,j+1}))
// and the periodic angular coupling is diagonalised by the discrete Fourier transform
// along theta: mode p of ring i sees  diag_i + 2 beta s_i cos(2 pi p / n),  and the
// rings of one mode form a tridiagonal system in r.  The origin couples to the mean
// (p = 0) only: its row sums o x_{1,j} over the angles, and ring 1 sees x_0 at every
// angle.  A solve is three kernels:
//   k_dft_rings (forward)  ring values -> Fourier coefficients X_ip, p = 0 .. n/2
//   k_modes                one thread per mode: tridiagonal (Thomas) solve along r;
//                          mode 0 adds the origin through a Schur step
//   k_dft_rings (inverse)  coefficients -> ring values
// The transform of a ring runs in shared memory: an iterative radix-2 FFT when n is a
// power of two, otherwise Bluestein's chirp-z form (a circular convolution of length
// M >= 2n - 1, a power of two, evaluated with three radix-2 FFTs; the transform of the
// chirp filter is precomputed once per mesh).  Inverse transforms use the forward one:
// x = conj(DFT(conj X)) / n.  All arithmetic is FP64.
#include <cmath>
#include <cstdint>
#include <vector>

#include "polar_fft.h"

namespace polar {

namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) {
  return __brev(v) >> (32 - bits);
}

// In-place forward FFT (X_k = sum_j x_j exp(-2 pi i j k / M)) of `rw` rings of length M
// held in shared memory (re, im: rw * M values, ring r at offset r * M), natural order in
// and out.  All threads of the CTA take part.
__device__ void fft_rings(double* re, double* im, int rw, int M, int logM, const double* twr,
                          const double* twi) {
  const int nt = blockDim.x;
  // bit-reversal permutation
  for (int t = threadIdx.x; t < rw * M; t += nt) {
    const int r = t / M, j = t - r * M;
    const int q = (int)bitrev((unsigned)j, logM);
    if (j < q) {
      const int a = r * M + j, b = r * M + q;
      const double xr = re[a], xi = im[a];
      re[a] = re[b];
      im[a] = im[b];
      re[b] = xr;
      im[b] = xi;
    }
  }
  __syncthreads();
  // decimation-in-time butterflies, stage s combines blocks of 2^s
  const int half_total = M >> 1;
  for (int s = 0; s < logM; ++s) {
    const int half = 1 << s;
    const int stride = half_total >> s;  // twiddle index step
    for (int t = threadIdx.x; t < rw * half_total; t += nt) {
      const int r = t / half_total, b = t - r * half_total;
      const int g = b >> s, pos = b & (half - 1);
      const int i0 = r * M + (g << (s + 1)) + pos, i1 = i0 + half;
      const double wr = twr[pos * stride], wi = twi[pos * stride];
      const double ur = re[i1], ui = im[i1];
      const double vr = fma(wr, ur, -wi * ui), vi = fma(wr, ui, wi * ur);
      const double ar = re[i0], ai = im[i0];
      re[i0] = ar + vr;
      im[i0] = ai + vi;
      re[i1] = ar - vr;
      im[i1] = ai - vi;
    }
    __syncthreads();
  }
}

// DFT of length n of every ring in shared memory (data in [0, n) of each ring's M slots,
// natural order), result in [0, n): the radix-2 FFT itself when M == n, else Bluestein:
//   a_j = x_j c_j (c_j = exp(-i pi j^2 / n)), zero padded to M;  A = FFT(a) * Bhat;
//   a = IFFT(A) = conj(FFT(conj A)) / M;  X_p = c_p a_p.
__device__ void dft_rings(double* re, double* im, int rw, const FftPlan& P) {
  const int M = P.M, n = P.n, nt = blockDim.x;
  if (M == n) {
    fft_rings(re, im, rw, M, P.logM, P.twr, P.twi);
    return;
  }
  for (int t = threadIdx.x; t < rw * M; t += nt) {
    const int r = t / M, j = t - r * M;
    const int a = r * M + j;
    if (j < n) {
      const double cr = P.chr[j], ci = P.chi[j];
      const double xr = re[a], xi = im[a];
      re[a] = fma(xr, cr, -xi * ci);
      im[a] = fma(xr, ci, xi * cr);
    } else {
      re[a] = 0.0;
      im[a] = 0.0;
    }
  }
  __syncthreads();
  fft_rings(re, im, rw, M, P.logM, P.twr, P.twi);
  // A * Bhat, conjugated for the inverse transform
  for (int t = threadIdx.x; t < rw * M; t += nt) {
    const int r = t / M, j = t - r * M;
    const int a = r * M + j;
    const double br = P.bhr[j], bi = P.bhi[j];
    const double xr = re[a], xi = im[a];
    re[a] = fma(xr, br, -xi * bi);
    im[a] = -fma(xr, bi, xi * br);
  }
  __syncthreads();
  fft_rings(re, im, rw, M, P.logM, P.twr, P.twi);
  const double inv = 1.0 / (double)M;
  for (int t = threadIdx.x; t < rw * n; t += nt) {
    const int r = t / n, j = t - r * n;
    const int a = r * M + j;
    const double xr = re[a] * inv, xi = -im[a] * inv;  // conj / M
    const double cr = P.chr[j], ci = P.chi[j];
    re[a] = fma(xr, cr, -xi * ci);
    im[a] = fma(xr, ci, xi * cr);
  }
  __syncthreads();
}

// Which parity block and which consecutive rings a CTA of a ring-group grid takes:
// CTAs [0, godd) take the odd rings RW at a time, the rest the even rings.
struct RingGroup {
  int parity, k0, count;
};
__device__ __forceinline__ RingGroup ring_group(const Shape& sh, int rw, int vb) {
  const int godd = (sh.no + rw - 1) / rw;
  RingGroup g;
  int b = vb;
  g.parity = b < godd ? 1 : 0;
  if (!g.parity) b -= godd;
  g.k0 = b * rw;
  const int nl = g.parity ? sh.no : sh.ne;
  g.count = min(rw, nl - g.k0);
  return g;
}

// forward: x (split layout) -> X_ip, p < nh;  inverse: X -> x
template <bool INVERSE>
__device__ __forceinline__ void dft_rings_body(const Shape& sh, const FftPlan& P, const double* x,
                                               double* Xr, double* Xi, double* y, int vb) {
  extern __shared__ double smem[];
  const int rw = P.rw, M = P.M, n = P.n, nh = P.nh, nt = blockDim.x;
  double* re = smem;
  double* im = smem + (size_t)rw * M;
  const RingGroup g = ring_group(sh, rw, vb);
  const size_t base = g.parity ? sh.odd0 : sh.even0;
  const int ld = g.parity ? sh.ldo : sh.lde;
  auto ring_of = [&](int r) { return g.parity ? 2 * (g.k0 + r) + 1 : 2 * (g.k0 + r) + 2; };
  if (!INVERSE) {
    // rings r < count at angle j are contiguous: consecutive threads read consecutive rings
    for (int t = threadIdx.x; t < rw * n; t += nt) {
      const int j = t / rw, r = t - j * rw;
      double v = 0.0;
      if (r < g.count) v = x[base + (size_t)j * ld + g.k0 + r];
      re[r * M + j] = v;
      im[r * M + j] = 0.0;
    }
  } else {
    // full spectrum from the half (X_{n-p} = conj X_p), conjugated: x = conj(DFT(conj X)) / n
    for (int t = threadIdx.x; t < rw * n; t += nt) {
      const int r = t / n, p = t - r * n;
      double vr = 0.0, vi = 0.0;
      if (r < g.count) {
        const size_t row = (size_t)(ring_of(r) - 1) * nh;
        if (p < nh) {
          vr = Xr[row + p];
          vi = -Xi[row + p];
        } else {
          vr = Xr[row + (n - p)];
          vi = Xi[row + (n - p)];
        }
      }
      re[r * M + p] = vr;
      im[r * M + p] = vi;
    }
  }
  __syncthreads();
  dft_rings(re, im, rw, P);
  if (!INVERSE) {
    for (int t = threadIdx.x; t < rw * nh; t += nt) {
      const int r = t / nh, p = t - r * nh;
      if (r >= g.count) continue;
      const size_t row = (size_t)(ring_of(r) - 1) * nh;
      Xr[row + p] = re[r * M + p];
      Xi[row + p] = im[r * M + p];
    }
  } else {
    const double inv = 1.0 / (double)n;
    for (int t = threadIdx.x; t < rw * n; t += nt) {
      const int j = t / rw, r = t - j * rw;
      if (r >= g.count) continue;
      y[base + (size_t)j * ld + g.k0 + r] = re[r * M + j] * inv;
    }
  }
}

template <bool INVERSE>
__global__ void __launch_bounds__(kFftThreads) k_dft_rings(Shape sh, FftPlan P, const double* x,
                                                           double* Xr, double* Xi, double* y) {
  dft_rings_body<INVERSE>(sh, P, x, Xr, Xi, y, blockIdx.x);
}

// One thread per Fourier mode p < nh: Thomas along r of
//   (diag_i + 2 beta s_i cos(2 pi p / n)) X_i + beta w_i X_{i-1} + beta e_i X_{i+1} = B_i
// for the real and imaginary parts (the same real matrix).  Mode 0 carries the origin:
// ring 1 sees n beta w_1 x_0 (x_0 at every angle), the origin row reads
// diag0 x_0 + beta o X_{1,0} = b_0; with y = T^{-1} B and z = T^{-1} (n beta w_1 e_1),
// x_0 = (b_0 - beta o y_1) / (diag0 - beta o z_1) and X = y - z x_0.
__device__ __forceinline__ void modes_body(const SepRings& R, const FftPlan& P, Params par,
                                           const double* b, double* x, double* Xr, double* Xi,
                                           double* cp, double* z, KrylovScalars* ks, int vb) {
  if (ks->done) return;
  const int p = vb * blockDim.x + threadIdx.x;
  const int m = R.m, nh = P.nh;
  if (p >= nh) return;
  const double alpha = par[0], beta = par[1];
  const double lam = 2.0 * beta * P.lam[p];
  auto dg = [&](int i) {  // i = 0 .. m-1 (ring i + 1)
    return fma(alpha, R.vol[i], beta * (R.rs[i] - R.w[i] - R.e[i] - 2.0 * R.s[i])) + lam * R.s[i];
  };
  // forward elimination; cp_i = c_i / den_i, the right-hand sides in place
  double cprev = 0.0, dr = 0.0, di = 0.0, dz = 0.0;
  for (int i = 0; i < m; ++i) {
    const size_t q = (size_t)i * nh + p;
    const double a = (i > 0) ? beta * R.w[i] : 0.0;
    const double c = (i < m - 1) ? beta * R.e[i] : 0.0;
    const double inv = 1.0 / (dg(i) - a * cprev);
    cprev = c * inv;
    cp[q] = cprev;
    dr = (Xr[q] - a * dr) * inv;
    di = (Xi[q] - a * di) * inv;
    Xr[q] = dr;
    Xi[q] = di;
    if (p == 0) {
      dz = ((i == 0 ? (double)P.n * beta * R.w[0] : 0.0) - a * dz) * inv;
      z[i] = dz;
    }
  }
  // back substitution
  double xr = 0.0, xi = 0.0, xz = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    const size_t q = (size_t)i * nh + p;
    const double c = cp[q];
    xr = Xr[q] - c * xr;
    xi = Xi[q] - c * xi;
    Xr[q] = xr;
    Xi[q] = xi;
    if (p == 0) {
      xz = z[i] - c * xz;
      z[i] = xz;
    }
  }
  if (p == 0) {
    // xr, xz now hold y_1 and z_1
    const double d0 = fma(alpha, R.vol0, beta * (R.rs0 - R.osum));
    const double x0 = (b[0] - beta * R.o * xr) / (d0 - beta * R.o * xz);
    x[0] = x0;
    for (int i = 0; i < m; ++i) Xr[(size_t)i * nh] -= z[i] * x0;
    ks->iters = 0;  // a direct solve: no Krylov iterations
    ks->done = 1;
  }
}

__global__ void __launch_bounds__(128) k_modes(SepRings R, FftPlan P, Params par, const double* b,
                                               double* x, double* Xr, double* Xi, double* cp,
                                               double* z, KrylovScalars* ks) {
  modes_body(R, P, par, b, x, Xr, Xi, cp, z, ks, blockIdx.x);
}

__global__ void k_pre_direct(KrylovScalars* ks) {
  ks->iters = 0;
  ks->done = 0;
}

// batched forms (per-instance DirectArgs; gate and work list as the other batched kernels)
// batched forms (per-slot DirectArgs; see BSlot): the set-up per active slot, the transforms
// over the slots' ring groups, the mode solves over their mode blocks
__global__ void k_pre_direct_b(const BSlot* S, int nslots, const int* mask,
                               KrylovScalars* const* ks) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
    if (!mask[S[s].inst]) continue;
    ks[s]->iters = 0;
    ks[s]->done = 0;
  }
}
template <bool INVERSE>
__global__ void __launch_bounds__(kFftThreads) k_dft_rings_b(const DirectArgs* A, const BSlot* S,
                                                             int nslots, const int* mask) {
  POLAR_BATCH_LOOP({
    const DirectArgs& a = A[s];
    const Shape sh = a.sh;
    const FftPlan P = a.P;
    dft_rings_body<INVERSE>(sh, P, a.b, a.Xr, a.Xi, a.x, vb);
    __syncthreads();  // the transform's shared memory is reused by the next item
  })
}
__global__ void __launch_bounds__(128) k_modes_b(const DirectArgs* A, const BSlot* S, int nslots,
                                                 const int* mask, KrylovScalars* const* ks) {
  POLAR_BATCH_LOOP({
    const DirectArgs& a = A[s];
    modes_body(a.R, a.P, a.par, a.b, a.x, a.Xr, a.Xi, a.cp, a.z, ks[s], vb);
  })
}

// Transform of the chirp filter b (b_k = conj c_k for |k| < n, circularly), once per mesh.
__global__ void __launch_bounds__(kFftThreads) k_chirp_filter(FftPlan P, double* bhr, double* bhi) {
  extern __shared__ double smem[];
  const int M = P.M, n = P.n;
  double* re = smem;
  double* im = smem + M;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    int src = -1;
    if (k < n) src = k;
    else if (k > M - n) src = M - k;
    re[k] = src >= 0 ? P.chr[src] : 0.0;
    im[k] = src >= 0 ? -P.chi[src] : 0.0;
  }
  __syncthreads();
  fft_rings(re, im, 1, M, P.logM, P.twr, P.twi);
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    bhr[k] = re[k];
    bhi[k] = im[k];
  }
}

}  // namespace

size_t dft_smem(const FftPlan& P) { return (size_t)P.rw * P.M * 2 * sizeof(double); }

bool fft_plan_sizes(int n, int* M, int* logM, int* rw) {
  int m2 = 1, lg = 0;
  while (m2 < n) {
    m2 <<= 1;
    ++lg;
  }
  if (m2 != n) {  // Bluestein: M >= 2n - 1
    while (m2 < 2 * n - 1) {
      m2 <<= 1;
      ++lg;
    }
  }
  if (m2 > kFftMaxM) return false;
  *M = m2;
  *logM = lg;
  // rings per CTA: a full 32-byte sector per angle (4 rings) where shared memory allows
  int r = 4;
  while (r > 1 && (size_t)r * m2 * 2 * sizeof(double) > kFftSmemCap) r >>= 1;
  *rw = r;
  return true;
}

void fft_host_tables(int n, int M, std::vector<double>& twr, std::vector<double>& twi,
                     std::vector<double>& chr, std::vector<double>& chi,
                     std::vector<double>& lam) {
  const double pi = 3.14159265358979323846;
  twr.resize(M / 2);
  twi.resize(M / 2);
  for (int k = 0; k < M / 2; ++k) {
    const double a = 2.0 * pi * (double)k / (double)M;
    twr[k] = std::cos(a);
    twi[k] = -std::sin(a);
  }
  chr.assign(n, 0.0);
  chi.assign(n, 0.0);
  if (M != n) {
    for (int k = 0; k < n; ++k) {
      // exp(-i pi k^2 / n) with k^2 reduced mod 2n exactly
      const int64_t q = ((int64_t)k * k) % (2 * (int64_t)n);
      const double a = pi * (double)q / (double)n;
      chr[k] = std::cos(a);
      chi[k] = -std::sin(a);
    }
  }
  const int nh = n / 2 + 1;
  lam.resize(nh);
  for (int p = 0; p < nh; ++p) lam[p] = std::cos(2.0 * pi * (double)p / (double)n);
}

int launch_chirp_filter(const FftPlan& P, double* bhr, double* bhi, cudaStream_t st) {
  const size_t smem = (size_t)P.M * 2 * sizeof(double);
  cudaFuncSetAttribute(k_chirp_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chirp_filter<<<1, kFftThreads, smem, st>>>(P, bhr, bhi);
  return 1;
}

int launch_direct_solve(const Shape& sh, const FftPlan& P, const SepRings& R, Params par,
                        const double* b, double* x, double* Xr, double* Xi, double* cp,
                        double* z, KrylovScalars* ks, cudaStream_t st) {
  const size_t smem = dft_smem(P);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dft_rings<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFftSmemCap);
    cudaFuncSetAttribute(k_dft_rings<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFftSmemCap);
    attr = true;
  }
  const int groups = (sh.no + P.rw - 1) / P.rw + (sh.ne + P.rw - 1) / P.rw;
  k_pre_direct<<<1, 1, 0, st>>>(ks);
  k_dft_rings<false><<<groups, kFftThreads, smem, st>>>(sh, P, b, Xr, Xi, nullptr);
  k_modes<<<(P.nh + 127) / 128, 128, 0, st>>>(R, P, par, b, x, Xr, Xi, cp, z, ks);
  k_dft_rings<true><<<groups, kFftThreads, smem, st>>>(sh, P, nullptr, Xr, Xi, x);
  return 4;
}


int launch_direct_b(const DirectArgs* A, const BSlot* Srings, const BSlot* Smodes, int nslots,
                    const int* mask, KrylovScalars* const* ks, int grid_rings, int grid_modes,
                    size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dft_rings_b<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFftSmemCap);
    cudaFuncSetAttribute(k_dft_rings_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kFftSmemCap);
    attr = true;
  }
  k_pre_direct_b<<<(nslots + 127) / 128, 128, 0, st>>>(Srings, nslots, mask, ks);
  k_dft_rings_b<false><<<grid_rings, kFftThreads, smem, st>>>(A, Srings, nslots, mask);
  k_modes_b<<<grid_modes, 128, 0, st>>>(A, Smodes, nslots, mask, ks);
  k_dft_rings_b<true><<<grid_rings, kFftThreads, smem, st>>>(A, Srings, nslots, mask);
  return 4;
}

}  // namespace polar
