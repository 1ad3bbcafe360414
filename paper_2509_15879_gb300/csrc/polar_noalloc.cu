// polar_apply_rows_noalloc: the 5-point polar operator applied from caller-supplied rows,
// for callers that cannot allocate device memory (a fixed device-memory budget they own,
// or a pipeline where an allocation call would stall the device).  See include/polar.h.
//
// Its only scratch is the file-scope array below: the origin row needs the sum over all
// angles of o_j (x_{1,j} - x_0); every thread on ring 1 stores its term at slot j, and the
// last block to finish adds the n slots in angle order (deterministic), then resets the
// arrival counter kept behind them.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/polar.h"

namespace polar {
int report_error(int code, const char* msg);  // polar_api.cu: sets polar_last_error()
}

namespace {

constexpr int kMaxAngles = 16384;            // largest n the array serves
constexpr int kCounterSlot = kMaxAngles;     // arrival counter (as unsigned int)
constexpr int kSlots = kMaxAngles + 32;      // 128 KB + 256 B

static __device__ __align__(256) double g_scratch[kSlots];

constexpr int kThreads = 256;
constexpr int kMaxGrid = 1024;
constexpr int kMaxDevices = 64;

int fail(int code, const std::string& msg) { return polar::report_error(code, msg.c_str()); }

__global__ void __launch_bounds__(kThreads)
    k_apply_rows(int m, int n, const double* __restrict__ R, const double* __restrict__ W,
                 const double* __restrict__ E, const double* __restrict__ S,
                 const double* __restrict__ Nn, const double* __restrict__ o, double alpha,
                 double beta, const double* __restrict__ x, double* __restrict__ y,
                 double* scratch) {
  const size_t Np = (size_t)m * n + 1;
  const double x0 = x[0];
  for (size_t q = 1 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < Np;
       q += (size_t)gridDim.x * blockDim.x) {
    const size_t t = q - 1;
    const int j = (int)(t / m);
    const int i = (int)(t - (size_t)j * m) + 1;
    const double xc = x[q];
    const double xw = (i == 1) ? x0 : x[q - 1];
    const double xe = (i == m) ? 0.0 : x[q + 1];
    const double xs = x[(j == 0) ? q + (size_t)(n - 1) * m : q - m];
    const double xn = x[(j == n - 1) ? q - (size_t)(n - 1) * m : q + m];
    double Lx = R[q] * xc;
    Lx = fma(W[q], xw - xc, Lx);
    Lx = fma(E[q], xe - xc, Lx);
    Lx = fma(S[q], xs - xc, Lx);
    Lx = fma(Nn[q], xn - xc, Lx);
    y[q] = fma(beta, Lx, alpha * xc);
    if (i == 1) scratch[j] = o[j] * (xc - x0);
  }
  // the last block to arrive finishes the origin row
  __shared__ unsigned int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounterSlot);
    last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double part[kThreads];
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += __ldcg(scratch + j);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) tot += part[k];
    y[0] = fma(beta, fma(R[0], x0, tot), alpha * x0);
    *reinterpret_cast<unsigned int*>(scratch + kCounterSlot) = 0u;
  }
}

// Device address of g_scratch on the current device.  In host code the name g_scratch
// is a host-side stand-in, not a device address, so the address is looked up with the
// device current.  The lookup is repeated on every call made while `st` is not being
// captured (a device reset or a new primary context can move the module); a call made
// during stream capture reuses the address of the last call on that device, and fails if
// there was none.
std::mutex g_lock;
double* g_addr[kMaxDevices] = {};

int scratch_address(cudaStream_t st, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return fail(POLAR_ECUDA, "no usable CUDA device");
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(POLAR_ECUDA, "cudaStreamIsCapturing failed on the given stream");
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(POLAR_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_addr[dev] = static_cast<double*>(p);
  } else if (!g_addr[dev]) {
    return fail(POLAR_ESTATE, "the first call on a device must come before any stream capture");
  }
  *out = g_addr[dev];
  return POLAR_OK;
}

}  // namespace

extern "C" {

int polar_apply_rows_noalloc(int32_t m, int32_t n, const double* R, const double* W,
                             const double* E, const double* S, const double* N, const double* o,
                             double alpha, double beta, const double* x, double* y,
                             void* stream) {
  if (m < 2 || n < 4) return fail(POLAR_EINVAL, "need m >= 2 and n >= 4");
  if (n > kMaxAngles)
    return fail(POLAR_EINVAL, "n above 16384: the origin row's scratch holds 16384 angles");
  if ((size_t)m * (size_t)n > ((size_t)1 << 31)) return fail(POLAR_EINVAL, "mesh too large");
  if (!R || !W || !E || !S || !N || !o || !x || !y) return fail(POLAR_EINVAL, "null argument");
  const size_t Np = (size_t)m * n + 1;
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  if (xa < ya + Np * sizeof(double) && ya < xa + Np * sizeof(double))
    return fail(POLAR_EINVAL, "x and y must not overlap");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  const int rc = scratch_address(st, &scratch);
  if (rc != POLAR_OK) return rc;
  // the arrival counter must start at zero (a failed earlier launch may have left it set)
  cudaError_t e = cudaMemsetAsync(scratch + kCounterSlot, 0, sizeof(double), st);
  if (e != cudaSuccess) return fail(POLAR_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const size_t work = (size_t)m * n;
  size_t grid = (work + kThreads - 1) / kThreads;
  if (grid > (size_t)kMaxGrid) grid = kMaxGrid;
  k_apply_rows<<<(unsigned)grid, kThreads, 0, st>>>(m, n, R, W, E, S, N, o, alpha, beta, x, y,
                                                    scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(POLAR_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return POLAR_OK;
}

}  // extern "C"
