// A coupling pass for callers that cannot allocate device memory.
//
// rapdb_coupling_pass needs a context, and creating one calls cudaMalloc for
// the padded copies, the solver state and the per-block partial sums.  Some
// callers cannot do that: code running inside another framework's memory
// pool or a fixed memory budget where every byte is pre-planned, real-time
// loops that must not enter the allocator, and code that records work into a
// CUDA graph where a new allocation would break the recording.  This entry
// point gives them the same products and dot products from the caller's own
// arrays, with the only scratch (the per-block FP64 partial dots) kept in a
// file-scope device array of fixed size.
#include <cuda_runtime.h>

#include "rapdb_device.cuh"

using namespace rapdb_dev;

namespace {

constexpr int NA_ROWS = 32;                       // rows per CTA
constexpr long long NA_MAX_PARTIALS = 1ll << 17;  // 131072 doubles = 1 MiB

// Scratch shared by every call on a device: per-(matrix, dot, row block)
// partial sums.  Each call overwrites every slot it later reads, so nothing
// in it has to start at zero.
static __device__ __align__(256) double g_na_partials[NA_MAX_PARTIALS];


__global__ void __launch_bounds__(NT) k_pass_noalloc(const float* __restrict__ Q, int n, int nrb,
                                                     const float* __restrict__ x, const float* __restrict__ v,
                                                     const float* __restrict__ uold, const float* __restrict__ c,
                                                     float* __restrict__ U, float* __restrict__ W,
                                                     double* __restrict__ part) {
  __shared__ double red[NWARP * NDOT];
  const int s = blockIdx.x / nrb;
  const int r = blockIdx.x - s * nrb;
  const int row0 = r * NA_ROWS;
  const int rows = min(NA_ROWS, n - row0);
  pass_block<RAPDB_F32, 4, 2>((const uint8_t*)(Q + (size_t)s * n * n), n, row0, rows, x, v, nullptr, nullptr,
                              nullptr, uold ? uold + (size_t)s * n : nullptr, c + (size_t)s * n,
                              U + (size_t)s * n, W + (size_t)s * n, part + (size_t)s * NDOT * nrb + r, nrb, red);
}

__global__ void __launch_bounds__(NT) k_dots_noalloc(const double* __restrict__ part, int M, int nrb,
                                                     double* __restrict__ dots) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pq = blockIdx.x * NWARP + warp; pq < M * NDOT; pq += gridDim.x * NWARP) {
    double t = 0.0;
    for (int rr = lane; rr < nrb; rr += 32) t += part[(size_t)pq * nrb + rr];
    t = warp_sum(t);
    if (lane == 0) dots[pq] = t;
  }
}

}  // namespace

extern "C" rapdb_status rapdb_coupling_pass_noalloc(int64_t n, int64_t m, const float* Q, const float* c,
                                                    const float* x, const float* v, const float* uold, float* U,
                                                    float* W, double* dots, void* stream) {
  if (n <= 0 || m < 0 || n > (1 << 24)) return RAPDB_ERR_INVALID;
  if (!Q || !c || !x || !v || !U || !W || !dots) return RAPDB_ERR_INVALID;
  if (n % 4 != 0) return RAPDB_ERR_INVALID;
  auto al16 = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
  if (!al16(Q) || !al16(x) || !al16(v)) return RAPDB_ERR_INVALID;
  const long long M = m + 1;
  const long long nrb = (n + NA_ROWS - 1) / NA_ROWS;
  if (M * NDOT * nrb > NA_MAX_PARTIALS) return RAPDB_ERR_INVALID;   // beyond the fixed scratch
  // The array's device address in the current device's context.  In host
  // code the symbol itself is only a stand-in, never a device address.  The
  // address is looked up on every call rather than remembered: after a
  // cudaDeviceReset, or with another context current on the device, the
  // library's device code is loaded again, possibly at another address.  The
  // first call on a device is the one that loads that code.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_partials) != cudaSuccess || !p) return RAPDB_ERR_CUDA;
  double* part = (double*)p;
  cudaStream_t st = (cudaStream_t)stream;
  k_pass_noalloc<<<(unsigned)(M * nrb), NT, 0, st>>>(Q, (int)n, (int)nrb, x, v, uold, c, U, W, part);
  k_dots_noalloc<<<(unsigned)((M * NDOT + NWARP - 1) / NWARP), NT, 0, st>>>(part, (int)M, (int)nrb, dots);
  return cudaGetLastError() == cudaSuccess ? RAPDB_OK : RAPDB_ERR_CUDA;
}
