// Self-test of the bounded mbarrier wait that guards every bulk-copy stage of
// the coupling pass.
//
// One CTA of one warp initialises an mbarrier in shared memory and waits on
// its first phase with the same helper the pass uses (mbar_wait_bounded),
// under a caller-chosen time limit.  With `complete` = 1 lane 0 also issues a
// real 16-byte bulk copy (cp.async.bulk, global -> shared) that completes the
// phase, so the wait returns normally.  With `complete` = 0 lane 0 announces
// 16 bytes on the barrier that no copy ever delivers: nothing completes the
// phase, so the wait must give up at the limit, set the error flag and return.
// No copy is in flight when the wait gives up, the CTA invalidates its barrier
// and exits, and the context stays usable.  This is how a stalled copy is
// detected without making the GPU fault or hang.
#include <cuda_runtime.h>

#include "rapdb_device.cuh"
#include "rapdb.h"

using namespace rapdb_dev;

namespace {

__device__ __align__(16) float g_st_src[4] = {1.0f, 2.0f, 3.0f, 4.0f};

__global__ void __launch_bounds__(32) k_wait_selftest(int complete, unsigned long long limit_ns, int* err,
                                                      float* got, unsigned long long* waited_ns) {
  __shared__ __align__(16) float buf[4];
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x;
  if (lane == 0) {
    buf[0] = buf[1] = buf[2] = buf[3] = 0.0f;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  __syncwarp();
  if (lane == 0) {
    mbar_expect_tx(&bar, 16);
    if (complete) bulk_g2s(buf, g_st_src, 16, &bar);
  }
  __syncwarp();
  const unsigned long long t0 = globaltimer();
  const bool ok = mbar_wait_bounded(&bar, 0u, err, limit_ns);
  const unsigned long long t1 = globaltimer();
  __syncwarp();
  if (lane == 0) {
    *waited_ns = t1 - t0;
    got[0] = ok ? buf[0] + buf[1] + buf[2] + buf[3] : -1.0f;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace

extern "C" rapdb_status rapdb_wait_selftest(int32_t complete, int64_t limit_us, int32_t* gave_up,
                                            double* waited_ms, float* copied_sum) {
  if (limit_us < 1 || limit_us > 2000000 || (complete != 0 && complete != 1)) return RAPDB_ERR_INVALID;
  struct Out {
    int err;
    float got;
    unsigned long long waited;
  };
  Out* d = nullptr;
  if (cudaMalloc(&d, sizeof(Out)) != cudaSuccess) return RAPDB_ERR_NOMEM;
  rapdb_status st = RAPDB_OK;
  Out h{};
  if (cudaMemset(d, 0, sizeof(Out)) != cudaSuccess) st = RAPDB_ERR_CUDA;
  if (st == RAPDB_OK) {
    k_wait_selftest<<<1, 32>>>(complete, (unsigned long long)limit_us * 1000ull, &d->err, &d->got, &d->waited);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&h, d, sizeof(Out), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = RAPDB_ERR_CUDA;
  }
  cudaFree(d);
  if (st != RAPDB_OK) return st;
  if (gave_up) *gave_up = h.err;
  if (waited_ms) *waited_ms = (double)h.waited * 1e-6;
  if (copied_sum) *copied_sum = h.got;
  return RAPDB_OK;
}
