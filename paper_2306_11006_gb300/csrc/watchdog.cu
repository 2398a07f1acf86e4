// watchdog.cu -- self-test of the device watchdog (the bounded mbarrier waits).
//
// Every wait of the blind-rotation kernels is bounded: after a limit it sets an
// abort flag shared by the CTA and the kDevTimeout bit of the device status word,
// and every other waiter of the CTA then gives up at its next check, so the
// kernel returns and the context stays usable; the host reads the word after the
// call and reports ARX_ETIMEOUT.  arx_watchdog_selftest runs that mechanism on
// purpose: one CTA of four warps waits, through the same two wait functions the
// kernels use (warps 0 and 2: the throughput kernel's, warps 1 and 3: the
// cluster kernels'), for one phase of an mbarrier that expects a single
// arrival.  With post_token set, thread 0 makes that arrival (the "token") and
// every wait completes; without it nothing arrives, the waits run out after
// limit_cycles and the status word records the expiry.  No counterpart in the
// paper: it tests the runtime, not the method.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "br_cluster_common.cuh"
#include "br_kernel.cuh"
#include "engine_internal.h"

namespace arx {
namespace {

constexpr int kWatchdogWarps = 4;

// result[w]: 1 = warp w's wait completed, 2 = it gave up.
__global__ void __launch_bounds__(32 * kWatchdogWarps, 1)
    watchdog_kernel(int post_token, long long limit, unsigned int *status, int *result) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    clu::mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (post_token && threadIdx.x == 0) clu::mbar_arrive_cta(&bar);
  const int warp = threadIdx.x >> 5;
  volatile int *ab = &abort_flag;
  const bool ok = (warp & 1) ? clu::mbar_wait(&bar, 0u, ab, status, limit)
                             : br::mbar_wait(&bar, 0u, ab, status, limit);
  if ((threadIdx.x & 31) == 0) result[warp] = ok ? 1 : 2;
}

}  // namespace
}  // namespace arx

using namespace arx;

extern "C" int arx_watchdog_selftest(int post_token, long long limit_cycles, int *waits_given_up) {
  if (limit_cycles < 1000 || limit_cycles > br::kWaitCycles)
    return fail(ARX_EINVAL, "limit_cycles %lld outside [1000, %lld]", limit_cycles, br::kWaitCycles);
  Engine &E = eng();
  std::lock_guard<std::mutex> lk(E.mu);
  int rc = ensure_init(E);
  if (rc) return rc;
  rc = read_status(E, E.stream);  // an expiry of an earlier call is not this test's
  if (rc) return rc;
  int *d_res = nullptr;
  cudaError_t e = cudaMalloc(&d_res, kWatchdogWarps * sizeof(int));
  if (e != cudaSuccess) return fail(ARX_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  int h_res[kWatchdogWarps] = {};
  e = cudaMemsetAsync(d_res, 0, sizeof(h_res), E.stream);
  if (e == cudaSuccess) {
    watchdog_kernel<<<1, 32 * kWatchdogWarps, 0, E.stream>>>(post_token, limit_cycles, E.status, d_res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_res, d_res, sizeof(h_res), cudaMemcpyDeviceToHost, E.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
  cudaFree(d_res);
  if (e != cudaSuccess) return fail(ARX_ECUDA, "watchdog self-test: %s", cudaGetErrorString(e));
  int gave_up = 0;
  for (int w = 0; w < kWatchdogWarps; ++w) {
    if (h_res[w] != 1 && h_res[w] != 2) return fail(ARX_ECUDA, "watchdog self-test: warp %d did not report", w);
    gave_up += h_res[w] == 2;
  }
  if (waits_given_up) *waits_given_up = gave_up;
  return read_status(E, E.stream);
}
