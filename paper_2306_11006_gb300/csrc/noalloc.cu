// noalloc.cu -- the key switch for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc while they run: a serving process that
// budgets every byte of HBM up front, a framework whose caching allocator must
// own all device memory, or a latency-critical loop where cudaMalloc / cudaFree
// would synchronise the device and stall other streams.  arx_keyswitch_noalloc
// gives them the split key-switch kernel without any allocation: the kernel's
// scratch (partial sums and per-gate counters) lives in the fixed-size device
// array below, which every GPU that loads the library holds until the process
// exits.  The caller passes the inputs (extracted LWE_N samples) and the output
// buffer; the key-switching key comes from a key set loaded earlier.
#include <cuda_runtime.h>

#include <mutex>

#include "arx_device.cuh"
#include "engine_internal.h"

namespace arx {
namespace {

constexpr int kNoallocMaxGates = ARX_KS_NOALLOC_MAX;  // gates per call
constexpr int kNoallocPartialRows = 1024;              // gates x splits rows of partial sums
constexpr int kKsThreadsNa = 160;                      // 160 x 4 words >= 632
constexpr int kKsVecNa = kKsRowStride / 4;             // 158 uint4 per row
constexpr size_t kNoallocWords = (size_t)kNoallocPartialRows * kKsRowStride + kNoallocMaxGates;
constexpr int kMaxDevices = 64;

// Partial sums [rows][632] followed by the per-gate counters [kNoallocMaxGates].
static __device__ __align__(256) uint32_t g_ks_scratch[kNoallocWords];

// Device address of g_ks_scratch, per device.  In host code the symbol's name is
// only a host-side stand-in, so the address is resolved with
// cudaGetSymbolAddress once per device, with that device current.
uint32_t *g_scratch_addr[kMaxDevices] = {};

// Same arithmetic as the key switch of the gate path: out = (0,...,0,b') minus
// the selected key rows, the N x 8 rows of a gate split over `splits` CTAs, the
// last CTA of a gate (per-gate counter) adding the partial sums.
__global__ void __launch_bounds__(kKsThreadsNa)
    ks_noalloc_kernel(const uint32_t *__restrict__ ksk_words, const uint32_t *__restrict__ lwe_N, int n,
                      uint32_t *__restrict__ out, int splits, uint32_t *partial_words, unsigned int *counters) {
  __shared__ uint32_t lwe[kN + 1];
  __shared__ int last;
  const int gate = blockIdx.x / splits, split = blockIdx.x - gate * splits;
  const int t = threadIdx.x;
  const int i0 = split * (kN / splits), i1 = i0 + kN / splits;
  const uint32_t *src = lwe_N + (size_t)gate * (kN + 1);
  for (int k = i0 + t; k < i1; k += kKsThreadsNa) lwe[k] = src[k];
  if (t == 0) lwe[kN] = src[kN];
  __syncthreads();
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  if (split == 0 && 4 * t <= n && n < 4 * t + 4) {
    const uint32_t b = lwe[kN];
    if (n == 4 * t) acc.x = b; else if (n == 4 * t + 1) acc.y = b; else if (n == 4 * t + 2) acc.z = b; else acc.w = b;
  }
  const bool live = t < kKsVecNa;
  const uint4 *__restrict__ ksk = reinterpret_cast<const uint4 *>(ksk_words);
#pragma unroll 1
  for (int i = i0; i < i1; i += 2) {
    uint4 r[16];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t y = lwe[i + u] + (1u << 15);
#pragma unroll
      for (int j = 1; j <= 8; ++j) {
        const uint32_t v = (y >> (32 - 2 * j)) & 3u;
        const size_t row = ((size_t)((i + u) * 8 + (j - 1)) * 3 + (v ? v - 1 : 0)) * kKsVecNa;
        r[u * 8 + j - 1] = (live && v) ? __ldg(ksk + row + t) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      acc.x -= r[q].x;
      acc.y -= r[q].y;
      acc.z -= r[q].z;
      acc.w -= r[q].w;
    }
  }
  uint32_t *dst = out + (size_t)gate * (n + 1);
  if (splits == 1) {
    if (live) {
      if (4 * t + 0 <= n) dst[4 * t + 0] = acc.x;
      if (4 * t + 1 <= n) dst[4 * t + 1] = acc.y;
      if (4 * t + 2 <= n) dst[4 * t + 2] = acc.z;
      if (4 * t + 3 <= n) dst[4 * t + 3] = acc.w;
    }
    return;
  }
  uint4 *part = reinterpret_cast<uint4 *>(partial_words) + (size_t)gate * splits * kKsVecNa;
  if (live) part[(size_t)split * kKsVecNa + t] = acc;
  __threadfence();
  __syncthreads();
  if (t == 0) last = atomicAdd(counters + gate, 1u) == (unsigned)(splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (live) {
    // eight loads in flight, eight partial sums (u32 additions mod 2^32 in any order)
    uint4 s8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] = make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < splits; q0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (q0 + u < splits) {
          const uint4 v = __ldcg(part + (size_t)(q0 + u) * kKsVecNa + t);
          s8[u].x += v.x;
          s8[u].y += v.y;
          s8[u].z += v.z;
          s8[u].w += v.w;
        }
      }
    }
    uint4 sum = s8[0];
#pragma unroll
    for (int u = 1; u < 8; ++u) {
      sum.x += s8[u].x;
      sum.y += s8[u].y;
      sum.z += s8[u].z;
      sum.w += s8[u].w;
    }
    if (4 * t + 0 <= n) dst[4 * t + 0] = sum.x;
    if (4 * t + 1 <= n) dst[4 * t + 1] = sum.y;
    if (4 * t + 2 <= n) dst[4 * t + 2] = sum.z;
    if (4 * t + 3 <= n) dst[4 * t + 3] = sum.w;
  }
  if (t == 0) counters[gate] = 0u;
}

}  // namespace
}  // namespace arx

using namespace arx;

// Allocation-free key switch; see include/arx.h for the contract.
extern "C" int arx_keyswitch_noalloc(const uint32_t *lwe_N, uint32_t *ct_out, size_t count, int keyset,
                                     void *stream) {
  Engine &E = eng();
  std::lock_guard<std::mutex> lk(E.mu);
  if (!E.ready) return fail(ARX_ENOKEYS, "no key set loaded");
  if (count == 0) return ARX_OK;
  if (count > (size_t)kNoallocMaxGates)
    return fail(ARX_EINVAL, "count %zu exceeds the allocation-free limit of %d gates", count, kNoallocMaxGates);
  if (!lwe_N || !ct_out) return fail(ARX_EINVAL, "null argument");
  if (!is_device_ptr(lwe_N) || !is_device_ptr(ct_out))
    return fail(ARX_EINVAL, "lwe_N and ct_out must be device memory");
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ARX_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(ARX_EINVAL, "device %d out of range", dev);
  if (!g_scratch_addr[dev]) {  // set-up, once per device, with that device current
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&g_scratch_addr[dev]), g_ks_scratch);
    if (e != cudaSuccess) {
      g_scratch_addr[dev] = nullptr;
      return fail(ARX_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
  }
  uint32_t *partial = g_scratch_addr[dev];
  unsigned int *counters = reinterpret_cast<unsigned int *>(partial + (size_t)kNoallocPartialRows * kKsRowStride);
  int splits = ks_splits((int)count, E.sms);
  while (splits > 1 && count * (size_t)splits > (size_t)kNoallocPartialRows) splits /= 2;
  cudaStream_t st = stream ? (cudaStream_t)stream : E.stream;
  // the counters must start at zero; the partial sums are overwritten before use
  e = cudaMemsetAsync(counters, 0, count * sizeof(unsigned int), st);
  if (e != cudaSuccess) return fail(ARX_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  ks_noalloc_kernel<<<(unsigned)(count * splits), kKsThreadsNa, 0, st>>>(ks->ksk, lwe_N, ks->n, ct_out, splits,
                                                                         partial, counters);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ARX_ECUDA, "ks_noalloc_kernel: %s", cudaGetErrorString(e));
  if (!stream) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ARX_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  }
  return ARX_OK;
}
