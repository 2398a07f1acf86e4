// probe.cu -- throughput of the integer pipes that bound the blind rotation:
// the measured side of its ALU roofline.
//
// Each probe kernel runs K independent dependency chains per thread for ITERS
// iterations with two 512-thread CTAs (32 warps) per SM, and times itself with
// clock64; the chains are nonlinear so that the compiler cannot fold them.  The
// result is lane operations per clock per SM:
//   0 IMAD (32-bit multiply-add, low word)       1 IMAD.HI (__umulhi)
//   2 IMAD.WIDE (32 x 32 -> 64-bit multiply-add) 3 plain ALU chain (one unit =
//     IADD3 + SHF + LOP)
//   4 Shoup butterfly modulo a 27-bit prime (the CRT arithmetic of the kernels)
//   5 Montgomery multiply-accumulate modulo a 27-bit prime (the key MAC)
//   6 butterfly modulo the paper's 64-bit prime 2^64 - 2^32 + 1 (Sec. 5.4),
//     multiplied by 2^64 = 2^32 - 1 and 2^96 = -1 (mod p) reduction
// No counterpart in the paper: it measures the device the roofline refers to.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/arx.h"

namespace arx {
namespace {

constexpr int kIters = 1024;
constexpr int kChains = 8;
constexpr int kProbeThreads = 512;
constexpr uint32_t kProbeQ = 134215681u;  // a 27-bit NTT prime (= 1 mod 2048)

__device__ __forceinline__ uint64_t gold_mul(uint64_t a, uint64_t b) {
  const uint64_t lo = a * b, hi = __umul64hi(a, b);
  const uint64_t h0 = hi & 0xffffffffull, h1 = hi >> 32;
  uint64_t r = lo - h1;                // 2^96 = -1
  if (lo < h1) r -= 0xffffffffull;     // + p = - (2^32 - 1) mod 2^64
  const uint64_t t = (h0 << 32) - h0;  // h0 2^64 = h0 (2^32 - 1)
  uint64_t s = r + t;
  if (s < t) s += 0xffffffffull;       // carry out: + 2^64 = + (2^32 - 1)
  return s;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(const uint32_t *in, uint32_t *out, long long *cyc) {
  const uint32_t w = in[0] | 1u, wp = in[1], c = in[2];
  uint32_t x[kChains], y[kChains];
  uint64_t gx[OP == 6 ? kChains : 1], gy[OP == 6 ? kChains : 1];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = in[3 + k] + threadIdx.x * 7u;
    y[k] = x[k] * 3u + 1u;
    if (OP == 6) {
      gx[k] = ((uint64_t)x[k] << 32) | y[k];
      gy[k] = ((uint64_t)y[k] << 32) ^ x[k];
    }
  }
  const uint64_t gw = ((uint64_t)wp << 32) | w, gp = 0xffffffff00000001ull;
  const long long t0 = clock64();
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) x[k] = x[k] * x[k] + c;
      if (OP == 1) x[k] = __umulhi(x[k], x[k] | w);
      if (OP == 2) {
        const uint64_t t = (uint64_t)x[k] * x[k] + c;
        x[k] = (uint32_t)(t >> 32) + (uint32_t)t;
      }
      if (OP == 3) x[k] = (x[k] + y[k] + c) ^ (x[k] >> 3);
      if (OP == 4) {
        const uint32_t t = w * y[k] - __umulhi(wp, y[k]) * kProbeQ;
        const uint32_t xn = x[k] + t;
        y[k] = x[k] - t + 2u * kProbeQ;
        x[k] = xn;
      }
      if (OP == 5) {
        const uint64_t t = (uint64_t)y[k] * w;
        const uint32_t m = (uint32_t)t * 0x8a2a0fffu;
        x[k] += (uint32_t)((t + (uint64_t)m * kProbeQ) >> 32);
        y[k] ^= x[k];
      }
      if (OP == 6) {
        const uint64_t t = gold_mul(gy[k], gw);
        uint64_t xn = gx[k] + t;
        if (xn < t || xn >= gp) xn -= gp;
        gy[k] = gx[k] >= t ? gx[k] - t : gx[k] - t + gp;
        gx[k] = xn;
      }
    }
  }
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= OP == 6 ? (uint32_t)(gx[k] ^ (gy[k] >> 32)) : (x[k] ^ y[k]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int OP>
cudaError_t run_probe(int sms, const uint32_t *din, uint32_t *dout, long long *dcyc, double *rate) {
  const int blocks = 2 * sms;
  for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
    probe_kernel<OP><<<blocks, kProbeThreads>>>(din, dout, dcyc);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
  }
  std::vector<long long> c(blocks);
  cudaError_t e = cudaMemcpy(c.data(), dcyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  double avg = 0;
  for (long long v : c) avg += (double)v;
  avg /= blocks;
  *rate = 2.0 * kProbeThreads * kIters * kChains / avg;  // lane operations per clock per SM
  return cudaSuccess;
}

}  // namespace
}  // namespace arx

// rate[i] for probe i < count (up to 7, listed in the header above).  Synchronous;
// uses the current device and the default stream.  ARX_OK, ARX_EINVAL or
// ARX_ECUDA.
extern "C" int arx_probe_alu(double *rate, int count) {
  using namespace arx;
  if (!rate || count < 0) return ARX_EINVAL;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) return ARX_ECUDA;
  const uint32_t h[16] = {0x9e3779b9u, 2147480000u, 777u, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13};
  uint32_t *din = nullptr, *dout = nullptr;
  long long *dcyc = nullptr;
  cudaError_t e = cudaMalloc(&din, sizeof(h));
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint32_t) * 2 * sms * kProbeThreads);
  if (e == cudaSuccess) e = cudaMalloc(&dcyc, sizeof(long long) * 2 * sms);
  if (e == cudaSuccess) e = cudaMemcpy(din, h, sizeof(h), cudaMemcpyHostToDevice);
  cudaError_t (*probes[7])(int, const uint32_t *, uint32_t *, long long *, double *) = {
      run_probe<0>, run_probe<1>, run_probe<2>, run_probe<3>, run_probe<4>, run_probe<5>, run_probe<6>};
  for (int i = 0; i < count && i < 7 && e == cudaSuccess; ++i) e = probes[i](sms, din, dout, dcyc, rate + i);
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dcyc);
  return e == cudaSuccess ? ARX_OK : ARX_ECUDA;
}
