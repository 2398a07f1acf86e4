// kernels.cu -- key load, key switch and gather kernels, and the shape dispatch
// of the blind-rotation kernel.
//
//   bsk_to_ntt_kernel   bootstrapping key -> NTT domain, once per key (the paper
//                       keeps the key resident and constant, Sec. 5.1)
//   ks_kernel           key switch (Fig. 2 "KeySwitch (Accum)") and the linear
//                       gates NOT / COPY / CONST (Sec. 2.2, Sec. 4.2)
//   gather_kernel       copies selected wires into an output array
#include <cuda_runtime.h>

#include <cstdint>

#include "arx_device.cuh"

namespace arx {

size_t br_smem_h1(int GT);
size_t br_smem_h2(int GT);
size_t br_smem_h3(int GT);
size_t br_smem_h6(int GT);
int br_occupancy_h1(int GT);
int br_occupancy_h2(int GT);
int br_occupancy_h3(int GT);
int br_occupancy_h6(int GT);

namespace {

// ---------------------------------------------------------------------------
// Key load: one warp per (key polynomial, prime).  Coefficients are read as
// centred Torus32 integers, transformed, scaled by N^-1 2^32 (the inverse
// transform's 1/N and the Montgomery factor of the MAC), fully reduced, and
// stored in the per-lane order the MAC reads: [e/4][lane][e%4].
// ---------------------------------------------------------------------------
template <int P>
__device__ void bsk_poly_to_ntt(const uint32_t *src, uint32_t *dst, uint32_t *xbuf, const TwiddleConst &tc,
                                const TwiddleGlobal *tg, int lane) {
  constexpr uint32_t q = Prime<P>::q;
  constexpr uint32_t kScale = 1u << 22;  // N^-1 2^32 mod q = 2^22
  uint32_t x[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    int32_t v = (int32_t)src[lane + 32 * e];
    int32_t m = v % (int32_t)q;
    x[e] = (uint32_t)(m < 0 ? m + (int32_t)q : m);
  }
  ntt_fwd<P>(x, xbuf, tc, tg->fwd2[P], lane);
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    uint32_t v = x[e] % q;
    dst[(e >> 2) * 128 + lane * 4 + (e & 3)] = (uint32_t)((uint64_t)v * kScale % q);
  }
}

__global__ void bsk_to_ntt_kernel(const uint32_t *__restrict__ bsk, int n, uint32_t *__restrict__ out,
                                  const __grid_constant__ TwiddleConst tc, const TwiddleGlobal *tg) {
  __shared__ uint32_t xbuf[4][kXpose];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * 4 + warp;
  const long long total = (long long)n * 12 * 2;
  if (wid >= total) return;
  const long long poly = wid >> 1;  // (i, r, c) in [0, n*12)
  const int P = (int)(wid & 1);
  const long long ir = poly >> 1;   // i*6 + r
  const int c = (int)(poly & 1);
  const uint32_t *src = bsk + poly * kN;
  uint32_t *dst = out + ir * kChunkWords + (size_t)(c * 2 + P) * kN;
  if (P == 0)
    bsk_poly_to_ntt<0>(src, dst, xbuf[warp], tc, tg, lane);
  else
    bsk_poly_to_ntt<1>(src, dst, xbuf[warp], tc, tg, lane);
}

// ---------------------------------------------------------------------------
// Key switch as a coalesced gather-accumulate: one CTA per gate, thread t owning
// output words t, t+128, ...; for each of the N x t (i, j) pairs the CTA reads
// the selected 632-word key row once.  The MUX sum (two extracted samples plus
// 1/8) and the linear gates are folded in.
// ---------------------------------------------------------------------------
constexpr int kKsThreads = 128;
constexpr int kKsPer = (kMaxLweN + 1 + kKsThreads - 1) / kKsThreads;  // 5

__global__ void __launch_bounds__(kKsThreads) ks_kernel(const __grid_constant__ KsArgs args) {
  __shared__ uint32_t lwe[kN + 1];
  const KsJob jb = args.jobs[blockIdx.x];
  const int n = args.n;
  const int t = threadIdx.x;
  uint32_t *dst = args.out + (size_t)jb.out * args.out_stride;
  if (jb.type == kGateNot || jb.type == kGateCopy) {
    const uint32_t *src = args.wires + (size_t)jb.ia * kWireStride;
    for (int k = t; k <= n; k += kKsThreads) dst[k] = jb.type == kGateNot ? 0u - src[k] : src[k];
    return;
  }
  if (jb.type == kGateConst0 || jb.type == kGateConst1) {
    for (int k = t; k <= n; k += kKsThreads) dst[k] = k < n ? 0u : (jb.type == kGateConst1 ? kMu : 0u - kMu);
    return;
  }
  const uint32_t *s0 = args.br_out + (size_t)jb.j0 * kOutStride;
  if (jb.type == kGateMux) {
    const uint32_t *s1 = args.br_out + (size_t)jb.j1 * kOutStride;
    for (int k = t; k <= kN; k += kKsThreads) lwe[k] = s0[k] + s1[k] + (k == kN ? kMu : 0u);
  } else {
    for (int k = t; k <= kN; k += kKsThreads) lwe[k] = s0[k];
  }
  __syncthreads();
  uint32_t acc[kKsPer];
#pragma unroll
  for (int m = 0; m < kKsPer; ++m) acc[m] = (t + m * kKsThreads == n) ? lwe[kN] : 0u;
  const uint32_t *__restrict__ ksk = args.ksk;
#pragma unroll 1
  for (int i = 0; i < kN; ++i) {
    const uint32_t y = lwe[i] + (1u << 15);  // round to 16 bits
#pragma unroll
    for (int j = 1; j <= 8; ++j) {
      const uint32_t v = (y >> (32 - 2 * j)) & 3u;
      const uint32_t *row = ksk + ((size_t)(i * 8 + (j - 1)) * 3 + (v ? v - 1 : 0)) * kKsRowStride;
#pragma unroll
      for (int m = 0; m < kKsPer; ++m) {
        const int k = t + m * kKsThreads;
        if (k <= n && v) acc[m] -= __ldg(row + k);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kKsPer; ++m) {
    const int k = t + m * kKsThreads;
    if (k <= n) dst[k] = acc[m];
  }
}

__global__ void gather_kernel(const uint32_t *__restrict__ wires, const uint32_t *__restrict__ idx, int count,
                              int n, uint32_t *__restrict__ dst, int dst_stride) {
  const int o = blockIdx.x;
  if (o >= count) return;
  const uint32_t *src = wires + (size_t)idx[o] * kWireStride;
  for (int k = threadIdx.x; k <= n; k += blockDim.x) dst[(size_t)o * dst_stride + k] = src[k];
}

}  // namespace

cudaError_t launch_bsk_to_ntt(const uint32_t *bsk_coef, int n, uint32_t *bsk_ntt, const TwiddleConst &tc,
                              const TwiddleGlobal *tg, cudaStream_t st) {
  const long long warps = (long long)n * 24;
  const int blocks = (int)((warps + 3) / 4);
  bsk_to_ntt_kernel<<<blocks, 128, 0, st>>>(bsk_coef, n, bsk_ntt, tc, tg);
  return cudaGetLastError();
}

cudaError_t launch_ks(const KsArgs &args, int num_jobs, cudaStream_t st) {
  if (num_jobs <= 0) return cudaSuccess;
  ks_kernel<<<num_jobs, kKsThreads, 0, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_gather(const uint32_t *wires, const uint32_t *idx, int count, int n, uint32_t *dst,
                          int dst_stride, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  gather_kernel<<<count, 128, 0, st>>>(wires, idx, count, n, dst, dst_stride);
  return cudaGetLastError();
}

size_t br_smem(BrShape s) {
  switch (s.H) {
    case 1: return br_smem_h1(s.GT);
    case 2: return br_smem_h2(s.GT);
    case 3: return br_smem_h3(s.GT);
    case 6: return br_smem_h6(s.GT);
    default: return 0;
  }
}

bool br_shape_supported(BrShape s) { return br_smem(s) != 0; }

int br_occupancy(BrShape s) {
  switch (s.H) {
    case 1: return br_occupancy_h1(s.GT);
    case 2: return br_occupancy_h2(s.GT);
    case 3: return br_occupancy_h3(s.GT);
    case 6: return br_occupancy_h6(s.GT);
    default: return 0;
  }
}

int br_threads(BrShape s) { return (2 * s.H * s.GT + 1) * 32; }

cudaError_t launch_br(const BrArgs &args, BrShape s, int grid, cudaStream_t st) {
  if (args.num_jobs <= 0) return cudaSuccess;
  switch (s.H) {
    case 1: return launch_br_h1(args, s.GT, grid, st);
    case 2: return launch_br_h2(args, s.GT, grid, st);
    case 3: return launch_br_h3(args, s.GT, grid, st);
    case 6: return launch_br_h6(args, s.GT, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace arx
