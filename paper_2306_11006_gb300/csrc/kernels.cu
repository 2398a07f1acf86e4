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

size_t br_smem_h1(int GT, int L);
size_t br_smem_h2(int GT, int L);
size_t br_smem_h3(int GT, int L);
size_t br_smem_h4(int GT, int L);
size_t br_smem_h6(int GT, int L);
int br_occupancy_h1(int GT, int L);
int br_occupancy_h2(int GT, int L);
int br_occupancy_h3(int GT, int L);
int br_occupancy_h4(int GT, int L);
int br_occupancy_h6(int GT, int L);

namespace {

// ---------------------------------------------------------------------------
// Key load: one warp per (key polynomial, prime).  Coefficients are read as
// centred Torus32 integers, transformed, scaled by N^-1 2^32 (the inverse
// transform's 1/N and the Montgomery factor of the MAC), fully reduced, and
// stored in the per-lane order the MAC reads: [e/4][lane][e%4].
// ---------------------------------------------------------------------------
__device__ void bsk_poly_to_ntt(const uint32_t *src, uint32_t *dst, uint32_t *xbuf, const TwiddleConst &tc,
                                const TwiddleGlobal *tg, int P, int lane) {
  const PrimeRT pr = prime_rt(P, tc);
  const uint32_t q = pr.q;
  constexpr uint32_t kScale = 1u << 22;  // N^-1 2^32 mod q = 2^22
  uint32_t x[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    const int32_t v = (int32_t)src[lane + 32 * e];
    const int32_t m = v % (int32_t)q;
    x[e] = (uint32_t)(m < 0 ? m + (int32_t)q : m);
  }
  ntt_fwd<0>(x, xbuf, tc.fwd1[P], tg->fwd2[P], pr, lane);
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    const uint32_t v = x[e] % q;
    dst[(e >> 2) * 128 + lane * 4 + (e & 3)] = (uint32_t)((uint64_t)v * kScale % q);
  }
}

__global__ void bsk_to_ntt_kernel(const uint32_t *__restrict__ bsk, int n, int rows, uint32_t *__restrict__ out,
                                  const __grid_constant__ TwiddleConst tc, const TwiddleGlobal *tg) {
  __shared__ __align__(16) uint32_t xbuf[4][kXpose];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * 4 + warp;
  const long long total = (long long)n * rows * 2 * 2;
  if (wid >= total) return;
  const long long poly = wid >> 1;  // (i, r, c) in [0, n rows 2)
  const int P = (int)(wid & 1);
  const long long ir = poly >> 1;   // i rows + r
  const int c = (int)(poly & 1);
  const uint32_t *src = bsk + poly * kN;
  uint32_t *dst = out + ir * kChunkWords + (size_t)(c * 2 + P) * kN;
  bsk_poly_to_ntt(src, dst, xbuf[warp], tc, tg, P, lane);
}

// ---------------------------------------------------------------------------
// Key switch as a coalesced gather-accumulate (Fig. 2 "KeySwitch (Accum)"):
// out = (0, ..., 0, b') - sum_i sum_j KSK[i][j][digit_ij].  A gate's N x t = 8192
// key rows are split over `splits` CTAs (narrow waves spread one gate over many
// SMs); thread t owns output words 4t .. 4t+3 and reads them with 128-bit loads,
// two input coefficients (16 rows) in flight per iteration.  With splits > 1
// each CTA writes its partial sum to scratch; the CTA that finishes last (per-gate
// atomic counter, no waiting) adds the partials, writes the output and re-arms the
// counter.  The MUX sum (two extracted samples plus 1/8) and the linear gates are
// folded in.
// ---------------------------------------------------------------------------
constexpr int kKsThreads = 160;             // 160 x 4 words >= 632
constexpr int kKsVec = kKsRowStride / 4;    // 158 uint4 per row

// acc -= the key rows selected by the base-4 digits of positions [i0, i1) of lwe
// (each rounded to 16 bits), columns 4 t .. 4 t + 3.  The CTA first writes the
// row of every (position, digit) pair into roff (uint4 offsets; digit 0: the
// zero row after the key rows, so that every load is unconditional): the digit
// and address arithmetic is done once per CTA instead of once per thread, and
// the loop is a broadcast shared-memory read, one load and four subtractions per
// row, 16 rows in flight (threads t >= kKsVec read in bounds and discard what
// they read).
__device__ __forceinline__ void ks_accumulate(uint4 &acc, const uint4 *__restrict__ ksk, const uint32_t *lwe,
                                              uint32_t *roff, int i0, int i1, int t) {
  const int cnt = (i1 - i0) * 8;  // a multiple of 16 (kN / S >= 16)
  for (int e = t; e < cnt; e += kKsThreads) {
    const int i = i0 + (e >> 3), j = (e & 7) + 1;
    const uint32_t y = lwe[i] + (1u << 15);  // round to 16 bits
    const uint32_t v = (y >> (32 - 2 * j)) & 3u;
    roff[e] = v ? (uint32_t)(((i * 8 + (j - 1)) * 3 + (int)(v - 1)) * kKsVec) : (uint32_t)(kN * 8 * 3 * kKsVec);
  }
  __syncthreads();
  const uint4 *kt = ksk + t;
#pragma unroll 1
  for (int e = 0; e < cnt; e += 16) {
    uint4 r[16];
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const uint4 o = reinterpret_cast<const uint4 *>(roff + e)[q4];
      r[4 * q4 + 0] = __ldg(kt + o.x);
      r[4 * q4 + 1] = __ldg(kt + o.y);
      r[4 * q4 + 2] = __ldg(kt + o.z);
      r[4 * q4 + 3] = __ldg(kt + o.w);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      acc.x -= r[q].x;
      acc.y -= r[q].y;
      acc.z -= r[q].z;
      acc.w -= r[q].w;
    }
  }
}

__global__ void __launch_bounds__(kKsThreads, 4) ks_kernel(const __grid_constant__ KsArgs args) {
  __shared__ uint32_t lwe[kN + 1];
  __shared__ __align__(16) uint32_t roff[kN * 8];  // key row of each (position, digit) pair of this CTA
  __shared__ int last;
  const int S = args.splits;
  const int gate = blockIdx.x / S, split = blockIdx.x - gate * S;
  const KsJob jb = args.jobs[gate];
  const int n = args.n;
  const int t = threadIdx.x;
  uint32_t *dst = args.out + (size_t)jb.out * args.out_stride;
  if (jb.type == kGateNot || jb.type == kGateCopy || jb.type == kGateConst0 || jb.type == kGateConst1) {
    if (split) return;
    const uint32_t *src = args.wires + (size_t)jb.ia * kWireStride;
    for (int k = t; k <= n; k += kKsThreads) {
      uint32_t v;
      if (jb.type == kGateNot) v = 0u - src[k];
      else if (jb.type == kGateCopy) v = src[k];
      else v = k < n ? 0u : (jb.type == kGateConst1 ? kMu : 0u - kMu);
      dst[k] = v;
    }
    return;
  }
  const int i0 = split * (kN / S), i1 = i0 + kN / S;
  const uint32_t *s0 = args.br_out + (size_t)jb.j0 * kOutStride;
  const uint32_t *s1 = args.br_out + (size_t)jb.j1 * kOutStride;
  const bool mux = jb.type == kGateMux;
  for (int k = i0 + t; k < i1; k += kKsThreads) lwe[k] = mux ? s0[k] + s1[k] : s0[k];
  if (t == 0) lwe[kN] = mux ? s0[kN] + s1[kN] + kMu : s0[kN];
  __syncthreads();
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  if (split == 0 && 4 * t <= n && n < 4 * t + 4) {
    const uint32_t b = lwe[kN];
    if (n == 4 * t) acc.x = b; else if (n == 4 * t + 1) acc.y = b; else if (n == 4 * t + 2) acc.z = b; else acc.w = b;
  }
  const bool live = t < kKsVec;
  ks_accumulate(acc, reinterpret_cast<const uint4 *>(args.ksk[jb.key]), lwe, roff, i0, i1, t);
  if (S == 1) {
    if (live) {
      if (4 * t + 0 <= n) dst[4 * t + 0] = acc.x;
      if (4 * t + 1 <= n) dst[4 * t + 1] = acc.y;
      if (4 * t + 2 <= n) dst[4 * t + 2] = acc.z;
      if (4 * t + 3 <= n) dst[4 * t + 3] = acc.w;
    }
    return;
  }
  uint4 *part = reinterpret_cast<uint4 *>(args.partial) + (size_t)gate * S * kKsVec;
  if (live) part[(size_t)split * kKsVec + t] = acc;
  __threadfence();
  __syncthreads();
  if (t == 0) last = atomicAdd(args.counters + gate, 1u) == (unsigned)(S - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (live) {
    // eight loads in flight, eight partial sums (u32 additions mod 2^32 in any order)
    uint4 s8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] = make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < S; q0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (q0 + u < S) {
          const uint4 v = __ldcg(part + (size_t)(q0 + u) * kKsVec + t);
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
  if (t == 0) args.counters[gate] = 0u;
}

__global__ void gather_kernel(const uint32_t *__restrict__ wires, const uint32_t *__restrict__ idx, int count,
                              int n, uint32_t *__restrict__ dst, int dst_stride) {
  const int o = blockIdx.x;
  if (o >= count) return;
  const uint32_t *src = wires + (size_t)idx[o] * kWireStride;
  for (int k = threadIdx.x; k <= n; k += blockDim.x) dst[(size_t)o * dst_stride + k] = src[k];
}

}  // namespace

cudaError_t launch_bsk_to_ntt(const uint32_t *bsk_coef, int n, int rows, uint32_t *bsk_ntt, const TwiddleConst &tc,
                              const TwiddleGlobal *tg, cudaStream_t st) {
  const long long warps = (long long)n * rows * 4;
  const int blocks = (int)((warps + 3) / 4);
  bsk_to_ntt_kernel<<<blocks, 128, 0, st>>>(bsk_coef, n, rows, bsk_ntt, tc, tg);
  return cudaGetLastError();
}

int ks_splits(int num_jobs, int sms) {
  // aim at about four CTAs per SM; splits divide N and stay in 1..64
  int s = 1;
  while (s < 64 && (long long)num_jobs * s < 4LL * sms) s *= 2;
  return s;
}

cudaError_t launch_ks(const KsArgs &args, int num_jobs, cudaStream_t st) {
  if (num_jobs <= 0) return cudaSuccess;
  if (args.splits < 1 || args.splits > 64 || (kN % args.splits) || (args.splits > 1 && (!args.partial || !args.counters)))
    return cudaErrorInvalidValue;
  ks_kernel<<<num_jobs * args.splits, kKsThreads, 0, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_gather(const uint32_t *wires, const uint32_t *idx, int count, int n, uint32_t *dst,
                          int dst_stride, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  gather_kernel<<<count, 128, 0, st>>>(wires, idx, count, n, dst, dst_stride);
  return cudaGetLastError();
}

size_t br_smem(BrShape s) {
  if (s.H == kClusterH) return s.GT == 1 ? br_cluster_smem() : 0;
  if (s.H == kCluster4H) return s.GT == 1 ? br_cluster4_smem() : 0;
  if (s.H == kCluster8H) return s.GT == 1 ? br_cluster8_smem() : 0;
  if (s.H == kCluster8L2H) return s.GT == 1 ? br_cluster8_l2_smem() : 0;
  if (s.H == kCluster16H) return s.GT == 1 ? br_cluster16_smem() : 0;
  if (s.H == kCluster16L2H) return s.GT == 1 ? br_cluster16_l2_smem() : 0;
  const int L = s.H > kGadget2 ? 2 : 3, H = s.H > kGadget2 ? s.H - kGadget2 : s.H;
  switch (H) {
    case 1: return br_smem_h1(s.GT, L);
    case 2: return br_smem_h2(s.GT, L);
    case 3: return br_smem_h3(s.GT, L);
    case 4: return br_smem_h4(s.GT, L);
    case 6: return br_smem_h6(s.GT, L);
    default: return 0;
  }
}

bool br_shape_supported(BrShape s) { return br_smem(s) != 0; }

int br_occupancy(BrShape s) {
  if (s.H == kClusterH) return s.GT == 1 ? br_cluster_occupancy() : 0;
  if (s.H == kCluster4H) return s.GT == 1 ? br_cluster4_occupancy() : 0;
  if (s.H == kCluster8H) return s.GT == 1 ? br_cluster8_occupancy() : 0;
  if (s.H == kCluster8L2H) return s.GT == 1 ? br_cluster8_l2_occupancy() : 0;
  if (s.H == kCluster16H) return s.GT == 1 ? br_cluster16_occupancy() : 0;
  if (s.H == kCluster16L2H) return s.GT == 1 ? br_cluster16_l2_occupancy() : 0;
  const int L = s.H > kGadget2 ? 2 : 3, H = s.H > kGadget2 ? s.H - kGadget2 : s.H;
  switch (H) {
    case 1: return br_occupancy_h1(s.GT, L);
    case 2: return br_occupancy_h2(s.GT, L);
    case 3: return br_occupancy_h3(s.GT, L);
    case 4: return br_occupancy_h4(s.GT, L);
    case 6: return br_occupancy_h6(s.GT, L);
    default: return 0;
  }
}

cudaError_t launch_br(const BrArgs &args, BrShape s, int grid, cudaStream_t st) {
  if (args.num_jobs <= 0) return cudaSuccess;
  if (s.H == kClusterH) return s.GT == 1 ? launch_br_cluster(args, grid, st) : cudaErrorInvalidValue;
  if (s.H == kCluster4H) return s.GT == 1 ? launch_br_cluster4(args, grid, st) : cudaErrorInvalidValue;
  if (s.H == kCluster8H) return s.GT == 1 ? launch_br_cluster8(args, grid, st) : cudaErrorInvalidValue;
  if (s.H == kCluster8L2H) return s.GT == 1 ? launch_br_cluster8_l2(args, grid, st) : cudaErrorInvalidValue;
  if (s.H == kCluster16H) return s.GT == 1 ? launch_br_cluster16(args, grid, st) : cudaErrorInvalidValue;
  if (s.H == kCluster16L2H) return s.GT == 1 ? launch_br_cluster16_l2(args, grid, st) : cudaErrorInvalidValue;
  const int L = s.H > kGadget2 ? 2 : 3, H = s.H > kGadget2 ? s.H - kGadget2 : s.H;
  switch (H) {
    case 1: return launch_br_h1(args, s.GT, L, grid, st);
    case 2: return launch_br_h2(args, s.GT, L, grid, st);
    case 3: return launch_br_h3(args, s.GT, L, grid, st);
    case 4: return launch_br_h4(args, s.GT, L, grid, st);
    case 6: return launch_br_h6(args, s.GT, L, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace arx
