// br_cluster_common.cuh -- device helpers shared by the cluster blind-rotation
// kernels (two-, four-, eight- and sixteen-CTA): cluster and mbarrier
// primitives, bulk copies between CTAs, the CRT recombination, and the split
// (quarter) transforms.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "arx_device.cuh"

namespace arx {
namespace clu {

constexpr long long kWaitCycles = 4000000000ll;  // bound of every mbarrier wait (about 2 s)
// rounding half of the 21-bit gadget plus the +64 offset of each 7-bit digit
constexpr uint32_t kDecOffset = (1u << 10) + (64u << 25) + (64u << 18) + (64u << 11);

constexpr uint32_t pow_mod(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1;
  b %= m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return (uint32_t)r;
}
constexpr uint32_t kQ0InvQ1 = pow_mod(kQ0, kQ1 - 2, kQ1);
constexpr uint32_t kQ0InvQ1Shoup = (uint32_t)(((uint64_t)kQ0InvQ1 << 32) / kQ1);
constexpr uint64_t kM = (uint64_t)kQ0 * kQ1;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Bulk copy from this CTA's shared memory into a peer CTA's shared memory; the
// bytes complete on the peer's mbarrier.  Both addresses 16-byte aligned, size a
// multiple of 16.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, const void *src, uint32_t bytes,
                                            uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst_cluster),
      "r"(smem_u32(src)), "r"(bytes), "r"(bar_cluster)
      : "memory");
}

// Bulk element-wise u32 addition of this CTA's shared memory into a peer CTA's
// shared memory (performed by the bulk copy engine); the bytes complete on the
// peer's mbarrier.  Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_add_s2peer(uint32_t dst_cluster, const void *src, uint32_t bytes,
                                                uint32_t bar_cluster) {
  asm volatile(
      "cp.reduce.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes.add.u32 [%0], [%1], %2, [%3];" ::"r"(
          dst_cluster),
      "r"(smem_u32(src)), "r"(bytes), "r"(bar_cluster)
      : "memory");
}

// Orders this thread's generic-proxy writes to shared memory before later
// async-proxy (bulk copy) reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}


__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of a phase (mbarrier.test_wait).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: a phase that has already completed returns at once (the abort
// flag is read only on the slow path, where a wait could otherwise last);
// returns false (and flags the CTA and the device status) once `limit` clock64
// cycles have passed (kWaitCycles in every blind-rotation kernel).  test_first:
// test the phase without blocking before the first blocking try_wait (a probe
// measured a try_wait on a phase completed earlier at ~200 cycles, a test_wait
// ~55 cycles less; used on the sixteen-CTA kernel's critical-path waits).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *status, long long limit = kWaitCycles,
                                          bool test_first = false) {
  if (test_first && mbar_test_wait(bar, parity)) return true;
  if (mbar_try_wait(bar, parity)) return true;
  if (*abort_flag) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(status, kDevTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void named_bar_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void named_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ uint32_t modswitch(uint32_t x) { return (x + (1u << 20)) >> 21; }

// Garner recombination of (x0 mod q0, x1 mod q1), each in [0, 2q), to the
// centred integer mod 2^32 (the reasoning is at br::crt_torus).
__device__ __forceinline__ uint32_t crt_torus(uint32_t x0, uint32_t x1) {
  const uint32_t d = x1 + 3u * kQ1 - x0;
  const uint32_t k = csub(shoup_mul(kQ0InvQ1, kQ0InvQ1Shoup, d, kQ1), kQ1);
  const uint32_t r = kQ0 * k + x0;
  return k >= kQ1 / 2 ? r - (uint32_t)kM : r;
}

// Word offset of position p in a buffer of 32-word rows: the 16-byte chunks of
// row p >> 5 are XOR-swizzled by the row index (see swz), so that storing 32
// consecutive positions, and 128-bit loads of 16 (or 8) consecutive positions per
// lane with the block order below, are free of bank conflicts.
__device__ __forceinline__ int swp(int p) { return swz(p >> 5, p & 31); }

// Butterfly between lanes (partner lane ^ mask): the lower lane holds x, the
// upper lane y; returns x + z y or x - z y + 2q.
__device__ __forceinline__ uint32_t xlane_bfly(uint32_t v, uint2 z, bool upper, int mask, const PrimeRT &pr) {
  const uint32_t o = __shfl_xor_sync(0xffffffffu, v, mask);
  const uint32_t y = upper ? v : o, x = upper ? o : v;
  const uint32_t t = shoup_mul(z.x, z.y, y, pr.q);
  return upper ? x - t + pr.q2 : x + t;
}

// Word offsets for the quarter transposes (positions 0 .. 255): sw1 XORs bits
// 3-4 with bits 6-7, so that a[lane + 32 e] and a[(lane mod 8) + 8 e +
// 64 (lane / 8)] (one e per access) are both free of bank conflicts; swp (see
// above) pairs the latter with 128-bit accesses of 8 consecutive positions.
__device__ __forceinline__ int sw1(int p) { return p ^ (((p >> 6) & 3) << 3); }

// Inverse quarter transform (cyclic Cooley-Tukey DIT with omega^-1) of spectral
// positions 256 Q .. 256 Q + 255, all stages but the last two (half-lengths
// 1 .. 128), in three register passes joined by two shared-memory transposes.
// In: x[e] = position 256 Q + 8 lane + e (< 12 q).  Out: x[e] = position
// lane + 32 e of the quarter's natural-order result (< 28 q).
__device__ __forceinline__ void inv_quarter(uint32_t (&x)[8], uint32_t *xbuf, const uint2 *tw1,
                                            const uint2 *__restrict__ twc, const uint2 *__restrict__ tw2,
                                            const PrimeRT &pr, int lane) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {  // half-lengths 1, 2, 4 on a[8 lane + e]: bits 0 .. 2 of e
    const int hh = 1 << t;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hh) == 0) ct_bfly(x[e], x[e + hh], tw1[(hh - 1) + (e & (hh - 1))], pr);
  }
  const int pc = (lane & 7) + 64 * (lane >> 3);  // middle pass: position pc + 8 e
  __syncwarp();
  uint4 *xb4 = reinterpret_cast<uint4 *>(xbuf);
#pragma unroll
  for (int c = 0; c < 2; ++c)
    xb4[swp(8 * lane + 4 * c) >> 2] = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[swp(pc + 8 * e)];
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // half-lengths 8, 16, 32: bits 0 .. 2 of e, per-lane twiddles
    const int hr = 1 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hr) == 0) ct_bfly(x[e], x[e + hr], __ldg(twc + ((hr - 1) + (e & (hr - 1))) * 32 + lane), pr);
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) xbuf[sw1(pc + 8 * e)] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[sw1(lane + 32 * e)];
#pragma unroll
  for (int s = 1; s < 3; ++s) {  // half-lengths 64, 128 on a[lane + 32 e]: bits 1, 2 of e
    const int hr = 1 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hr) == 0) ct_bfly(x[e], x[e + hr], __ldg(tw2 + ((hr - 1) + (e & (hr - 1))) * 32 + lane), pr);
  }
}

// Block of 8 positions that lane l holds after the forward quarter transform
// (makes the key loads and the product stores conflict-free).
__device__ __forceinline__ int fwd_block8(int lane) { return 4 * (lane & 7) + (lane >> 3); }

// The first two forward stages (distances 512 and 256) of spectral quarter Qf,
// taken while loading packed digit bytes: Dr[k] holds the bytes u = d + 64 of
// positions k, k+256, k+512, k+768 (one row).  Out: x[e] = the stage-2 output at
// p = lane + 32 e of the quarter (< 5q + 128); the -64 offsets ride on dc, dd.
__device__ __forceinline__ void load_first2(uint32_t (&x)[8], const uint32_t *Dr, uint2 z1, uint2 z23, int Qf,
                                            const PrimeRT &pr, int lane) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint32_t d4 = Dr[lane + 32 * e];
    const uint32_t t0 = shoup_mul(z1.x, z1.y, __byte_perm(d4, 0u, 0x4442u), pr.q);
    const uint32_t t1 = shoup_mul(z1.x, z1.y, __byte_perm(d4, 0u, 0x4443u), pr.q);
    const uint32_t u0 = __byte_perm(d4, 0u, 0x4440u), u1 = __byte_perm(d4, 0u, 0x4441u);
    // stage 1 (distance 512): the upper spectral half takes the differences
    const uint32_t a = Qf < 2 ? u0 + t0 + pr.dc : u0 - t0 + pr.q2 + pr.dd;
    const uint32_t b = Qf < 2 ? u1 + t1 + pr.dc : u1 - t1 + pr.q2 + pr.dd;
    // stage 2 (distance 256) with zeta[2] or zeta[3]
    const uint32_t t2 = shoup_mul(z23.x, z23.y, b, pr.q);
    x[e] = (Qf & 1) ? a - t2 + pr.q2 : a + t2;
  }
}

// Twist of quarter Q's inverse outputs before they are posted: x[e] (position
// k = lane + 32 e, < 28q) -> psi^-(c_Q k) x[e] in [0, 2q), c = (1, 5, 3, 7).
__device__ __forceinline__ void quarter_twist(uint32_t (&x)[8], const uint2 *__restrict__ fint, const PrimeRT &pr,
                                              int lane) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint2 f = __ldg(fint + lane + 32 * e);
    x[e] = shoup_mul(f.x, f.y, x[e], pr.q);
  }
}

// Last two inverse stages and the output twist for one prime: outputs k,
// k + 256, k + 512, k + 768 (each in [0, 2q), what crt_torus takes) from the
// twisted quarter outputs t = (psi^-k u_0, psi^-5k u_1, psi^-3k u_2,
// psi^-7k u_3) at k, each in [0, 2q).
__device__ __forceinline__ void inv_last(uint32_t (&o)[4], const uint32_t (&t)[4], uint2 m512, uint2 m256,
                                         uint32_t q) {
  const uint32_t s01 = t[0] + t[1], d01 = t[0] - t[1] + 2u * q;  // < 4q
  const uint32_t s23 = t[2] + t[3], d23 = t[2] - t[3] + 2u * q;
  o[0] = csub(csub(s01 + s23, 4u * q), 2u * q);
  o[2] = shoup_mul(m512.x, m512.y, s01 - s23 + 4u * q, q);
  const uint32_t e23 = shoup_mul(m512.x, m512.y, d23, q), e01 = shoup_mul(m512.x, m512.y, d01, q);
  o[1] = shoup_mul(m256.x, m256.y, d01 + e23, q);
  o[3] = shoup_mul(m256.x, m256.y, e01 + d23, q);
}

// Gadget digits of X^a ACC - ACC (Fig. 2), packed for the split forward
// transforms: D[r][k] holds the digit bytes d + 64 of row r at positions k,
// k + 256, k + 512, k + 768 (bytes 0 .. 3).
__device__ __forceinline__ void make_digits4(uint32_t *D, const uint32_t *A, uint32_t a, int tid, int nthreads) {
  for (int k = tid; k < 256; k += nthreads) {
    uint32_t pk[4];  // bytes 0, 1, 2: digits of rows 0, 1, 2 at position k + 256 m
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t pos = (uint32_t)k + 256u * m;
      const uint32_t j = (pos - a) & 2047u;
      uint32_t v = A[j & 1023u];
      v = (j & 1024u) ? 0u - v : v;
      const uint32_t y = v - A[pos] + kDecOffset;
      pk[m] = (y >> 25) | ((y >> 10) & 0x7F00u) | ((y << 5) & 0x7F0000u);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const uint32_t sel = (uint32_t)r | ((4u + r) << 4);
      D[r * 256 + k] = __byte_perm(__byte_perm(pk[0], pk[1], sel), __byte_perm(pk[2], pk[3], sel), 0x5410u);
    }
  }
}

// Rounding half of the 20-bit gadget of the variant l = 2, Bg = 2^10, plus the
// +512 offset of each 10-bit digit.
constexpr uint32_t kDecOffset2 = (1u << 11) + (512u << 22) + (512u << 12);

// Forward quarter transform with its per-lane twiddles in registers (zc: middle
// pass, lengths 32, 16, 8; zq: last pass, lengths 4, 2, 1; same entries as the
// global tables fwdc / fwdq).  In / out as the four-CTA kernel's fwd_quarter:
// x[e] at p = lane + 32 e (< 5q + 1024: 7- or 10-bit digits) -> spectral position 256 Q + 8 b + e,
// b = fwd_block8(lane) (< 22q).
__device__ __forceinline__ void fwd_quarter_r(uint32_t (&x)[8], uint32_t *xbuf, const uint2 *tw1,
                                              const uint2 (&zc)[7], const uint2 (&zq)[7], int Q, const PrimeRT &pr,
                                              int lane) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {  // lengths 128, 64 on a[lane + 32 e]: bits 2, 1 of e
    const int lr = 4 >> s, m = 4 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & lr) == 0) ct_bfly(x[e], x[e + lr], tw1[m + (m >> 2) * Q + e / (2 * lr)], pr);
  }
  const int pc = (lane & 7) + 64 * (lane >> 3);  // middle pass: position pc + 8 e
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) xbuf[sw1(lane + 32 * e)] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[sw1(pc + 8 * e)];
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // lengths 32, 16, 8: bits 2 .. 0 of e
    const int lr = 4 >> s, k0 = (1 << s) - 1;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & lr) == 0) ct_bfly(x[e], x[e + lr], zc[k0 + e / (2 * lr)], pr);
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) xbuf[swp(pc + 8 * e)] = x[e];
  __syncwarp();
  const uint4 *xb4 = reinterpret_cast<const uint4 *>(xbuf);
  const int b = fwd_block8(lane);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const uint4 v = xb4[swp(8 * b + 4 * c) >> 2];
    x[4 * c + 0] = v.x;
    x[4 * c + 1] = v.y;
    x[4 * c + 2] = v.z;
    x[4 * c + 3] = v.w;
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // lengths 4, 2, 1 on a[8 b + e]
    const int len = 4 >> s, k0 = (1 << s) - 1;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & len) == 0) ct_bfly(x[e], x[e + len], zq[k0 + e / (2 * len)], pr);
  }
}

// Inverse quarter transform with its per-lane twiddles in registers (zi: middle
// pass, half-lengths 8, 16, 32, entries of invc; z2: half-lengths 64 and 128,
// entries 1 .. 6 of inv2), followed by the quarter's share of the output twist
// (zt[e] = psi^-(c_Q k) at k = lane + 32 e).  In / out as inv_quarter +
// quarter_twist: x[e] = position 256 Q + 8 lane + e (< 12 q) -> the twisted
// natural-order result at lane + 32 e (< 2q).
__device__ __forceinline__ void inv_quarter_r(uint32_t (&x)[8], uint32_t *xbuf, const uint2 *tw1,
                                              const uint2 (&zi)[7], const uint2 (&z2)[6], const uint2 (&zt)[8],
                                              const PrimeRT &pr, int lane) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {  // half-lengths 1, 2, 4 on a[8 lane + e]
    const int hh = 1 << t;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hh) == 0) ct_bfly(x[e], x[e + hh], tw1[(hh - 1) + (e & (hh - 1))], pr);
  }
  const int pc = (lane & 7) + 64 * (lane >> 3);
  __syncwarp();
  uint4 *xb4 = reinterpret_cast<uint4 *>(xbuf);
#pragma unroll
  for (int c = 0; c < 2; ++c)
    xb4[swp(8 * lane + 4 * c) >> 2] = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[swp(pc + 8 * e)];
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // half-lengths 8, 16, 32
    const int hr = 1 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hr) == 0) ct_bfly(x[e], x[e + hr], zi[(hr - 1) + (e & (hr - 1))], pr);
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) xbuf[sw1(pc + 8 * e)] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[sw1(lane + 32 * e)];
#pragma unroll
  for (int s = 1; s < 3; ++s) {  // half-lengths 64, 128: entries (hr - 1) + j of inv2, stored from entry 1
    const int hr = 1 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & hr) == 0) ct_bfly(x[e], x[e + hr], z2[(hr - 2) + (e & (hr - 1))], pr);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = shoup_mul(zt[e].x, zt[e].y, x[e], pr.q);
}

// Gadget digits of X^a ACC - ACC (Fig. 2) with the first two forward stages
// (distances 512 and 256) of spectral quarter Qf taken at once, for each of NP
// primes: S[p][r][k] = the stage-2 output at position k of quarter Qf for row r
// in prime p (< 5q + 2^bits), from the digits u = d + 2^(bits-1) at k, k + 256,
// k + 512, k + 768 (the offsets ride on pr[p].dc, pr[p].dd).  L = 3: 7-bit
// digits (Bg = 2^7); L = 2: 10-bit digits (Bg = 2^10).  Run by all of a CTA's
// threads, it takes these stages off the forward warps' path (for L = 3 the
// values are those make_digits4 and load_first2 give).
template <int L, int NP>
__device__ __forceinline__ void make_stage2(uint32_t *S, const uint32_t *A, uint32_t a, const uint2 (&z1)[NP],
                                            const uint2 (&z23)[NP], int Qf, const PrimeRT (&pr)[NP], int tid,
                                            int nthreads) {
  static_assert(L == 2 || L == 3, "gadget length");
  for (int k = tid; k < 256; k += nthreads) {
    uint32_t u[4][L];  // u[m][r]: digit + offset of row r at position k + 256 m
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t pos = (uint32_t)k + 256u * m;
      const uint32_t j = (pos - a) & 2047u;
      uint32_t v = A[j & 1023u];
      v = (j & 1024u) ? 0u - v : v;
      if constexpr (L == 3) {
        const uint32_t y = v - A[pos] + kDecOffset;
        u[m][0] = y >> 25;
        u[m][1] = (y >> 18) & 0x7Fu;
        u[m][2] = (y >> 11) & 0x7Fu;
      } else {
        const uint32_t y = v - A[pos] + kDecOffset2;
        u[m][0] = y >> 22;
        u[m][1] = (y >> 12) & 0x3FFu;
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int r = 0; r < L; ++r) {
        const uint32_t t0 = shoup_mul(z1[p].x, z1[p].y, u[2][r], pr[p].q);
        const uint32_t t1 = shoup_mul(z1[p].x, z1[p].y, u[3][r], pr[p].q);
        // stage 1 (distance 512): the upper spectral half takes the differences
        const uint32_t s0 = Qf < 2 ? u[0][r] + t0 + pr[p].dc : u[0][r] - t0 + pr[p].q2 + pr[p].dd;
        const uint32_t s1 = Qf < 2 ? u[1][r] + t1 + pr[p].dc : u[1][r] - t1 + pr[p].q2 + pr[p].dd;
        // stage 2 (distance 256) with zeta[2] or zeta[3]
        const uint32_t t2 = shoup_mul(z23[p].x, z23[p].y, s1, pr[p].q);
        S[(p * L + r) * 256 + k] = (Qf & 1) ? s0 - t2 + pr[p].q2 : s0 + t2;
      }
    }
  }
}

// make_stage2 for one prime on a CTA of 256 threads whose thread k holds its
// column of ACC, acc4[m] = A[k + 256 m], in registers (the previous CMux's CRT
// pass computed them): only the rotated values come from shared memory.
template <int L>
__device__ __forceinline__ void make_stage2_col(uint32_t *S, const uint32_t *A, const uint32_t (&acc4)[4], uint32_t a,
                                                uint2 z1, uint2 z23, int Qf, const PrimeRT &pr, int k) {
  static_assert(L == 2 || L == 3, "gadget length");
  uint32_t u[4][L];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const uint32_t pos = (uint32_t)k + 256u * m;
    const uint32_t j = (pos - a) & 2047u;
    uint32_t v = A[j & 1023u];
    v = (j & 1024u) ? 0u - v : v;
    if constexpr (L == 3) {
      const uint32_t y = v - acc4[m] + kDecOffset;
      u[m][0] = y >> 25;
      u[m][1] = (y >> 18) & 0x7Fu;
      u[m][2] = (y >> 11) & 0x7Fu;
    } else {
      const uint32_t y = v - acc4[m] + kDecOffset2;
      u[m][0] = y >> 22;
      u[m][1] = (y >> 12) & 0x3FFu;
    }
  }
#pragma unroll
  for (int r = 0; r < L; ++r) {
    const uint32_t t0 = shoup_mul(z1.x, z1.y, u[2][r], pr.q);
    const uint32_t t1 = shoup_mul(z1.x, z1.y, u[3][r], pr.q);
    const uint32_t s0 = Qf < 2 ? u[0][r] + t0 + pr.dc : u[0][r] - t0 + pr.q2 + pr.dd;
    const uint32_t s1 = Qf < 2 ? u[1][r] + t1 + pr.dc : u[1][r] - t1 + pr.q2 + pr.dd;
    const uint32_t t2 = shoup_mul(z23.x, z23.y, s1, pr.q);
    S[r * 256 + k] = (Qf & 1) ? s0 - t2 + pr.q2 : s0 + t2;
  }
}

// crt_update for a CTA of 256 threads whose thread k keeps its column of ACC in
// acc4 (updated here and stored back to A for the other threads' rotations).
__device__ __forceinline__ void crt_update_col(uint32_t *A, uint32_t (&acc4)[4], const uint32_t *const (&post0)[4],
                                               int poff1, const BrArgs &args, int k) {
  uint32_t t[4], o0[4], o1[4];
#pragma unroll
  for (int Q = 0; Q < 4; ++Q) t[Q] = post0[Q][k];
  inv_last(o0, t, args.tc.psi512[0], args.tc.psi256[0], kQ0);
#pragma unroll
  for (int Q = 0; Q < 4; ++Q) t[Q] = post0[Q][k + poff1];
  inv_last(o1, t, args.tc.psi512[1], args.tc.psi256[1], kQ1);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    acc4[m] += crt_torus(o0[m], o1[m]);
    A[k + 256 * m] = acc4[m];
  }
}

// The inverse quarter transform on a pair of warps (w = 0, 1 of the pair, t =
// lane + 32 w): the butterflies, twiddles and stage order of inv_quarter_r, in
// four register passes of two stages on 4 values per lane (half-lengths 1-2,
// 4-8, 16-32, 64-128), joined by re-layouts through two shared buffers of 256
// words (XOR-swizzled by isw: every write and read conflict-free).  Stages up to
// half-length 64 stay inside the warp's half of the quarter (positions
// [128 w, 128 w + 128)), so the first two re-layouts need only __syncwarp; the
// last, before half-length 128, goes through the pair's named barrier.  Each
// butterfly's twiddle depends only on (h, p mod h); the per-lane values come
// from the same tables (load_inv_pair).
// In: x[e] at position 4 t + e (< 12 q); out: the twisted result at t + 64 e (< 2q).
struct InvPairTw {
  uint2 a[3];     // h = 1 (j = 0), h = 2 (j = 0, 1): inv1[0 .. 2]
  uint2 b4;       // h = 4, j = t & 3
  uint2 b8[2];    // h = 8, j = (t & 3) + 4 m
  uint2 c16;      // h = 16, j = t & 15
  uint2 c32[2];   // h = 32, j = (t & 15) + 16 m
  uint2 d64;      // h = 64, j = t
  uint2 d128[2];  // h = 128, j = t + 64 m
  uint2 tw[4];    // output twist of quarter Q at t + 64 e
};

__device__ __forceinline__ int isw(int p) { return p ^ ((p >> 2) & 31); }

__device__ __forceinline__ InvPairTw load_inv_pair(const BrArgs &args, int P, int Q, int t) {
  InvPairTw z;
#pragma unroll
  for (int k = 0; k < 3; ++k) z.a[k] = args.tc.inv1[P][k];
  z.b4 = args.tc.inv1[P][3 + (t & 3)];
  const uint2 *invc = args.tg->invc[P], *inv2 = args.tg->inv2[P];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    z.b8[m] = __ldg(invc + (t & 3) + 4 * m);
    const int j32 = (t & 15) + 16 * m, j128 = t + 64 * m;
    z.c32[m] = __ldg(invc + (3 + (j32 >> 3)) * 32 + (j32 & 7));
    z.d128[m] = __ldg(inv2 + (3 + (j128 >> 5)) * 32 + (j128 & 31));
  }
  z.c16 = __ldg(invc + (1 + ((t & 15) >> 3)) * 32 + (t & 7));
  z.d64 = __ldg(inv2 + (1 + (t >> 5)) * 32 + (t & 31));
#pragma unroll
  for (int e = 0; e < 4; ++e) z.tw[e] = __ldg(args.tg->fint[P][Q] + t + 64 * e);
  return z;
}

__device__ __forceinline__ void inv_quarter_pair(uint32_t (&x)[4], uint32_t *buf0, uint32_t *buf1,
                                                 const InvPairTw &z, const PrimeRT &pr, int t, int bar) {
  // pass A: half-lengths 1, 2 on positions 4 t + e
  ct_bfly(x[0], x[1], z.a[0], pr);
  ct_bfly(x[2], x[3], z.a[0], pr);
  ct_bfly(x[0], x[2], z.a[1], pr);
  ct_bfly(x[1], x[3], z.a[2], pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) buf0[isw(4 * t + e)] = x[e];
  __syncwarp();
  const int pb = (t & 3) + 16 * (t >> 2);  // pass B: positions pb + 4 e
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = buf0[isw(pb + 4 * e)];
  ct_bfly(x[0], x[1], z.b4, pr);
  ct_bfly(x[2], x[3], z.b4, pr);
  ct_bfly(x[0], x[2], z.b8[0], pr);
  ct_bfly(x[1], x[3], z.b8[1], pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) buf1[isw(pb + 4 * e)] = x[e];
  __syncwarp();
  const int pcc = (t & 15) + 64 * (t >> 4);  // pass C: positions pcc + 16 e
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = buf1[isw(pcc + 16 * e)];
  ct_bfly(x[0], x[1], z.c16, pr);
  ct_bfly(x[2], x[3], z.c16, pr);
  ct_bfly(x[0], x[2], z.c32[0], pr);
  ct_bfly(x[1], x[3], z.c32[1], pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) buf0[isw(pcc + 16 * e)] = x[e];
  named_bar(bar, 64);
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = buf0[isw(t + 64 * e)];  // pass D: positions t + 64 e
  ct_bfly(x[0], x[1], z.d64, pr);
  ct_bfly(x[2], x[3], z.d64, pr);
  ct_bfly(x[0], x[2], z.d128[0], pr);
  ct_bfly(x[1], x[3], z.d128[1], pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = shoup_mul(z.tw[e].x, z.tw[e].y, x[e], pr.q);
}

// Conflict-free word offsets of the forward pair's three re-layouts (checked
// for every access pattern below: 32 distinct banks per warp access).
__device__ __forceinline__ int s_ab(int p) { return p ^ (((p >> 6) & 1) << 4); }
__device__ __forceinline__ int s_bc(int p) { return p ^ (((p >> 5) & 1) << 2) ^ (((p >> 6) & 1) * 24); }
__device__ __forceinline__ int s_cd(int p) { return p ^ (((p >> 5) & 1) * 5) ^ (((p >> 6) & 1) * 10); }
// 16-byte slot of positions 4 j .. 4 j + 3 in the product buffers (own, oth and
// the receive slot): conflict-free for the forward pair's stores (j = 32 w +
// 8 (lane mod 4) + lane / 4), a one-warp forward transform's stores (j =
// 2 fwd_block8(lane) + c), the inverse pair's loads (j = t) and a one-warp
// inverse's loads (j = 2 lane + c); each warp's half of a pair (j < 32,
// j >= 32) stays contiguous for its bulk reduction.
__device__ __forceinline__ int s_j(int j) {
  return j ^ (((j >> 3) & 1) * 3) ^ (((j >> 4) & 1) * 4) ^ ((j >> 5) & 1);
}

// Per-thread twiddles of the forward quarter transform on a pair of warps.  The
// butterfly of length len on global spectral position g (bit len of g clear)
// takes zeta[512 / len + g / (2 len)], g = 256 Q + p; see fwd_quarter_pair for
// the positions each thread holds.
struct FwdPairTw {
  uint2 a128, a64[2];  // lengths 128, 64 (the same on every thread)
  uint2 b32, b16[2];   // 32, 16
  uint2 c8, c4[2];     // 8, 4
  uint2 d2, d1[2];     // 2, 1
};

__device__ __forceinline__ FwdPairTw load_fwd_pair(const BrArgs &args, int P, int Q, int w, int lane) {
  const uint2 *z = args.tg->fwdz[P];
  const int l4 = lane >> 4, l2 = lane >> 2, j = 32 * w + 8 * (lane & 3) + l2;
  FwdPairTw f;
  f.a128 = __ldg(z + 4 + Q);
  f.b32 = __ldg(z + 16 + 4 * Q + 2 * w + l4);
  f.c8 = __ldg(z + 64 + 16 * Q + 8 * w + l2);
  f.d2 = __ldg(z + 256 + 64 * Q + j);
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    f.a64[m] = __ldg(z + 8 + 2 * Q + m);
    f.b16[m] = __ldg(z + 32 + 8 * Q + 4 * w + 2 * l4 + m);
    f.c4[m] = __ldg(z + 128 + 32 * Q + 16 * w + 2 * l2 + m);
    f.d1[m] = __ldg(z + 512 + 128 * Q + 2 * j + m);
  }
  return f;
}

// Two stages on four values: lengths 2 d (pairs x0-x2, x1-x3, twiddle zo) and
// d (pairs x0-x1 with zi[0], x2-x3 with zi[1]).
__device__ __forceinline__ void fwd_radix4(uint32_t (&x)[4], uint2 zo, const uint2 (&zi)[2], const PrimeRT &pr) {
  ct_bfly(x[0], x[2], zo, pr);
  ct_bfly(x[1], x[3], zo, pr);
  ct_bfly(x[0], x[1], zi[0], pr);
  ct_bfly(x[2], x[3], zi[1], pr);
}

// The last eight forward stages (lengths 128 .. 1) of spectral quarter Q on a
// pair of warps (w = 0, 1 of the pair, t = lane + 32 w): the butterflies and
// twiddles of fwd_quarter_r in four register passes of two stages on 4 values
// per lane, joined by three re-layouts.  Pass A (lengths 128, 64) reads
// positions t + 64 e straight from the stage-2 row Dr; from pass B on, warp w
// holds positions [128 w, 128 w + 128), so only the A -> B re-layout (through
// the pair buffer pbuf, 256 words) needs the pair's named barrier; B -> C and
// C -> D go through the warp's own 256 words wbuf.  Out: x[e] = spectral
// position 256 Q + 4 j + e, j = 32 w + 8 (lane mod 4) + lane / 4 (< 22 q, as
// fwd_quarter_r).
__device__ __forceinline__ void fwd_quarter_pair(uint32_t (&x)[4], const uint32_t *Dr, uint32_t *pbuf,
                                                 uint32_t *wbuf, const FwdPairTw &z, const PrimeRT &pr, int w,
                                                 int lane, int bar) {
  const int t = lane + 32 * w;
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = Dr[t + 64 * e];
  fwd_radix4(x, z.a128, z.a64, pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) pbuf[s_ab(t + 64 * e)] = x[e];
  named_bar(bar, 64);
  const int pb = (lane & 15) + 64 * (lane >> 4);  // pass B: local positions pb + 16 e
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = pbuf[s_ab(128 * w + pb + 16 * e)];
  fwd_radix4(x, z.b32, z.b16, pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) wbuf[s_bc(pb + 16 * e)] = x[e];
  __syncwarp();
  const int pc = (lane & 3) + 16 * (lane >> 2);  // pass C: local positions pc + 4 e
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = wbuf[s_bc(pc + 4 * e)];
  fwd_radix4(x, z.c8, z.c4, pr);
#pragma unroll
  for (int e = 0; e < 4; ++e) wbuf[128 + s_cd(pc + 4 * e)] = x[e];
  __syncwarp();
  const int jl = 8 * (lane & 3) + (lane >> 2);  // pass D: local positions 4 jl + e
#pragma unroll
  for (int e = 0; e < 4; ++e) x[e] = wbuf[128 + s_cd(4 * jl + e)];
  fwd_radix4(x, z.d2, z.d1, pr);
}

// Last two inverse stages and CRT of both primes, then ACC += the Torus32
// result: post0[Q] holds quarter Q of prime 0 (twisted, natural order), prime 1
// lies poff1 words above it.
__device__ __forceinline__ void crt_update(uint32_t *A, const uint32_t *const (&post0)[4], int poff1,
                                           const BrArgs &args, int tid, int nthreads) {
  for (int k = tid; k < kN / 4; k += nthreads) {
    uint32_t t[4], o0[4], o1[4];
#pragma unroll
    for (int Q = 0; Q < 4; ++Q) t[Q] = post0[Q][k];
    inv_last(o0, t, args.tc.psi512[0], args.tc.psi256[0], kQ0);
#pragma unroll
    for (int Q = 0; Q < 4; ++Q) t[Q] = post0[Q][k + poff1];
    inv_last(o1, t, args.tc.psi512[1], args.tc.psi256[1], kQ1);
#pragma unroll
    for (int m = 0; m < 4; ++m) A[k + 256 * m] += crt_torus(o0[m], o1[m]);
  }
}

}  // namespace clu
}  // namespace arx
