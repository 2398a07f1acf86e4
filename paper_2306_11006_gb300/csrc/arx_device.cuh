// arx_device.cuh -- device-side arithmetic for GB300 (sm_103a) CGGI bootstrapping.
//
// Exact negacyclic polynomial products (Sec. 2.2: "TGSW BK_i x TLWE temp" of
// Fig. 2) through number-theoretic transforms (Sec. 5.4 motivates the NTT over
// the FFT because it is exact).  The paper's A100 design used one 64-bit prime;
// here each product is carried modulo two 27-bit primes (CRT), so every modular
// multiply is a native 32-bit IMAD / IMAD.HI sequence:
//   q0 = 134215681, q1 = 134203393, both = 1 (mod 2048), q0 q1 > 2^53,
// while the exact products are bounded by 6 * 1024 * 64 * 2^31 < 2^50 for the
// gadget l = 3 (Bg = 2^7) and by 4 * 1024 * 512 * 2^31 = 2^52 for l = 2
// (Bg = 2^10): both below q0 q1 / 2 > 2^53.
//
// Warp-per-transform layout: a 1024-point transform is held by one warp, 32
// values per lane.  Forward (negacyclic Cooley-Tukey with merged twist, natural
// order in, bit-reversed order out): pass 1 (lengths 512..32) on
// x[e] = a[lane + 32 e] with warp-uniform twiddles from the kernel parameter bank,
// a swizzled shared-memory transpose, pass 2 (lengths 16..1) on a[32 lane + e]
// with per-lane twiddles.  Inverse of the warp transforms (ntt_inv_gs):
// Gentleman-Sande with the psi^-1 twist merged into its twiddles, bit-reversed
// in, natural out, pass 1 (half-lengths 1..16) on a[32 lane + e] with per-lane
// twiddles, transpose, pass 2 (32..512) with warp-uniform ones; the split
// transforms of the cluster kernels keep a cyclic inverse and a separate twist.
// The forward grows lazily by < 2q per stage with no correction: it starts below
// 3q + 1024 after its first stage (or 4q + 128 after the first two, taken from
// digit tables for Bg = 2^7) and ends below 22q.  The inverse starts below 12q
// (six Montgomery products) and reduces every butterfly output to [0, 2q).
#pragma once
#include <cstdint>

#include "arx_kernels.h"

namespace arx {

constexpr int kRows = 6;               // (k+1) l TGSW rows, l = 3
constexpr uint32_t kMu = 0x20000000u;  // +1/8
constexpr int kXpose = 1024;           // words per transpose buffer (swizzled, unpadded)

__host__ __device__ constexpr uint32_t neg_inv32(uint32_t q) {
  uint32_t x = q;  // correct to 3 bits for odd q; Newton doubles the bits
  for (int i = 0; i < 5; ++i) x *= 2u - q * x;
  return 0u - x;
}

// One CRT prime, in registers (the same code serves both primes).
struct PrimeRT {
  uint32_t q, q2, qni;  // q, 2q, -q^-1 mod 2^32
  uint32_t dc, dd;      // first-stage offsets for raw digit bytes (see ntt_fwd)
};

__device__ __forceinline__ PrimeRT prime_rt(int P, const TwiddleConst &tc) {
  PrimeRT r;
  r.q = P ? kQ1 : kQ0;
  r.q2 = 2u * r.q;
  r.qni = P ? neg_inv32(kQ1) : neg_inv32(kQ0);
  r.dc = tc.dig_c[P];
  r.dd = tc.dig_d[P];
  return r;
}

// ---- device-side launch timing (autotuner) --------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void stamp_start(unsigned long long *stamps) {
  if (stamps) atomicMin(stamps, global_ns());
}
__device__ __forceinline__ void stamp_end(unsigned long long *stamps) {
  if (stamps) atomicMax(stamps + 1, global_ns());
}

// ---- modular helpers ----------------------------------------------------
// Shoup: w * y mod q in [0, 2q) for any 32-bit y, given wp = floor(w 2^32 / q).
__device__ __forceinline__ uint32_t shoup_mul(uint32_t w, uint32_t wp, uint32_t y, uint32_t q) {
  return w * y - __umulhi(wp, y) * q;
}

// Montgomery: a b 2^-32 mod q in [0, 2q) for a b < 2^32 q.
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const PrimeRT &pr) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t m = (uint32_t)t * pr.qni;
  return (uint32_t)((t + (uint64_t)m * pr.q) >> 32);
}

// Montgomery reduction of an exact sum of products: T 2^-32 mod q, below
// T / 2^32 + q, for T < 2^63 (the sum of up to six products x b with x < 22q,
// b < q is below 132 q^2 < 2^62, reduced below 5.2q).
__device__ __forceinline__ uint32_t mont_redc(uint64_t t, const PrimeRT &pr) {
  const uint32_t m = (uint32_t)t * pr.qni;
  return (uint32_t)((t + (uint64_t)m * pr.q) >> 32);
}

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

__device__ __forceinline__ void ct_bfly(uint32_t &x, uint32_t &y, uint2 z, const PrimeRT &pr) {
  const uint32_t t = shoup_mul(z.x, z.y, y, pr.q);
  y = x - t + pr.q2;
  x = x + t;
}

// Element (row r, column c) of a 32 x 32 transpose buffer: 16-byte chunks of a
// row are XOR-swizzled by r & 7, so that a column write (32 lanes, one row) and a
// 128-bit row read (8 lanes per wavefront, 8 rows) are both conflict-free.
__device__ __forceinline__ int swz(int r, int c) { return r * 32 + ((((c >> 2) ^ (r & 7))) << 2) + (c & 3); }

// ---- warp transforms ----------------------------------------------------
// Forward.  kDig = 0: x[e] < q.  kDig = 1: x[e] holds raw gadget digits u =
// d + Bg/2 in [0, Bg) of a[lane + 32 e]; the -Bg/2 offsets ride on the first
// stage's constants, and the first stage's products zeta[1] u come from dtab[u]
// (zeta[1] u mod q, fully reduced, built once per CTA: a shared-memory load
// instead of a Shoup product).  kDig = 2 (7-bit digits, Bg = 2^7): the first two
// stages at once, as four sums of table products -- with z1 = zeta[1] and z2,
// z3 = zeta[2], zeta[3], the radix-4 group (u0, u1, u2, u3) = x[e, e+8, e+16,
// e+24] gives u0 + z1 u2 +- (z2 u1 + z2 z1 u3) and u0 - z1 u2 +- (z3 u1 - z3 z1 u3),
// the five products from dtab[t][u], t = (z1, z2, z2 z1, z3, z3 z1), and the
// digit offsets and 2q (outputs 1 .. 3, which subtract two table values) from
// dk[0 .. 3]: each output is below 4q + Bg before stage 3.  Output: x[e] =
// A[32 lane + e] < 22 q.
template <int kDig>
__device__ __forceinline__ void ntt_fwd(uint32_t (&x)[32], uint32_t *xbuf, const uint2 *tw1,
                                        const uint2 *__restrict__ tw2, const PrimeRT &pr, int lane,
                                        const uint32_t *dtab = nullptr, const uint32_t *dk = nullptr) {
  if constexpr (kDig == 2) {
    const uint32_t k0 = dk[0], k1 = dk[1], k2 = dk[2], k3 = dk[3];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t u0 = x[e], u1 = x[e + 8], u2 = x[e + 16], u3 = x[e + 24];
      const uint32_t a = dtab[u2], b = dtab[128 + u1], c = dtab[256 + u3], d = dtab[384 + u1], f = dtab[512 + u3];
      const uint32_t s = u0 + a, t = u0 - a;  // t wraps; every output below is a non-negative integer < 2^32
      x[e] = s + b + c + k0;
      x[e + 8] = s - b - c + k1;
      x[e + 16] = t + d - f + k2;
      x[e + 24] = t - d + f + k3;
    }
  } else {
    const uint2 z = tw1[1];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if (kDig == 1) {
        const uint32_t t = dtab[x[e + 16]];
        const uint32_t u = x[e];
        x[e] = u + t + pr.dc;
        x[e + 16] = u - t + pr.q2 + pr.dd;
      } else {
        ct_bfly(x[e], x[e + 16], z, pr);
      }
    }
  }
#pragma unroll
  for (int s = kDig == 2 ? 2 : 1; s < 5; ++s) {
    const int lr = 16 >> s;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & lr) == 0) ct_bfly(x[e], x[e + lr], tw1[(1 << s) + e / (2 * lr)], pr);
    }
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) xbuf[swz(e, lane)] = x[e];
  __syncwarp();
  const uint4 *xb4 = reinterpret_cast<const uint4 *>(xbuf);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 v = xb4[lane * 8 + (c ^ (lane & 7))];
    x[4 * c + 0] = v.x;
    x[4 * c + 1] = v.y;
    x[4 * c + 2] = v.z;
    x[4 * c + 3] = v.w;
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int len = 16 >> s;      // 16, 8, 4, 2, 1
    const int k0 = (1 << s) - 1;  // 0, 1, 3, 7, 15: first per-lane zeta of the stage
    uint2 z;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & len) == 0) {
        if ((e & (2 * len - 1)) == 0) z = __ldg(tw2 + (k0 + e / (2 * len)) * 32 + lane);
        ct_bfly(x[e], x[e + len], z, pr);
      }
    }
  }
}

// Gentleman-Sande butterfly of the merged inverse: (x, y) -> (x + y, (x - y) z),
// both in [0, 2q).  Inputs x, y < kIn q: 12 for the first stage after
// per-product Montgomery MACs (six products, each below 2q), 8 after the exact
// 64-bit MAC sums (one reduction per row group, below 7.2q in every shape that
// uses them), 2 for every later stage.
template <int kIn>
__device__ __forceinline__ void gs_bfly(uint32_t &x, uint32_t &y, uint2 z, const PrimeRT &pr) {
  static_assert(kIn == 2 || kIn == 8 || kIn == 12, "input bound");
  uint32_t s = x + y;
  const uint32_t d = x - y + (kIn / 2) * pr.q2;
  if (kIn == 12) s = csub(s, 8u * pr.q2);  // < 24q -> < 16q
  if (kIn >= 8) {
    s = csub(s, 4u * pr.q2);  // < 16q -> < 8q
    s = csub(s, 2u * pr.q2);  // < 8q -> < 4q
  }
  x = csub(s, pr.q2);
  y = shoup_mul(z.x, z.y, d, pr.q);
}

// Inverse with the output twist merged into the butterflies (Gentleman-Sande,
// psi^-1 powers: no separate twist pass; the 1/N factor rides on the stored
// key).  Pass 1 (half-lengths 1..16) on a[32 lane + e] with per-lane twiddles
// gs1, transpose, pass 2 (half-lengths 32..512) on a[lane + 32 e] with the
// warp-uniform gs2 (kernel parameter bank).  In: x[e] = A[32 lane + e] < 12 q
// (bit-reversed spectral order, as ntt_fwd leaves it).  Out: x[e] = a[lane +
// 32 e] in [0, 2q) (what crt_torus takes); every butterfly output is reduced to
// [0, 2q) (one conditional subtraction on the sum, the Shoup product on the
// difference).
template <int kIn0>  // input bound in q (see gs_bfly)
__device__ __forceinline__ void ntt_inv_gs(uint32_t (&x)[32], uint32_t *xbuf, const uint2 *__restrict__ gs1,
                                           const uint2 *gs2, const PrimeRT &pr, int lane) {
  constexpr int kOff[5] = {0, 16, 24, 28, 30};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int t = 1 << s;  // half-length 1, 2, 4, 8, 16
    uint2 z;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & t) == 0) {
        if ((e & (2 * t - 1)) == 0) z = __ldg(gs1 + (kOff[s] + e / (2 * t)) * 32 + lane);
        if (s == 0)
          gs_bfly<kIn0>(x[e], x[e + t], z, pr);
        else
          gs_bfly<2>(x[e], x[e + t], z, pr);
      }
    }
  }
  __syncwarp();
  uint4 *xb4 = reinterpret_cast<uint4 *>(xbuf);
#pragma unroll
  for (int c = 0; c < 8; ++c)
    xb4[lane * 8 + (c ^ (lane & 7))] = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) x[e] = xbuf[swz(e, lane)];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int hr = 1 << s;  // half-length / 32: 1, 2, 4, 8, 16
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & hr) == 0) gs_bfly<2>(x[e], x[e + hr], gs2[16 / hr + e / (2 * hr)], pr);
    }
  }
}

}  // namespace arx
