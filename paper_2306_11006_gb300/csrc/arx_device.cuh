// arx_device.cuh -- device-side arithmetic for GB300 (sm_103a) CGGI bootstrapping.
//
// Exact negacyclic polynomial products (Sec. 2.2: "TGSW BK_i x TLWE temp" of
// Fig. 2) through number-theoretic transforms (Sec. 5.4 motivates the NTT over
// the FFT because it is exact).  The paper's A100 design used one 64-bit prime;
// here each product is carried modulo two 28-bit primes (CRT), so every modular
// multiply is a native 32-bit IMAD / IMAD.HI sequence:
//   q0 = 195198977, q1 = 195188737, both = 1 (mod 2048), q0*q1 > 2^55,
// while the exact products are bounded by 6 * 1024 * 64 * 2^31 < 2^50.
//
// Warp-per-transform layout: a 1024-point transform is held by one warp, 32
// values per lane.  Pass 1 (lengths 512..32) runs on x[e] = a[lane + 32 e] with
// warp-uniform twiddles read from the constant bank; a padded shared-memory
// transpose moves lane to a[32 lane + e]; pass 2 (lengths 16..1) uses per-lane
// twiddles.  The inverse runs the mirror image.  Values are kept lazily reduced:
// the forward pass needs no correction at all (inputs < 2q, each stage adds < 2q,
// 22 q < 2^32), the inverse uses Harvey's [0, 2q) Gentleman-Sande butterfly.
#pragma once
#include <cstdint>

#include "arx_kernels.h"

namespace arx {

constexpr int kRows = 6;          // (k+1) l TGSW rows, l = 3
constexpr uint32_t kMu = 0x20000000u;  // +1/8
constexpr int kPad = 33;                           // transpose row pitch (words)
constexpr int kXpose = 32 * kPad;                  // 1056 words per transpose buffer


__host__ __device__ constexpr uint32_t neg_inv32(uint32_t q) {
  uint32_t x = q;  // correct to 3 bits for odd q; Newton doubles the bits
  for (int i = 0; i < 5; ++i) x *= 2u - q * x;
  return 0u - x;
}

template <int P> struct Prime;
template <> struct Prime<0> {
  static constexpr uint32_t q = kQ0;
  static constexpr uint32_t qneg_inv = neg_inv32(kQ0);
};
template <> struct Prime<1> {
  static constexpr uint32_t q = kQ1;
  static constexpr uint32_t qneg_inv = neg_inv32(kQ1);
};

// ---- modular helpers ----------------------------------------------------
// Shoup: w * y mod q in [0, 2q) for any 32-bit y, given wp = floor(w 2^32 / q).
template <int P>
__device__ __forceinline__ uint32_t shoup_mul(uint32_t w, uint32_t wp, uint32_t y) {
  uint32_t qhat = __umulhi(wp, y);
  return w * y - qhat * Prime<P>::q;
}

// Montgomery: a b 2^-32 mod q in [0, 2q) for a b < 2^32 q.
template <int P>
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b) {
  uint64_t t = (uint64_t)a * b;
  uint32_t m = (uint32_t)t * Prime<P>::qneg_inv;
  return (uint32_t)((t + (uint64_t)m * Prime<P>::q) >> 32);
}

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

template <int P>
__device__ __forceinline__ void ct_bfly(uint32_t &x, uint32_t &y, uint2 z) {
  uint32_t t = shoup_mul<P>(z.x, z.y, y);
  y = x - t + 2u * Prime<P>::q;
  x = x + t;
}

template <int P>
__device__ __forceinline__ void gs_bfly(uint32_t &x, uint32_t &y, uint2 z) {
  uint32_t s = csub(x + y, 2u * Prime<P>::q);
  uint32_t d = x - y + 2u * Prime<P>::q;
  x = s;
  y = shoup_mul<P>(z.x, z.y, d);
}

// ---- warp transforms ----------------------------------------------------
// Forward: x[e] = a[lane + 32 e] with a < 2q  ->  x[e] = A[32 lane + e] < 22 q.
template <int P>
__device__ __forceinline__ void ntt_fwd(uint32_t (&x)[32], uint32_t *xbuf, const TwiddleConst &tc,
                                        const uint2 *__restrict__ tw2, int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int lr = 16 >> s;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & lr) == 0) ct_bfly<P>(x[e], x[e + lr], tc.fwd1[P][(1 << s) + e / (2 * lr)]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) xbuf[lane + kPad * e] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) x[e] = xbuf[kPad * lane + e];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int len = 16 >> s;       // 16, 8, 4, 2, 1
    const int k0 = (1 << s) - 1;   // 0, 1, 3, 7, 15: first per-lane zeta of the stage
    uint2 z;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & len) == 0) {
        if ((e & (2 * len - 1)) == 0) z = __ldg(tw2 + (k0 + e / (2 * len)) * 32 + lane);
        ct_bfly<P>(x[e], x[e + len], z);
      }
    }
  }
}

// Inverse (without the 1/N factor, which the stored key carries):
// x[e] = A[32 lane + e] < 2q  ->  x[e] = a[lane + 32 e] < 2q.
template <int P>
__device__ __forceinline__ void ntt_inv(uint32_t (&x)[32], uint32_t *xbuf, const TwiddleConst &tc,
                                        const uint2 *__restrict__ tw1, int lane) {
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int len = 1 << t;        // 1, 2, 4, 8, 16
    const int blocks = 16 >> t;    // 16, 8, 4, 2, 1
    const int k0 = blocks - 1;     // 15, 7, 3, 1, 0
    uint2 z;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & len) == 0) {
        if ((e & (2 * len - 1)) == 0) z = __ldg(tw1 + (k0 + e / (2 * len)) * 32 + lane);
        gs_bfly<P>(x[e], x[e + len], z);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) xbuf[kPad * lane + e] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 32; ++e) x[e] = xbuf[lane + kPad * e];
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int lr = 1 << t;  // 1, 2, 4, 8, 16: undoes forward pass-1 stage m = 16 >> t
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      if ((e & lr) == 0) gs_bfly<P>(x[e], x[e + lr], tc.inv2[P][(16 >> t) + e / (2 * lr)]);
    }
  }
}

}  // namespace arx
