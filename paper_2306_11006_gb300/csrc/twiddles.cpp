// twiddles.cpp -- twiddle tables of the device NTTs for the CRT primes q0, q1.
//
// Forward (negacyclic, merged twist): zeta[k] = psi^bitrev10(k) for k = 1..1023,
// psi a primitive 2048-th root of unity mod q (psi^1024 = -1); the stage with m
// blocks uses zeta[m + block].  Inverse of the warp transforms (Gentleman-Sande,
// merged twist): the stage of half-length t uses psi^-bitrev10(512 / t + block).
// Inverse of the split transforms (cyclic DIT on the bit-reversed spectrum,
// omega = psi^2): the stage of half-length h uses omega^-(j 512 / h) for the j-th
// pair of each block, followed by the twist psi^-p at output p.  Every entry
// carries its Shoup companion floor(w 2^32 / q).
//
// Split transforms of the cluster kernel.  Forward: two warps per transform, half
// w holds positions 512 w .. 512 w + 511; in pass 2 lane l holds the 16
// positions of block b = 2 (l mod 16) + l / 16, and stage s (length 8 >> s),
// block-part c < 2^s uses zeta[(64 << s) + (32 << s) w + (1 << s) b + c].
// Inverse: four warps per transform (quarters Q of 256 spectral positions), the
// last two stages and the twist folded together: with u_Q the quarters'
// outputs at k < 256 and t = (psi^-k u_0, psi^-5k u_1, psi^-3k u_2, psi^-7k u_3),
//   out_k       = t0 + t1 + t2 + t3
//   out_(k+512) = psi^-512 (t0 + t1 - t2 - t3)
//   out_(k+256) = psi^-256 ((t0 - t1) + psi^-512 (t2 - t3))
//   out_(k+768) = psi^-256 (psi^-512 (t0 - t1) + (t2 - t3)).
// The four-CTA kernel also splits the forward transform in quarters Q (the
// first two stages taken on load).  Its middle pass holds positions
// (l mod 8) + 8 e + 64 g, g = l / 8: stage s (length 32 >> s), block-part c < 2^s
// uses zeta[(16 << s) + (4 << s) Q + (1 << s) g + c].  In its last pass lane l
// holds the 8 positions of block b = 4 (l mod 8) + l / 8, and stage s (length
// 4 >> s) uses zeta[(128 << s) + (32 << s) Q + (1 << s) b + c].
#include <cstdint>
#include <stdexcept>

#include "arx_kernels.h"

namespace arx {
namespace {

uint64_t pw(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1;
  b %= m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

uint32_t bitrev10(uint32_t k) {
  uint32_t r = 0;
  for (int i = 0; i < 10; ++i) r |= ((k >> i) & 1u) << (9 - i);
  return r;
}

uint2 entry(uint64_t w, uint64_t q) {
  uint2 e;
  e.x = (uint32_t)w;
  e.y = (uint32_t)((w << 32) / q);
  return e;
}

void fill(int P, uint64_t q, TwiddleConst *tc, TwiddleGlobal *tg) {
  uint64_t psi = 0;
  for (uint64_t x = 2; x < q; ++x) {
    uint64_t c = pw(x, (q - 1) / 2048, q);
    if (pw(c, 1024, q) == q - 1) {
      psi = c;
      break;
    }
  }
  if (!psi) throw std::runtime_error("no 2048-th root of unity");
  const uint64_t psi_inv = pw(psi, q - 2, q);
  const uint64_t omega_inv = psi_inv * psi_inv % q;
  uint64_t zeta[1024];
  for (uint32_t k = 1; k < 1024; ++k) zeta[k] = pw(psi, bitrev10(k), q);
  zeta[0] = 1;
  for (int zi = 0; zi < 32; ++zi) tc->fwd1[P][zi] = entry(zeta[zi], q);
  for (int k = 0; k < 1024; ++k) tg->fwdz[P][k] = entry(zeta[k], q);
  tc->dig_c[P] = (uint32_t)((2 * q - 64 - 64 * zeta[1] % q) % q);
  tc->dig_d[P] = (uint32_t)((64 * zeta[1] % q + q - 64) % q);
  tc->dig_c2[P] = (uint32_t)((2 * q - 512 - 512 * zeta[1] % q) % q);
  tc->dig_d2[P] = (uint32_t)((512 * zeta[1] % q + q - 512) % q);
  {  // stages 1 and 2 on raw digits u = d + 64: output j carries -64 (its sum of
     // +-1, +-z1, +-z2 or z3, +-z2 z1 or z3 z1); outputs 1 .. 3 add 2q (see ntt_fwd)
    const uint64_t z1 = zeta[1], z2 = zeta[2], z3 = zeta[3], z21 = z2 * z1 % q, z31 = z3 * z1 % q;
    auto off = [q](uint64_t plus, uint64_t minus) {  // 64 (minus - plus) mod q
      return (uint32_t)((64 * (minus % q) % q + q - 64 * (plus % q) % q) % q);
    };
    tc->dig4[P][0] = off(1 + z1 + z2 + z21, 0);
    tc->dig4[P][1] = (uint32_t)(2 * q) + off(1 + z1, z2 + z21);
    tc->dig4[P][2] = (uint32_t)(2 * q) + off(1 + z3, z1 + z31);
    tc->dig4[P][3] = (uint32_t)(2 * q) + off(1 + z31, z1 + z3);
  }
  // forward pass 2, per lane: stage s (length 16 >> s) has 2^s blocks per lane;
  // block b of lane l is zeta index 2^s (32 + l) + b, stored at [(2^s - 1 + b)][l].
  for (int s = 0; s < 5; ++s)
    for (int b = 0; b < (1 << s); ++b)
      for (int lane = 0; lane < 32; ++lane)
        tg->fwd2[P][((1 << s) - 1 + b) * 32 + lane] = entry(zeta[(1 << s) * (32 + lane) + b], q);
  // inverse pass 1 (half-lengths 1..16 within a lane): omega^-(j 512 / h)
  for (int zi = 0; zi < 32; ++zi) tc->inv1[P][zi] = entry(1, q);
  for (int t = 0; t < 5; ++t) {
    const int h = 1 << t;
    for (int j = 0; j < h; ++j) tc->inv1[P][(h - 1) + j] = entry(pw(omega_inv, (uint64_t)j * (512 / h), q), q);
  }
  // inverse pass 2 (half-lengths 32..512 across e): pair index j = lane + 32 b,
  // b < h / 32, twiddle omega^-(j 512 / h), stored at [(h/32 - 1) + b][lane]
  for (int s = 0; s < 5; ++s) {
    const int hr = 1 << s, h = 32 * hr;
    for (int b = 0; b < hr; ++b)
      for (int lane = 0; lane < 32; ++lane)
        tg->inv2[P][(hr - 1 + b) * 32 + lane] = entry(pw(omega_inv, (uint64_t)(lane + 32 * b) * (512 / h), q), q);
  }
  for (int w = 0; w < 2; ++w)
    for (int s = 0; s < 4; ++s)
      for (int c = 0; c < (1 << s); ++c)
        for (int lane = 0; lane < 32; ++lane) {
          const int b = 2 * (lane & 15) + (lane >> 4);
          tg->fwdh[P][w][((1 << s) - 1 + c) * 32 + lane] =
              entry(zeta[(64 << s) + (32 << s) * w + (1 << s) * b + c], q);
        }
  for (int Q = 0; Q < 4; ++Q)
    for (int s = 0; s < 3; ++s)
      for (int c = 0; c < (1 << s); ++c)
        for (int lane = 0; lane < 32; ++lane) {
          const int b = 4 * (lane & 7) + (lane >> 3);
          tg->fwdq[P][Q][((1 << s) - 1 + c) * 32 + lane] =
              entry(zeta[(128 << s) + (32 << s) * Q + (1 << s) * b + c], q);
          tg->fwdc[P][Q][((1 << s) - 1 + c) * 32 + lane] =
              entry(zeta[(16 << s) + (4 << s) * Q + (1 << s) * (lane >> 3) + c], q);
        }
  // inverse quarter, middle pass on positions (l mod 8) + 8 e + 64 (l / 8): stage s
  // (half-length 8 << s) pairs j = (l mod 8) + 8 c, c < 2^s, twiddle omega^-(j 512 / h)
  for (int s = 0; s < 3; ++s)
    for (int c = 0; c < (1 << s); ++c)
      for (int lane = 0; lane < 32; ++lane)
        tg->invc[P][((1 << s) - 1 + c) * 32 + lane] =
            entry(pw(omega_inv, (uint64_t)((lane & 7) + 8 * c) * (512 / (8 << s)), q), q);
  const int cQ[4] = {1, 5, 3, 7};
  for (int Q = 0; Q < 4; ++Q)
    for (int k = 0; k < 256; ++k) tg->fint[P][Q][k] = entry(pw(psi_inv, (uint64_t)cQ[Q] * k, q), q);
  tc->psi512[P] = entry(pw(psi_inv, 512, q), q);
  tc->psi256[P] = entry(pw(psi_inv, 256, q), q);
  // merged inverse (Gentleman-Sande, bit-reversed in, natural out): the butterfly
  // of half-length t on block i (positions 2 t i .. 2 t i + 2t - 1) takes
  // psi^-bitrev10(512 / t + i).  Pass 1 (t = 1..16, lane l holds positions
  // 32 l + e): block i = l 16 / t + b, b < 16 / t, stored at [off_s + b][l],
  // off = 0, 16, 24, 28, 30; pass 2 (t = 32..512, positions l + 32 e): the block
  // does not depend on the lane, index 512 / t + e / (t / 16) in gsi2.
  {
    const int off[5] = {0, 16, 24, 28, 30};
    for (int s = 0; s < 5; ++s) {
      const int t = 1 << s;
      for (int b = 0; b < 16 / t; ++b)
        for (int lane = 0; lane < 32; ++lane)
          tg->gsi1[P][(off[s] + b) * 32 + lane] =
              entry(pw(psi_inv, bitrev10((uint32_t)(512 / t + lane * (16 / t) + b)), q), q);
    }
    tc->gsi2[P][0] = entry(1, q);
    for (uint32_t k = 1; k < 32; ++k) tc->gsi2[P][k] = entry(pw(psi_inv, bitrev10(k), q), q);
  }
}

}  // namespace

void make_twiddles(TwiddleConst *tc, TwiddleGlobal *tg) {
  fill(0, kQ0, tc, tg);
  fill(1, kQ1, tc, tg);
}

}  // namespace arx
