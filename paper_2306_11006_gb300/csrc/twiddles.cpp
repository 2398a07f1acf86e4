// twiddles.cpp -- twiddle tables of the device NTTs for the CRT primes q0, q1.
//
// zeta[k] = psi^bitrev10(k) for k = 1..1023, psi a primitive 2048-th root of
// unity mod q (psi^1024 = -1), so the negacyclic Cooley-Tukey stage with m blocks
// uses zeta[m + block]; the inverse uses zeta^-1 at the same positions.  Each
// entry carries its Shoup companion floor(w 2^32 / q).
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
  uint64_t zeta[1024], zinv[1024];
  for (uint32_t k = 1; k < 1024; ++k) {
    zeta[k] = pw(psi, bitrev10(k), q);
    zinv[k] = pw(zeta[k], q - 2, q);
  }
  zeta[0] = zinv[0] = 1;
  for (int zi = 0; zi < 32; ++zi) {
    tc->fwd1[P][zi] = entry(zeta[zi], q);
    tc->inv2[P][zi] = entry(zinv[zi], q);
  }
  // per-lane tables: stage s (length 16 >> s) has 2^s blocks per lane; block b of
  // lane l is zeta index 2^s (32 + l) + b, stored at [(2^s - 1 + b)][l].
  for (int s = 0; s < 5; ++s) {
    for (int b = 0; b < (1 << s); ++b) {
      for (int lane = 0; lane < 32; ++lane) {
        const int zi = (1 << s) * (32 + lane) + b;
        const int k = (1 << s) - 1 + b;
        tg->fwd2[P][k * 32 + lane] = entry(zeta[zi], q);
        tg->inv1[P][k * 32 + lane] = entry(zinv[zi], q);
      }
    }
  }
}

}  // namespace

void make_twiddles(TwiddleConst *tc, TwiddleGlobal *tg) {
  fill(0, kQ0, tc, tg);
  fill(1, kQ1, tc, tg);
}

}  // namespace arx
