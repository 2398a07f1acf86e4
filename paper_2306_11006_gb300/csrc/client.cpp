// client.cpp -- client-side key generation, encryption and decryption (host).
//
// The data owner holds the secret keys, encrypts its inputs and decrypts the
// results; the server (the GPU engine) only sees ciphertexts, the bootstrapping
// key and the key-switching key (App. D, threat model).  All randomness is an
// argument, so that a caller can reproduce keys bit for bit.
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/arx.h"

namespace {

constexpr int kN = ARX_N;

// body += a * K  mod (X^N + 1, 2^32), K binary: add a rotated by each set bit.
void add_times_binary(const uint32_t *a, const uint8_t *K, uint32_t *body) {
  for (int j = 0; j < kN; ++j) {
    if (!K[j]) continue;
    for (int k = 0; k < j; ++k) body[k] -= a[k - j + kN];
    for (int k = j; k < kN; ++k) body[k] += a[k - j];
  }
}

template <class F>
void parallel_for(int count, F f) {
  unsigned hw = std::thread::hardware_concurrency();
  int T = (int)(hw ? hw : 1);
  if (T > count) T = count > 0 ? count : 1;
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t)
    th.emplace_back([=] {
      for (int i = t; i < count; i += T) f(i);
    });
  for (auto &x : th) x.join();
}

}  // namespace

extern "C" int arx_client_keygen_gadget(int n, int l, int bg_bits, const uint8_t *s, const uint8_t *K,
                                        const uint32_t *bsk_mask, const int32_t *bsk_noise, const uint32_t *ksk_mask,
                                        const int32_t *ksk_noise, uint32_t *bsk, uint32_t *ksk) {
  if (n < 1 || n > ARX_LWE_N || !s || !K || !bsk_mask || !bsk_noise || !ksk_mask || !ksk_noise || !bsk || !ksk)
    return ARX_EINVAL;
  if (!((l == 3 && bg_bits == 7) || (l == 2 && bg_bits == 10))) return ARX_EINVAL;
  const int rows = 2 * l;
  // BSK_i = TGSW_K(s_i): row (c, p) is (a, a K + e) plus s_i 2^(32 - p bg_bits) on component c.
  parallel_for(n, [&](int i) {
    for (int r = 0; r < rows; ++r) {
      const int c = r / l, p = r % l + 1;
      const size_t src = ((size_t)i * rows + r) * kN;
      uint32_t *mask = bsk + (((size_t)i * rows + r) * 2 + 0) * kN;
      uint32_t *body = bsk + (((size_t)i * rows + r) * 2 + 1) * kN;
      std::memcpy(mask, bsk_mask + src, sizeof(uint32_t) * kN);
      for (int k = 0; k < kN; ++k) body[k] = (uint32_t)bsk_noise[src + k];
      add_times_binary(mask, K, body);
      const uint32_t h = s[i] ? (1u << (32 - bg_bits * p)) : 0u;
      (c == 0 ? mask : body)[0] += h;
    }
  });
  // KSK[i][j][v] = LWE_s(v K_i 2^(32-2j)); the v = 0 rows are left zero.
  const size_t row = (size_t)n + 1;
  parallel_for(kN, [&](int i) {
    for (int j = 1; j <= ARX_KS_T; ++j) {
      uint32_t *blk = ksk + ((size_t)i * ARX_KS_T + (j - 1)) * ARX_KS_BASE * row;
      std::memset(blk, 0, sizeof(uint32_t) * row);
      for (int v = 1; v < ARX_KS_BASE; ++v) {
        const size_t idx = ((size_t)i * ARX_KS_T + (j - 1)) * 3 + (v - 1);
        const uint32_t *a = ksk_mask + idx * (size_t)n;
        uint32_t *out = blk + (size_t)v * row;
        uint32_t b = (uint32_t)ksk_noise[idx] + (K[i] ? (uint32_t)v << (32 - 2 * j) : 0u);
        for (int q = 0; q < n; ++q) {
          out[q] = a[q];
          if (s[q]) b += a[q];
        }
        out[n] = b;
      }
    }
  });
  return ARX_OK;
}

extern "C" int arx_client_keygen(int n, const uint8_t *s, const uint8_t *K, const uint32_t *bsk_mask,
                                 const int32_t *bsk_noise, const uint32_t *ksk_mask, const int32_t *ksk_noise,
                                 uint32_t *bsk, uint32_t *ksk) {
  return arx_client_keygen_gadget(n, 3, 7, s, K, bsk_mask, bsk_noise, ksk_mask, ksk_noise, bsk, ksk);
}

extern "C" int arx_client_encrypt(int n, const uint8_t *s, const uint32_t *mask, const int32_t *noise,
                                  const uint8_t *bits, size_t count, uint32_t *ct) {
  if (n < 1 || n > ARX_LWE_N || (count && (!s || !mask || !noise || !bits || !ct))) return ARX_EINVAL;
  for (size_t g = 0; g < count; ++g) {
    const uint32_t *a = mask + g * (size_t)n;
    uint32_t *out = ct + g * ((size_t)n + 1);
    uint32_t b = (uint32_t)noise[g] + (bits[g] ? ARX_MU : 0u - ARX_MU);
    for (int q = 0; q < n; ++q) {
      out[q] = a[q];
      if (s[q]) b += a[q];
    }
    out[n] = b;
  }
  return ARX_OK;
}

extern "C" int arx_client_decrypt(int n, const uint8_t *s, const uint32_t *ct, size_t count, uint8_t *bits) {
  if (n < 1 || n > ARX_LWE_N || (count && (!s || !ct || !bits))) return ARX_EINVAL;
  for (size_t g = 0; g < count; ++g) {
    const uint32_t *c = ct + g * ((size_t)n + 1);
    uint32_t phase = c[n];
    for (int q = 0; q < n; ++q)
      if (s[q]) phase -= c[q];
    bits[g] = (int32_t)phase > 0;
  }
  return ARX_OK;
}
