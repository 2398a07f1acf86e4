/*
 * cggi_oracle.c -- plain, slow CPU oracle for CGGI gate bootstrapping.
 *
 * TEST INFRASTRUCTURE ONLY: the independent reference the CUDA path is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant generator with the
 * product library.
 *
 * Written for a reader checking it against the paper (ArctyrEX, arXiv
 * 2306.11006) by eye: no blocking, no fusion, no reordering beyond what the
 * definitions state.  Each function names the passage it follows.
 */
#include "cggi_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Goldilocks field.  Sec. 5.4: "we utilize the modulus Q = 2^64 - 2^32 + 1,   */
/* which simplifies modular reduction", and "the primitive element g".        */
/* ------------------------------------------------------------------------- */
static const uint64_t GL_Q = 0xFFFFFFFF00000001ull;
static const uint64_t GL_G = 12037493425763644479ull;

static uint64_t gl_add(uint64_t a, uint64_t b) {
  unsigned __int128 s = (unsigned __int128)a + b;
  if (s >= GL_Q) s -= GL_Q;
  return (uint64_t)s;
}

static uint64_t gl_sub(uint64_t a, uint64_t b) { return a >= b ? a - b : a + (GL_Q - b); }

/* x mod Q for x < 2^128, from 2^64 = 2^32 - 1 and 2^96 = -1 (mod Q). */
static uint64_t gl_reduce(unsigned __int128 x) {
  uint64_t lo = (uint64_t)x;
  uint64_t hi = (uint64_t)(x >> 64);
  uint64_t h0 = hi & 0xFFFFFFFFull;
  uint64_t h1 = hi >> 32;
  __int128 r = (__int128)lo + (__int128)h0 * 0xFFFFFFFFll - (__int128)h1;
  while (r < 0) r += (__int128)GL_Q;
  while (r >= (__int128)GL_Q) r -= (__int128)GL_Q;
  return (uint64_t)r;
}

uint64_t orc_gl_mul(uint64_t a, uint64_t b) { return gl_reduce((unsigned __int128)a * b); }

uint64_t orc_gl_pow(uint64_t a, uint64_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = orc_gl_mul(r, a);
    a = orc_gl_mul(a, a);
    e >>= 1;
  }
  return r;
}

static uint64_t gl_inv(uint64_t a) { return orc_gl_pow(a, GL_Q - 2); }

/* integer in (-Q, Q) -> residue */
static uint64_t gl_from_i64(int64_t v) {
  return v >= 0 ? (uint64_t)v % GL_Q : GL_Q - ((uint64_t)(-v) % GL_Q);
}

/* residue -> centred representative in (-Q/2, Q/2] */
static int64_t gl_centred(uint64_t x) {
  return x > GL_Q / 2 ? -(int64_t)(GL_Q - x) : (int64_t)x;
}

/* ------------------------------------------------------------------------- */
/* Negacyclic NTT (textbook form).  psi_m = g^(2^32/(2m)) has order 2m because */
/* g has order 2^32.  Forward: twist a[j] by psi^j, then the cyclic transform  */
/* with omega = psi^2 (bit reversal + radix-2 Cooley-Tukey), so that           */
/* A[k] = sum_j a[j] psi^((2k+1) j).  Inverse undoes each step in reverse.      */
/* ------------------------------------------------------------------------- */
static void bit_reverse(uint64_t *a, int m) {
  for (int i = 1, j = 0; i < m; i++) {
    int bit = m >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      uint64_t t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
}

/* A[k] = sum_j a[j] w^(jk), with pw[e] = w^e for e < m. */
static void ntt_cyclic(uint64_t *a, int m, const uint64_t *pw) {
  bit_reverse(a, m);
  for (int len = 2; len <= m; len <<= 1) {
    int step = m / len;
    for (int i = 0; i < m; i += len) {
      for (int j = 0; j < len / 2; j++) {
        uint64_t u = a[i + j];
        uint64_t v = orc_gl_mul(a[i + j + len / 2], pw[j * step]);
        a[i + j] = gl_add(u, v);
        a[i + j + len / 2] = gl_sub(u, v);
      }
    }
  }
}

typedef struct {
  int m;
  uint64_t psi_pow[2 * ORC_N];     /* psi^j, j < 2m */
  uint64_t psi_inv_pow[2 * ORC_N]; /* psi^-j */
  uint64_t w_pow[ORC_N];           /* omega^e = psi^(2e), e < m */
  uint64_t w_inv_pow[ORC_N];
  uint64_t m_inv;
} ntt_tables;

static void ntt_tables_init(ntt_tables *t, int m) {
  uint64_t psi = orc_gl_pow(GL_G, (1ull << 32) / (2ull * (uint64_t)m));
  uint64_t psi_inv = gl_inv(psi);
  t->m = m;
  t->psi_pow[0] = 1;
  t->psi_inv_pow[0] = 1;
  for (int j = 1; j < 2 * m; j++) {
    t->psi_pow[j] = orc_gl_mul(t->psi_pow[j - 1], psi);
    t->psi_inv_pow[j] = orc_gl_mul(t->psi_inv_pow[j - 1], psi_inv);
  }
  for (int e = 0; e < m; e++) {
    t->w_pow[e] = t->psi_pow[(2 * e) % (2 * m)];
    t->w_inv_pow[e] = t->psi_inv_pow[(2 * e) % (2 * m)];
  }
  t->m_inv = gl_inv((uint64_t)m);
}

static ntt_tables g_tab1024;
static pthread_once_t g_tab_once = PTHREAD_ONCE_INIT;
static void tab1024_init(void) { ntt_tables_init(&g_tab1024, ORC_N); }

static void ntt_with(const ntt_tables *t, uint64_t *a, int inverse) {
  int m = t->m;
  if (!inverse) {
    for (int j = 0; j < m; j++) a[j] = orc_gl_mul(a[j], t->psi_pow[j]);
    ntt_cyclic(a, m, t->w_pow);
  } else {
    ntt_cyclic(a, m, t->w_inv_pow);
    for (int j = 0; j < m; j++) a[j] = orc_gl_mul(orc_gl_mul(a[j], t->m_inv), t->psi_inv_pow[j]);
  }
}

void orc_ntt(uint64_t *a, int m, int inverse) {
  if (m == ORC_N) {
    pthread_once(&g_tab_once, tab1024_init);
    ntt_with(&g_tab1024, a, inverse);
    return;
  }
  ntt_tables *t = (ntt_tables *)malloc(sizeof(ntt_tables));
  ntt_tables_init(t, m);
  ntt_with(t, a, inverse);
  free(t);
}

void orc_negacyclic_mul_ntt(const int64_t *a, const int64_t *b, int64_t *c, int m) {
  uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
  uint64_t *B = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
  for (int j = 0; j < m; j++) {
    A[j] = gl_from_i64(a[j]);
    B[j] = gl_from_i64(b[j]);
  }
  orc_ntt(A, m, 0);
  orc_ntt(B, m, 0);
  for (int j = 0; j < m; j++) A[j] = orc_gl_mul(A[j], B[j]);
  orc_ntt(A, m, 1);
  for (int j = 0; j < m; j++) c[j] = gl_centred(A[j]);
  free(A);
  free(B);
}

/* c[k] = sum_{i+j=k} a_i b_j - sum_{i+j=k+m} a_i b_j  (X^m = -1) */
void orc_negacyclic_mul_schoolbook(const int64_t *a, const int64_t *b, int64_t *c, int m) {
  for (int k = 0; k < m; k++) {
    __int128 s = 0;
    for (int i = 0; i < m; i++) {
      int j = k - i;
      if (j >= 0)
        s += (__int128)a[i] * b[j];
      else
        s -= (__int128)a[i] * b[j + m];
    }
    c[k] = (int64_t)s;
  }
}

/* ------------------------------------------------------------------------- */
/* Scalar pieces (the paper is silent on these; readings c6, c10, c13).        */
/* ------------------------------------------------------------------------- */

/* Mod switch of a Torus32 value to Z_2N, round half up: the exponents of X in  */
/* "Accum = out x X^-b" and "X^a[i]" of Fig. 2.  2N = 2^11, so drop 21 bits.    */
uint32_t orc_modswitch(uint32_t x) {
  uint32_t rounded = x + (1u << 20);
  return rounded >> 21;
}

/* Signed gadget decomposition (Bg = 2^7, l = 3 by default): round x to its top */
/* l log2(Bg) bits (21) and write that as sum_p d_p 2^(32 - p log2 Bg) with     */
/* d_p in [-Bg/2, Bg/2), p = 1 first.                                           */
void orc_decompose(uint32_t x, int32_t digits[ORC_L]) {
  const int total = ORC_BG_BITS * ORC_L; /* 21 (20 for l = 2, Bg = 2^10) */
  uint32_t offset = 0;
  for (int p = 1; p <= ORC_L; p++) offset += (1u << (ORC_BG_BITS - 1)) << (32 - ORC_BG_BITS * p);
  uint32_t y = x + (1u << (32 - total - 1)) + offset;
  for (int p = 1; p <= ORC_L; p++) {
    uint32_t u = (y >> (32 - ORC_BG_BITS * p)) & ((1u << ORC_BG_BITS) - 1);
    digits[p - 1] = (int32_t)u - (1 << (ORC_BG_BITS - 1));
  }
}

/* Key-switch digits: round x to 16 bits, then base-4 digits, j = 1 first.      */
void orc_ks_digits(uint32_t x, uint32_t digits[ORC_KS_T]) {
  const int total = ORC_KS_BITS * ORC_KS_T; /* 16 */
  uint32_t y = x + (1u << (32 - total - 1));
  for (int j = 1; j <= ORC_KS_T; j++) digits[j - 1] = (y >> (32 - ORC_KS_BITS * j)) & 3u;
}

/* ------------------------------------------------------------------------- */
/* Polynomial helpers over Torus32 (Z / 2^32).                                 */
/* ------------------------------------------------------------------------- */

/* out = X^e * p  mod (X^N + 1), e in [0, 2N) */
static void poly_mul_monomial(const uint32_t *p, uint32_t e, uint32_t *out) {
  for (int j = 0; j < ORC_N; j++) {
    uint32_t m = ((uint32_t)j + e) % (2 * ORC_N);
    if (m < ORC_N)
      out[m] = p[j];
    else
      out[m - ORC_N] = 0u - p[j];
  }
}

/* exact negacyclic product of a Torus32 poly (read as int32) and a binary poly */
static void torus_times_binary(const uint32_t *a, const uint8_t *K, uint32_t *out) {
  int64_t A[ORC_N], B[ORC_N], C[ORC_N];
  for (int j = 0; j < ORC_N; j++) {
    A[j] = (int32_t)a[j];
    B[j] = K[j];
  }
  orc_negacyclic_mul_ntt(A, B, C, ORC_N);
  for (int j = 0; j < ORC_N; j++) out[j] = (uint32_t)C[j];
}

/* ------------------------------------------------------------------------- */
/* Keys and LWE encryption (Sec. 2.2: LWE, TLWE and TGSW samples).             */
/* ------------------------------------------------------------------------- */
void orc_keygen(int n, const uint8_t *s, const uint8_t *K, const uint32_t *bsk_mask,
                const int32_t *bsk_noise, const uint32_t *ksk_mask, const int32_t *ksk_noise,
                uint32_t *bsk, uint32_t *ksk) {
  /* Bootstrapping key: BSK_i = TGSW_K(s_i).  Row r = c*l + (p-1) is a TLWE      */
  /* encryption of 0 under K, (a, a*K + e), plus s_i * 2^(32-7p) on component c. */
  for (int i = 0; i < n; i++) {
    for (int c = 0; c < 2; c++) {
      for (int p = 1; p <= ORC_L; p++) {
        int r = c * ORC_L + (p - 1);
        size_t src = ((size_t)i * ORC_ROWS + r) * ORC_N;
        uint32_t *mask = bsk + (((size_t)i * ORC_ROWS + r) * 2 + 0) * ORC_N;
        uint32_t *body = bsk + (((size_t)i * ORC_ROWS + r) * 2 + 1) * ORC_N;
        memcpy(mask, bsk_mask + src, sizeof(uint32_t) * ORC_N);
        torus_times_binary(mask, K, body);
        for (int k = 0; k < ORC_N; k++) body[k] += (uint32_t)bsk_noise[src + k];
        uint32_t h = 1u << (32 - ORC_BG_BITS * p);
        if (c == 0)
          mask[0] += s[i] ? h : 0u;
        else
          body[0] += s[i] ? h : 0u;
      }
    }
  }
  /* Key-switching key: KSK[i][j][v] = LWE_s(v K_i 2^(32-2j)), v = 0 unused.     */
  for (int i = 0; i < ORC_N; i++) {
    for (int j = 1; j <= ORC_KS_T; j++) {
      for (int v = 0; v < 4; v++) {
        uint32_t *row = ksk + (((size_t)i * ORC_KS_T + (j - 1)) * 4 + v) * (size_t)(n + 1);
        if (v == 0) {
          memset(row, 0, sizeof(uint32_t) * (size_t)(n + 1));
          continue;
        }
        size_t src = ((size_t)i * ORC_KS_T + (j - 1)) * 3 + (v - 1);
        const uint32_t *a = ksk_mask + src * (size_t)n;
        uint32_t b = (uint32_t)ksk_noise[src] + (uint32_t)v * (uint32_t)K[i] * (1u << (32 - ORC_KS_BITS * j));
        for (int q = 0; q < n; q++) {
          row[q] = a[q];
          b += a[q] * (uint32_t)s[q];
        }
        row[n] = b;
      }
    }
  }
}

void orc_encrypt(int n, const uint8_t *s, const uint32_t *mask, const int32_t *noise,
                 const uint8_t *bits, size_t count, uint32_t *ct) {
  for (size_t g = 0; g < count; g++) {
    uint32_t *out = ct + g * (size_t)(n + 1);
    const uint32_t *a = mask + g * (size_t)n;
    uint32_t b = (uint32_t)noise[g] + (bits[g] ? ORC_MU : 0u - ORC_MU);
    for (int q = 0; q < n; q++) {
      out[q] = a[q];
      b += a[q] * (uint32_t)s[q];
    }
    out[n] = b;
  }
}

void orc_decrypt(int n, const uint8_t *s, const uint32_t *ct, size_t count, uint8_t *bits,
                 int32_t *phase) {
  for (size_t g = 0; g < count; g++) {
    const uint32_t *c = ct + g * (size_t)(n + 1);
    uint32_t ph = c[n];
    for (int q = 0; q < n; q++) ph -= c[q] * (uint32_t)s[q];
    if (bits) bits[g] = (int32_t)ph > 0;
    if (phase) phase[g] = (int32_t)ph;
  }
}

/* ------------------------------------------------------------------------- */
/* Bootstrapping context: the BSK lifted to integers (centred Torus32) and     */
/* carried into the Goldilocks NTT domain once, as the key is constant.        */
/* ------------------------------------------------------------------------- */
struct orc_ctx {
  int n;
  uint64_t *bsk_hat; /* [n][6][2][N] */
  uint32_t *ksk;     /* [N][8][4][n+1] */
};

orc_ctx *orc_ctx_create(int n, const uint32_t *bsk, const uint32_t *ksk) {
  pthread_once(&g_tab_once, tab1024_init);
  orc_ctx *ctx = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  ctx->n = n;
  size_t polys = (size_t)n * ORC_ROWS * 2;
  ctx->bsk_hat = (uint64_t *)malloc(sizeof(uint64_t) * polys * ORC_N);
  for (size_t q = 0; q < polys; q++) {
    uint64_t *dst = ctx->bsk_hat + q * ORC_N;
    for (int k = 0; k < ORC_N; k++) dst[k] = gl_from_i64((int32_t)bsk[q * ORC_N + k]);
    orc_ntt(dst, ORC_N, 0);
  }
  size_t ksk_words = (size_t)ORC_N * ORC_KS_T * 4 * (size_t)(n + 1);
  ctx->ksk = (uint32_t *)malloc(sizeof(uint32_t) * ksk_words);
  memcpy(ctx->ksk, ksk, sizeof(uint32_t) * ksk_words);
  return ctx;
}

void orc_ctx_destroy(orc_ctx *ctx) {
  if (!ctx) return;
  free(ctx->bsk_hat);
  free(ctx->ksk);
  free(ctx);
}

/* Fig. 2 "4 Forward DFTs / TGSW BK_i x TLWE temp / 2 Inverse DFTs", with l = 3: */
/* decompose both polynomials of temp, forward-transform the 6 digit polys,    */
/* multiply-accumulate with the 6 x 2 key polys, inverse-transform the 2 sums.  */
/* The sums are exact integers (|sum| < 2^50 << Q/2), reduced mod 2^32.         */
void orc_external_product(const orc_ctx *ctx, int i, const uint32_t *t0, const uint32_t *t1,
                          uint32_t *out0, uint32_t *out1) {
  const uint32_t *temp[2] = {t0, t1};
  uint32_t *outp[2] = {out0, out1};
  uint64_t *D = (uint64_t *)malloc(sizeof(uint64_t) * ORC_ROWS * ORC_N);
  uint64_t *S = (uint64_t *)malloc(sizeof(uint64_t) * 2 * ORC_N);
  for (int c = 0; c < 2; c++) {
    for (int k = 0; k < ORC_N; k++) {
      int32_t d[ORC_L];
      orc_decompose(temp[c][k], d);
      for (int p = 1; p <= ORC_L; p++) D[(c * ORC_L + p - 1) * ORC_N + k] = gl_from_i64(d[p - 1]);
    }
  }
  for (int r = 0; r < ORC_ROWS; r++) orc_ntt(D + r * ORC_N, ORC_N, 0);
  for (int co = 0; co < 2; co++) {
    uint64_t *acc = S + co * ORC_N;
    for (int k = 0; k < ORC_N; k++) acc[k] = 0;
    for (int r = 0; r < ORC_ROWS; r++) {
      const uint64_t *B = ctx->bsk_hat + (((size_t)i * ORC_ROWS + r) * 2 + co) * ORC_N;
      for (int k = 0; k < ORC_N; k++) acc[k] = gl_add(acc[k], orc_gl_mul(D[r * ORC_N + k], B[k]));
    }
    orc_ntt(acc, ORC_N, 1);
    for (int k = 0; k < ORC_N; k++) outp[co][k] = (uint32_t)gl_centred(acc[k]);
  }
  free(D);
  free(S);
}

/* Fig. 2: "Accum = out x X^-b", then n times "temp = X^a[i] x Accum - Accum",  */
/* external product with BK_i, and "+" back into Accum.  The accumulator starts */
/* as the trivial TLWE (0, testv) with testv = mu (1 + X + ... + X^(N-1)).      */
void orc_blind_rotate(const orc_ctx *ctx, const uint32_t *abar, uint32_t bbar, uint32_t *acc) {
  uint32_t testv[ORC_N], rot[ORC_N], temp[2][ORC_N], ext[2][ORC_N];
  for (int k = 0; k < ORC_N; k++) testv[k] = ORC_MU;
  memset(acc, 0, sizeof(uint32_t) * ORC_N);
  poly_mul_monomial(testv, (2 * ORC_N - bbar) % (2 * ORC_N), acc + ORC_N);
  for (int i = 0; i < ctx->n; i++) {
    for (int c = 0; c < 2; c++) {
      poly_mul_monomial(acc + c * ORC_N, abar[i], rot);
      for (int k = 0; k < ORC_N; k++) temp[c][k] = rot[k] - acc[c * ORC_N + k];
    }
    orc_external_product(ctx, i, temp[0], temp[1], ext[0], ext[1]);
    for (int c = 0; c < 2; c++)
      for (int k = 0; k < ORC_N; k++) acc[c * ORC_N + k] += ext[c][k];
  }
}

/* Coefficient 0 of the TLWE phase b - a*K is b_0 - (a_0 K_0 - sum_{j>0} a_{N-j} K_j), */
/* so the N-dim LWE sample is a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0 (reading c12).      */
void orc_sample_extract(const uint32_t *acc, uint32_t *lwe_N) {
  lwe_N[0] = acc[0];
  for (int j = 1; j < ORC_N; j++) lwe_N[j] = 0u - acc[ORC_N - j];
  lwe_N[ORC_N] = acc[ORC_N];
}

/* Fig. 2 "KeySwitch (Accum)": out = (0,...,0,b') - sum_i sum_j KSK[i][j][digit_ij]. */
void orc_keyswitch(const orc_ctx *ctx, const uint32_t *lwe_N, uint32_t *lwe_n) {
  int n = ctx->n;
  memset(lwe_n, 0, sizeof(uint32_t) * (size_t)(n + 1));
  lwe_n[n] = lwe_N[ORC_N];
  for (int i = 0; i < ORC_N; i++) {
    uint32_t d[ORC_KS_T];
    orc_ks_digits(lwe_N[i], d);
    for (int j = 1; j <= ORC_KS_T; j++) {
      const uint32_t *row = ctx->ksk + (((size_t)i * ORC_KS_T + (j - 1)) * 4 + d[j - 1]) * (size_t)(n + 1);
      for (int q = 0; q <= n; q++) lwe_n[q] -= row[q];
    }
  }
}

void orc_bootstrap_to_N(const orc_ctx *ctx, const uint32_t *ct, uint32_t *out) {
  int n = ctx->n;
  uint32_t *abar = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * ORC_N);
  for (int i = 0; i < n; i++) abar[i] = orc_modswitch(ct[i]);
  orc_blind_rotate(ctx, abar, orc_modswitch(ct[n]), acc);
  orc_sample_extract(acc, out);
  free(abar);
  free(acc);
}

/* Fig. 2 top box ("LWE out = Enc(0) - ct1 - ct2" for NAND), with the trivial   */
/* constant (0, +-1/8) or (0, +-1/4) of each gate (reading c5).                  */
void orc_gate_linear(int n, int type, const uint32_t *a, const uint32_t *b, uint32_t *out) {
  const uint32_t eighth = ORC_MU, quarter = 2 * ORC_MU;
  int32_t sign = 1, scale = 1;
  uint32_t cst = 0;
  switch (type) {
    case ORC_AND:  sign = 1;  scale = 1; cst = 0u - eighth; break;
    case ORC_NAND: sign = -1; scale = 1; cst = eighth; break;
    case ORC_OR:   sign = 1;  scale = 1; cst = eighth; break;
    case ORC_NOR:  sign = -1; scale = 1; cst = 0u - eighth; break;
    case ORC_XOR:  sign = 1;  scale = 2; cst = quarter; break;
    case ORC_XNOR: sign = -1; scale = 2; cst = 0u - quarter; break;
    default: break;
  }
  uint32_t f = (uint32_t)(sign * scale);
  for (int q = 0; q <= n; q++) out[q] = f * (a[q] + b[q]);
  out[n] += cst;
}

/* MUX (reading c15): two bootstraps without key switch, AND(sel, t) and         */
/* AND(not sel, f), summed with (0, 1/8) on the N-dim samples, one key switch.   */
void orc_gate(const orc_ctx *ctx, int type, const uint32_t *a, const uint32_t *b,
              const uint32_t *c, uint32_t *out) {
  int n = ctx->n;
  if (type == ORC_NOT || type == ORC_COPY) {
    for (int q = 0; q <= n; q++) out[q] = type == ORC_NOT ? 0u - a[q] : a[q];
    return;
  }
  if (type == ORC_CONST0 || type == ORC_CONST1) {
    memset(out, 0, sizeof(uint32_t) * (size_t)n);
    out[n] = type == ORC_CONST1 ? ORC_MU : 0u - ORC_MU;
    return;
  }
  uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint32_t *u1 = (uint32_t *)malloc(sizeof(uint32_t) * (ORC_N + 1));
  if (type == ORC_MUX) {
    uint32_t *u2 = (uint32_t *)malloc(sizeof(uint32_t) * (ORC_N + 1));
    uint32_t *nsel = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    orc_gate_linear(n, ORC_AND, a, b, lin);
    orc_bootstrap_to_N(ctx, lin, u1);
    for (int q = 0; q <= n; q++) nsel[q] = 0u - a[q];
    orc_gate_linear(n, ORC_AND, nsel, c, lin);
    orc_bootstrap_to_N(ctx, lin, u2);
    for (int q = 0; q <= ORC_N; q++) u1[q] += u2[q];
    u1[ORC_N] += ORC_MU;
    orc_keyswitch(ctx, u1, out);
    free(u2);
    free(nsel);
  } else {
    orc_gate_linear(n, type, a, b, lin);
    orc_bootstrap_to_N(ctx, lin, u1);
    orc_keyswitch(ctx, u1, out);
  }
  free(lin);
  free(u1);
}

/* ------------------------------------------------------------------------- */
/* Independent gates on a pool of POSIX threads (one gate per task).           */
/* ------------------------------------------------------------------------- */
typedef struct {
  const orc_ctx *ctx;
  const uint8_t *types;
  const uint32_t *const *a, *const *b, *const *c;
  uint32_t *const *out;
  size_t count;
  int tid, nthreads;
} gate_job;

static void *gate_worker(void *arg) {
  gate_job *j = (gate_job *)arg;
  for (size_t g = (size_t)j->tid; g < j->count; g += (size_t)j->nthreads)
    orc_gate(j->ctx, j->types[g], j->a[g], j->b[g], j->c ? j->c[g] : NULL, j->out[g]);
  return NULL;
}

static void run_gates(const orc_ctx *ctx, const uint8_t *types, const uint32_t *const *a,
                      const uint32_t *const *b, const uint32_t *const *c, uint32_t *const *out,
                      size_t count, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > count) nthreads = count ? (int)count : 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  gate_job *jobs = (gate_job *)malloc(sizeof(gate_job) * (size_t)nthreads);
  for (int t = 0; t < nthreads; t++) {
    gate_job j = {ctx, types, a, b, c, out, count, t, nthreads};
    jobs[t] = j;
    pthread_create(&th[t], NULL, gate_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

void orc_gates(const orc_ctx *ctx, const uint8_t *types, const uint32_t *a, const uint32_t *b,
               const uint32_t *c, uint32_t *out, size_t count, int nthreads) {
  size_t w = (size_t)ctx->n + 1;
  const uint32_t **pa = (const uint32_t **)malloc(sizeof(void *) * (count + 1));
  const uint32_t **pb = (const uint32_t **)malloc(sizeof(void *) * (count + 1));
  const uint32_t **pc = (const uint32_t **)malloc(sizeof(void *) * (count + 1));
  uint32_t **po = (uint32_t **)malloc(sizeof(void *) * (count + 1));
  for (size_t g = 0; g < count; g++) {
    pa[g] = a + g * w;
    pb[g] = b ? b + g * w : a + g * w;
    pc[g] = c ? c + g * w : a + g * w;
    po[g] = out + g * w;
  }
  run_gates(ctx, types, pa, pb, pc, po, count, nthreads);
  free(pa);
  free(pb);
  free(pc);
  free(po);
}

/* ------------------------------------------------------------------------- */
/* Netlists: the wave levelization of Sec. 4.2.  Successor lists and          */
/* predecessor counts, a FIFO of ready gates; a gate with no gate inputs goes  */
/* to wave 0, any other to 1 + the largest wave of its predecessors.           */
/* ------------------------------------------------------------------------- */
static int gate_arity(int type) {
  switch (type) {
    case ORC_NOT: case ORC_COPY: return 1;
    case ORC_CONST0: case ORC_CONST1: return 0;
    case ORC_MUX: return 3;
    default: return 2;
  }
}

int orc_levelize(uint32_t num_inputs, uint32_t num_gates, const uint8_t *type,
                 const uint32_t *in0, const uint32_t *in1, const uint32_t *in2, uint32_t *wave) {
  const uint32_t *ins[3] = {in0, in1, in2};
  uint64_t wires = (uint64_t)num_inputs + num_gates;
  uint32_t *npred = (uint32_t *)calloc(num_gates + 1, sizeof(uint32_t));
  uint32_t *nsucc = (uint32_t *)calloc(num_gates + 1, sizeof(uint32_t));
  for (uint32_t g = 0; g < num_gates; g++) {
    if (type[g] > ORC_CONST1) { free(npred); free(nsucc); return -1; }
    for (int s = 0; s < gate_arity(type[g]); s++) {
      uint32_t w = ins[s][g];
      if (w >= wires) { free(npred); free(nsucc); return -1; }
      if (w >= num_inputs) { npred[g]++; nsucc[w - num_inputs]++; }
    }
  }
  /* successor lists in compressed form */
  uint32_t *start = (uint32_t *)calloc(num_gates + 1, sizeof(uint32_t));
  for (uint32_t g = 0; g < num_gates; g++) start[g + 1] = start[g] + nsucc[g];
  uint32_t *succ = (uint32_t *)malloc(sizeof(uint32_t) * (start[num_gates] + 1));
  uint32_t *fill = (uint32_t *)calloc(num_gates + 1, sizeof(uint32_t));
  for (uint32_t g = 0; g < num_gates; g++)
    for (int s = 0; s < gate_arity(type[g]); s++) {
      uint32_t w = ins[s][g];
      if (w >= num_inputs) {
        uint32_t p = w - num_inputs;
        succ[start[p] + fill[p]++] = g;
      }
    }
  uint32_t *fifo = (uint32_t *)malloc(sizeof(uint32_t) * (num_gates + 1));
  uint32_t head = 0, tail = 0;
  for (uint32_t g = 0; g < num_gates; g++)
    if (npred[g] == 0) fifo[tail++] = g;
  while (head < tail) {
    uint32_t g = fifo[head++];
    uint32_t wv = 0;
    int has_pred = 0;
    for (int s = 0; s < gate_arity(type[g]); s++) {
      uint32_t w = ins[s][g];
      if (w >= num_inputs) {
        uint32_t pw = wave[w - num_inputs];
        if (!has_pred || pw + 1 > wv) wv = pw + 1;
        has_pred = 1;
      }
    }
    wave[g] = wv;
    for (uint32_t e = start[g]; e < start[g + 1]; e++)
      if (--npred[succ[e]] == 0) fifo[tail++] = succ[e];
  }
  int rc = head == num_gates ? 0 : -2;
  free(npred); free(nsucc); free(start); free(succ); free(fill); free(fifo);
  return rc;
}

int orc_eval_netlist(const orc_ctx *ctx, uint32_t num_inputs, uint32_t num_gates,
                     const uint8_t *type, const uint32_t *in0, const uint32_t *in1,
                     const uint32_t *in2, uint32_t num_outputs, const uint32_t *outputs,
                     const uint32_t *ct_in, uint32_t *ct_out, int nthreads) {
  size_t w = (size_t)ctx->n + 1;
  uint32_t *wave = (uint32_t *)malloc(sizeof(uint32_t) * (num_gates + 1));
  int rc = orc_levelize(num_inputs, num_gates, type, in0, in1, in2, wave);
  if (rc) { free(wave); return rc; }
  for (uint32_t o = 0; o < num_outputs; o++)
    if (outputs[o] >= (uint64_t)num_inputs + num_gates) { free(wave); return -1; }
  uint32_t *wires = (uint32_t *)malloc(sizeof(uint32_t) * w * ((size_t)num_inputs + num_gates));
  memcpy(wires, ct_in, sizeof(uint32_t) * w * num_inputs);
  uint32_t depth = 0;
  for (uint32_t g = 0; g < num_gates; g++)
    if (wave[g] + 1 > depth) depth = wave[g] + 1;
  const uint32_t **pa = (const uint32_t **)malloc(sizeof(void *) * (num_gates + 1));
  const uint32_t **pb = (const uint32_t **)malloc(sizeof(void *) * (num_gates + 1));
  const uint32_t **pc = (const uint32_t **)malloc(sizeof(void *) * (num_gates + 1));
  uint32_t **po = (uint32_t **)malloc(sizeof(void *) * (num_gates + 1));
  uint8_t *ty = (uint8_t *)malloc(num_gates + 1);
  for (uint32_t lv = 0; lv < depth; lv++) {
    size_t cnt = 0;
    for (uint32_t g = 0; g < num_gates; g++) {
      if (wave[g] != lv) continue;
      int ar = gate_arity(type[g]);
      pa[cnt] = wires + (size_t)(ar > 0 ? in0[g] : 0) * w;
      pb[cnt] = wires + (size_t)(ar > 1 ? in1[g] : 0) * w;
      pc[cnt] = wires + (size_t)(ar > 2 ? in2[g] : 0) * w;
      po[cnt] = wires + ((size_t)num_inputs + g) * w;
      ty[cnt] = type[g];
      cnt++;
    }
    run_gates(ctx, ty, pa, pb, pc, po, cnt, nthreads);
  }
  for (uint32_t o = 0; o < num_outputs; o++)
    memcpy(ct_out + (size_t)o * w, wires + (size_t)outputs[o] * w, sizeof(uint32_t) * w);
  free(wave); free(wires); free(pa); free(pb); free(pc); free(po); free(ty);
  return 0;
}
