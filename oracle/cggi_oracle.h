/*
 * cggi_oracle.h -- plain, slow CPU oracle for CGGI gate bootstrapping.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links,
 * includes or calls anything here, and nothing here is shared with it.
 *
 * What it computes (paper: "ArctyrEX", arXiv 2306.11006):
 *   - gate evaluation as drawn in Fig. 2 (Sec. 2.2): a linear pre-combination of
 *     the LWE inputs, blind rotation by n CMux external products (TGSW x TLWE,
 *     "Repeat n times"), then a key switch;
 *   - polynomial products through an exact negacyclic NTT over the prime
 *     Q = 2^64 - 2^32 + 1 with the element g = 12037493425763644479 (Sec. 5.4);
 *   - the wave levelization of Sec. 4.2 (FIFO topological sort).
 * Points the paper leaves open (mod switch, decomposition, sample extraction,
 * key-switch digits, test vector, MUX construction) follow the readings listed
 * in the design notes; each function below states the reading it takes.
 *
 * Parameters: N = 1024, k = 1, Bg = 2^7, l = 3, key-switch base 2^2 with t = 8,
 * Torus32 = uint32 mod 2^32.  The LWE dimension n is a runtime argument
 * (1 <= n <= 1024; the standard set uses 630, Sec. 2.2).  Building with
 * -DORC_L=2 -DORC_BG_BITS=10 gives the variant with l = 2 (the paper's Fig. 2
 * draws 4 forward DFTs, i.e. (k+1) l = 4) and Bg = 2^10; the arrays documented
 * with 6 rows then have 2 l = 4.
 *
 * Parity status: every function here is pinned by a CPU test (closed forms,
 * brute force, special cases); none is "parity unpinned".
 */
#ifndef CGGI_ORACLE_H
#define CGGI_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_N 1024          /* TLWE ring degree (Sec. 2.2: "1024-degree polynomials") */
#ifndef ORC_L               /* the default set; a second build takes l = 2, Bg = 2^10 */
#define ORC_BG_BITS 7       /* gadget base Bg = 2^7 */
#define ORC_L 3             /* gadget length l */
#endif
#define ORC_ROWS (2 * ORC_L) /* (k+1) l rows of a TGSW sample */
#define ORC_KS_BITS 2       /* key-switch base 2^2 */
#define ORC_KS_T 8          /* key-switch digits */
#define ORC_MU 0x20000000u  /* encoding of "true": +1/8 of the torus */

/* gate opcodes (the same numbering as the product's C-ABI) */
enum { ORC_AND = 0, ORC_NAND, ORC_OR, ORC_NOR, ORC_XOR, ORC_XNOR,
       ORC_NOT, ORC_MUX, ORC_COPY, ORC_CONST0, ORC_CONST1 };

/* ---- Goldilocks field (Sec. 5.4) ---- */
uint64_t orc_gl_mul(uint64_t a, uint64_t b);
uint64_t orc_gl_pow(uint64_t a, uint64_t e);
/* In-place negacyclic NTT of length m (power of two, 2 <= m <= 1024) over Q,
 * built from psi_m = g^(2^32 / 2m).  Forward output is in natural order:
 * A[k] = sum_j a[j] psi^((2k+1) j).  inverse != 0 computes the inverse. */
void orc_ntt(uint64_t *a, int m, int inverse);
/* Exact negacyclic product c = a * b mod (X^m + 1) over the integers for
 * int64 inputs whose exact result lies in (-Q/2, Q/2); via the NTT. */
void orc_negacyclic_mul_ntt(const int64_t *a, const int64_t *b, int64_t *c, int m);
/* Same product by the schoolbook definition (int128 accumulation). */
void orc_negacyclic_mul_schoolbook(const int64_t *a, const int64_t *b, int64_t *c, int m);

/* ---- scalar pieces ---- */
uint32_t orc_modswitch(uint32_t x);                    /* round(x 2N / 2^32) mod 2N */
void orc_decompose(uint32_t x, int32_t digits[ORC_L]); /* signed gadget digits, p = 1 first */
void orc_ks_digits(uint32_t x, uint32_t digits[ORC_KS_T]); /* unsigned base-4 digits, j = 1 first */

/* ---- keys / encryption (client side; all randomness is passed in) ----
 * s[n] in {0,1}; K[N] in {0,1}.
 * bsk_mask [n][6][N] u32 uniform, bsk_noise [n][6][N] i32 (already in Torus32 units).
 * ksk_mask [N][8][3][n] u32 uniform, ksk_noise [N][8][3] i32.
 * Output bsk [n][6][2][N] u32: row r = c*l + (p-1), component 0 = mask, 1 = body.
 * Output ksk [N][8][4][n+1] u32: entry [i][j-1][v] = LWE_s(v K_i 2^(32-2j)); v = 0 rows zero. */
void orc_keygen(int n, const uint8_t *s, const uint8_t *K,
                const uint32_t *bsk_mask, const int32_t *bsk_noise,
                const uint32_t *ksk_mask, const int32_t *ksk_noise,
                uint32_t *bsk, uint32_t *ksk);
/* ct [count][n+1] = (a, b = <a,s> + e + (bit ? +1/8 : -1/8)). */
void orc_encrypt(int n, const uint8_t *s, const uint32_t *mask, const int32_t *noise,
                 const uint8_t *bits, size_t count, uint32_t *ct);
/* phase = b - <a,s> as int32; bit = phase > 0.  Either output may be NULL. */
void orc_decrypt(int n, const uint8_t *s, const uint32_t *ct, size_t count,
                 uint8_t *bits, int32_t *phase);

/* ---- bootstrapping context ---- */
typedef struct orc_ctx orc_ctx;
orc_ctx *orc_ctx_create(int n, const uint32_t *bsk, const uint32_t *ksk);
void orc_ctx_destroy(orc_ctx *ctx);

/* One external product out = BSK_i [x] (t0, t1) (Fig. 2 "TGSW BK_i x TLWE temp"). */
void orc_external_product(const orc_ctx *ctx, int i, const uint32_t *t0, const uint32_t *t1,
                          uint32_t *out0, uint32_t *out1);
/* Blind rotation of mod-switched values abar[n], bbar; acc [2][N] out. */
void orc_blind_rotate(const orc_ctx *ctx, const uint32_t *abar, uint32_t bbar, uint32_t *acc);
/* Sample extraction of coefficient 0: acc [2][N] -> lwe_N [N+1]. */
void orc_sample_extract(const uint32_t *acc, uint32_t *lwe_N);
/* Key switch lwe_N [N+1] -> lwe_n [n+1]. */
void orc_keyswitch(const orc_ctx *ctx, const uint32_t *lwe_N, uint32_t *lwe_n);
/* mod switch + blind rotation + extraction of one LWE_n sample: out [N+1]. */
void orc_bootstrap_to_N(const orc_ctx *ctx, const uint32_t *ct, uint32_t *out);
/* Linear pre-combination of a two-input gate (Fig. 2 top box). */
void orc_gate_linear(int n, int type, const uint32_t *a, const uint32_t *b, uint32_t *out);
/* Full gate.  ct_c is only read by MUX (sel = a, true-input = b, false-input = c). */
void orc_gate(const orc_ctx *ctx, int type, const uint32_t *a, const uint32_t *b,
              const uint32_t *c, uint32_t *out);
/* count independent gates, nthreads POSIX threads (<= 0: one). */
void orc_gates(const orc_ctx *ctx, const uint8_t *types, const uint32_t *a, const uint32_t *b,
               const uint32_t *c, uint32_t *out, size_t count, int nthreads);

/* ---- netlists (Sec. 4.2) ----
 * Wire ids: 0..num_inputs-1 are inputs, num_inputs + g is gate g's output.
 * wave[g] receives the gate's wave index.  Returns 0, or -1 on a bad wire id,
 * -2 on a cycle. */
int orc_levelize(uint32_t num_inputs, uint32_t num_gates, const uint8_t *type,
                 const uint32_t *in0, const uint32_t *in1, const uint32_t *in2, uint32_t *wave);
/* Evaluate wave by wave; ct_in [num_inputs][n+1], ct_out [num_outputs][n+1]. */
int orc_eval_netlist(const orc_ctx *ctx, uint32_t num_inputs, uint32_t num_gates,
                     const uint8_t *type, const uint32_t *in0, const uint32_t *in1,
                     const uint32_t *in2, uint32_t num_outputs, const uint32_t *outputs,
                     const uint32_t *ct_in, uint32_t *ct_out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
