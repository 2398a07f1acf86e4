// br_kernel.cuh -- the blind-rotation kernel of CGGI gate bootstrapping on GB300.
//
//   br_kernel<H, GT, L>: gate pre-combination, mod switch, blind rotation through n
//   CMux external products, sample extraction (Fig. 2 and Sec. 2.2 of the paper).
//   Each br_h*.cu translation unit instantiates the shapes of one H.
//
// Blind rotation kernel organisation.  A gate is processed by 2H warps: warp
// (P, h) carries prime P of the CRT pair and the h-th group of 2L/H TGSW rows
// (gadget length L: 3 for Bg = 2^7, 2 for the paper's own Bg = 2^10).
// GT gates share a CTA so that every bootstrapping-key row (16 KiB: two output
// polynomials x two primes) is brought into shared memory once per CTA
// (cp.async.bulk into a 4..8-stage mbarrier ring) and read by all 2 GT warps that
// use it.  There is no producer warp: the last of those warps to finish with a
// slot refills it with the row kStages ahead, so a CTA of 12 warps keeps three
// warps per scheduler and 168 registers a thread.  The MAC keeps each
// coefficient's exact 64-bit sum of row products, reduced once per CMux: in
// registers in CTAs of at most 8 warps (255 registers a thread), in tensor
// memory (TMEM, tcgen05.alloc / ld / st) in the 12-warp shapes whose warps take
// two or more rows.  Every wait is bounded: on a
// timeout the kernel records kDevTimeout in the device status word, stops
// waiting, runs to the end, lets its copies in flight land and returns.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "arx_device.cuh"

namespace arx {
namespace br {

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
static_assert(32ull * kQ0 < (1ull << 32) && 32ull * kQ1 < (1ull << 32), "lazy transform bounds");
static_assert(2ull * kQ0 < 3ull * kQ1 && 5ull * kQ1 < (1ull << 32), "CRT difference stays in (0, 2^32)");
static_assert(6ull * 1024 * 64 * (1ull << 31) * 2 < kM / 4, "CRT range must hold the exact products");

// Gadget decomposition offset: 2^10 rounds to the top 21 bits, 64 * 2^(32-7p)
// recentres each 7-bit digit into [-64, 64).
constexpr uint32_t kDecOffset = (1u << 10) + (64u << 25) + (64u << 18) + (64u << 11);
// The same for the gadget variant l = 2, Bg = 2^10: 2^11 rounds to the top 20
// bits, 512 * 2^(32-10p) recentres each 10-bit digit into [-512, 512).
constexpr uint32_t kDecOffset2 = (1u << 11) + (512u << 22) + (512u << 12);

constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at GB300 clocks

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
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

// Bounded wait: a phase that has already completed returns at once (the abort
// flag is read only on the slow path); returns false (and flags the CTA and the
// device status) once `limit` clock64 cycles have passed (kWaitCycles in the
// kernel).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *status, long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  if (*abort_flag) return false;
  long long t0 = clock64();
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

__device__ __forceinline__ void named_bar(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// ---- tensor memory (TMEM) as a spill space for the MAC sums ---------------
// A warp may address only its quadrant of the 128 TMEM lanes: lanes
// 32 (w mod 4) .. + 31 for warp w of the CTA; lane i of the warp holds TMEM lane
// 32 (w mod 4) + i.  Address: lane << 16 | column.  Each helper waits for its
// own access, so registers are free (store) or valid (load) on return.
__device__ __forceinline__ void tmem_ld64(uint32_t (&r)[64], uint32_t taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64};\n"
      "tcgen05.wait::st.sync.aligned;"
      :
      : "r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]),
        "r"(r[32]), "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]), "r"(r[37]), "r"(r[38]), "r"(r[39]),
        "r"(r[40]), "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]), "r"(r[46]), "r"(r[47]),
        "r"(r[48]), "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]), "r"(r[55]),
        "r"(r[56]), "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63])
      );
}

// One warp allocates `cols` TMEM columns (a power of two, 32 .. 512) and gives up
// the CTA's right to allocate more; the address lands in *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// w[2i], w[2i + 1]: low and high word of a 64-bit sum; adds x b in place (a
// carry chain on the two words: no register moves between the TMEM blocks and
// 64-bit pairs; measured 1.6-2.2 % faster on a full wave than a 64-bit add).
__device__ __forceinline__ void mac64(uint32_t (&w)[64], int i, uint32_t x, uint32_t b) {
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
      : "+r"(w[2 * i]), "+r"(w[2 * i + 1])
      : "r"(x), "r"(b));
}

__device__ __forceinline__ uint64_t pair64(const uint32_t (&w)[64], int i) {
  return ((uint64_t)w[2 * i + 1] << 32) | w[2 * i];
}

__device__ __forceinline__ uint32_t modswitch(uint32_t x) { return (x + (1u << 20)) >> 21; }

// (x0 mod q0, x1 mod q1), each in [0, 2q) -> the centred integer V, mod 2^32.
// Garner: X = x0 + q0 k, k = (x1 - x0) q0^-1 mod q1 fully reduced (d stays in
// (0, 2^32) for these input ranges).  |V| < 2^50 for the gadget l = 3 and
// |V| <= 2^52 for l = 2, so the coefficient K of V's representative in
// [0, q0 q1) is below 2^23 (l = 3) or 2^25 + 2^12 (l = 2; 2^52 / q0 is just
// above 2^25) when V >= 0, and above q1 minus those when V < 0; q1 / 2 > 2^26
// lies between (a margin of 8x for l = 3, 2x for l = 2): V is negative exactly
// when k >= q1 / 2, and
// then X - q0 q1 = V.  An x0 one q0 above its residue gives k = K - 1; for
// K = 0 (0 <= V < q0) that wraps to q1 - 1, X = V + q0 q1, and the same rule
// returns V.  (The worst cases of both gadgets are checked on the CPU in
// tests/test_crt_bounds.py.)
__device__ __forceinline__ uint32_t crt_torus(uint32_t x0, uint32_t x1) {
  const uint32_t d = x1 + 3u * kQ1 - x0;
  const uint32_t k = csub(shoup_mul(kQ0InvQ1, kQ0InvQ1Shoup, d, kQ1), kQ1);
  const uint32_t r = kQ0 * k + x0;
  return k >= kQ1 / 2 ? r - (uint32_t)kM : r;
}

// Gadget digits of temp = X^a ACC - ACC for both polynomials, computed by the
// gate's threads into dig[c]: for L = 3 three biased 7-bit fields (digit + 64)
// with p = 1 in the low byte; for L = 2 two biased 10-bit fields (digit + 512)
// with p = 1 in the low half.  Position k = r + 32 e (r = k mod 32) sits in row
// r, 16-byte chunk (e / 4) XOR (r mod 8), word e mod 4 of a 32 x 32 word block:
// lane r of a warp reads its positions r + 32 e as eight 16-byte loads, and a
// thread stores the four positions of one chunk as one 16-byte store (both
// free of bank conflicts).
template <int kGateThreads, int L>
__device__ __forceinline__ void make_digits(uint32_t *dig, const uint32_t *A, uint32_t a, int tid_g) {
#pragma unroll 1
  for (int it = tid_g; it < 2 * 256; it += kGateThreads) {  // (c, chunk j, row r)
    const uint32_t r = (uint32_t)it & 31u, j = ((uint32_t)it >> 5) & 7u, c = (uint32_t)it >> 8;
    const uint32_t *P = A + c * kN;
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t k = r + 32u * (4u * j + (uint32_t)i);
      const uint32_t jr = (k - a) & 2047u;
      uint32_t v = P[jr & 1023u];
      v = (jr & 1024u) ? 0u - v : v;
      if constexpr (L == 3) {
        const uint32_t y = v - P[k] + kDecOffset;
        w[i] = (y >> 25) | ((y >> 10) & 0x7F00u) | ((y << 5) & 0x7F0000u);
      } else {
        const uint32_t y = v - P[k] + kDecOffset2;
        w[i] = (y >> 22) | (((y >> 12) & 0x3FFu) << 16);
      }
    }
    reinterpret_cast<uint4 *>(dig + c * kN)[r * 8u + (j ^ (r & 7u))] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

struct BrShared {
  uint32_t *ring;     // kStages x kChunkWords
  uint32_t *dtab;     // [prime][digit_tab_words]: table products of digit values (see ntt_fwd)
  uint32_t *acc;      // GT x [2][N]
  uint32_t *dig;      // GT x [2][N] packed gadget digits
  uint32_t *scratch;  // consumer warps x kScratch
  uint16_t *abar;     // GT x kAbarPitch
  uint64_t *full;     // kStages: row landed (transaction count)
  uint32_t *cnt;      // kStages: warps done with the slot's current row
  uint32_t *issued;   // kStages: 1 + the last row copied into the slot
  volatile int *abort_flag;
  uint32_t *tmem;     // TMEM base address written by tcgen05.alloc (tmem_mac shapes)
};

constexpr int kAbarPitch = 640;
constexpr size_t kSmemLimit = 227 * 1024;  // opt-in shared memory per CTA

template <int H>
__host__ __device__ constexpr int scratch_words() { return (H == 1 ? 1 : 2) * kXpose; }

// Digit values of the gadget: Bg (7-bit digits for L = 3, 10-bit for L = 2).
template <int L>
__host__ __device__ constexpr int digit_values() { return L == 3 ? 128 : 1024; }

// Words of a prime's digit tables: for L = 3 the products of the first two
// forward stages, [z1, z2, z2 z1, z3, z3 z1][u] (ntt_fwd<2>); for L = 2 zeta[1] u
// (ntt_fwd<1>).
template <int L>
__host__ __device__ constexpr int digit_tab_words() { return L == 3 ? 5 * 128 : 1024; }

template <int H, int GT, int L = 3>
constexpr size_t br_fixed_bytes() {
  return (size_t)GT * 4 * kN * 4 + (size_t)2 * H * GT * scratch_words<H>() * 4 + (size_t)GT * kAbarPitch * 2 +
         (size_t)2 * digit_tab_words<L>() * 4 + 2 * 8 * 8 + 16;
}

// Ring depth: as many key rows in flight as shared memory allows, 4..8.
template <int H, int GT, int L = 3>
__host__ __device__ constexpr int br_stages() {
  return (kSmemLimit - br_fixed_bytes<H, GT, L>()) / kChunkBytes >= 8 ? 8
         : (int)((kSmemLimit - br_fixed_bytes<H, GT, L>()) / kChunkBytes);
}

template <int H, int GT, int L = 3>
constexpr size_t br_smem_bytes() {
  return (size_t)br_stages<H, GT, L>() * kChunkBytes + br_fixed_bytes<H, GT, L>();
}

template <int H, int GT, int L = 3>
__device__ __forceinline__ BrShared br_carve(uint8_t *smem) {
  constexpr int kStages = br_stages<H, GT, L>();
  BrShared s;
  s.ring = reinterpret_cast<uint32_t *>(smem);
  s.dtab = s.ring + kStages * kChunkWords;
  s.acc = s.dtab + 2 * digit_tab_words<L>();
  s.dig = s.acc + GT * 2 * kN;
  s.scratch = s.dig + GT * 2 * kN;
  s.abar = reinterpret_cast<uint16_t *>(s.scratch + 2 * H * GT * scratch_words<H>());
  s.full = reinterpret_cast<uint64_t *>(s.abar + GT * kAbarPitch);
  s.cnt = reinterpret_cast<uint32_t *>(s.full + kStages);
  s.issued = s.cnt + kStages;
  s.abort_flag = reinterpret_cast<volatile int *>(s.issued + kStages);
  s.tmem = reinterpret_cast<uint32_t *>(s.issued + kStages + 1);
  return s;
}

// MAC forms.  wide_mac: CTAs of at most 8 warps (a thread may hold 255
// registers) keep each coefficient's exact 64-bit sum of row products in
// registers.  tmem_mac: the 12-warp shapes whose warps take at least two rows
// (168 registers a thread) keep those sums in tensor memory between rows, 128
// columns per warp (three warps share each lane quadrant: 384 of the 512
// columns allocated).  Both reduce once per CMux.  Otherwise (one row per warp)
// each product is reduced on its own.
template <int H, int GT, int L>
__host__ __device__ constexpr bool wide_mac() { return 2 * H * GT <= 8; }
template <int H, int GT, int L>
__host__ __device__ constexpr bool tmem_mac() { return !wide_mac<H, GT, L>() && 2 * L / H >= 2; }
constexpr uint32_t kTmemCols = 512;

// Key rows this CTA consumes: 2L n per tile of GT gates (2L TGSW rows per CMux).
template <int GT, int L>
__device__ __forceinline__ uint32_t cta_rows(const BrArgs &args) {
  const int tiles = (args.num_jobs + GT - 1) / GT;
  const int mine = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  return (uint32_t)mine * (2u * L) * (uint32_t)args.n;
}

// Copy key row jc of the CTA's sequence (row jc mod 2Ln of the key of its tile
// jc / 2Ln: CMux i, TGSW row r) into its ring slot.  The gates of a tile share
// one key set (the host groups them so).
// it_hint / bsk_hint: the caller's tile iteration and that tile's key (a row of
// another tile looks its key up).
template <int kStages, int GT, int L>
__device__ __forceinline__ void issue_row(const BrShared &S, const BrArgs &args, uint32_t jc, uint32_t it_hint = ~0u,
                                          const uint32_t *bsk_hint = nullptr) {
  const uint32_t slot = jc % kStages;
  const uint32_t per_tile = 2u * L * (uint32_t)args.n;
  const uint32_t it = jc / per_tile;
  const uint32_t tile = blockIdx.x + it * gridDim.x;
  const uint32_t *bsk = it == it_hint ? bsk_hint : args.bsk[args.jobs[tile * GT].key];
  S.issued[slot] = jc + 1u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic reads of the slot before the copy
  mbar_expect_tx(S.full + slot, kChunkBytes);
  bulk_g2s(S.ring + slot * kChunkWords, bsk + (size_t)(jc % per_tile) * kChunkWords, kChunkBytes, S.full + slot);
}

// One warp (prime P, row group h) over all tiles of the launch.  The
// same code serves both primes; the owner of output c (warp (P, c) for H > 1,
// both outputs for H = 1) keeps that output's accumulator in acc0.
template <int H, int GT, int L>
__device__ __forceinline__ void br_consumer(const BrShared &S, const BrArgs &args, int g, int h, int P, int lane,
                                            uint32_t taddr) {
  constexpr int kRows = 2 * L;  // TGSW rows per CMux
  static_assert(kRows % H == 0, "row groups");
  constexpr int kRpg = kRows / H;
  constexpr int kScr = scratch_words<H>();
  constexpr int kGateThreads = 64 * H;
  constexpr int kStages = br_stages<H, GT, L>();
  constexpr bool kWide = wide_mac<H, GT, L>();
  constexpr bool kTmem = tmem_mac<H, GT, L>();  // taddr: this warp's 128 TMEM columns
  constexpr int kInvIn = kWide || kTmem ? 8 : 12;  // the inverse's input bound in q (gs_bfly)
  const int n = args.n;
  const int bar_id = 1 + g;
  const int role = h * 2 + P;
  const int wbase = g * 2 * H;  // first warp of this gate
  const int tid_g = role * 32 + lane;
  const int cA = h < 2 ? h : 0;  // output held in acc0
  uint32_t *A = S.acc + g * 2 * kN;
  uint32_t *D = S.dig + g * 2 * kN;
  uint16_t *abar = S.abar + g * kAbarPitch;
  uint32_t *myscr = S.scratch + (wbase + role) * kScr;
  PrimeRT pr = prime_rt(P, args.tc);
  if (L == 2) {  // first-stage offsets of 10-bit digits
    pr.dc = args.tc.dig_c2[P];
    pr.dd = args.tc.dig_d2[P];
  }
  const uint2 *tw1f = args.tc.fwd1[P];
  const uint2 *tw2f = args.tg->fwd2[P];
  const uint2 *gsi1 = args.tg->gsi1[P];
  const int tiles = (args.num_jobs + GT - 1) / GT;
  const uint32_t rows = cta_rows<GT, L>(args);
  uint32_t it = 0;

  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
    const int job_idx = tile * GT + g;
    const bool active = job_idx < args.num_jobs;
    const BrJob jb = args.jobs[active ? job_idx : args.num_jobs - 1];
    const uint32_t *tile_bsk = args.bsk[args.jobs[tile * GT].key];  // the tile's gates share one key set
    const uint32_t *wa = args.wires + (size_t)jb.ia * kWireStride;
    const uint32_t *wb = args.wires + (size_t)jb.ib * kWireStride;
    const uint32_t sa = (uint32_t)(int32_t)jb.sa, sb = (uint32_t)(int32_t)jb.sb;
    // Fig. 2 top box: linear pre-combination, then the mod switch to Z_2N.
    for (int k = tid_g; k < n; k += kGateThreads) abar[k] = (uint16_t)modswitch(sa * wa[k] + sb * wb[k]);
    const uint32_t bbar = modswitch(jb.cst + sa * wa[n] + sb * wb[n]);
    // ACC = X^-bbar (0, testv), testv = mu (1 + X + ... + X^(N-1)).
    const uint32_t shift = (2u * kN - bbar) & (2u * kN - 1);
    for (int k = tid_g; k < 2 * kN; k += kGateThreads) {
      uint32_t v = 0;
      if (k >= kN) v = (((uint32_t)(k - kN) - shift) & (2u * kN - 1)) < (uint32_t)kN ? kMu : 0u - kMu;
      A[k] = v;
    }
    named_bar(bar_id, kGateThreads);

    for (int i = 0; i < n; ++i) {
      make_digits<kGateThreads, L>(D, A, abar[i], tid_g);
      named_bar(bar_id, kGateThreads);  // B0: digits ready
      uint32_t acc0[32], acc1[32];
      // kWide: the MAC keeps the exact 64-bit sum of the row products (one
      // 32 x 32 -> 64-bit multiply-add per product) and reduces it once after the rows
      uint64_t wacc0[kWide ? 32 : 1], wacc1[kWide ? 32 : 1];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        if constexpr (kWide) {
          wacc0[e] = wacc1[e] = 0;
        } else if constexpr (!kTmem) {
          acc0[e] = acc1[e] = 0;
        }
      }
#pragma unroll 1
      for (int rr = 0; rr < kRpg; ++rr) {
        const int r = h * kRpg + rr;
        const int c = r / L, p = r - L * (r / L);
        // positions lane + 32 e, e = 4 q .. 4 q + 3, from chunk q of row lane (make_digits)
        const uint4 *dc = reinterpret_cast<const uint4 *>(D + c * kN) + lane * 8;
        uint32_t x[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint4 v = dc[q ^ (lane & 7)];
          if constexpr (L == 3) {
            const uint32_t sel = 0x4440u | (uint32_t)p;  // byte p of the packed digits, zero-extended
            x[4 * q + 0] = __byte_perm(v.x, 0u, sel);
            x[4 * q + 1] = __byte_perm(v.y, 0u, sel);
            x[4 * q + 2] = __byte_perm(v.z, 0u, sel);
            x[4 * q + 3] = __byte_perm(v.w, 0u, sel);
          } else {
            const uint32_t sh = 16u * (uint32_t)p;  // half p of the packed digits
            x[4 * q + 0] = (v.x >> sh) & 0xFFFFu;
            x[4 * q + 1] = (v.y >> sh) & 0xFFFFu;
            x[4 * q + 2] = (v.z >> sh) & 0xFFFFu;
            x[4 * q + 3] = (v.w >> sh) & 0xFFFFu;
          }
        }
        ntt_fwd<L == 3 ? 2 : 1>(x, myscr, tw1f, tw2f, pr, lane, S.dtab + P * digit_tab_words<L>(), args.tc.dig4[P]);
        // MAC with the NTT-domain key row staged in the ring.
        const uint32_t jc = (it * (uint32_t)n + (uint32_t)i) * (uint32_t)kRows + (uint32_t)r;
        const uint32_t slot = jc % kStages;
        mbar_wait(S.full + slot, (jc / kStages) & 1u, S.abort_flag, args.status);
        const uint4 *B0 = reinterpret_cast<const uint4 *>(S.ring + slot * kChunkWords + (cA * 2 + P) * kN);
        const uint4 *B1 = reinterpret_cast<const uint4 *>(S.ring + slot * kChunkWords + ((1 - cA) * 2 + P) * kN);
        if constexpr (kWide) {
#pragma unroll
          for (int e4 = 0; e4 < 8; ++e4) {
            const uint4 b0 = B0[e4 * 32 + lane];
            const uint4 b1 = B1[e4 * 32 + lane];
            wacc0[4 * e4 + 0] += (uint64_t)x[4 * e4 + 0] * b0.x;
            wacc0[4 * e4 + 1] += (uint64_t)x[4 * e4 + 1] * b0.y;
            wacc0[4 * e4 + 2] += (uint64_t)x[4 * e4 + 2] * b0.z;
            wacc0[4 * e4 + 3] += (uint64_t)x[4 * e4 + 3] * b0.w;
            wacc1[4 * e4 + 0] += (uint64_t)x[4 * e4 + 0] * b1.x;
            wacc1[4 * e4 + 1] += (uint64_t)x[4 * e4 + 1] * b1.y;
            wacc1[4 * e4 + 2] += (uint64_t)x[4 * e4 + 2] * b1.z;
            wacc1[4 * e4 + 3] += (uint64_t)x[4 * e4 + 3] * b1.w;
          }
        } else if constexpr (kTmem) {
          // this row's products join the exact sums kept in TMEM: output cA in
          // columns 0 .. 63 of the warp's block, 1 - cA in 64 .. 127
#pragma unroll 1
          for (int o = 0; o < 2; ++o) {
            const uint4 *B = o == 0 ? B0 : B1;
            uint32_t w[64];
            __syncwarp();
            if (rr == 0) {
#pragma unroll
              for (int k = 0; k < 64; ++k) w[k] = 0u;
            } else {
              tmem_ld64(w, taddr + 64u * (uint32_t)o);
            }
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
              const uint4 b = B[e4 * 32 + lane];
              mac64(w, 4 * e4 + 0, x[4 * e4 + 0], b.x);
              mac64(w, 4 * e4 + 1, x[4 * e4 + 1], b.y);
              mac64(w, 4 * e4 + 2, x[4 * e4 + 2], b.z);
              mac64(w, 4 * e4 + 3, x[4 * e4 + 3], b.w);
            }
            tmem_st64(taddr + 64u * (uint32_t)o, w);
          }
        } else {
#pragma unroll
          for (int e4 = 0; e4 < 8; ++e4) {
            const uint4 b0 = B0[e4 * 32 + lane];
            const uint4 b1 = B1[e4 * 32 + lane];
            acc0[4 * e4 + 0] += mont_mul(x[4 * e4 + 0], b0.x, pr);
            acc0[4 * e4 + 1] += mont_mul(x[4 * e4 + 1], b0.y, pr);
            acc0[4 * e4 + 2] += mont_mul(x[4 * e4 + 2], b0.z, pr);
            acc0[4 * e4 + 3] += mont_mul(x[4 * e4 + 3], b0.w, pr);
            acc1[4 * e4 + 0] += mont_mul(x[4 * e4 + 0], b1.x, pr);
            acc1[4 * e4 + 1] += mont_mul(x[4 * e4 + 1], b1.y, pr);
            acc1[4 * e4 + 2] += mont_mul(x[4 * e4 + 2], b1.z, pr);
            acc1[4 * e4 + 3] += mont_mul(x[4 * e4 + 3], b1.w, pr);
          }
        }
        __syncwarp();
        if (lane == 0) {  // the slot's last user refills it
          __threadfence_block();
          if (atomicAdd(S.cnt + slot, 1u) == 2u * GT - 1u) {
            __threadfence_block();
            S.cnt[slot] = 0u;
            if (jc + kStages < rows) issue_row<kStages, GT, L>(S, args, jc + kStages, it, tile_bsk);
          }
        }
      }
      if constexpr (kWide) {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          acc0[e] = mont_redc(wacc0[e], pr);
          acc1[e] = mont_redc(wacc1[e], pr);
        }
      }
      if constexpr (kTmem) {
        uint32_t w[64];
        __syncwarp();
        tmem_ld64(w, taddr);
#pragma unroll
        for (int e = 0; e < 32; ++e) acc0[e] = mont_redc(pair64(w, e), pr);
        tmem_ld64(w, taddr + 64u);
#pragma unroll
        for (int e = 0; e < 32; ++e) acc1[e] = mont_redc(pair64(w, e), pr);
      }

      // prime P combines coefficients e in [16 P, 16 P + 16) and sends the other half;
      // register arrays need static indices, hence the selects on P
      if constexpr (H == 1) {
        // both outputs: one inverse code path, the accumulators swapped between uses
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
          ntt_inv_gs<kInvIn>(acc0, myscr, gsi1, args.tc.gsi2[P], pr, lane);
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const uint32_t t = acc0[e];
            acc0[e] = acc1[e];
            acc1[e] = t;
          }
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          myscr[e * 32 + lane] = P ? acc0[e] : acc0[16 + e];
          myscr[512 + e * 32 + lane] = P ? acc1[e] : acc1[16 + e];
        }
        named_bar(bar_id, kGateThreads);  // B2: CRT halves posted
        const uint32_t *peer = S.scratch + (wbase + (1 - P)) * kScr;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const uint32_t m0 = P ? acc0[16 + e] : acc0[e], m1 = P ? acc1[16 + e] : acc1[e];
          const uint32_t o0 = peer[e * 32 + lane], o1 = peer[512 + e * 32 + lane];
          const int pos = lane + 32 * (16 * P + e);
          A[pos] += P == 0 ? crt_torus(m0, o0) : crt_torus(o0, m0);
          A[kN + pos] += P == 0 ? crt_torus(m1, o1) : crt_torus(o1, m1);
        }
        named_bar(bar_id, kGateThreads);  // B3: ACC updated
      } else {
        // partial sums meet in the owner warp (P, c) of each output c: half c of a
        // warp's scratch holds its partial of output c (the owner's own half c
        // stays free for its inverse transform and CRT exchange)
        __syncwarp();
        if (h >= 2) {
#pragma unroll
          for (int e = 0; e < 32; ++e) myscr[cA * kXpose + e * 32 + lane] = acc0[e];
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) myscr[(1 - cA) * kXpose + e * 32 + lane] = acc1[e];
        named_bar(bar_id, kGateThreads);  // B1: partials posted
        if (h < 2) {
          uint32_t *half = myscr + h * kXpose;
          for (int hp = 0; hp < H; ++hp) {
            if (hp == h) continue;
            const uint32_t *src = S.scratch + (wbase + hp * 2 + P) * kScr + h * kXpose;
#pragma unroll
            for (int e = 0; e < 32; ++e) acc0[e] += src[e * 32 + lane];
          }
          ntt_inv_gs<kInvIn>(acc0, half, gsi1, args.tc.gsi2[P], pr, lane);
          __syncwarp();
#pragma unroll
          for (int e = 0; e < 16; ++e) half[e * 32 + lane] = P ? acc0[e] : acc0[16 + e];
        }
        named_bar(bar_id, kGateThreads);  // B2: CRT halves posted
        if (h < 2) {
          const uint32_t *peer = S.scratch + (wbase + h * 2 + (1 - P)) * kScr + h * kXpose;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const uint32_t m = P ? acc0[16 + e] : acc0[e];
            const uint32_t o = peer[e * 32 + lane];
            A[h * kN + lane + 32 * (16 * P + e)] += P == 0 ? crt_torus(m, o) : crt_torus(o, m);
          }
        }
        named_bar(bar_id, kGateThreads);  // B3: ACC updated
      }
    }

    // Sample extraction of coefficient 0: a'_0 = a_0, a'_j = -a_(N-j), b' = b_0.
    if (active) {
      uint32_t *o = args.out + (size_t)job_idx * kOutStride;
      for (int k = tid_g; k <= kN; k += kGateThreads)
        o[k] = k == 0 ? A[0] : (k < kN ? 0u - A[kN - k] : A[kN]);
    }
    named_bar(bar_id, kGateThreads);
  }
}

template <int H, int GT, int L>
__global__ void __launch_bounds__(2 * H * GT * 32, 1) br_kernel(const __grid_constant__ BrArgs args) {
  extern __shared__ __align__(128) uint8_t smem[];
  BrShared S = br_carve<H, GT, L>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kStages = br_stages<H, GT, L>();
  static_assert(kStages >= 4 && kStages <= 8, "ring depth");
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(S.full + s, 1);
      S.cnt[s] = 0u;
      S.issued[s] = 0u;
    }
    *S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < 2 * digit_tab_words<L>(); k += blockDim.x) {  // digit tables per prime
    const int P = k / digit_tab_words<L>(), j = k - P * digit_tab_words<L>();
    const uint64_t q = P ? kQ1 : kQ0;
    uint64_t z = args.tc.fwd1[P][1].x;  // L = 2: zeta[1]
    if (L == 3) {
      const uint64_t z1 = args.tc.fwd1[P][1].x, z2 = args.tc.fwd1[P][2].x, z3 = args.tc.fwd1[P][3].x;
      const int t = j >> 7;
      z = t == 0 ? z1 : t == 1 ? z2 : t == 2 ? z2 * z1 % q : t == 3 ? z3 : z3 * z1 % q;
    }
    S.dtab[k] = (uint32_t)(z * (uint64_t)(j & (digit_values<L>() - 1)) % q);
  }
  __syncthreads();
  if (threadIdx.x == 0) stamp_start(args.stamps);
  if (args.num_jobs <= 0) return;
  constexpr bool kTmem = tmem_mac<H, GT, L>();
  static_assert(!kTmem || 2 * H * GT == 12, "TMEM columns: three warps per lane quadrant, 128 columns each");
  uint32_t tbase = 0;
  if constexpr (kTmem) {  // freed below on every path that reaches this point
    if (warp == 0) tmem_alloc(S.tmem, kTmemCols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    tbase = *S.tmem;
  }
  if (threadIdx.x == 0) {  // the first kStages rows; later ones are issued by the warps
    const uint32_t rows = cta_rows<GT, L>(args);
    for (uint32_t jc = 0; jc < (uint32_t)kStages && jc < rows; ++jc) issue_row<kStages, GT, L>(S, args, jc);
  }
  const int g = warp / (2 * H), role = warp % (2 * H);
  // warp w: TMEM lanes 32 (w mod 4) .. + 31, columns 128 (w / 4) .. + 127
  const uint32_t taddr = tbase + ((32u * (uint32_t)(warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
  br_consumer<H, GT, L>(S, args, g, role >> 1, role & 1, lane, taddr);
  if constexpr (kTmem) tmem_fence_before_sync();
  __syncthreads();
  if constexpr (kTmem) {
    if (warp == 0) {
      tmem_fence_after_sync();
      tmem_dealloc(tbase, kTmemCols);
    }
  }
  if (threadIdx.x == 0 && *S.abort_flag) {  // after a timeout: let copies in flight land (bounded)
    for (int s = 0; s < kStages; ++s) {
      const uint32_t k = S.issued[s];
      if (k == 0u) continue;
      const long long t0 = clock64();
      while (!mbar_try_wait(S.full + s, ((k - 1u) / kStages) & 1u) && clock64() - t0 < kWaitCycles) {
      }
    }
  }
  if (lane == 0) stamp_end(args.stamps);
}

template <int H, int GT, int L>
cudaError_t prepare_shape() {
  static bool done = false;  // calls are serialised by the engine lock
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(br_kernel<H, GT, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)br_smem_bytes<H, GT, L>());
  if (e == cudaSuccess) done = true;
  return e;
}

template <int H, int GT, int L = 3>
cudaError_t launch_shape(const BrArgs &args, int grid, cudaStream_t st) {
  cudaError_t e = prepare_shape<H, GT, L>();
  if (e != cudaSuccess) return e;
  br_kernel<H, GT, L><<<grid, 2 * H * GT * 32, br_smem_bytes<H, GT, L>(), st>>>(args);
  return cudaGetLastError();
}

// Resident CTAs per SM of a shape (0 if it cannot launch on this device).
template <int H, int GT, int L = 3>
int occupancy_shape() {
  if (prepare_shape<H, GT, L>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, br_kernel<H, GT, L>, 2 * H * GT * 32,
                                                    br_smem_bytes<H, GT, L>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

}  // namespace br
}  // namespace arx
