// br_cluster8.cu -- blind rotation of one gate on a cluster of eight CTAs (eight
// SMs), for the narrowest waves (at most as many gates as eight-CTA clusters fit).
//
// The paper runs one gate per SM and names spreading a gate over several SMs as
// the remedy for thin waves (Sec. 8).  Here CTA (h, Q) of the cluster (rank
// 2 Q + h) owns accumulator component ACC_h, the three TGSW rows whose digits
// come from it (rows 3h .. 3h+2), and spectral quarter Q, for both CRT primes.
//
// Per CMux: all warps compute the gadget digits of the CTA's rows and take the
// first two forward stages of quarter Q in both primes at once (make_stage2:
// the quarters of a negacyclic transform are independent after those two
// stages); six forward warps (row, prime) run the rest of their quarter-Q
// transform.
// Each adds its key products for output 1-h into CTA (1-h, Q)'s receive slot
// with a bulk reduction (1 KiB).  With the products it receives, the CTA holds
// quarter Q of both primes' sums of output h; two warps run the two inverse
// quarter transforms (all stages but the last two, then their share of the
// output twist) and post them here and at the three CTAs (h, Q') (1 KiB each).
// All four CTAs of component h then fold the last two stages, run the CRT and
// update identical copies of ACC_h.  Every cross-CTA dependency is a transaction
// count on an mbarrier (double-buffered by CMux parity); every wait is bounded.
// With nine warps per CTA the loop-invariant per-lane twiddles of each warp stay
// in registers.  The kernel is a template on the gadget length L: 3 (Bg = 2^7,
// 7-bit digits, six forward warps) or 2 (Bg = 2^10, 10-bit digits, four forward
// warps and the TGSW rows 2h, 2h+1 of the paper's own parameter set).
#include <cuda_runtime.h>

#include <cstdint>

#include "br_cluster_common.cuh"

namespace arx {
namespace brc8 {

using namespace clu;

constexpr int kCons = 8;                    // forward warps + helpers for the digits and the CRT pass
constexpr int kThreads = (kCons + 1) * 32;  // + producer warp
constexpr int kConsThreads = kCons * 32;    // 256
constexpr int kStages = 6;                  // ring of 16 KiB key rows: two CMux ahead (L = 3)
constexpr int kAbarPitch = 640;
constexpr int kQuarter = 256;
constexpr uint32_t kPartnerBytes = 3 * 2 * kQuarter * 4;      // three partners x two primes

template <int L>
struct Cfg {
  static constexpr int kFwd = 2 * L;                              // forward warps: (row) x (prime)
  static constexpr uint32_t kPeerBytes = kFwd * kQuarter * 4;     // the peer's product quarters
  // shared memory (bytes)
  static constexpr size_t kRingBytes = (size_t)kStages * kChunkBytes;
  static constexpr size_t kAccBytes = kN * 4;                     // ACC_h
  static constexpr size_t kDigBytes = (size_t)2 * L * 256 * 4;    // [prime][row][k] stage-2 values (make_stage2)
  static constexpr size_t kOwnBytes = 2 * L * kQuarter * 4;       // [prime][row][quarter Q] products for output h
  static constexpr size_t kOthBytes = 2 * 2 * L * kQuarter * 4;   // [parity][prime][row][quarter Q] for output 1-h
  static constexpr size_t kSlotBytes = 2 * 2 * kQuarter * 4;      // [parity][prime][quarter Q] the peer's row sums
  static constexpr size_t kPostBytes = 2 * 2 * 4 * kQuarter * 4;  // [parity][prime][quarter][k] inverse quarters
  static constexpr bool kInvPair = L == 2;  // the inverse on a pair of warps (measured faster only for L = 2)
  static constexpr size_t kScrBytes = (size_t)(kFwd + (kInvPair ? 2 : 0)) * kQuarter * 4;
  static constexpr size_t kAbarBytes = kAbarPitch * 2;
  static constexpr size_t kBarBytes = (2 * kStages + 4) * 8 + 16;
  static constexpr size_t kSmem = kRingBytes + kAccBytes + kDigBytes + kOwnBytes + kOthBytes + kSlotBytes +
                                  kPostBytes + kScrBytes + kAbarBytes + kBarBytes;
};

template <int L>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(kThreads, 1)
    br_cluster8_kernel(const __grid_constant__ BrArgs args) {
  using C = Cfg<L>;
  constexpr int kFwd = C::kFwd;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint32_t *A = reinterpret_cast<uint32_t *>(smem + C::kRingBytes);
  uint32_t *D = A + kN;                          // [prime][row][k] stage-2 values
  uint32_t *own = D + C::kDigBytes / 4;          // [prime][row][256], swizzled (swp)
  uint32_t *oth = own + 2 * L * kQuarter;        // [parity][prime][row][256], same layout
  uint32_t *slots = oth + 4 * L * kQuarter;      // [parity][prime][256], same layout, zero between uses
  uint32_t *post = slots + 4 * kQuarter;         // [parity][prime][quarter][256], natural order
  uint32_t *scratch = post + 16 * kQuarter;      // [forward warp][256]
  uint16_t *abar = reinterpret_cast<uint16_t *>(scratch + C::kScrBytes / 4);
  uint64_t *full = reinterpret_cast<uint64_t *>(abar + kAbarPitch);
  uint64_t *empty = full + kStages;
  uint64_t *done1 = empty + kStages;             // [parity]: the peer's row sums in place
  uint64_t *done2 = done1 + 2;                   // [parity]: the partners' inverse quarters in place
  volatile int *abort_flag = reinterpret_cast<volatile int *>(done2 + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t h = rank & 1u;                  // accumulator component
  const int Q = (int)(rank >> 1);                // spectral quarter
  const uint32_t peer = rank ^ 1u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 2);  // the two forward warps (primes) of a row
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(done1 + p, 1);  // one local arrival (with the expected bytes) per CMux
      mbar_init(done2 + p, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < 4 * kQuarter; k += kThreads) slots[k] = 0u;
  fence_proxy_async_smem();
  cluster_sync_all();  // all eight CTAs initialised before any remote access
  if (threadIdx.x == 0) stamp_start(args.stamps);

  const int n = args.n;
  const int nclusters = gridDim.x / 8, cid = blockIdx.x / 8;
  const int tiles = args.num_jobs;

  if (warp == kCons) {  // producer: stream the L key rows of component h for every CMux
    if (lane == 0 && tiles > 0) {
      uint32_t jc = 0;
      bool ok = true;
      for (int tile = cid; tile < tiles && ok; tile += nclusters) {
        for (int i = 0; i < n && ok; ++i) {
          for (int rr = 0; rr < L; ++rr, ++jc) {
            const uint32_t slot = jc % kStages;
            if (jc >= (uint32_t)kStages &&
                !mbar_wait(empty + slot, ((jc / kStages) - 1) & 1u, abort_flag, args.status)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full + slot, kChunkBytes);
            bulk_g2s(ring + slot * kChunkWords, args.bsk[args.jobs[tile].key] + ((size_t)i * 2 * L + L * h + rr) * kChunkWords,
                     kChunkBytes, full + slot);
          }
        }
      }
      if (!ok) {
        for (uint32_t k = jc > (uint32_t)kStages ? jc - kStages : 0; k < jc; ++k) {
          const long long t0 = clock64();
          while (!mbar_try_wait(full + (k % kStages), (k / kStages) & 1u) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (tiles > 0) {
    const bool fwd = warp < kFwd;
    const int rr = fwd ? warp >> 1 : 0, P = warp & 1;  // forward warps: row L h + rr, prime P
    const int tid = threadIdx.x;                         // 0 .. 255
    const PrimeRT pr = prime_rt(P, args.tc);
    PrimeRT prs[2] = {prime_rt(0, args.tc), prime_rt(1, args.tc)};
    if (L == 2) {  // first-stage offsets of 10-bit digits
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        prs[p].dc = args.tc.dig_c2[p];
        prs[p].dd = args.tc.dig_d2[p];
      }
    }
    const uint2 z1s[2] = {args.tc.fwd1[0][1], args.tc.fwd1[1][1]};
    const uint2 z23s[2] = {args.tc.fwd1[0][2 + (Q >> 1)], args.tc.fwd1[1][2 + (Q >> 1)]};
    uint32_t *myscr = scratch + (fwd ? warp : 0) * kQuarter;
    const uint2 *tw1f = args.tc.fwd1[P], *tw1i = args.tc.inv1[P];
    // L = 2: the inverse of prime P on the pair of forward warps P (rows rr = 0)
    // and 2 + P (rr = 1), each holding half of the quarter
    const int t = lane + (warp >= 2 ? 32 : 0);
    const int fb = fwd_block8(lane);
    // loop-invariant per-lane twiddles
    uint2 zc[7], zq[7], zi[7], z2[6], zt[8];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      zc[k] = __ldg(args.tg->fwdc[P][Q] + k * 32 + lane);
      zq[k] = __ldg(args.tg->fwdq[P][Q] + k * 32 + lane);
      zi[k] = __ldg(args.tg->invc[P] + k * 32 + lane);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) z2[k] = __ldg(args.tg->inv2[P] + (k + 1) * 32 + lane);
#pragma unroll
    for (int e = 0; e < 8; ++e) zt[e] = __ldg(args.tg->fint[P][Q] + lane + 32 * e);
    const InvPairTw zp = load_inv_pair(args, P, Q, t);
    uint32_t it = 0, cm = 0;  // tile counter, CMux counter
    for (int tile = cid; tile < tiles; tile += nclusters, ++it) {
      const BrJob jb = args.jobs[tile];
      const uint32_t *wa = args.wires + (size_t)jb.ia * kWireStride;
      const uint32_t *wb = args.wires + (size_t)jb.ib * kWireStride;
      const uint32_t sa = (uint32_t)(int32_t)jb.sa, sb = (uint32_t)(int32_t)jb.sb;
      for (int k = tid; k < n; k += kConsThreads) abar[k] = (uint16_t)modswitch(sa * wa[k] + sb * wb[k]);
      const uint32_t bbar = modswitch(jb.cst + sa * wa[n] + sb * wb[n]);
      const uint32_t shift = (2u * kN - bbar) & (2u * kN - 1);
      // ACC_0 = 0, ACC_1 = X^-bbar testv
      for (int k = tid; k < kN; k += kConsThreads)
        A[k] = h == 0 ? 0u : ((((uint32_t)k - shift) & (2u * kN - 1)) < (uint32_t)kN ? kMu : 0u - kMu);
      named_bar(1, kConsThreads);

      for (int i = 0; i < n; ++i, ++cm) {
        const uint32_t par = cm & 1u, ph = (cm >> 1) & 1u;
        make_stage2<L, 2>(D, A, abar[i], z1s, z23s, Q, prs, tid, kConsThreads);
        named_bar(1, kConsThreads);
        if (fwd) {
          uint32_t x[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) x[e] = D[(P * L + rr) * 256 + lane + 32 * e];
          fwd_quarter_r(x, myscr, tw1f, zc, zq, Q, pr, lane);
          const uint32_t jc = (it * (uint32_t)n + (uint32_t)i) * (uint32_t)L + (uint32_t)rr;
          const uint32_t slot = jc % kStages;
          mbar_wait(full + slot, (jc / kStages) & 1u, abort_flag, args.status);
          // key row layout: position 32 L + E at word ((E >> 2) * 32 + L) * 4 + (E & 3)
          const uint4 *Bown = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + (h * 2 + P) * kN);
          const uint4 *Both = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + ((1 - h) * 2 + P) * kN);
          uint32_t *oq = oth + ((par * 2 + P) * L + rr) * kQuarter;
          uint4 *oth4 = reinterpret_cast<uint4 *>(oq);
          uint4 *own4 = reinterpret_cast<uint4 *>(own + (P * L + rr) * kQuarter);
          // products for the peer's output first: added into its slot while the rest runs
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const uint4 b1 = Both[(2 * (fb & 3) + c) * 32 + 8 * Q + (fb >> 2)];
            oth4[swp(8 * fb + 4 * c) >> 2] =
                make_uint4(mont_mul(x[4 * c + 0], b1.x, pr), mont_mul(x[4 * c + 1], b1.y, pr),
                           mont_mul(x[4 * c + 2], b1.z, pr), mont_mul(x[4 * c + 3], b1.w, pr));
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0)
            bulk_add_s2peer(map_peer(smem_u32(slots + (par * 2 + P) * kQuarter), peer), oq, kQuarter * 4u,
                            map_peer(smem_u32(done1 + par), peer));
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const uint4 b0 = Bown[(2 * (fb & 3) + c) * 32 + 8 * Q + (fb >> 2)];
            own4[swp(8 * fb + 4 * c) >> 2] =
                make_uint4(mont_mul(x[4 * c + 0], b0.x, pr), mont_mul(x[4 * c + 1], b0.y, pr),
                           mont_mul(x[4 * c + 2], b0.z, pr), mont_mul(x[4 * c + 3], b0.w, pr));
          }
          __syncwarp();
          if (lane == 0) mbar_arrive_cta(empty + slot);
          named_bar(2 + P, 32 * L);  // the L rows of output h, prime P, quarter Q, in place
          if (warp == 0 && lane == 0) {
            mbar_expect_tx(done1 + par, C::kPeerBytes);
            mbar_expect_tx(done2 + par, kPartnerBytes);
          }
          if constexpr (C::kInvPair) {
            if (warp < 4) {
              // quarter Q of output h in prime P: L local rows and the peer's sum, at 4 t + e
              mbar_wait(done1 + par, ph, abort_flag, args.status);
              uint32_t y[4] = {0u, 0u, 0u, 0u};
              const int ci = swp(4 * t) >> 2;
#pragma unroll
              for (int r4 = 0; r4 <= L; ++r4) {
                uint4 *sl = reinterpret_cast<uint4 *>(r4 < L ? own + (P * L + r4) * kQuarter : slots + (par * 2 + P) * kQuarter);
                const uint4 q = sl[ci];
                y[0] += q.x;
                y[1] += q.y;
                y[2] += q.z;
                y[3] += q.w;
                if (r4 == L) sl[ci] = make_uint4(0u, 0u, 0u, 0u);  // the slot starts its next use at zero
              }
              fence_proxy_async_smem();  // the zeroes precede the peer's next bulk additions
              inv_quarter_pair(y, scratch + P * kQuarter, scratch + (kFwd + P) * kQuarter, zp, pr, t, 4 + P);
              // post the quarter here and at the three CTAs (h, Q')
              uint32_t *pq = post + ((par * 2 + P) * 4 + Q) * kQuarter;
#pragma unroll
              for (int e = 0; e < 4; ++e) pq[t + 64 * e] = y[e];
              fence_proxy_async_smem();
              named_bar(4 + P, 64);  // both halves in place
              if (warp < 2 && lane < 3) {
                const uint32_t dst = rank ^ (2u * (uint32_t)(lane + 1));  // (h, Q ^ (lane + 1))
                bulk_s2peer(map_peer(smem_u32(pq), dst), pq, kQuarter * 4u, map_peer(smem_u32(done2 + par), dst));
              }
            }
          } else if (rr == 0) {
            // quarter Q of output h in prime P: L local rows and the peer's sum
            mbar_wait(done1 + par, ph, abort_flag, args.status);
            uint32_t y[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) y[e] = 0u;
#pragma unroll
            for (int r4 = 0; r4 <= L; ++r4) {
              uint4 *sl = reinterpret_cast<uint4 *>(r4 < L ? own + (P * L + r4) * kQuarter : slots + (par * 2 + P) * kQuarter);
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                const int ci = swp(8 * lane + 4 * c) >> 2;
                const uint4 q = sl[ci];
                y[4 * c + 0] += q.x;
                y[4 * c + 1] += q.y;
                y[4 * c + 2] += q.z;
                y[4 * c + 3] += q.w;
                if (r4 == L) sl[ci] = make_uint4(0u, 0u, 0u, 0u);  // the slot starts its next use at zero
              }
            }
            fence_proxy_async_smem();  // the zeroes precede the peer's next bulk additions
            inv_quarter_r(y, myscr, tw1i, zi, z2, zt, pr, lane);
            // post the quarter here and at the three CTAs (h, Q')
            uint32_t *pq = post + ((par * 2 + P) * 4 + Q) * kQuarter;
#pragma unroll
            for (int e = 0; e < 8; ++e) pq[lane + 32 * e] = y[e];
            fence_proxy_async_smem();
            __syncwarp();
            if (lane < 3) {
              const uint32_t dst = rank ^ (2u * (uint32_t)(lane + 1));  // (h, Q ^ (lane + 1))
              bulk_s2peer(map_peer(smem_u32(pq), dst), pq, kQuarter * 4u, map_peer(smem_u32(done2 + par), dst));
            }
          }
        }
        mbar_wait(done2 + par, ph, abort_flag, args.status);
        named_bar(1, kConsThreads);  // all four quarters of both primes posted
        {
          const uint32_t *pp = post + par * 2 * 4 * kQuarter;
          const uint32_t *post0[4] = {pp, pp + kQuarter, pp + 2 * kQuarter, pp + 3 * kQuarter};
          crt_update(A, post0, 4 * kQuarter, args, tid, kConsThreads);
        }
        named_bar(1, kConsThreads);  // ACC_h updated
      }
      // sample extraction (quarter 0 only): CTA (0, 0) holds the mask a' (from ACC_0), CTA (1, 0) the body b'
      uint32_t *o = args.out + (size_t)tile * kOutStride;
      if (Q == 0) {
        if (h == 0) {
          for (int k = tid; k < kN; k += kConsThreads) o[k] = k == 0 ? A[0] : 0u - A[kN - k];
        } else if (tid == 0) {
          o[kN] = A[0];
        }
      }
      named_bar(1, kConsThreads);
    }
  }
  __syncwarp();
  cluster_sync_all();  // no CTA leaves while another may still touch its shared memory
  if (threadIdx.x == 0) stamp_end(args.stamps);
}

}  // namespace brc8

namespace {
template <int L>
cudaError_t launch8(const BrArgs &args, int clusters, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(brc8::br_cluster8_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)brc8::Cfg<L>::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  brc8::br_cluster8_kernel<L><<<8 * clusters, brc8::kThreads, brc8::Cfg<L>::kSmem, st>>>(args);
  return cudaGetLastError();
}

template <int L>
int occupancy8() {
  if (cudaFuncSetAttribute(brc8::br_cluster8_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)brc8::Cfg<L>::kSmem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(8, 1, 1);
  cfg.blockDim = dim3(brc8::kThreads, 1, 1);
  cfg.dynamicSmemBytes = brc8::Cfg<L>::kSmem;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 8;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, brc8::br_cluster8_kernel<L>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}
}  // namespace

size_t br_cluster8_smem() { return brc8::Cfg<3>::kSmem; }
cudaError_t launch_br_cluster8(const BrArgs &args, int clusters, cudaStream_t st) { return launch8<3>(args, clusters, st); }
int br_cluster8_occupancy() { return occupancy8<3>(); }
size_t br_cluster8_l2_smem() { return brc8::Cfg<2>::kSmem; }
cudaError_t launch_br_cluster8_l2(const BrArgs &args, int clusters, cudaStream_t st) {
  return launch8<2>(args, clusters, st);
}
int br_cluster8_l2_occupancy() { return occupancy8<2>(); }

}  // namespace arx
