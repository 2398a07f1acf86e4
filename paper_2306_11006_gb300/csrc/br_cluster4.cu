// br_cluster4.cu -- blind rotation of one gate on a cluster of four CTAs (four
// SMs), for the narrowest waves.
//
// The paper runs one gate per SM and names spreading a gate over several SMs as
// the remedy for thin waves (Sec. 8).  Here CTA (h, w) of the cluster (rank
// 2 w + h) owns accumulator component ACC_h, the three TGSW rows whose digits
// come from it (rows 3h .. 3h+2), and spectral half w, for both CRT primes.
//
// Per CMux: the first two forward stages (distances 512 and 256) are taken while
// loading the packed digits, after which the four quarters of a transform are
// independent 256-point transforms; the CTA runs its two quarters of the three
// rows in both primes on twelve warps (row, prime, quarter).  Each warp adds its
// key products for output 1-h into CTA (1-h, w)'s receive slot with a bulk
// reduction (1 KiB; the receiver zeroes the slot after use); with the products
// it receives, the CTA holds half w of both
// primes' sums of output h and runs their inverse quarters (all stages but the
// last two, then the output twist) on four warps.  It sends those quarters to
// CTA (h, 1-w) (4 KiB) and receives the other two, so both CTAs of component h
// run the folded last stages and the CRT on all four quarters and update
// identical copies of ACC_h.  Every cross-CTA dependency is a transaction count on an mbarrier
// (double-buffered by CMux parity); every wait is bounded.
#include <cuda_runtime.h>

#include <cstdint>

#include "br_cluster_common.cuh"

namespace arx {
namespace brc4 {

using namespace clu;

constexpr int kCons = 12;                   // consumer warps: (row 0..2) x (prime 0..1) x (quarter 0..1)
constexpr int kThreads = (kCons + 1) * 32;  // + producer warp
constexpr int kConsThreads = kCons * 32;
constexpr int kStages = 6;                  // ring of 16 KiB key rows: two CMux ahead
constexpr int kAbarPitch = 640;
constexpr int kHalfW = 512;                 // words of a half spectrum
constexpr int kQuarter = 256;
constexpr uint32_t kPeerBytes = kCons * kQuarter * 4;  // the peer's twelve product quarters
constexpr uint32_t kPartnerBytes = 2 * 2 * kQuarter * 4;  // two inverse quarters, both primes

// shared memory (bytes)
constexpr size_t kRingBytes = (size_t)kStages * kChunkBytes;
constexpr size_t kAccBytes = kN * 4;                 // ACC_h
constexpr size_t kDigBytes = 3 * 256 * 4;            // [row][k] digit bytes of k, k+256, k+512, k+768
constexpr size_t kOwnBytes = 2 * 3 * kHalfW * 4;     // [prime][row][half w] products for output h
constexpr size_t kOthBytes = 2 * 2 * 3 * kHalfW * 4; // [parity][prime][row][half w] products for output 1-h
constexpr size_t kSlotBytes = 2 * 2 * kHalfW * 4;    // [parity][prime][half w] the peer's row sums
constexpr size_t kPostBytes = 2 * 2 * 4 * kQuarter * 4;  // [parity][prime][quarter][k] inverse quarters
constexpr size_t kScrBytes = (size_t)kCons * kQuarter * 4;
constexpr size_t kAbarBytes = kAbarPitch * 2;
constexpr size_t kBarBytes = (2 * kStages + 4) * 8 + 16;
constexpr size_t kSmem = kRingBytes + kAccBytes + kDigBytes + kOwnBytes + kOthBytes + kSlotBytes + kPostBytes +
                         kScrBytes + kAbarBytes + kBarBytes;

// Forward quarter transform (negacyclic Cooley-Tukey, merged twist), spectral
// block Qf (positions 256 Qf + p), in three register passes joined by two
// shared-memory transposes.  In: x[e] = the output of the first two stages at
// p = lane + 32 e (< 5q + 128).  Out: x[e] = spectral position 256 Qf + 8 b + e,
// b = fwd_block8(lane) (< 22q), bit-reversed order.
__device__ __forceinline__ void fwd_quarter(uint32_t (&x)[8], uint32_t *xbuf, const uint2 *tw1,
                                            const uint2 *__restrict__ twc, const uint2 *__restrict__ twq, int Qf,
                                            const PrimeRT &pr, int lane) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {  // lengths 128, 64 on a[lane + 32 e]: bits 2, 1 of e
    const int lr = 4 >> s, m = 4 << s;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if ((e & lr) == 0) ct_bfly(x[e], x[e + lr], tw1[m + (m >> 2) * Qf + e / (2 * lr)], pr);
  }
  const int pc = (lane & 7) + 64 * (lane >> 3);  // middle pass: position pc + 8 e
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) xbuf[sw1(lane + 32 * e)] = x[e];
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = xbuf[sw1(pc + 8 * e)];
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // lengths 32, 16, 8: bits 2 .. 0 of e, per-lane twiddles
    const int lr = 4 >> s, k0 = (1 << s) - 1;
    uint2 z;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if ((e & lr) == 0) {
        if ((e & (2 * lr - 1)) == 0) z = __ldg(twc + (k0 + e / (2 * lr)) * 32 + lane);
        ct_bfly(x[e], x[e + lr], z, pr);
      }
    }
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
  for (int s = 0; s < 3; ++s) {  // lengths 4, 2, 1 on a[8 b + e], per-lane twiddles
    const int len = 4 >> s, k0 = (1 << s) - 1;
    uint2 z;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if ((e & len) == 0) {
        if ((e & (2 * len - 1)) == 0) z = __ldg(twq + (k0 + e / (2 * len)) * 32 + lane);
        ct_bfly(x[e], x[e + len], z, pr);
      }
    }
  }
}

__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(kThreads, 1)
    br_cluster4_kernel(const __grid_constant__ BrArgs args) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint32_t *A = reinterpret_cast<uint32_t *>(smem + kRingBytes);
  uint32_t *D = A + kN;                          // [row][256]
  uint32_t *own = D + 3 * 256;                   // [prime][row][512], swizzled (swp)
  uint32_t *oth = own + 6 * kHalfW;              // [parity][prime][row][512], same layout
  uint32_t *slots = oth + 12 * kHalfW;           // [parity][prime][512], same layout, zero between uses
  uint32_t *post = slots + 4 * kHalfW;           // [parity][prime][quarter][256], natural order
  uint32_t *scratch = post + 16 * kQuarter;      // [warp][256]
  uint16_t *abar = reinterpret_cast<uint16_t *>(scratch + kCons * kQuarter);
  uint64_t *full = reinterpret_cast<uint64_t *>(abar + kAbarPitch);
  uint64_t *empty = full + kStages;
  uint64_t *done1 = empty + kStages;             // [parity]: the peer's row sums in place
  uint64_t *done2 = done1 + 2;                   // [parity]: the partner's inverse quarters in place
  volatile int *abort_flag = reinterpret_cast<volatile int *>(done2 + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t h = rank & 1u, w = rank >> 1;   // accumulator component, spectral half
  const uint32_t peer = rank ^ 1u, partner = rank ^ 2u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 4);  // the four warps (prime, quarter) of a row
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(done1 + p, 1);  // one local arrival (with the expected bytes) per CMux
      mbar_init(done2 + p, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < 4 * kHalfW; k += kThreads) slots[k] = 0u;
  fence_proxy_async_smem();
  cluster_sync_all();  // all four CTAs initialised before any remote access
  if (threadIdx.x == 0) stamp_start(args.stamps);

  const int n = args.n;
  const int nclusters = gridDim.x / 4, cid = blockIdx.x / 4;
  const int tiles = args.num_jobs;

  if (warp == kCons) {  // producer: stream the three key rows of component h for every CMux
    if (lane == 0 && tiles > 0) {
      uint32_t jc = 0;
      bool ok = true;
      for (int tile = cid; tile < tiles && ok; tile += nclusters) {
        for (int i = 0; i < n && ok; ++i) {
          for (int rr = 0; rr < 3; ++rr, ++jc) {
            const uint32_t slot = jc % kStages;
            if (jc >= (uint32_t)kStages &&
                !mbar_wait(empty + slot, ((jc / kStages) - 1) & 1u, abort_flag, args.status)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full + slot, kChunkBytes);
            bulk_g2s(ring + slot * kChunkWords, args.bsk[args.jobs[tile].key] + ((size_t)i * 6 + 3 * h + rr) * kChunkWords, kChunkBytes,
                     full + slot);
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
    const int rr = warp >> 2, P = (warp >> 1) & 1, v = warp & 1;  // row 3h + rr, prime P, quarter v of half w
    const int Qf = 2 * (int)w + v;                                 // spectral quarter
    const int tid = threadIdx.x;                                   // 0 .. 383
    const PrimeRT pr = prime_rt(P, args.tc);
    uint32_t *myscr = scratch + warp * kQuarter;
    const uint2 *tw1f = args.tc.fwd1[P], *tw1i = args.tc.inv1[P];
    const uint2 *tw2i = args.tg->inv2[P], *twc = args.tg->fwdc[P][Qf], *twq = args.tg->fwdq[P][Qf];
    const uint2 z1 = args.tc.fwd1[P][1], z23 = args.tc.fwd1[P][2 + (Qf >> 1)];
    const int fb = fwd_block8(lane);
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
        make_digits4(D, A, abar[i], tid, kConsThreads);
        named_bar(1, kConsThreads);
        uint32_t x[8];
        load_first2(x, D + rr * 256, z1, z23, Qf, pr, lane);
        fwd_quarter(x, myscr, tw1f, twc, twq, Qf, pr, lane);
        const uint32_t jc = (it * (uint32_t)n + (uint32_t)i) * 3u + (uint32_t)rr;
        const uint32_t slot = jc % kStages;
        mbar_wait(full + slot, (jc / kStages) & 1u, abort_flag, args.status);
        // key row layout: position 32 L + E at word ((E >> 2) * 32 + L) * 4 + (E & 3)
        const uint4 *Bown = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + (h * 2 + P) * kN);
        const uint4 *Both = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + ((1 - h) * 2 + P) * kN);
        uint4 *own4 = reinterpret_cast<uint4 *>(own + (P * 3 + rr) * kHalfW);
        uint32_t *oq = oth + ((par * 2 + P) * 3 + rr) * kHalfW + kQuarter * v;  // quarter v of this row
        uint4 *oth4 = reinterpret_cast<uint4 *>(oth + ((par * 2 + P) * 3 + rr) * kHalfW);
        // products for the peer's output first: added into its slot while the rest runs
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint4 b1 = Both[(2 * (fb & 3) + c) * 32 + 8 * Qf + (fb >> 2)];
          oth4[swp(256 * v + 8 * fb + 4 * c) >> 2] =
              make_uint4(mont_mul(x[4 * c + 0], b1.x, pr), mont_mul(x[4 * c + 1], b1.y, pr),
                         mont_mul(x[4 * c + 2], b1.z, pr), mont_mul(x[4 * c + 3], b1.w, pr));
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
          bulk_add_s2peer(map_peer(smem_u32(slots + (par * 2 + P) * kHalfW + kQuarter * v), peer), oq,
                          kQuarter * 4u, map_peer(smem_u32(done1 + par), peer));
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint4 b0 = Bown[(2 * (fb & 3) + c) * 32 + 8 * Qf + (fb >> 2)];
          own4[swp(256 * v + 8 * fb + 4 * c) >> 2] =
              make_uint4(mont_mul(x[4 * c + 0], b0.x, pr), mont_mul(x[4 * c + 1], b0.y, pr),
                         mont_mul(x[4 * c + 2], b0.z, pr), mont_mul(x[4 * c + 3], b0.w, pr));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(empty + slot);
        named_bar(2 + P, kConsThreads / 2);  // the three rows of output h, prime P, half w, in place
        if (warp == 0 && lane == 0) {
          mbar_expect_tx(done1 + par, kPeerBytes);
          mbar_expect_tx(done2 + par, kPartnerBytes);
        }
        if (rr == 0) {
          // quarter Qf of output h in prime P: three local rows and the peer's sum
          mbar_wait(done1 + par, ph, abort_flag, args.status);
          uint32_t y[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) y[e] = 0u;
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            uint4 *sl = reinterpret_cast<uint4 *>(r4 < 3 ? own + (P * 3 + r4) * kHalfW : slots + (par * 2 + P) * kHalfW);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int ci = swp(256 * v + 8 * lane + 4 * c) >> 2;
              const uint4 q = sl[ci];
              y[4 * c + 0] += q.x;
              y[4 * c + 1] += q.y;
              y[4 * c + 2] += q.z;
              y[4 * c + 3] += q.w;
              if (r4 == 3) sl[ci] = make_uint4(0u, 0u, 0u, 0u);  // the slot starts its next use at zero
            }
          }
          fence_proxy_async_smem();  // the zeroes precede the peer's next bulk additions
          inv_quarter(y, myscr, tw1i, args.tg->invc[P], tw2i, pr, lane);
          quarter_twist(y, args.tg->fint[P][Qf], pr, lane);
          // post the quarter here and at CTA (h, 1-w)
          uint32_t *pq = post + ((par * 2 + P) * 4 + Qf) * kQuarter;
#pragma unroll
          for (int e = 0; e < 8; ++e) pq[lane + 32 * e] = y[e];
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0)
            bulk_s2peer(map_peer(smem_u32(pq), partner), pq, kQuarter * 4u,
                        map_peer(smem_u32(done2 + par), partner));
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
      // sample extraction (half 0 only): CTA (0, 0) holds the mask a' (from ACC_0), CTA (1, 0) the body b'
      uint32_t *o = args.out + (size_t)tile * kOutStride;
      if (w == 0) {
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

}  // namespace brc4

size_t br_cluster4_smem() { return brc4::kSmem; }

cudaError_t launch_br_cluster4(const BrArgs &args, int clusters, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(brc4::br_cluster4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)brc4::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  brc4::br_cluster4_kernel<<<4 * clusters, brc4::kThreads, brc4::kSmem, st>>>(args);
  return cudaGetLastError();
}

int br_cluster4_occupancy() {
  if (cudaFuncSetAttribute(brc4::br_cluster4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)brc4::kSmem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(4, 1, 1);
  cfg.blockDim = dim3(brc4::kThreads, 1, 1);
  cfg.dynamicSmemBytes = brc4::kSmem;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 4;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, brc4::br_cluster4_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}

}  // namespace arx
