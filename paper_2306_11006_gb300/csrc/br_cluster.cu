// br_cluster.cu -- blind rotation of one gate on a cluster of two CTAs (two SMs),
// for waves too narrow to fill the GPU.
//
// The paper runs one gate per SM and names spreading a gate over several SMs as
// the remedy for thin waves (Sec. 8).  Here the two TLWE components split the
// work: CTA h of the cluster owns accumulator polynomial ACC_h and the three TGSW
// rows whose digits come from ACC_h (rows 3h .. 3h+2), for both CRT primes.  Each
// forward 1024-point transform is split over two warps (halves w = 0, 1): its
// first stage (distance 512) is taken while loading the digits, after which the
// halves are independent 512-point transforms.  Each inverse transform is split
// over four warps (quarters of the spectrum, each applying its part of the
// output twist); the last two stages are folded into the CRT pass that all warps
// share.  So twelve
// consumer warps per CTA: (row, prime, half); eight of them run the inverses.
//
// Each warp writes its key products for both outputs to local shared memory;
// after a barrier of the six warps of its prime, each adds the three rows of
// output 1-h over a sixth of the coefficients into a staging buffer and has the
// bulk copy engine move it into the peer's shared memory (distributed shared
// memory, 8 KiB per CMux and CTA), completing its bytes on the peer's mbarrier.
// So CTA h ends each CMux holding the complete sums of output h in both primes:
// it runs the inverse transforms, the CRT and the update of ACC_h by itself, and
// never needs ACC_{1-h}.  The only cross-SM dependency per CMux is that
// transaction count (one mbarrier per CMux parity in each CTA); no thread fences
// at cluster scope, and the owner warps wait with a bounded wait.
#include <cuda_runtime.h>

#include <cstdint>

#include "br_cluster_common.cuh"

namespace arx {
namespace brc {

using namespace clu;

constexpr int kCons = 12;                     // consumer warps: (row 0..2) x (prime 0..1) x (half 0..1)
constexpr int kThreads = (kCons + 1) * 32;    // + producer warp
constexpr int kStages = 4;                    // ring of 16 KiB key rows (smaller ring, larger L1 for twiddles)
constexpr int kAbarPitch = 640;
constexpr uint32_t kPeerBytes = 2 * kN * 4;  // the peer's row sums (both primes) per CMux

// shared memory (bytes)
constexpr size_t kRingBytes = (size_t)kStages * kChunkBytes;
constexpr size_t kAccBytes = kN * 4;                // ACC_h
constexpr size_t kDigBytes = 3 * 256 * 4;           // digits of ACC_h: [row][k] bytes of k, k+256, k+512, k+768
constexpr size_t kSumBytes = 2 * 2 * 3 * kN * 4;    // [output own/other][prime 2][row 3][N] products
constexpr size_t kSlotBytes = 2 * 2 * kN * 4;       // [parity 2][prime 2][N] the peer's row sums
constexpr size_t kStageBytes = 2 * 2 * kN * 4;      // [parity 2][prime 2][N] row sums sent to the peer
constexpr int kHalf = 512;                    // words per half transform
constexpr size_t kScrBytes = (size_t)kCons * kHalf * 4;
constexpr size_t kAbarBytes = kAbarPitch * 2;
constexpr size_t kBarBytes = (2 * kStages + 2) * 8 + 16;
constexpr size_t kSmem =
    kRingBytes + kAccBytes + kDigBytes + kSumBytes + kSlotBytes + kStageBytes + kScrBytes + kAbarBytes + kBarBytes;

// Block of 16 positions that lane l holds after the forward transpose.
__device__ __forceinline__ int fwd_block(int lane) { return 2 * (lane & 15) + (lane >> 4); }

// Forward half transform (negacyclic Cooley-Tukey, merged twist), positions
// 512 w + p.  In: x[e] = stage-1 output at p = lane + 32 e (< 3q + 128).
// Out: x[e] = spectral position 512 w + 16 b + e, b = fwd_block(lane) (< 22q),
// bit-reversed order.
__device__ __forceinline__ void fwd_half(uint32_t (&x)[16], uint32_t *xbuf, const uint2 *tw1,
                                         const uint2 *__restrict__ tw2, const uint2 *__restrict__ twh, int w,
                                         const PrimeRT &pr, int lane) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {  // lengths 256, 128, 64, 32: bits 3 .. 0 of e
    const int lr = 8 >> s, m = 2 << s;
#pragma unroll
    for (int e = 0; e < 16; ++e)
      if ((e & lr) == 0) ct_bfly(x[e], x[e + lr], tw1[m + (m >> 1) * w + e / (2 * lr)], pr);
  }
  {  // length 16: lane bit 4, zeta[32 + 16 w + e]
    const bool up = (lane & 16) != 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) x[e] = xlane_bfly(x[e], __ldg(tw2 + 16 * w + e), up, 16, pr);
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 16; ++e) xbuf[swp(lane + 32 * e)] = x[e];
  __syncwarp();
  const uint4 *xb4 = reinterpret_cast<const uint4 *>(xbuf);
  const int b = fwd_block(lane);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 v = xb4[swp(16 * b + 4 * c) >> 2];
    x[4 * c + 0] = v.x;
    x[4 * c + 1] = v.y;
    x[4 * c + 2] = v.z;
    x[4 * c + 3] = v.w;
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {  // lengths 8, 4, 2, 1 with per-lane twiddles
    const int len = 8 >> s, k0 = (1 << s) - 1;
    uint2 z;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if ((e & len) == 0) {
        if ((e & (2 * len - 1)) == 0) z = __ldg(twh + (k0 + e / (2 * len)) * 32 + lane);
        ct_bfly(x[e], x[e + len], z, pr);
      }
    }
  }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    br_cluster_kernel(const __grid_constant__ BrArgs args) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint32_t *A = reinterpret_cast<uint32_t *>(smem + kRingBytes);
  uint32_t *D = A + kN;                             // [row][256]
  uint32_t *sums = D + 3 * 256;                         // [output own/other][prime][row][N], halves swizzled (swh)
  uint32_t *slots = sums + 12 * kN;                 // [parity][prime][N], same layout
  uint32_t *stage = slots + 4 * kN;                 // [parity][prime][N], same layout
  uint32_t *scratch = stage + 4 * kN;               // [warp][kHalf]; the inverse warps post here
  uint16_t *abar = reinterpret_cast<uint16_t *>(scratch + kCons * kHalf);
  uint64_t *full = reinterpret_cast<uint64_t *>(abar + kAbarPitch);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;                 // [parity]: the peer's row sums of a CMux in place
  volatile int *abort_flag = reinterpret_cast<volatile int *>(done + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t h = cluster_rank();                // accumulator component owned here
  const uint32_t peer = h ^ 1u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 4);  // the four warps (prime, half) of a row
    }
    mbar_init(done + 0, 1);  // one local arrival (with the expected bytes) per CMux
    mbar_init(done + 1, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync_all();  // both CTAs initialised before any remote access
  if (threadIdx.x == 0) stamp_start(args.stamps);

  const int n = args.n;
  const int nclusters = gridDim.x / 2, cid = blockIdx.x / 2;
  const int tiles = args.num_jobs;
  constexpr int kConsThreads = kCons * 32;

  if (warp == kCons) {  // producer: stream this CTA's three key rows of every CMux
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
    const int rr = warp >> 2, P = (warp >> 1) & 1, w = warp & 1;  // row 3h + rr, prime P, half w
    const int tid = threadIdx.x;                                   // 0 .. 383
    const PrimeRT pr = prime_rt(P, args.tc);
    uint32_t *myscr = scratch + warp * kHalf;
    const uint2 *tw1f = args.tc.fwd1[P], *tw1i = args.tc.inv1[P];
    const uint2 *tw2f = args.tg->fwd2[P], *tw2i = args.tg->inv2[P], *twh = args.tg->fwdh[P][w];
    const uint2 z1 = args.tc.fwd1[P][1];
    // chunks [c0, c0 + nc) of a prime's row sum are this warp's to send
    const int c0 = (rr * 2 + w) * 43, nc = c0 + 43 <= 256 ? 43 : 256 - c0;
    const int fb = fwd_block(lane);
    // inverse: warps of rows 0, 1 take quarter Q = 2 rr + w of prime P
    const int Qd = 2 * rr + w;
    // quarter Q of prime P is posted by warp ((Q >> 1) * 2 + P) * 2 + (Q & 1); prime 1 lies 2 kHalf above prime 0
    const uint32_t *post0[4];
#pragma unroll
    for (int Q = 0; Q < 4; ++Q) post0[Q] = scratch + ((Q >> 1) * 4 + (Q & 1)) * kHalf;
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
        // gadget digits of X^a ACC_h - ACC_h
        const uint32_t a = abar[i];
        make_digits4(D, A, a, tid, kConsThreads);
        named_bar(1, kConsThreads);
        // digit bytes u = d + 64 of row rr; the first stage (distance 512) on load
        uint32_t x[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t d4 = D[rr * 256 + lane + 32 * e];  // positions p, p + 256, p + 512, p + 768
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const uint32_t u = __byte_perm(d4, 0u, 0x4440u | g);
            const uint32_t t = shoup_mul(z1.x, z1.y, __byte_perm(d4, 0u, 0x4442u | g), pr.q);
            x[e + 8 * g] = w ? u - t + pr.q2 + pr.dd : u + t + pr.dc;
          }
        }
        fwd_half(x, myscr, tw1f, tw2f, twh, w, pr, lane);
        const uint32_t jc = (it * (uint32_t)n + (uint32_t)i) * 3u + (uint32_t)rr;
        const uint32_t slot = jc % kStages;
        mbar_wait(full + slot, (jc / kStages) & 1u, abort_flag, args.status);
        // key row layout: position 32 L + E at word ((E >> 2) * 32 + L) * 4 + (E & 3)
        const uint4 *Bown = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + (h * 2 + P) * kN);
        const uint4 *Both = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + ((1 - h) * 2 + P) * kN);
        uint4 *own = reinterpret_cast<uint4 *>(sums + (P * 3 + rr) * kN);
        uint4 *oth = reinterpret_cast<uint4 *>(sums + ((2 + P) * 3 + rr) * kN);
        // products for the peer's output first, so that their transfer overlaps
        // the products for this CTA's output
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 b1 = Both[(4 * (fb & 1) + c) * 32 + 16 * w + (fb >> 1)];
          oth[128 * w + (swp(16 * fb + 4 * c) >> 2)] =
              make_uint4(mont_mul(x[4 * c + 0], b1.x, pr), mont_mul(x[4 * c + 1], b1.y, pr),
                         mont_mul(x[4 * c + 2], b1.z, pr), mont_mul(x[4 * c + 3], b1.w, pr));
        }
        named_bar(2 + P, kConsThreads / 2);  // the three rows of output 1-h, prime P, in place
        {
          // output 1-h: add the three rows over this warp's chunks and send them
          const uint4 *o0 = reinterpret_cast<const uint4 *>(sums + ((2 + P) * 3) * kN);
          uint32_t *st = stage + ((cm & 1u) * 2 + P) * kN;
          uint4 *st4 = reinterpret_cast<uint4 *>(st);
          for (int c = c0 + lane; c < c0 + nc; c += 32) {
            const uint4 u = o0[c], v = o0[256 + c], t = o0[512 + c];
            st4[c] = make_uint4(u.x + v.x + t.x, u.y + v.y + t.y, u.z + v.z + t.z, u.w + v.w + t.w);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0)
            bulk_s2peer(map_peer(smem_u32(slots + ((cm & 1u) * 2 + P) * kN + c0 * 4), peer), st + c0 * 4,
                        (uint32_t)nc * 16u, map_peer(smem_u32(done + (cm & 1u)), peer));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 b0 = Bown[(4 * (fb & 1) + c) * 32 + 16 * w + (fb >> 1)];
          own[128 * w + (swp(16 * fb + 4 * c) >> 2)] =
              make_uint4(mont_mul(x[4 * c + 0], b0.x, pr), mont_mul(x[4 * c + 1], b0.y, pr),
                         mont_mul(x[4 * c + 2], b0.z, pr), mont_mul(x[4 * c + 3], b0.w, pr));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(empty + slot);
        named_bar(2 + P, kConsThreads / 2);  // the three rows of output h, prime P, in place
        if (rr < 2) {
          // quarter Qd of output h in prime P: three local rows and the peer's sum
          if (warp == 0 && lane == 0) mbar_expect_tx(done + (cm & 1u), kPeerBytes);
          mbar_wait(done + (cm & 1u), (cm >> 1) & 1u, abort_flag, args.status);
          uint32_t y[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) y[e] = 0u;
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const uint4 *sl = reinterpret_cast<const uint4 *>(r4 < 3 ? sums + (P * 3 + r4) * kN
                                                                     : slots + ((cm & 1u) * 2 + P) * kN);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const uint4 v = sl[128 * (Qd >> 1) + (swp(256 * (Qd & 1) + 8 * lane + 4 * c) >> 2)];
              y[4 * c + 0] += v.x;
              y[4 * c + 1] += v.y;
              y[4 * c + 2] += v.z;
              y[4 * c + 3] += v.w;
            }
          }
          inv_quarter(y, myscr, tw1i, args.tg->invc[P], tw2i, pr, lane);
          quarter_twist(y, args.tg->fint[P][Qd], pr, lane);
          __syncwarp();
#pragma unroll
          for (int e = 0; e < 8; ++e) myscr[lane + 32 * e] = y[e];  // natural positions of the quarter
        }
        named_bar(1, kConsThreads);  // both primes' quarters posted
        crt_update(A, post0, 2 * kHalf, args, tid, kConsThreads);
        named_bar(1, kConsThreads);  // ACC_h updated
      }
      // sample extraction: CTA 0 holds the mask a' (from ACC_0), CTA 1 the body b'
      uint32_t *o = args.out + (size_t)tile * kOutStride;
      if (h == 0) {
        for (int k = tid; k < kN; k += kConsThreads) o[k] = k == 0 ? A[0] : 0u - A[kN - k];
      } else if (tid == 0) {
        o[kN] = A[0];
      }
      named_bar(1, kConsThreads);
    }
  }
  __syncwarp();
  cluster_sync_all();  // neither CTA leaves while the peer may still touch its shared memory
  if (threadIdx.x == 0) stamp_end(args.stamps);
}

}  // namespace brc

size_t br_cluster_smem() { return brc::kSmem; }

cudaError_t launch_br_cluster(const BrArgs &args, int clusters, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(brc::br_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)brc::kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  brc::br_cluster_kernel<<<2 * clusters, brc::kThreads, brc::kSmem, st>>>(args);
  return cudaGetLastError();
}

int br_cluster_occupancy() {
  if (cudaFuncSetAttribute(brc::br_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)brc::kSmem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(brc::kThreads, 1, 1);
  cfg.dynamicSmemBytes = brc::kSmem;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 2;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, brc::br_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}

}  // namespace arx
