// br_cluster.cu -- blind rotation of one gate on a cluster of two CTAs (two SMs),
// for waves too narrow to fill the GPU.
//
// The paper runs one gate per SM and names spreading a gate over several SMs as
// the remedy for thin waves (Sec. 8).  Here the two TLWE components split the
// work: CTA h of the cluster owns accumulator polynomial ACC_h and the three TGSW
// rows whose digits come from ACC_h (rows 3h .. 3h+2), for both CRT primes (six
// consumer warps, one forward transform each per CMux).  Each warp writes its
// row's key products for both outputs to local shared memory; after a barrier
// of the three warps of its prime, each of them adds the three rows of output
// 1-h over one third of the coefficients and stores that third into the peer's
// shared memory (distributed shared memory, 8 KiB per CMux and CTA).  So CTA h
// ends each CMux holding the complete sums of output h in both primes: it runs
// the inverse transforms, the CRT and the update of ACC_h by itself, and never
// needs ACC_{1-h}.  The only cross-SM dependency per CMux is one mbarrier in
// each CTA that the peer's warps arrive on remotely (one release at cluster
// scope per warp) after their stores; the two owner warps wait on it with a
// bounded wait, and all six warps then share the CRT.
#include <cuda_runtime.h>

#include <cstdint>

#include "arx_device.cuh"

namespace arx {
namespace brc {

constexpr int kCons = 6;                      // consumer warps: (row 0..2) x (prime 0..1)
constexpr int kThreads = (kCons + 1) * 32;    // + producer warp
constexpr int kStages = 6;                    // ring of 16 KiB key rows: two CMux ahead
constexpr int kAbarPitch = 640;
constexpr long long kWaitCycles = 4000000000ll;
constexpr uint32_t kArrivals = kCons;        // the peer's consumer warps, per CMux
constexpr uint32_t kDecOffset = (1u << 10) + (64u << 25) + (64u << 18) + (64u << 11);

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

// shared memory (bytes)
constexpr size_t kRingBytes = (size_t)kStages * kChunkBytes;
constexpr size_t kAccBytes = kN * 4;                // ACC_h
constexpr size_t kDigBytes = kN * 4;                // packed digits of ACC_h
constexpr size_t kSumBytes = 2 * 2 * 3 * kN * 4;    // [output own/other][prime 2][row 3][N] products
constexpr size_t kSlotBytes = 2 * 2 * kN * 4;       // [parity 2][prime 2][N] the peer's row sums
constexpr size_t kScrBytes = (size_t)kCons * kXpose * 4;
constexpr size_t kAbarBytes = kAbarPitch * 2;
constexpr size_t kBarBytes = (2 * kStages + 1) * 8 + 16;
constexpr size_t kSmem =
    kRingBytes + kAccBytes + kDigBytes + kSumBytes + kSlotBytes + kScrBytes + kAbarBytes + kBarBytes;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void st_remote_v4(uint32_t caddr, uint4 v) {
  asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(caddr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

// Arrive on an mbarrier of any CTA of the cluster, releasing this thread's prior
// writes (and those ordered before them) at cluster scope.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

template <bool kCluster>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *status) {
  if (*abort_flag) return false;
  auto probe = [&] { return kCluster ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity); };
  if (probe()) return true;
  const long long t0 = clock64();
  while (!probe()) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
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

__device__ __forceinline__ uint32_t modswitch(uint32_t x) { return (x + (1u << 20)) >> 21; }

__device__ __forceinline__ uint32_t crt_torus(uint32_t x0, uint32_t x1) {
  const uint32_t d = x1 + 2u * kQ1 - x0;
  const uint32_t k = csub(shoup_mul(kQ0InvQ1, kQ0InvQ1Shoup, d, kQ1), kQ1);
  const uint32_t r = kQ0 * k + x0;
  return k >= kQ1 / 2 ? r - (uint32_t)kM : r;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    br_cluster_kernel(const __grid_constant__ BrArgs args) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
  uint32_t *A = reinterpret_cast<uint32_t *>(smem + kRingBytes);
  uint32_t *D = A + kN;
  uint32_t *sums = D + kN;                          // [output][prime][row][N], 16-byte chunks swizzled
  uint32_t *slots = sums + 12 * kN;                 // [parity][prime][N], same chunk order
  uint32_t *scratch = slots + 4 * kN;               // [warp][kXpose]
  uint16_t *abar = reinterpret_cast<uint16_t *>(scratch + kCons * kXpose);
  uint64_t *full = reinterpret_cast<uint64_t *>(abar + kAbarPitch);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;                 // the peer's row sums of a CMux in place
  volatile int *abort_flag = reinterpret_cast<volatile int *>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t h = cluster_rank();                // accumulator component owned here
  const uint32_t peer = h ^ 1u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 2);
    }
    mbar_init(done, kArrivals);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync_all();  // both CTAs initialised before any remote access

  const int n = args.n;
  const int nclusters = gridDim.x / 2, cid = blockIdx.x / 2;
  const int tiles = args.num_jobs;

  if (warp == kCons) {  // producer: stream this CTA's three key rows of every CMux
    if (lane == 0 && tiles > 0) {
      uint32_t jc = 0;
      bool ok = true;
      for (int tile = cid; tile < tiles && ok; tile += nclusters) {
        for (int i = 0; i < n && ok; ++i) {
          for (int rr = 0; rr < 3; ++rr, ++jc) {
            const uint32_t slot = jc % kStages;
            if (jc >= (uint32_t)kStages &&
                !mbar_wait<false>(empty + slot, ((jc / kStages) - 1) & 1u, abort_flag, args.status)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full + slot, kChunkBytes);
            bulk_g2s(ring + slot * kChunkWords, args.bsk + ((size_t)i * 6 + 3 * h + rr) * kChunkWords, kChunkBytes,
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
    const int rr = warp >> 1, P = warp & 1;         // row 3h + rr, prime P
    const int tid = threadIdx.x;                    // 0 .. 191
    const PrimeRT pr = prime_rt(P, args.tc);
    uint32_t *myscr = scratch + warp * kXpose;
    const uint2 *tw1f = args.tc.fwd1[P], *tw1i = args.tc.inv1[P];
    const uint2 *tw2f = args.tg->fwd2[P], *tw2i = args.tg->inv2[P], *twist = args.tg->twist[P];
    const uint32_t done_remote = map_peer(smem_u32(done), peer);
    uint32_t it = 0, cm = 0;  // tile counter, CMux counter
    for (int tile = cid; tile < tiles; tile += nclusters, ++it) {
      const BrJob jb = args.jobs[tile];
      const uint32_t *wa = args.wires + (size_t)jb.ia * kWireStride;
      const uint32_t *wb = args.wires + (size_t)jb.ib * kWireStride;
      const uint32_t sa = (uint32_t)(int32_t)jb.sa, sb = (uint32_t)(int32_t)jb.sb;
      for (int k = tid; k < n; k += kCons * 32) abar[k] = (uint16_t)modswitch(sa * wa[k] + sb * wb[k]);
      const uint32_t bbar = modswitch(jb.cst + sa * wa[n] + sb * wb[n]);
      const uint32_t shift = (2u * kN - bbar) & (2u * kN - 1);
      // ACC_0 = 0, ACC_1 = X^-bbar testv
      for (int k = tid; k < kN; k += kCons * 32)
        A[k] = h == 0 ? 0u : ((((uint32_t)k - shift) & (2u * kN - 1)) < (uint32_t)kN ? kMu : 0u - kMu);
      named_bar(1, kCons * 32);

      for (int i = 0; i < n; ++i, ++cm) {
        // gadget digits of X^a ACC_h - ACC_h
        const uint32_t a = abar[i];
        for (int k = tid; k < kN; k += kCons * 32) {
          const uint32_t j = ((uint32_t)k - a) & 2047u;
          uint32_t v = A[j & 1023u];
          v = (j & 1024u) ? 0u - v : v;
          const uint32_t y = v - A[k] + kDecOffset;
          D[k] = (y >> 25) | ((y >> 10) & 0x7F00u) | ((y << 5) & 0x7F0000u);
        }
        named_bar(1, kCons * 32);
        uint32_t x[32];
        const uint32_t sel = 0x4440u | (uint32_t)rr;
#pragma unroll
        for (int e = 0; e < 32; ++e) x[e] = __byte_perm(D[lane + 32 * e], 0u, sel);
        ntt_fwd<true>(x, myscr, tw1f, tw2f, pr, lane);
        const uint32_t jc = (it * (uint32_t)n + (uint32_t)i) * 3u + (uint32_t)rr;
        const uint32_t slot = jc % kStages;
        mbar_wait<false>(full + slot, (jc / kStages) & 1u, abort_flag, args.status);
        const uint4 *Bown = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + (h * 2 + P) * kN);
        const uint4 *Both = reinterpret_cast<const uint4 *>(ring + slot * kChunkWords + ((1 - h) * 2 + P) * kN);
        // row rr's products for both outputs; row `lane` of a product holds
        // positions 32 lane + e, as 16-byte chunks swizzled by lane
        uint4 *own = reinterpret_cast<uint4 *>(sums + (P * 3 + rr) * kN);
        uint4 *oth = reinterpret_cast<uint4 *>(sums + ((2 + P) * 3 + rr) * kN);
#pragma unroll
        for (int e4 = 0; e4 < 8; ++e4) {
          const uint4 b0 = Bown[e4 * 32 + lane];
          const uint4 b1 = Both[e4 * 32 + lane];
          const int chunk = lane * 8 + (e4 ^ (lane & 7));
          own[chunk] = make_uint4(mont_mul(x[4 * e4 + 0], b0.x, pr), mont_mul(x[4 * e4 + 1], b0.y, pr),
                                  mont_mul(x[4 * e4 + 2], b0.z, pr), mont_mul(x[4 * e4 + 3], b0.w, pr));
          oth[chunk] = make_uint4(mont_mul(x[4 * e4 + 0], b1.x, pr), mont_mul(x[4 * e4 + 1], b1.y, pr),
                                  mont_mul(x[4 * e4 + 2], b1.z, pr), mont_mul(x[4 * e4 + 3], b1.w, pr));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(empty + slot);
        named_bar(2 + P, 96);  // the three rows of prime P in place
        {
          // output 1-h: add the three rows over chunks rr, rr + 3, ... and send them
          const uint4 *o0 = reinterpret_cast<const uint4 *>(sums + ((2 + P) * 3) * kN);
          const uint32_t rslot = map_peer(smem_u32(slots + ((cm & 1u) * 2 + P) * kN), peer);
          for (int c = rr * 32 + lane; c < 256; c += 96) {
            const uint4 u = o0[c], v = o0[256 + c], w = o0[512 + c];
            st_remote_v4(rslot + (uint32_t)c * 16u,
                         make_uint4(u.x + v.x + w.x, u.y + v.y + w.y, u.z + v.z + w.z, u.w + v.w + w.w));
          }
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(done_remote);
        }
        if (rr == 0) {
          // owner of output h in prime P: the three local rows and the peer's sum
          mbar_wait<true>(done, cm & 1u, abort_flag, args.status);
#pragma unroll
          for (int e = 0; e < 32; ++e) x[e] = 0u;
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const uint4 *sl = reinterpret_cast<const uint4 *>(
                r4 < 3 ? sums + (P * 3 + r4) * kN : slots + ((cm & 1u) * 2 + P) * kN);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint4 v = sl[lane * 8 + (c ^ (lane & 7))];
              x[4 * c + 0] += v.x;
              x[4 * c + 1] += v.y;
              x[4 * c + 2] += v.z;
              x[4 * c + 3] += v.w;
            }
          }
          ntt_inv(x, myscr, tw1i, tw2i, twist, pr, lane);
          __syncwarp();
#pragma unroll
          for (int e = 0; e < 32; ++e) myscr[e * 32 + lane] = x[e];  // natural position lane + 32 e
        }
        named_bar(1, kCons * 32);  // both primes' results posted
        {
          const uint32_t *r0 = scratch, *r1 = scratch + kXpose;  // owner warps 0 (prime 0) and 1 (prime 1)
          for (int k = tid; k < kN; k += kCons * 32) A[k] += crt_torus(r0[k], r1[k]);
        }
        named_bar(1, kCons * 32);  // ACC_h updated
      }
      // sample extraction: CTA 0 holds the mask a' (from ACC_0), CTA 1 the body b'
      uint32_t *o = args.out + (size_t)tile * kOutStride;
      if (h == 0) {
        for (int k = tid; k < kN; k += kCons * 32) o[k] = k == 0 ? A[0] : 0u - A[kN - k];
      } else if (tid == 0) {
        o[kN] = A[0];
      }
      named_bar(1, kCons * 32);
    }
  }
  __syncwarp();
  cluster_sync_all();  // neither CTA leaves while the peer may still touch its shared memory
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
