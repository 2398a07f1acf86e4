// br_cluster16.cu -- blind rotation of one gate on a cluster of sixteen CTAs
// (sixteen SMs, a non-portable cluster size), for the narrowest waves.
//
// The paper runs one gate per SM and names spreading a gate over several SMs as
// the remedy for thin waves (Sec. 8).  Here CTA (h, Q, P) of the cluster (rank
// 4 Q + 2 P + h) owns accumulator component ACC_h, the TGSW rows whose digits
// come from it (rows L h .. L h + L - 1), spectral quarter Q and one CRT prime P:
// the eight-CTA kernel's work split once more, by prime, so that a CTA's
// forward and inverse transforms can each run on a pair of warps.
//
// Per CMux: all warps compute the gadget digits of the CTA's three rows and
// take the first two forward stages of quarter Q in prime P at once
// (make_stage2); three pairs of forward warps (one pair per row) run the rest
// of the quarter-Q transform of their row (fwd_quarter_pair); each warp copies
// its half of the key products for output 1-h into its row's receive slot at
// CTA (1-h, Q, P) (a plain bulk copy of 512 bytes: measured faster than bulk
// reduce-adds into one slot) and keeps those for output h.  A pair of inverse
// warps on two schedulers (two of the forward warps) sums the L local rows and
// the L received ones (quarter Q of output h in prime P), runs the inverse
// quarter transform split between them (inv_quarter_pair: all stages but the
// last two, then the quarter's share of the output twist) and stores it here;
// seven consumer warps then post it to the seven CTAs (h, Q', P') (1 KiB each,
// one bulk copy per warp).  All eight CTAs of component h
// then fold the last two stages, run the CRT and update identical copies of
// ACC_h.  Every
// cross-CTA dependency is a transaction count on an mbarrier (double-buffered
// by CMux parity); every wait is bounded.  The kernel is a template on the
// gadget length L: 3 (Bg = 2^7: six forward warps, the inverse pair on warps 3
// and 4) or 2 (Bg = 2^10, the paper's own set: four forward warps, one per
// scheduler, the inverse pair on warps 1 and 2).
#include <cuda_runtime.h>

#include <cstdint>

#include "br_cluster_common.cuh"

namespace arx {
namespace brc16 {

using namespace clu;

constexpr int kClusterSize = 16;
constexpr int kCons = 8;                    // forward warps (two of them the inverse pair), helpers
constexpr int kThreads = (kCons + 1) * 32;  // + producer warp
constexpr int kConsThreads = kCons * 32;    // 256
constexpr int kStages = 6;                  // ring of 8 KiB key rows (one prime, both outputs)
constexpr int kRowWords = 2 * kN;
constexpr uint32_t kRowBytes = kRowWords * 4;
constexpr int kAbarPitch = 640;
constexpr int kQuarter = 256;
constexpr uint32_t kPartnerBytes = 7 * kQuarter * 4;  // seven partners, one quarter each

template <int L>  // TGSW rows per accumulator component (gadget length)
struct Cfg {
  static constexpr int kFwd = 2 * L;                 // forward pair of row r: warps r and r + L
  static constexpr int kInvWarp = L == 3 ? 3 : 1;    // inverse pair: warps kInvWarp, kInvWarp + 1
  static_assert(kInvWarp + 1 < kFwd, "the inverse pair is two of the forward warps");
  static constexpr uint32_t kPeerBytes = L * kQuarter * 4;         // the peer's L row products
  static constexpr size_t kRingBytes = (size_t)kStages * kRowBytes;
  static constexpr size_t kAccBytes = kN * 4;
  static constexpr size_t kDigBytes = (size_t)L * 256 * 4;        // [row][k] stage-2 values of quarter Q
  static constexpr size_t kOwnBytes = (size_t)L * kQuarter * 4;       // [row][quarter Q] products for output h
  static constexpr size_t kOthBytes = (size_t)2 * L * kQuarter * 4;   // [parity][row] for output 1-h
  static constexpr size_t kSlotBytes = (size_t)2 * L * kQuarter * 4;  // [parity][row] the peer's products
  static constexpr size_t kPostBytes = (size_t)2 * 2 * 4 * kQuarter * 4;  // [parity][prime][quarter][k]
  static constexpr size_t kScrBytes = (size_t)kCons * kQuarter * 4;
  static constexpr size_t kPairBytes = (size_t)L * kQuarter * 4;      // [row] the pass A -> B exchange
  static constexpr size_t kAbarBytes = kAbarPitch * 2;
  static constexpr size_t kBarBytes = (2 * kStages + 4) * 8 + 16;
  static constexpr size_t kSmem = kRingBytes + kAccBytes + kDigBytes + kOwnBytes + kOthBytes + kSlotBytes +
                                  kPostBytes + kScrBytes + kPairBytes + kAbarBytes + kBarBytes;
};

template <int L>
__global__ void __launch_bounds__(kThreads, 1) br_cluster16_kernel(const __grid_constant__ BrArgs args) {
  using C = Cfg<L>;  // shared-memory layout
  constexpr int kFwd = C::kFwd, kInvWarp = C::kInvWarp;
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem);  // [stage][output][N]
  uint32_t *A = reinterpret_cast<uint32_t *>(smem + C::kRingBytes);
  uint32_t *D = A + kN;                          // [row][k] stage-2 values (make_stage2)
  uint32_t *own = D + C::kDigBytes / 4;          // [row][256], swizzled (swp)
  uint32_t *oth = own + L * kQuarter;            // [parity][row][256], same layout
  uint32_t *slots = oth + 2 * L * kQuarter;      // [parity][row][256], same layout
  uint32_t *post = slots + 2 * L * kQuarter;     // [parity][prime][quarter][256], natural order
  uint32_t *scratch = post + 16 * kQuarter;      // [warp][256]
  uint32_t *pairbuf = scratch + kCons * kQuarter;  // [row][256]
  uint16_t *abar = reinterpret_cast<uint16_t *>(pairbuf + L * kQuarter);
  uint64_t *full = reinterpret_cast<uint64_t *>(abar + kAbarPitch);
  uint64_t *empty = full + kStages;
  uint64_t *done1 = empty + kStages;             // [parity]: the peer's L rows in place
  uint64_t *done2 = done1 + 2;                   // [parity]: the partners' inverse quarters in place
  volatile int *abort_flag = reinterpret_cast<volatile int *>(done2 + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t h = rank & 1u;                  // accumulator component
  const int P = (int)((rank >> 1) & 1u);         // CRT prime
  const int Q = (int)(rank >> 2);                // spectral quarter
  const uint32_t peer = rank ^ 1u;               // (1-h, Q, P)
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 2);  // the forward pair of the row
    }
    for (int p = 0; p < 2; ++p) {
      mbar_init(done1 + p, 1);  // one local arrival (with the expected bytes) per CMux
      mbar_init(done2 + p, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync_all();  // all sixteen CTAs initialised before any remote access
  if (threadIdx.x == 0) stamp_start(args.stamps);

  const int n = args.n;
  const int nclusters = gridDim.x / kClusterSize, cid = blockIdx.x / kClusterSize;
  const int tiles = args.num_jobs;

  if (warp == kCons) {  // producer: the L key rows of component h, prime P, for every CMux
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
            mbar_expect_tx(full + slot, kRowBytes);
            const uint32_t *row = args.bsk[args.jobs[tile].key] + ((size_t)i * 2 * L + L * h + rr) * kChunkWords;
#pragma unroll
            for (int c = 0; c < 2; ++c)  // key row layout [output][prime][N]
              bulk_g2s(ring + slot * kRowWords + c * kN, row + (c * 2 + P) * kN, kN * 4u, full + slot);
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
    const int rr = fwd ? warp % L : 0;  // forward pairs: row L h + rr on warps rr, rr + L
    const int fw = fwd ? warp / L : 0;  // the warp's half of the pair
    const int tid = threadIdx.x;        // 0 .. 255
    PrimeRT pr = prime_rt(P, args.tc);
    if (L == 2) {  // first-stage offsets of 10-bit digits
      pr.dc = args.tc.dig_c2[P];
      pr.dd = args.tc.dig_d2[P];
    }
    const uint2 z1 = args.tc.fwd1[P][1], z23 = args.tc.fwd1[P][2 + (Q >> 1)];
    const int jl = 8 * (lane & 3) + (lane >> 2);  // the forward pair's output block (see fwd_quarter_pair)
    const int jf = 32 * fw + jl;
    const FwdPairTw zf = load_fwd_pair(args, P, Q, fw, lane);  // loop-invariant per-lane twiddles
    const bool inv = warp == kInvWarp || warp == kInvWarp + 1;
    const int t = lane + 32 * (warp == kInvWarp + 1 ? 1 : 0);  // position index within the inverse pair
    const InvPairTw zp = load_inv_pair(args, P, Q, t);
    uint32_t cm = 0;  // CMux counter over this cluster's tiles
    for (int tile = cid; tile < tiles; tile += nclusters) {
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
      uint32_t acc4[4];  // this thread's column of ACC_h: A[tid + 256 m], kept across CMuxes
#pragma unroll
      for (int m = 0; m < 4; ++m) acc4[m] = A[tid + 256 * m];

      for (int i = 0; i < n; ++i, ++cm) {
        const uint32_t par = cm & 1u, ph = (cm >> 1) & 1u;
        // key row of this CMux: waited for here only for the first CMux; later ones
        // are waited for during the previous CMux's wait for the partners
        if (fwd && cm == 0) mbar_wait(full + rr % kStages, 0u, abort_flag, args.status, kWaitCycles, true);
        make_stage2_col<L>(D, A, acc4, abar[i], z1, z23, Q, pr, tid);
        named_bar(1, kConsThreads);
        if (fwd) {
          uint32_t x[4];
          fwd_quarter_pair(x, D + rr * 256, pairbuf + rr * kQuarter, scratch + warp * kQuarter, zf, pr, fw, lane,
                           4 + rr);
          const uint32_t jc = cm * (uint32_t)L + (uint32_t)rr;
          const uint32_t slot = jc % kStages;
          // key row layout: position 32 L + E at word ((E >> 2) * 32 + L) * 4 + (E & 3), so
          // positions 256 Q + 4 j .. + 3 are 16-byte word (j mod 8) * 32 + 8 Q + j / 8
          const uint4 *Bown = reinterpret_cast<const uint4 *>(ring + slot * kRowWords + h * kN);
          const uint4 *Both = reinterpret_cast<const uint4 *>(ring + slot * kRowWords + (1 - h) * kN);
          const int kj = (jf & 7) * 32 + 8 * Q + (jf >> 3);
          uint32_t *oq = oth + (par * L + rr) * kQuarter;
          // products for the peer's output first: copied into its slot of this row while the rest runs
          const uint4 b1 = Both[kj];
          reinterpret_cast<uint4 *>(oq)[s_j(jf)] =
              make_uint4(mont_mul(x[0], b1.x, pr), mont_mul(x[1], b1.y, pr), mont_mul(x[2], b1.z, pr),
                         mont_mul(x[3], b1.w, pr));
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0)  // this warp's half: positions 128 fw .. 128 fw + 127, 512 bytes
            bulk_s2peer(map_peer(smem_u32(slots + (par * L + rr) * kQuarter + 128 * fw), peer), oq + 128 * fw,
                        kQuarter * 2u, map_peer(smem_u32(done1 + par), peer));
          const uint4 b0 = Bown[kj];
          reinterpret_cast<uint4 *>(own + rr * kQuarter)[s_j(jf)] =
              make_uint4(mont_mul(x[0], b0.x, pr), mont_mul(x[1], b0.y, pr), mont_mul(x[2], b0.z, pr),
                         mont_mul(x[3], b0.w, pr));
          __syncwarp();
          if (lane == 0) mbar_arrive_cta(empty + slot);
          if (!inv) named_bar_arrive(2, 32 * kFwd);  // the L rows of output h, quarter Q, in place
        }
        if (inv) {
          if (warp == kInvWarp && lane == 0) {
            mbar_expect_tx(done1 + par, C::kPeerBytes);
            mbar_expect_tx(done2 + par, kPartnerBytes);
          }
          named_bar(2, 32 * kFwd);
          // quarter Q of output h in prime P: L local rows and the peer's L rows, at 4 t + e
          // (the slots are read before this CTA's posts below, so before the peer can
          // refill them two CMuxes later)
          // (the local rows are summed before the wait for the peer's)
          uint32_t y[4] = {0u, 0u, 0u, 0u};
          const int ci = s_j(t);
#pragma unroll
          for (int r4 = 0; r4 < 2 * L; ++r4) {
            if (r4 == L) mbar_wait(done1 + par, ph, abort_flag, args.status, kWaitCycles, true);
            const uint4 *sl =
                reinterpret_cast<const uint4 *>(r4 < L ? own + r4 * kQuarter : slots + (par * L + r4 - L) * kQuarter);
            const uint4 q = sl[ci];
            y[0] += q.x;
            y[1] += q.y;
            y[2] += q.z;
            y[3] += q.w;
          }
          inv_quarter_pair(y, scratch + kInvWarp * kQuarter, scratch + (kInvWarp + 1) * kQuarter, zp, pr, t, 3);
          // post the quarter here and at the seven CTAs (h, Q', P') (ranks rank ^ 2 j)
          uint32_t *pq = post + ((par * 2 + P) * 4 + Q) * kQuarter;
#pragma unroll
          for (int e = 0; e < 4; ++e) pq[t + 64 * e] = y[e];
          fence_proxy_async_smem();
        }
        // the quarter is in place: consumer warps 0 .. 6 post it to the seven CTAs
        // (h, Q', P') (ranks rank ^ 2 (w + 1)), one bulk copy each (seven warps
        // measured 0.3 % faster per step than seven lanes of one warp)
        named_bar(7, kConsThreads);
        if (warp < 7 && lane == 0) {
          const uint32_t *pq = post + ((par * 2 + P) * 4 + Q) * kQuarter;
          const uint32_t dst = rank ^ (2u * (uint32_t)(warp + 1));
          bulk_s2peer(map_peer(smem_u32(pq), dst), pq, kQuarter * 4u, map_peer(smem_u32(done2 + par), dst));
        }
        if (fwd && (i + 1 < n || tile + nclusters < tiles)) {  // the next CMux's key row
          const uint32_t jn = (cm + 1u) * (uint32_t)L + (uint32_t)rr;
          mbar_wait(full + jn % kStages, (jn / kStages) & 1u, abort_flag, args.status, kWaitCycles, true);
        }
        // every thread waits for the partners' quarters itself (the local one is
        // behind barrier 7), so no barrier is needed before the CRT pass
        mbar_wait(done2 + par, ph, abort_flag, args.status, kWaitCycles, true);
        {
          const uint32_t *pp = post + par * 2 * 4 * kQuarter;
          const uint32_t *post0[4] = {pp, pp + kQuarter, pp + 2 * kQuarter, pp + 3 * kQuarter};
          crt_update_col(A, acc4, post0, 4 * kQuarter, args, tid);
        }
        named_bar(1, kConsThreads);  // ACC_h updated
      }
      // sample extraction (quarter 0, prime 0): CTA (0, 0, 0) holds the mask a' (from ACC_0), CTA (1, 0, 0) the body b'
      uint32_t *o = args.out + (size_t)tile * kOutStride;
      if (Q == 0 && P == 0) {
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

}  // namespace brc16

namespace {
template <int L>
cudaError_t prepare16() {
  static bool attr = false;  // calls are serialised by the engine lock
  if (attr) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(brc16::br_cluster16_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)brc16::Cfg<L>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(brc16::br_cluster16_kernel<L>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) attr = true;
  return e;
}

template <int L>
cudaLaunchConfig_t config16(int clusters, cudaStream_t st, cudaLaunchAttribute *at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(brc16::kClusterSize * clusters, 1, 1);
  cfg.blockDim = dim3(brc16::kThreads, 1, 1);
  cfg.dynamicSmemBytes = brc16::Cfg<L>::kSmem;
  cfg.stream = st;
  at->id = cudaLaunchAttributeClusterDimension;
  at->val.clusterDim.x = brc16::kClusterSize;
  at->val.clusterDim.y = 1;
  at->val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <int L>
cudaError_t launch16(const BrArgs &args, int clusters, cudaStream_t st) {
  cudaError_t e = prepare16<L>();
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at;
  cudaLaunchConfig_t cfg = config16<L>(clusters, st, &at);
  return cudaLaunchKernelEx(&cfg, brc16::br_cluster16_kernel<L>, args);
}

// Co-resident sixteen-CTA clusters (0 where the device does not allow them).
template <int L>
int occupancy16() {
  if (prepare16<L>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute at;
  cudaLaunchConfig_t cfg = config16<L>(1, nullptr, &at);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, brc16::br_cluster16_kernel<L>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}
}  // namespace

size_t br_cluster16_smem() { return brc16::Cfg<3>::kSmem; }
cudaError_t launch_br_cluster16(const BrArgs &args, int clusters, cudaStream_t st) {
  return launch16<3>(args, clusters, st);
}
int br_cluster16_occupancy() { return occupancy16<3>(); }
size_t br_cluster16_l2_smem() { return brc16::Cfg<2>::kSmem; }
cudaError_t launch_br_cluster16_l2(const BrArgs &args, int clusters, cudaStream_t st) {
  return launch16<2>(args, clusters, st);
}
int br_cluster16_l2_occupancy() { return occupancy16<2>(); }

}  // namespace arx
