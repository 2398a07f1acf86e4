// arx_kernels.h -- internal interface between the host engine and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace arx {

constexpr int kN = 1024;          // TLWE ring degree
constexpr int kMaxLweN = 630;     // largest LWE dimension the device layouts hold
constexpr int kWireStride = 632;  // words per LWE_n ciphertext in device buffers
constexpr int kOutStride = 1028;  // words per extracted LWE_N sample
constexpr int kKsRowStride = 632; // words per key-switching-key row
constexpr int kKsZeroWords = 640; // zero words after the key-switching-key rows (read for digit 0)
constexpr int kChunkWords = 2 * 2 * kN;       // one BSK row: [c_out 2][prime 2][N]
constexpr int kChunkBytes = kChunkWords * 4;  // 16 KiB
constexpr uint32_t kQ0 = 134215681u;  // CRT primes: = 1 mod 2048, 32 q < 2^32
constexpr uint32_t kQ1 = 134203393u;


// Twiddles.  Forward zeta[k] = psi^bitrev10(k) (k = 1..1023), psi a primitive
// 2048-th root of unity mod q; the stage with m blocks uses zeta[m + block].
// Inverse of the split transforms: omega = psi^2, the DIT stage of half-length h
// uses omega^-(j 512 / h) for the j-th pair of a block, then the output twist
// psi^-p; of the warp transforms: Gentleman-Sande, the stage of half-length t
// uses psi^-bitrev10(512 / t + block).  Every entry is
// (w, floor(w 2^32 / q)).  The warp-uniform ones travel in the kernel parameter
// block (constant bank), the per-lane ones in global memory.
struct TwiddleConst {
  uint2 fwd1[2][32];      // forward pass 1: zeta[1..31]
  uint2 inv1[2][32];      // inverse pass 1: index (h - 1) + j, h = 1, 2, 4, 8, 16, j < h
  uint32_t dig_c[2];      // (-64 - 64 zeta[1]) mod q: first-stage offset for raw digits
  uint32_t dig_d[2];      // (64 zeta[1] - 64) mod q
  uint32_t dig_c2[2];     // the same for 10-bit digits (gadget l = 2, Bg = 2^10): (-512 - 512 zeta[1]) mod q
  uint32_t dig_d2[2];     // (512 zeta[1] - 512) mod q
  uint32_t dig4[2][4];    // first two forward stages of raw 7-bit digits: the constant parts (ntt_fwd<2>)
  uint2 gsi2[2][32];      // merged inverse pass 2 (half-lengths 32..512): psi^-bitrev10(k), k = 1..31
  uint2 psi512[2];        // psi^-512 and psi^-256 (last stages of the split inverse)
  uint2 psi256[2];
};

struct TwiddleGlobal {
  uint2 fwd2[2][31 * 32];   // forward pass 2, per lane: [(2^s - 1) + block][lane]
  uint2 inv2[2][31 * 32];   // inverse pass 2, per lane: [(h/32 - 1) + j mod (h/32)][lane]
  uint2 gsi1[2][31 * 32];   // merged inverse pass 1 (half-lengths 1..16), per lane: [off_s + block][lane]
  // split transforms of the cluster kernel
  uint2 fwdh[2][2][15 * 32];  // forward pass 2 of half w: [prime][w][(2^s - 1) + block][lane]
  uint2 fwdc[2][4][7 * 32];   // forward middle pass of quarter Q (lengths 32, 16, 8): [prime][Q][(2^s - 1) + block][lane]
  uint2 fwdq[2][4][7 * 32];   // forward last pass of quarter Q (lengths 4, 2, 1): [prime][Q][(2^s - 1) + block][lane]
  uint2 invc[2][7 * 32];      // inverse quarter, middle pass (half-lengths 8, 16, 32): [prime][(2^s - 1) + j][lane]
  uint2 fint[2][4][256];      // split inverse, twist of quarter Q at k < 256: psi^-(c_Q k), c = (1, 5, 3, 7)
  uint2 fwdz[2][1024];        // every forward twiddle zeta[k] = psi^bitrev10(k) (pair transforms)
};

enum : uint32_t {
  kGateAnd = 0, kGateNand, kGateOr, kGateNor, kGateXor, kGateXnor,
  kGateNot, kGateMux, kGateCopy, kGateConst0, kGateConst1, kGateTypes
};

constexpr unsigned int kDevTimeout = 1u;

// Key sets one launch may mix (each job names its key set by an index into the
// launch's table of key pointers).
constexpr int kMaxLaunchKeys = 16;

// One blind rotation: input = cst + sa * W[ia] + sb * W[ib] (LWE_n, Torus32),
// with the bootstrapping key bsk[key] of the launch.
struct BrJob {
  uint32_t ia, ib, cst;
  int8_t sa, sb;
  uint16_t key;
};
static_assert(sizeof(BrJob) == 16, "BrJob layout");

struct BrArgs {
  const uint32_t *bsk[kMaxLaunchKeys];  // NTT-domain keys: [n][2l] rows of [c_out 2][prime 2][N] (per-lane order)
  const uint32_t *wires;  // [*][632] LWE_n ciphertexts
  const BrJob *jobs;
  int num_jobs;
  int n;
  uint32_t *out;          // [num_jobs][1028] extracted LWE_N samples
  const TwiddleGlobal *tg;
  unsigned int *status;   // device status word (kDevTimeout on a watchdog expiry)
  unsigned long long *stamps;  // optional {first CTA start, last warp end} in global-timer ns (autotuner)
  TwiddleConst tc;        // warp-uniform twiddles, read from the parameter bank
};

// One gate output.  Bootstrapped gates key-switch br_out[j0] (+ br_out[j1] + 1/8
// for MUX) with the key-switching key ksk[key] of the launch; NOT / COPY read
// wire ia; CONST writes a trivial sample.
struct KsJob {
  uint32_t type, j0, j1, ia, out, key;
};

struct KsArgs {
  const uint32_t *ksk[kMaxLaunchKeys];  // [N][8][3][632] rows for digits 1..3
  const uint32_t *br_out;  // [*][1028]
  const uint32_t *wires;   // [*][632]
  const KsJob *jobs;
  int n;
  uint32_t *out;           // destination rows (out_stride words apart)
  int out_stride;
  int splits;              // CTAs per gate: each sums N / splits of the key rows
  uint32_t *partial;       // scratch [jobs][splits][632] (splits > 1)
  unsigned int *counters;  // scratch [jobs], zero between launches (splits > 1)
};

struct BrShape {
  int H;   // row groups per prime: 2H warps per gate
  int GT;  // gates per CTA
};

// Twiddle tables for the two CRT primes (computed on the host, once).
void make_twiddles(TwiddleConst *tc, TwiddleGlobal *tg);

// rows = (k+1) l TGSW rows per key index (6, or 4 for the gadget l = 2)
cudaError_t launch_bsk_to_ntt(const uint32_t *bsk_coef, int n, int rows, uint32_t *bsk_ntt, const TwiddleConst &tc,
                              const TwiddleGlobal *tg, cudaStream_t st);
size_t br_smem(BrShape s);
bool br_shape_supported(BrShape s);
int br_occupancy(BrShape s);  // resident CTAs per SM (0: cannot launch)
cudaError_t launch_br(const BrArgs &args, BrShape s, int grid, cudaStream_t st);
cudaError_t launch_ks(const KsArgs &args, int num_jobs, cudaStream_t st);
// Splits of the key-switch gather for a wave of num_jobs gates on sms SMs.
int ks_splits(int num_jobs, int sms);
cudaError_t launch_gather(const uint32_t *wires, const uint32_t *idx, int count, int n, uint32_t *dst,
                          int dst_stride, cudaStream_t st);

// Cluster shape {kClusterH, 1}: one gate on a cluster of two CTAs (two SMs);
// its grid is counted in clusters.
constexpr int kClusterH = 12;
size_t br_cluster_smem();
cudaError_t launch_br_cluster(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster_occupancy();  // co-resident clusters on the device (0: cannot launch)
// Cluster shape {kCluster4H, 1}: one gate on a cluster of four CTAs (four SMs).
constexpr int kCluster4H = 24;
size_t br_cluster4_smem();
cudaError_t launch_br_cluster4(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster4_occupancy();
// Cluster shape {kCluster8H, 1}: one gate on a cluster of eight CTAs (eight SMs).
constexpr int kCluster8H = 48;
size_t br_cluster8_smem();
cudaError_t launch_br_cluster8(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster8_occupancy();
// Shape {kCluster8L2H, 1}: the eight-CTA kernel for key sets with gadget l = 2
// (Bg = 2^10); chosen automatically for such key sets, never by an override.
constexpr int kCluster8L2H = 40;
size_t br_cluster8_l2_smem();
cudaError_t launch_br_cluster8_l2(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster8_l2_occupancy();
// Cluster shape {kCluster16H, 1}: one gate on a cluster of sixteen CTAs (a
// non-portable cluster size; occupancy 0 where the device refuses it).
constexpr int kCluster16H = 96;
size_t br_cluster16_smem();
cudaError_t launch_br_cluster16(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster16_occupancy();
// Shape {kCluster16L2H, 1}: the sixteen-CTA kernel for key sets with gadget
// l = 2; chosen automatically for such key sets, never by an override.
constexpr int kCluster16L2H = 80;
size_t br_cluster16_l2_smem();
cudaError_t launch_br_cluster16_l2(const BrArgs &args, int clusters, cudaStream_t st);
int br_cluster16_l2_occupancy();
inline bool is_cluster_shape(BrShape s) {
  return s.H == kClusterH || s.H == kCluster4H || s.H == kCluster8H || s.H == kCluster8L2H || s.H == kCluster16H ||
         s.H == kCluster16L2H;
}
// Shapes {kGadget2 + H, GT}: the throughput kernel br_kernel<H, GT, 2> for key
// sets with gadget l = 2 (H in 1, 2, 4).
constexpr int kGadget2 = 100;
// Shapes reserved for key sets with gadget l = 2 (never an override).
inline bool is_l2_shape(BrShape s) { return s.H == kCluster8L2H || s.H == kCluster16L2H || s.H > kGadget2; }

// per-shape launchers (one translation unit per H)
cudaError_t launch_br_h1(const BrArgs &args, int GT, int L, int grid, cudaStream_t st);
cudaError_t launch_br_h2(const BrArgs &args, int GT, int L, int grid, cudaStream_t st);
cudaError_t launch_br_h3(const BrArgs &args, int GT, int L, int grid, cudaStream_t st);
cudaError_t launch_br_h4(const BrArgs &args, int GT, int L, int grid, cudaStream_t st);
cudaError_t launch_br_h6(const BrArgs &args, int GT, int L, int grid, cudaStream_t st);

}  // namespace arx
