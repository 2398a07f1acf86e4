// engine_internal.h -- host-side state of libarx shared by engine.cpp and serve.cpp.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/arx.h"
#include "arx_kernels.h"

namespace arx {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t bytes);
  void release();
  template <class T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

struct Keyset {
  bool used = false;
  int n = 0;
  int l = 3;                // gadget length: 3 (Bg = 2^7) or 2 (Bg = 2^10)
  uint32_t *bsk = nullptr;  // NTT-domain bootstrapping key
  uint32_t *ksk = nullptr;  // [N][8][3][632]
  int refs = 0;             // plans referencing it
};

struct Workspace {
  DevBuf wires, brjobs, ksjobs, brout, out, kspart, kscnt;
};

struct Level {
  int br_off = 0, br_cnt = 0, ks_off = 0, ks_cnt = 0;
  BrShape shape{1, 1};
  int grid = 1;
  // a level split over two blind-rotation launches: the first br_split jobs on
  // `shape`, the rest on shape2 (br_split = 0: one launch of all br_cnt)
  int br_split = 0;
  BrShape shape2{0, 0};
  int grid2 = 0;
  int ks_splits = 1;
};

struct Plan {
  int keyset = -1, n = 0, mode = 0, l = 3;
  uint32_t num_inputs = 0, num_gates = 0;
  std::vector<uint32_t> outputs;
  std::vector<Level> levels;
  uint64_t bootstraps = 0;
  DevBuf wires, brjobs, ksjobs, brout, outidx, outstage, kspart, kscnt;
  cudaGraphExec_t exec = nullptr;
};

struct TuneEntry {
  BrShape shape{1, 1};
  double wave_ms_per_cmux = 0;
  int gates_per_wave = 0;
};

// Launch-shape choice: the autotuned table (one LWE dimension), resident CTAs
// per SM of every shape, and an optional override.  Copyable, so that the
// serving thread can use a snapshot without the engine lock.
struct ShapePolicy {
  int sms = 0;
  int clusters16 = 0, clusters8 = 0, clusters4 = 0, clusters2 = 0;  // co-resident 16- / 8- / 4- / 2-CTA clusters
  int clusters16l2 = 0;  // co-resident sixteen-CTA clusters of the l = 2 kernel
  std::vector<TuneEntry> tune;
  int tuned_n = -1;
  std::vector<std::pair<BrShape, int>> occ;
  BrShape forced{0, 0};
  int occupancy(BrShape s);
  BrShape heuristic(int jobs) const;
  BrShape wide(int jobs) const;  // the throughput shapes of the heuristic
  BrShape pick(int jobs, int n) const;
  // Autotuned cost (ms per CMux) of `jobs` blind rotations as one launch of the
  // best shape (the one pick takes, stored in *s).
  double launch_cost(int jobs, BrShape *s) const;
  // The cheapest way, by the autotuned table, to run `jobs` blind rotations as at
  // most two launches: rounds of one throughput shape (*bulk, the first
  // *bulk_jobs) and the rest on the best shape for them (*tail; {0, 0} when one
  // launch is cheapest).  Returns its cost (ms per CMux).
  double split(int jobs, BrShape *bulk, int *bulk_jobs, BrShape *tail) const;
  // The most blind rotations one level takes at the cost of a level of `jobs`
  // (gadget length l): a cluster kernel's wave costs the same for every count up
  // to its co-resident clusters, so the rest of that width is free; with the
  // autotuned table the costs are the measured ones, of the level's launches as
  // split chooses them.
  int free_capacity(int jobs, int n, int l) const;
  // Key sets with gadget l = 2 (given the shape chosen for l = 3 and the wave's
  // blind rotations): their own sixteen-CTA kernel while the wave's gates fit
  // its co-resident clusters, else their eight-CTA kernel while a wave takes at
  // most two rounds of its clusters, else the throughput kernel
  // br_kernel<H, GT, 2> on the matching shape.  An override of a cluster shape
  // maps to the l = 2 kernel of the same cluster size (sixteen), else to the
  // eight-CTA one.
  BrShape for_gadget(int l, BrShape s, int jobs) const;
  int grid(BrShape s, int jobs);
};

struct Engine {
  std::mutex mu;
  bool ready = false;
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  TwiddleConst tc{};
  TwiddleGlobal *tg = nullptr;
  unsigned int *status = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<Keyset> keysets;
  int last = -1;
  size_t budget = 0;  // HBM budget for resident keys (0 = none)
  std::map<cudaStream_t, Workspace> ws;
  std::vector<std::unique_ptr<Plan>> plans;
  ShapePolicy policy;
  size_t resident_bytes() const;
};

Engine &eng();
int fail(int code, const char *fmt, ...);
int ensure_init(Engine &E);
bool is_device_ptr(const void *p);
int resolve_keyset(Engine &E, int keyset, Keyset **out);
int read_status(Engine &E, cudaStream_t st);
int gate_arity(uint32_t type);
void emit_gate(uint32_t type, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t out, std::vector<BrJob> &br,
               std::vector<KsJob> &ks, uint32_t br_base);
int calibrate(Engine &E, int n);
int levelize(const arx_netlist *nl, uint32_t *wave, uint32_t *depth);
// Moves gates between their earliest wave (wave[g] from levelize) and their
// latest one so that each launch is filled up to its free capacity
// (cap_of(blind rotations) = the most blind rotations at the same cost); the
// depth is unchanged and every gate still follows its inputs.
void balance_levels(const arx_netlist *nl, uint32_t depth, const std::function<long long(long long)> &cap_of,
                    uint32_t *wave);
size_t keyset_bytes(int n, int l = 3);
int reserve_ks_scratch(DevBuf &part, DevBuf &cnt, size_t jobs, int splits);

}  // namespace arx
