// engine.cpp -- host side of libarx: device state, key sets, workspaces, the wave
// scheduler for netlists, plans with CUDA-graph replay, the launch-shape
// autotuner, and the C-ABI entry points declared in include/arx.h.
//
// Runtime structure follows Sec. 4.2 / Sec. 5 of the paper, re-designed for one
// GB300: the netlist is levelized once into waves (FIFO topological sort); each
// wave becomes one blind-rotation launch over all of its bootstrapped gates (of any
// gate type, with a per-gate descriptor) and one key-switch launch; wires stay in
// HBM for the whole evaluation (instead of pinned host memory); the per-wave
// descriptor arrays are built on the host ahead of time and stay on the device
// (instead of per-stream buffers filled by host callbacks); waves are ordered by
// stream order, or replayed as a single CUDA graph (instead of event fences).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "../../include/arx.h"
#include "arx_kernels.h"
#include "engine_internal.h"

namespace arx {

thread_local std::string t_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? ARX_ENOMEM : ARX_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                  \
    }                                                                                       \
  } while (0)

cudaError_t DevBuf::reserve(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t want = bytes + bytes / 4;  // grow with headroom
  cudaError_t e = cudaMalloc(&p, want);
  if (e == cudaSuccess) cap = want;
  return e;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

Engine &eng() {
  static Engine *e = new Engine;  // intentionally never destroyed (no teardown after the CUDA runtime)
  return *e;
}

int ensure_init(Engine &E) {
  if (E.ready) return ARX_OK;
  CK(cudaGetDevice(&E.device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, E.device));
  if (prop.major < 10)
    return fail(ARX_ECUDA, "device %s (sm_%d%d): libarx is built for sm_103a", prop.name, prop.major, prop.minor);
  E.sms = prop.multiProcessorCount;
  E.policy.sms = E.sms;
  E.policy.clusters16 = E.policy.occupancy(BrShape{kCluster16H, 1});
  E.policy.clusters16l2 = E.policy.occupancy(BrShape{kCluster16L2H, 1});
  E.policy.clusters8 = E.policy.occupancy(BrShape{kCluster8H, 1});
  E.policy.clusters4 = E.policy.occupancy(BrShape{kCluster4H, 1});
  E.policy.clusters2 = E.policy.occupancy(BrShape{kClusterH, 1});
  E.smem_optin = prop.sharedMemPerBlockOptin;
  std::unique_ptr<TwiddleGlobal> tg(new TwiddleGlobal);
  make_twiddles(&E.tc, tg.get());
  CK(cudaMalloc(&E.tg, sizeof(TwiddleGlobal)));
  CK(cudaMemcpy(E.tg, tg.get(), sizeof(TwiddleGlobal), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&E.status, sizeof(unsigned int)));
  CK(cudaMemset(E.status, 0, sizeof(unsigned int)));
  CK(cudaStreamCreateWithFlags(&E.stream, cudaStreamNonBlocking));
  E.ready = true;
  return ARX_OK;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int resolve_keyset(Engine &E, int keyset, Keyset **out) {
  if (keyset < 0) keyset = E.last;
  if (keyset < 0 || keyset >= (int)E.keysets.size() || !E.keysets[keyset].used)
    return fail(ARX_ENOKEYS, "no key set %d loaded", keyset);
  *out = &E.keysets[keyset];
  return ARX_OK;
}

int read_status(Engine &E, cudaStream_t st) {
  unsigned int v = 0;
  CK(cudaMemcpyAsync(&v, E.status, sizeof(v), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (v) {
    CK(cudaMemsetAsync(E.status, 0, sizeof(unsigned int), st));
    CK(cudaStreamSynchronize(st));
    return fail(ARX_ETIMEOUT, "device watchdog expired (status 0x%x)", v);
  }
  return ARX_OK;
}

// --------------------------------------------------------------------------
// gate linear parts (Fig. 2 top box; constants as in the design notes)
// --------------------------------------------------------------------------
bool gate_linear(uint32_t type, int8_t *sa, int8_t *sb, uint32_t *cst) {
  const uint32_t e = ARX_MU, q = 2u * ARX_MU;
  switch (type) {
    case ARX_AND: *sa = 1; *sb = 1; *cst = 0u - e; return true;
    case ARX_NAND: *sa = -1; *sb = -1; *cst = e; return true;
    case ARX_OR: *sa = 1; *sb = 1; *cst = e; return true;
    case ARX_NOR: *sa = -1; *sb = -1; *cst = 0u - e; return true;
    case ARX_XOR: *sa = 2; *sb = 2; *cst = q; return true;
    case ARX_XNOR: *sa = -2; *sb = -2; *cst = 0u - q; return true;
    default: return false;
  }
}

int gate_arity(uint32_t type) {
  switch (type) {
    case ARX_NOT: case ARX_COPY: return 1;
    case ARX_CONST0: case ARX_CONST1: return 0;
    case ARX_MUX: return 3;
    default: return 2;
  }
}

// Appends the blind-rotation jobs and the key-switch job of one gate.
void emit_gate(uint32_t type, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t out, std::vector<BrJob> &br,
               std::vector<KsJob> &ks, uint32_t br_base) {
  KsJob k{type, 0, 0, w0, out};
  BrJob j{};
  if (type == ARX_MUX) {
    // MUX(s, t, f): AND(s, t) and AND(not s, f) blind-rotated, summed with 1/8, one KS.
    j = BrJob{w0, w1, 0u - ARX_MU, 1, 1};
    k.j0 = (uint32_t)br.size() - br_base;
    br.push_back(j);
    j = BrJob{w0, w2, 0u - ARX_MU, -1, 1};
    k.j1 = (uint32_t)br.size() - br_base;
    br.push_back(j);
  } else if (gate_linear(type, &j.sa, &j.sb, &j.cst)) {
    j.ia = w0;
    j.ib = w1;
    k.j0 = (uint32_t)br.size() - br_base;
    br.push_back(j);
  }
  ks.push_back(k);
}

// --------------------------------------------------------------------------
// launch shapes: heuristic and autotuned
// --------------------------------------------------------------------------
const BrShape kShapes[] = {{kCluster16H, 1}, {kCluster8H, 1}, {kCluster4H, 1}, {kClusterH, 1}, {6, 1}, {3, 1}, {3, 2}, {2, 1}, {2, 3}, {1, 1}, {1, 2}, {1, 4}, {1, 6}};

int ShapePolicy::occupancy(BrShape s) {
  for (auto &kv : occ)
    if (kv.first.H == s.H && kv.first.GT == s.GT) return kv.second;
  const int o = br_occupancy(s);
  occ.push_back({s, o});
  return o;
}

// Plain mode: a sixteen-, eight-, four-, then two-SM cluster per gate while all of the
// wave's clusters fit on the device at once (larger clusters pack less densely:
// a cluster must sit in one GPC), then about twelve consumer warps per SM with
// more gates per CTA as the wave widens.
BrShape ShapePolicy::heuristic(int jobs) const {
  if (forced.H) return forced;
  if (jobs <= clusters16) return {kCluster16H, 1};
  if (jobs <= clusters8) return {kCluster8H, 1};
  if (jobs <= clusters4) return {kCluster4H, 1};
  if (jobs <= std::max(clusters2, sms / 2)) return {kClusterH, 1};
  return wide(jobs);
}

BrShape ShapePolicy::wide(int jobs) const {
  const int per_sm = (jobs + sms - 1) / sms;
  if (per_sm <= 1) return {6, 1};
  if (per_sm == 2) return {3, 2};
  if (per_sm == 3) return {2, 3};
  if (per_sm <= 4) return {1, 4};
  return {1, 6};
}

BrShape ShapePolicy::for_gadget(int l, BrShape s, int jobs) const {
  if (l != 2) return s;
  const bool cluster = is_cluster_shape(s);
  // (each cluster kernel only where the device co-schedules its clusters)
  if (!forced.H) {
    if (clusters16l2 > 0 && jobs <= clusters16l2) return {kCluster16L2H, 1};
    if (clusters8 > 0 && jobs <= 2 * clusters8) return {kCluster8L2H, 1};
  } else if (cluster) {
    if (s.H == kCluster16H && clusters16l2 > 0) return {kCluster16L2H, 1};
    if (clusters8 > 0) return {kCluster8L2H, 1};
  }
  if (cluster) s = wide(jobs);
  // rows per warp as close as the 4 rows of l = 2 allow: H 6 -> 4, 3 and 2 -> 2
  switch (s.H) {
    case 1: return {kGadget2 + 1, s.GT};
    case 2: return {kGadget2 + 2, s.GT};
    case 3: return {kGadget2 + 2, s.GT == 1 ? 1 : 3};
    default: return {kGadget2 + 4, 1};
  }
}

// Autotuned: the shape minimising waves x measured time per wave.
BrShape ShapePolicy::pick(int jobs, int n) const {
  if (forced.H) return forced;
  if (tune.empty() || tuned_n != n) return heuristic(jobs);
  BrShape out = tune.front().shape;
  launch_cost(jobs, &out);
  return out;
}

double ShapePolicy::launch_cost(int jobs, BrShape *s) const {
  double best = 1e300;
  for (const TuneEntry &t : tune) {
    const int waves = (jobs + t.gates_per_wave - 1) / t.gates_per_wave;
    const double cost = waves * t.wave_ms_per_cmux;
    if (cost < best * 0.999) {
      best = cost;
      if (s) *s = t.shape;
    }
  }
  return best;
}

// A persistent launch costs whole rounds of its shape, so a level whose width is
// not a multiple of any shape's round pays a full round for its remainder; here
// the remainder may take a second launch on a shape sized for it (the 912-gate
// rounds of (1, 6) and 8 left over: a sixteen-CTA launch for the 8).
double ShapePolicy::split(int jobs, BrShape *bulk, int *bulk_jobs, BrShape *tail) const {
  BrShape s1 = tune.empty() ? BrShape{1, 1} : tune.front().shape;
  double best = launch_cost(jobs, &s1);
  *bulk = s1;
  *bulk_jobs = jobs;
  *tail = BrShape{0, 0};
  for (const TuneEntry &t : tune) {
    if (is_cluster_shape(t.shape) || t.gates_per_wave <= 0) continue;
    for (long long k = 1; k * t.gates_per_wave < jobs; ++k) {
      BrShape s2 = t.shape;
      const double c = k * t.wave_ms_per_cmux + launch_cost(jobs - (int)(k * t.gates_per_wave), &s2);
      if (c < best * 0.999) {
        best = c;
        *bulk = t.shape;
        *bulk_jobs = (int)(k * t.gates_per_wave);
        *tail = s2;
      }
    }
  }
  return best;
}

int ShapePolicy::free_capacity(int jobs, int n, int l) const {
  if (jobs <= 0) return 0;
  if (forced.H) return jobs;
  if (l == 3 && !tune.empty() && tuned_n == n) {
    // cost of the level as split runs it, then the widest level within that cost:
    // k rounds of a throughput shape and whole rounds of any shape for the rest
    BrShape b, t2;
    int bj = 0;
    const double budget = split(jobs, &b, &bj, &t2) * (1.0 + 1e-9);
    long long cap = jobs;
    for (const TuneEntry &t1 : tune) {
      const bool bulk_ok = !is_cluster_shape(t1.shape) && t1.wave_ms_per_cmux > 0.0;
      for (long long k = 0; k == 0 || (bulk_ok && k * t1.wave_ms_per_cmux <= budget); ++k) {
        const double rest = budget - k * t1.wave_ms_per_cmux;
        long long tail = 0;
        for (const TuneEntry &t : tune)
          if (t.wave_ms_per_cmux > 0.0) tail = std::max(tail, (long long)(rest / t.wave_ms_per_cmux) * t.gates_per_wave);
        cap = std::max(cap, k * t1.gates_per_wave + tail);
      }
    }
    return (int)std::min<long long>(cap, INT_MAX / 2);
  }
  // the heuristic's cluster classes (rounds of co-resident clusters)
  const int c16 = l == 2 ? clusters16l2 : clusters16;
  if (c16 > 0 && jobs <= c16) return c16;
  if (clusters8 > 0 && jobs <= clusters8) return clusters8;
  if (l == 2) return clusters8 > 0 && jobs <= 2 * clusters8 ? 2 * clusters8 : jobs;
  if (clusters4 > 0 && jobs <= clusters4) return clusters4;
  const int c2 = std::max(clusters2, sms / 2);
  if (jobs <= c2) return c2;
  return jobs;
}

// Grid of a launch: CTAs, or clusters for the cluster shapes.
int ShapePolicy::grid(BrShape s, int jobs) {
  if (is_cluster_shape(s)) return std::max(1, std::min(jobs, std::max(1, occupancy(s))));
  const int tiles = (jobs + s.GT - 1) / s.GT;
  const int cap = sms * std::max(1, occupancy(s));
  return std::max(1, std::min(tiles, cap));
}

// Autotuner: time one full wave of every shape once per (device, n) with short
// synthetic blind rotations (timing is data-independent) of two lengths, and
// take the time per CMux as the slope between them (the launch's fixed start-up
// -- ring fill, twiddle loads -- drops out, as it does in a 630-CMux wave); then
// pick the shape minimising waves x time-per-wave for each launch width.
int calibrate(Engine &E, int n) {
  if (E.policy.tuned_n == n) return ARX_OK;
  const int ncal = std::min(n, 40), nshort = std::min(ncal, 8);
  int max_jobs = 0;
  for (BrShape s : kShapes) max_jobs = std::max(max_jobs, is_cluster_shape(s) ? E.policy.occupancy(s) : E.sms * s.GT * std::max(1, E.policy.occupancy(s)));
  DevBuf bsk, wires, jobs, out;
  CK(bsk.reserve((size_t)ncal * 6 * kChunkBytes));
  CK(wires.reserve((size_t)kWireStride * 4 * 2));
  CK(jobs.reserve(sizeof(BrJob) * max_jobs));
  CK(out.reserve((size_t)kOutStride * 4 * max_jobs));
  CK(cudaMemset(bsk.p, 0, (size_t)ncal * 6 * kChunkBytes));
  CK(cudaMemset(wires.p, 0, (size_t)kWireStride * 4 * 2));
  std::vector<BrJob> hj(max_jobs, BrJob{0, 1, ARX_MU, 1, 1});
  CK(cudaMemcpy(jobs.p, hj.data(), sizeof(BrJob) * max_jobs, cudaMemcpyHostToDevice));
  // device-side timing (global timer, first CTA start to last warp end): free of
  // launch overhead and of anything a profiler adds around a launch
  DevBuf stamps;
  CK(stamps.reserve(2 * sizeof(unsigned long long)));
  E.policy.tune.clear();
  for (BrShape s : kShapes) {
    if (!E.policy.occupancy(s)) continue;
    BrArgs args{};
    args.bsk[0] = bsk.as<uint32_t>();
    args.wires = wires.as<uint32_t>();
    args.jobs = jobs.as<BrJob>();
    args.num_jobs = is_cluster_shape(s) ? E.policy.occupancy(s) : E.sms * s.GT * E.policy.occupancy(s);
    args.n = ncal;
    args.out = out.as<uint32_t>();
    args.tg = E.tg;
    args.status = E.status;
    args.tc = E.tc;
    args.stamps = stamps.as<unsigned long long>();
    const int grid = E.policy.grid(s, args.num_jobs);
    double best[2] = {1e30, 1e30};  // shortest time over the repetitions, for nshort and ncal CMux
    for (int len = 0; len < 2; ++len) {
      args.n = len ? ncal : nshort;
      for (int rep = 0; rep < 4; ++rep) {
        CK(cudaMemsetAsync(stamps.p, 0xFF, sizeof(unsigned long long), E.stream));
        CK(cudaMemsetAsync(stamps.as<unsigned long long>() + 1, 0, sizeof(unsigned long long), E.stream));
        CK(launch_br(args, s, grid, E.stream));
        unsigned long long t[2] = {0, 0};
        CK(cudaMemcpyAsync(t, stamps.p, sizeof(t), cudaMemcpyDeviceToHost, E.stream));
        CK(cudaStreamSynchronize(E.stream));
        const double ms = t[1] > t[0] ? (t[1] - t[0]) * 1e-6 : 1e30;
        if (rep) best[len] = std::min(best[len], ms);
      }
    }
    TuneEntry t;
    t.shape = s;
    const double slope = ncal > nshort ? (best[1] - best[0]) / (ncal - nshort) : 0.0;
    t.wave_ms_per_cmux = slope > 0.0 ? slope : best[1] / ncal;
    t.gates_per_wave = args.num_jobs;
    E.policy.tune.push_back(t);
  }
  stamps.release();
  bsk.release();
  wires.release();
  jobs.release();
  out.release();
  int rc = read_status(E, E.stream);
  if (rc) return rc;
  E.policy.tuned_n = n;
  return ARX_OK;
}

// --------------------------------------------------------------------------
// levelization (Sec. 4.2): successor lists, predecessor counts, a FIFO of ready
// gates; wave = 0 without gate inputs, else 1 + max wave of the gate inputs.
// --------------------------------------------------------------------------
int validate_netlist(const arx_netlist *nl) {
  if (!nl) return fail(ARX_EINVAL, "null netlist");
  if (nl->num_gates && (!nl->type || !nl->in0)) return fail(ARX_EINVAL, "netlist arrays missing");
  if (nl->num_outputs && !nl->outputs) return fail(ARX_EINVAL, "netlist outputs missing");
  const uint64_t wires = (uint64_t)nl->num_inputs + nl->num_gates;
  for (uint32_t g = 0; g < nl->num_gates; ++g) {
    const uint32_t t = nl->type[g];
    if (t > ARX_CONST1) return fail(ARX_EINVAL, "gate %u: bad type %u", g, t);
    const int ar = gate_arity(t);
    if (ar >= 2 && !nl->in1) return fail(ARX_EINVAL, "netlist in1 missing");
    if (ar >= 3 && !nl->in2) return fail(ARX_EINVAL, "netlist in2 missing");
    const uint32_t *ins[3] = {nl->in0, nl->in1, nl->in2};
    for (int s = 0; s < ar; ++s)
      if (ins[s][g] >= wires) return fail(ARX_EINVAL, "gate %u input %d: wire %u out of range", g, s, ins[s][g]);
  }
  for (uint32_t o = 0; o < nl->num_outputs; ++o)
    if (nl->outputs[o] >= wires) return fail(ARX_EINVAL, "output %u: wire %u out of range", o, nl->outputs[o]);
  return ARX_OK;
}

int levelize(const arx_netlist *nl, uint32_t *wave, uint32_t *depth) {
  int rc = validate_netlist(nl);
  if (rc) return rc;
  const uint32_t G = nl->num_gates, I = nl->num_inputs;
  const uint32_t *ins[3] = {nl->in0, nl->in1, nl->in2};
  std::vector<uint32_t> npred(G, 0), start(G + 1, 0);
  for (uint32_t g = 0; g < G; ++g)
    for (int s = 0; s < gate_arity(nl->type[g]); ++s)
      if (ins[s][g] >= I) {
        npred[g]++;
        start[ins[s][g] - I + 1]++;
      }
  for (uint32_t g = 0; g < G; ++g) start[g + 1] += start[g];
  std::vector<uint32_t> succ(start[G]), fill(start.begin(), start.end() - 1);
  for (uint32_t g = 0; g < G; ++g)
    for (int s = 0; s < gate_arity(nl->type[g]); ++s)
      if (ins[s][g] >= I) succ[fill[ins[s][g] - I]++] = g;
  std::vector<uint32_t> fifo;
  fifo.reserve(G);
  for (uint32_t g = 0; g < G; ++g)
    if (!npred[g]) fifo.push_back(g);
  uint32_t d = 0;
  for (size_t head = 0; head < fifo.size(); ++head) {
    const uint32_t g = fifo[head];
    uint32_t w = 0;
    for (int s = 0; s < gate_arity(nl->type[g]); ++s)
      if (ins[s][g] >= I) w = std::max(w, wave[ins[s][g] - I] + 1);
    wave[g] = w;
    d = std::max(d, w + 1);
    for (uint32_t e = start[g]; e < start[g + 1]; ++e)
      if (--npred[succ[e]] == 0) fifo.push_back(succ[e]);
  }
  if (fifo.size() != G) return fail(ARX_ECYCLE, "netlist has a cycle (%zu of %u gates ordered)", fifo.size(), G);
  if (depth) *depth = d;
  return ARX_OK;
}

// Launch widths within slack.  latest[g] is the last level at which gate g can
// run without deepening the netlist (depth - 1 for a gate no other gate reads,
// else one before its earliest reader's latest level).  Level by level, the
// launch takes every ready gate whose latest level it is, then -- earliest
// deadline first -- more ready gates while the launch's cost does not grow
// (cap_of on the blind rotations: MUX two, linear gates none).  By
// induction a gate's inputs are placed by the level before its latest one, so
// every gate is placed by its latest level: the depth stays, each gate still
// runs after its inputs, and the results are those of the paper's levelization.
void balance_levels(const arx_netlist *nl, uint32_t depth, const std::function<long long(long long)> &cap_of,
                    uint32_t *wave) {
  const uint32_t G = nl->num_gates, I = nl->num_inputs;
  if (!G || depth < 2) return;
  const uint32_t *ins[3] = {nl->in0, nl->in1, nl->in2};
  std::vector<uint32_t> start(G + 1, 0), npred(G, 0), weight(G);
  for (uint32_t g = 0; g < G; ++g) {
    const uint32_t t = nl->type[g];
    weight[g] = t == ARX_MUX ? 2u : gate_arity(t) == 2 ? 1u : 0u;
    for (int s = 0; s < gate_arity(t); ++s)
      if (ins[s][g] >= I) {
        npred[g]++;
        start[ins[s][g] - I + 1]++;
      }
  }
  for (uint32_t g = 0; g < G; ++g) start[g + 1] += start[g];
  std::vector<uint32_t> succ(start[G]), fill(start.begin(), start.end() - 1);
  for (uint32_t g = 0; g < G; ++g)
    for (int s = 0; s < gate_arity(nl->type[g]); ++s)
      if (ins[s][g] >= I) succ[fill[ins[s][g] - I]++] = g;
  // latest levels, readers first (by decreasing earliest level)
  std::vector<uint32_t> by(G), cnt(depth + 1, 0);
  for (uint32_t g = 0; g < G; ++g) cnt[wave[g] + 1]++;
  for (uint32_t w = 0; w < depth; ++w) cnt[w + 1] += cnt[w];
  for (uint32_t g = 0; g < G; ++g) by[cnt[wave[g]]++] = g;
  std::vector<uint32_t> latest(G, depth - 1);
  for (uint32_t k = G; k-- > 0;) {
    const uint32_t g = by[k];
    for (uint32_t e = start[g]; e < start[g + 1]; ++e) latest[g] = std::min(latest[g], latest[succ[e]] - 1);
  }
  typedef std::pair<uint32_t, uint32_t> Item;  // (latest level, gate)
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> ready;
  for (uint32_t g = 0; g < G; ++g)
    if (!npred[g]) ready.push(Item(latest[g], g));
  std::vector<uint32_t> taken, next;
  for (uint32_t L = 0; L < depth; ++L) {
    taken.clear();
    long long jobs = 0;
    while (!ready.empty() && ready.top().first <= L) {  // due now
      taken.push_back(ready.top().second);
      jobs += weight[ready.top().second];
      ready.pop();
    }
    const long long cap = jobs > 0 ? cap_of(jobs) : 0;
    while (!ready.empty() && jobs + weight[ready.top().second] <= cap) {  // free room, earliest deadline first
      taken.push_back(ready.top().second);
      jobs += weight[ready.top().second];
      ready.pop();
    }
    next.clear();
    for (uint32_t g : taken) {
      wave[g] = L;
      for (uint32_t e = start[g]; e < start[g + 1]; ++e)
        if (--npred[succ[e]] == 0) next.push_back(succ[e]);
    }
    for (uint32_t g : next) ready.push(Item(latest[g], g));
  }
}

// Key-switch scratch: partial sums [jobs][splits][632] and zeroed counters [jobs].
int reserve_ks_scratch(DevBuf &part, DevBuf &cnt, size_t jobs, int splits) {
  if (splits <= 1 || !jobs) return ARX_OK;
  const size_t pbytes = jobs * (size_t)splits * kKsRowStride * 4;
  if (pbytes > part.cap) CK(part.reserve(pbytes));
  if (jobs * 4 > cnt.cap) {
    CK(cnt.reserve(jobs * 4));
    CK(cudaMemset(cnt.p, 0, cnt.cap));
  }
  return ARX_OK;
}

// --------------------------------------------------------------------------
// plans
// --------------------------------------------------------------------------
int plan_build(Engine &E, const arx_netlist *nl, int keyset, int mode, std::unique_ptr<Plan> &out) {
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  std::vector<uint32_t> wave(nl->num_gates ? nl->num_gates : 1);
  uint32_t depth = 0;
  rc = levelize(nl, wave.data(), &depth);
  if (rc) return rc;
  if (mode == ARX_MODE_GRAPH) {  // autotuned shapes, launch widths balanced within slack
    if (ks->l == 3) {
      rc = calibrate(E, ks->n);
      if (rc) return rc;
    }
    const ShapePolicy &pol = E.policy;
    const int n = ks->n, l = ks->l;
    balance_levels(
        nl, depth, [&](long long j) { return (long long)pol.free_capacity((int)std::min<long long>(j, INT_MAX / 2), n, l); },
        wave.data());
  }
  std::unique_ptr<Plan> P(new Plan);
  P->keyset = keyset < 0 ? E.last : keyset;
  P->n = ks->n;
  P->l = ks->l;
  P->mode = mode;
  P->num_inputs = nl->num_inputs;
  P->num_gates = nl->num_gates;
  P->outputs.assign(nl->outputs, nl->outputs + nl->num_outputs);
  // bucket gates by wave, keeping gate order inside a wave
  std::vector<uint32_t> cnt(depth + 1, 0), order(nl->num_gates);
  for (uint32_t g = 0; g < nl->num_gates; ++g) cnt[wave[g] + 1]++;
  for (uint32_t w = 0; w < depth; ++w) cnt[w + 1] += cnt[w];
  std::vector<uint32_t> pos(cnt.begin(), cnt.end() - 1);
  for (uint32_t g = 0; g < nl->num_gates; ++g) order[pos[wave[g]]++] = g;
  std::vector<BrJob> br;
  std::vector<KsJob> ksj;
  int max_br = 0;
  for (uint32_t w = 0; w < depth; ++w) {
    if (cnt[w + 1] == cnt[w]) continue;  // a level the balancing emptied
    Level L{};
    L.br_off = (int)br.size();
    L.ks_off = (int)ksj.size();
    for (uint32_t k = cnt[w]; k < cnt[w + 1]; ++k) {
      const uint32_t g = order[k];
      const uint32_t t = nl->type[g];
      const int ar = gate_arity(t);
      emit_gate(t, ar > 0 ? nl->in0[g] : 0, ar > 1 ? nl->in1[g] : 0, ar > 2 ? nl->in2[g] : 0,
                nl->num_inputs + g, br, ksj, (uint32_t)L.br_off);
    }
    L.br_cnt = (int)br.size() - L.br_off;
    L.ks_cnt = (int)ksj.size() - L.ks_off;
    max_br = std::max(max_br, L.br_cnt);
    P->levels.push_back(L);
  }
  P->bootstraps = br.size();
  size_t ks_part_max = 0, ks_gate_max = 0;
  const bool tuned = mode == ARX_MODE_GRAPH && P->l == 3 && !E.policy.forced.H && !E.policy.tune.empty() &&
                     E.policy.tuned_n == P->n;
  for (Level &L : P->levels) {
    if (tuned && L.br_cnt > 0) {  // autotuned, possibly as a bulk launch and a tail launch
      BrShape tail{0, 0};
      int bulk_jobs = L.br_cnt;
      E.policy.split(L.br_cnt, &L.shape, &bulk_jobs, &tail);
      if (tail.H && bulk_jobs > 0 && bulk_jobs < L.br_cnt) {
        L.br_split = bulk_jobs;
        L.shape2 = tail;
        L.grid2 = E.policy.grid(tail, L.br_cnt - bulk_jobs);
      }
    } else {
      L.shape = E.policy.for_gadget(
          P->l, mode == ARX_MODE_GRAPH ? E.policy.pick(L.br_cnt, P->n) : E.policy.heuristic(L.br_cnt), L.br_cnt);
    }
    L.grid = E.policy.grid(L.shape, std::max(1, L.br_split ? L.br_split : L.br_cnt));
    L.ks_splits = ks_splits(L.ks_cnt, E.sms);
    if (L.ks_splits > 1) {
      ks_part_max = std::max(ks_part_max, (size_t)L.ks_cnt * L.ks_splits);
      ks_gate_max = std::max(ks_gate_max, (size_t)L.ks_cnt);
    }
  }
  if (ks_part_max) {
    CK(P->kspart.reserve(ks_part_max * kKsRowStride * 4));
    CK(P->kscnt.reserve(ks_gate_max * 4));
    CK(cudaMemset(P->kscnt.p, 0, P->kscnt.cap));
  }

  const size_t wires = (size_t)nl->num_inputs + nl->num_gates;
  CK(P->wires.reserve(std::max<size_t>(wires, 1) * kWireStride * 4));
  CK(P->brjobs.reserve(std::max<size_t>(br.size(), 1) * sizeof(BrJob)));
  CK(P->ksjobs.reserve(std::max<size_t>(ksj.size(), 1) * sizeof(KsJob)));
  CK(P->brout.reserve((size_t)std::max(max_br, 1) * kOutStride * 4));
  CK(P->outidx.reserve(std::max<size_t>(P->outputs.size(), 1) * 4));
  if (!br.empty()) CK(cudaMemcpy(P->brjobs.p, br.data(), br.size() * sizeof(BrJob), cudaMemcpyHostToDevice));
  if (!ksj.empty()) CK(cudaMemcpy(P->ksjobs.p, ksj.data(), ksj.size() * sizeof(KsJob), cudaMemcpyHostToDevice));
  if (!P->outputs.empty())
    CK(cudaMemcpy(P->outidx.p, P->outputs.data(), P->outputs.size() * 4, cudaMemcpyHostToDevice));
  out = std::move(P);
  return ARX_OK;
}

// The blind-rotation launches of a level: one, or the bulk and the tail of a
// split (the tail's jobs and outputs follow the bulk's).  *launches counts them.
int launch_level_br(Engine &E, const Plan &P, const Level &L, const Keyset &ks, cudaStream_t st,
                     uint32_t *launches) {
  if (!L.br_cnt) return ARX_OK;
  const int first = L.br_split ? L.br_split : L.br_cnt;
  BrArgs a{};
  a.bsk[0] = ks.bsk;
  a.wires = P.wires.as<uint32_t>();
  a.jobs = P.brjobs.as<BrJob>() + L.br_off;
  a.num_jobs = first;
  a.n = P.n;
  a.out = P.brout.as<uint32_t>();
  a.tg = E.tg;
  a.status = E.status;
  a.tc = E.tc;
  CK(launch_br(a, L.shape, L.grid, st));
  if (launches) ++*launches;
  if (L.br_split) {
    a.jobs += first;
    a.num_jobs = L.br_cnt - first;
    a.out += (size_t)first * kOutStride;
    CK(launch_br(a, L.shape2, L.grid2, st));
    if (launches) ++*launches;
  }
  return ARX_OK;
}

int plan_launch_levels(Engine &E, Plan &P, cudaStream_t st) {
  Keyset &ks = E.keysets[P.keyset];
  for (const Level &L : P.levels) {
    const int rc = launch_level_br(E, P, L, ks, st, nullptr);
    if (rc) return rc;
    KsArgs k{};
    k.ksk[0] = ks.ksk;
    k.br_out = P.brout.as<uint32_t>();
    k.wires = P.wires.as<uint32_t>();
    k.jobs = P.ksjobs.as<KsJob>() + L.ks_off;
    k.n = P.n;
    k.out = P.wires.as<uint32_t>();
    k.out_stride = kWireStride;
    k.splits = L.ks_splits;
    k.partial = P.kspart.as<uint32_t>();
    k.counters = P.kscnt.as<unsigned int>();
    CK(launch_ks(k, L.ks_cnt, st));
  }
  return ARX_OK;
}

int plan_exec(Engine &E, Plan &P, const uint32_t *ct_in, uint32_t *ct_out, cudaStream_t user_st) {
  cudaStream_t st = user_st ? user_st : E.stream;
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, P.keyset, &ks);
  if (rc) return rc;
  const size_t row = (size_t)P.n + 1;
  if (P.num_inputs) {
    if (!ct_in) return fail(ARX_EINVAL, "ct_in is null");
    CK(cudaMemcpy2DAsync(P.wires.p, kWireStride * 4, ct_in, row * 4, row * 4, P.num_inputs, cudaMemcpyDefault, st));
  }
  if (P.mode == ARX_MODE_GRAPH) {
    if (!P.exec) {
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int lrc = plan_launch_levels(E, P, cs);
      cudaError_t ce = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (lrc) return lrc;
      CK(ce);
      ce = cudaGraphInstantiate(&P.exec, g, 0);
      cudaGraphDestroy(g);
      CK(ce);
    }
    CK(cudaGraphLaunch(P.exec, st));
  } else {
    rc = plan_launch_levels(E, P, st);
    if (rc) return rc;
  }
  const int nout = (int)P.outputs.size();
  if (nout) {
    if (!ct_out) return fail(ARX_EINVAL, "ct_out is null");
    if (is_device_ptr(ct_out)) {
      CK(launch_gather(P.wires.as<uint32_t>(), P.outidx.as<uint32_t>(), nout, P.n, ct_out, (int)row, st));
    } else {
      CK(P.outstage.reserve((size_t)nout * row * 4));
      CK(launch_gather(P.wires.as<uint32_t>(), P.outidx.as<uint32_t>(), nout, P.n, P.outstage.as<uint32_t>(),
                       (int)row, st));
      CK(cudaMemcpyAsync(ct_out, P.outstage.p, (size_t)nout * row * 4, cudaMemcpyDeviceToHost, st));
    }
  }
  if (!user_st) return read_status(E, st);
  return ARX_OK;
}

void plan_free(Plan &P) {
  if (P.exec) cudaGraphExecDestroy(P.exec);
  P.exec = nullptr;
  P.wires.release();
  P.brjobs.release();
  P.ksjobs.release();
  P.brout.release();
  P.outidx.release();
  P.outstage.release();
  P.kspart.release();
  P.kscnt.release();
}

// --------------------------------------------------------------------------
// independent gates
// --------------------------------------------------------------------------
int bootstrap_gates(Engine &E, const uint8_t *types, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                    uint32_t *out, size_t count, int keyset, cudaStream_t user_st) {
  if (count == 0) return ARX_OK;
  if (!types || !a || !out) return fail(ARX_EINVAL, "null argument");
  if (count > (1u << 24)) return fail(ARX_EINVAL, "count %zu too large", count);
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  bool need_b = false, need_c = false;
  for (size_t g = 0; g < count; ++g) {
    if (types[g] > ARX_CONST1) return fail(ARX_EINVAL, "gate %zu: bad type %u", g, types[g]);
    need_b |= gate_arity(types[g]) >= 2;
    need_c |= types[g] == ARX_MUX;
  }
  if (need_b && !b) return fail(ARX_EINVAL, "ct_b is null but a gate needs it");
  if (need_c && !c) return fail(ARX_EINVAL, "ct_c is null but a MUX needs it");
  cudaStream_t st = user_st ? user_st : E.stream;
  Workspace &W = E.ws[st];
  const size_t row = (size_t)ks->n + 1;
  const uint32_t cnt = (uint32_t)count;
  std::vector<BrJob> br;
  std::vector<KsJob> ksj;
  br.reserve(count);
  ksj.reserve(count);
  for (uint32_t g = 0; g < cnt; ++g) emit_gate(types[g], g, cnt + g, 2 * cnt + g, g, br, ksj, 0);
  const int nin = need_c ? 3 : (need_b ? 2 : 1);
  CK(W.wires.reserve((size_t)nin * count * kWireStride * 4));
  CK(W.brjobs.reserve(std::max<size_t>(br.size(), 1) * sizeof(BrJob)));
  CK(W.ksjobs.reserve(ksj.size() * sizeof(KsJob)));
  CK(W.brout.reserve(std::max<size_t>(br.size(), 1) * kOutStride * 4));
  const uint32_t *srcs[3] = {a, b, c};
  for (int s = 0; s < nin; ++s)
    CK(cudaMemcpy2DAsync(W.wires.as<uint32_t>() + (size_t)s * count * kWireStride, kWireStride * 4, srcs[s],
                         row * 4, row * 4, count, cudaMemcpyDefault, st));
  if (!br.empty()) CK(cudaMemcpyAsync(W.brjobs.p, br.data(), br.size() * sizeof(BrJob), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(W.ksjobs.p, ksj.data(), ksj.size() * sizeof(KsJob), cudaMemcpyHostToDevice, st));
  if (!br.empty()) {
    BrArgs args{};
    args.bsk[0] = ks->bsk;
    args.wires = W.wires.as<uint32_t>();
    args.jobs = W.brjobs.as<BrJob>();
    args.num_jobs = (int)br.size();
    args.n = ks->n;
    args.out = W.brout.as<uint32_t>();
    args.tg = E.tg;
    args.status = E.status;
    args.tc = E.tc;
    const BrShape s = E.policy.for_gadget(ks->l, E.policy.pick(args.num_jobs, ks->n), args.num_jobs);
    CK(launch_br(args, s, E.policy.grid(s, args.num_jobs), st));
  }
  const bool dev_out = is_device_ptr(out);
  if (!dev_out) CK(W.out.reserve(count * row * 4));
  KsArgs k{};
  k.ksk[0] = ks->ksk;
  k.br_out = W.brout.as<uint32_t>();
  k.wires = W.wires.as<uint32_t>();
  k.jobs = W.ksjobs.as<KsJob>();
  k.n = ks->n;
  k.out = dev_out ? out : W.out.as<uint32_t>();
  k.out_stride = (int)row;
  k.splits = ks_splits((int)count, E.sms);
  rc = reserve_ks_scratch(W.kspart, W.kscnt, count, k.splits);
  if (rc) return rc;
  k.partial = W.kspart.as<uint32_t>();
  k.counters = W.kscnt.as<unsigned int>();
  CK(launch_ks(k, (int)count, st));
  if (!dev_out) CK(cudaMemcpyAsync(out, W.out.p, count * row * 4, cudaMemcpyDeviceToHost, st));
  if (!user_st) return read_status(E, st);
  return ARX_OK;
}

// --------------------------------------------------------------------------
// keys
// --------------------------------------------------------------------------
size_t keyset_bytes(int n, int l) {
  return (size_t)n * 2 * l * kChunkBytes + ((size_t)kN * 8 * 3 * kKsRowStride + kKsZeroWords) * 4;
}

int load_keys(Engine &E, const uint32_t *bsk, const uint32_t *ksk, int n, int l, cudaStream_t user_st) {
  if (!bsk || !ksk) return fail(ARX_EINVAL, "null key pointer");
  if (n < 1 || n > kMaxLweN) return fail(ARX_EINVAL, "lwe_n %d outside 1..%d", n, kMaxLweN);
  if (l != 3 && l != 2) return fail(ARX_EINVAL, "gadget length %d: only 3 (Bg = 2^7) or 2 (Bg = 2^10)", l);
  if (E.budget && E.resident_bytes() + keyset_bytes(n, l) > E.budget)
    return fail(ARX_ENOMEM, "key set would exceed the HBM budget");
  cudaStream_t st = user_st ? user_st : E.stream;
  Keyset K;
  K.n = n;
  K.l = l;
  const int rows = 2 * l;
  const size_t bsk_ntt = (size_t)n * rows * kChunkBytes;
  const size_t ksk_dev = ((size_t)kN * 8 * 3 * kKsRowStride + kKsZeroWords) * 4;  // + the zero row
  const size_t bsk_coef = (size_t)n * rows * 2 * kN * 4;
  cudaError_t e = cudaMalloc(&K.bsk, bsk_ntt);
  if (e == cudaSuccess) e = cudaMalloc(&K.ksk, ksk_dev);
  uint32_t *tmp = nullptr;
  const uint32_t *src = bsk;
  if (e == cudaSuccess && !is_device_ptr(bsk)) {
    e = cudaMalloc(&tmp, bsk_coef);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, bsk, bsk_coef, cudaMemcpyHostToDevice, st);
    src = tmp;
  }
  if (e == cudaSuccess) e = launch_bsk_to_ntt(src, n, rows, K.bsk, E.tc, E.tg, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(K.ksk, 0, ksk_dev, st);
  const size_t row = (size_t)n + 1;
  for (int v = 1; v < 4 && e == cudaSuccess; ++v)
    e = cudaMemcpy2DAsync(K.ksk + (size_t)(v - 1) * kKsRowStride, 3 * kKsRowStride * 4, ksk + (size_t)v * row,
                          4 * row * 4, row * 4, (size_t)kN * 8, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) {
    if (K.bsk) cudaFree(K.bsk);
    if (K.ksk) cudaFree(K.ksk);
    return fail(e == cudaErrorMemoryAllocation ? ARX_ENOMEM : ARX_ECUDA, "loading keys: %s", cudaGetErrorString(e));
  }
  K.used = true;
  int slot = -1;
  for (int i = 0; i < (int)E.keysets.size(); ++i)
    if (!E.keysets[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) {
    slot = (int)E.keysets.size();
    E.keysets.push_back(K);
  } else {
    E.keysets[slot] = K;
  }
  E.last = slot;
  return slot;
}

int unload_keys(Engine &E, int id) {
  if (id < 0 || id >= (int)E.keysets.size() || !E.keysets[id].used) return fail(ARX_ENOKEYS, "no key set %d", id);
  Keyset &K = E.keysets[id];
  if (K.refs) return fail(ARX_EBUSY, "key set %d is referenced by %d plan(s)", id, K.refs);
  cudaDeviceSynchronize();
  cudaFree(K.bsk);
  cudaFree(K.ksk);
  K = Keyset{};
  if (E.last == id) {
    E.last = -1;
    for (int i = (int)E.keysets.size() - 1; i >= 0; --i)
      if (E.keysets[i].used) {
        E.last = i;
        break;
      }
  }
  return ARX_OK;
}

size_t Engine::resident_bytes() const {
  size_t s = 0;
  for (const Keyset &k : keysets)
    if (k.used) s += keyset_bytes(k.n, k.l);
  return s;
}

}  // namespace arx

// ============================================================================
// C-ABI
// ============================================================================
using namespace arx;

#define API_BEGIN                       \
  Engine &E = eng();                    \
  std::lock_guard<std::mutex> lk(E.mu); \
  {                                     \
    int rc_ = ensure_init(E);           \
    if (rc_) return rc_;                \
  }

extern "C" int arx_load_keys(const uint32_t *bsk, const uint32_t *ksk) {
  API_BEGIN
  return load_keys(E, bsk, ksk, ARX_LWE_N, 3, nullptr);
}

extern "C" int arx_load_keys_ex(const uint32_t *bsk, const uint32_t *ksk, int lwe_n, void *stream) {
  API_BEGIN
  return load_keys(E, bsk, ksk, lwe_n, 3, (cudaStream_t)stream);
}

extern "C" int arx_load_keys_gadget(const uint32_t *bsk, const uint32_t *ksk, int lwe_n, int l, int bg_bits,
                                    void *stream) {
  API_BEGIN
  if (!((l == 3 && bg_bits == 7) || (l == 2 && bg_bits == 10)))
    return fail(ARX_EINVAL, "gadget (l %d, Bg 2^%d): only (3, 2^7) and (2, 2^10)", l, bg_bits);
  return load_keys(E, bsk, ksk, lwe_n, l, (cudaStream_t)stream);
}

extern "C" int arx_keyset_dims(int keyset, int *lwe_n, int *l) {
  API_BEGIN
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  if (lwe_n) *lwe_n = ks->n;
  if (l) *l = ks->l;
  return ARX_OK;
}

extern "C" int arx_unload_keys(int keyset) {
  API_BEGIN
  return unload_keys(E, keyset);
}

extern "C" int arx_use_keys(int keyset) {
  API_BEGIN
  Keyset *ks = nullptr;
  if (keyset < 0) return fail(ARX_ENOKEYS, "no key set %d", keyset);
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  E.last = keyset;
  return ARX_OK;
}

extern "C" size_t arx_resident_bytes(void) {
  Engine &E = eng();
  std::lock_guard<std::mutex> lk(E.mu);
  return E.resident_bytes();
}

extern "C" size_t arx_keyset_bytes(int lwe_n) { return lwe_n < 1 || lwe_n > kMaxLweN ? 0 : keyset_bytes(lwe_n); }

extern "C" int arx_bootstrap_gates(const uint8_t *types, const uint32_t *ct_a, const uint32_t *ct_b,
                                   uint32_t *ct_out, size_t count) {
  API_BEGIN
  for (size_t g = 0; g < count && types; ++g)
    if (types[g] == ARX_MUX) return fail(ARX_EINVAL, "MUX needs arx_bootstrap_gates_ex (third input)");
  return bootstrap_gates(E, types, ct_a, ct_b, nullptr, ct_out, count, -1, nullptr);
}

extern "C" int arx_bootstrap_gates_ex(const uint8_t *types, const uint32_t *ct_a, const uint32_t *ct_b,
                                      const uint32_t *ct_c, uint32_t *ct_out, size_t count, int keyset,
                                      void *stream) {
  API_BEGIN
  return bootstrap_gates(E, types, ct_a, ct_b, ct_c, ct_out, count, keyset, (cudaStream_t)stream);
}

extern "C" int arx_levelize(const arx_netlist *nl, uint32_t *wave, uint32_t *depth) {
  if (!wave && nl && nl->num_gates) return fail(ARX_EINVAL, "wave is null");
  uint32_t dummy = 0;
  return levelize(nl, wave ? wave : &dummy, depth);
}

extern "C" int arx_levelize_balanced(const arx_netlist *nl, const uint32_t *caps, uint32_t ncaps, uint32_t *wave,
                                     uint32_t *depth) {
  if (!wave && nl && nl->num_gates) return fail(ARX_EINVAL, "wave is null");
  if (ncaps && !caps) return fail(ARX_EINVAL, "caps is null");
  for (uint32_t k = 1; k < ncaps; ++k)
    if (caps[k] <= caps[k - 1]) return fail(ARX_EINVAL, "caps must increase");
  uint32_t dummy = 0, d = 0;
  int rc = levelize(nl, wave ? wave : &dummy, &d);
  if (rc) return rc;
  if (depth) *depth = d;
  if (!nl->num_gates) return ARX_OK;
  balance_levels(
      nl, d,
      [&](long long j) {
        for (uint32_t k = 0; k < ncaps; ++k)
          if (j <= (long long)caps[k]) return (long long)caps[k];
        return j;
      },
      wave);
  return ARX_OK;
}

extern "C" int arx_split_wave(const double *ms, const uint32_t *gates, const uint8_t *cluster, uint32_t shapes,
                               uint32_t jobs, uint32_t *bulk, uint32_t *bulk_jobs, int32_t *tail, double *cost,
                               uint32_t *cap) {
  if (!ms || !gates || !cluster || shapes < 1 || shapes > 64 || jobs < 1 || jobs > (1u << 30))
    return fail(ARX_EINVAL, "bad split arguments");
  ShapePolicy pol;  // a table of synthetic shapes; shape s is (H, s + 1), H marking cluster shapes
  pol.tuned_n = 1;
  for (uint32_t s = 0; s < shapes; ++s) {
    if (!(ms[s] > 0.0) || !gates[s]) return fail(ARX_EINVAL, "shape %u: ms and gates must be positive", s);
    TuneEntry t;
    t.shape = BrShape{cluster[s] ? kCluster16H : 1, (int)s + 1};
    t.wave_ms_per_cmux = ms[s];
    t.gates_per_wave = (int)gates[s];
    pol.tune.push_back(t);
  }
  BrShape b{1, 1}, t2{0, 0};
  int bj = 0;
  const double c = pol.split((int)jobs, &b, &bj, &t2);
  if (bulk) *bulk = (uint32_t)(b.GT - 1);
  if (bulk_jobs) *bulk_jobs = (uint32_t)bj;
  if (tail) *tail = t2.H ? t2.GT - 1 : -1;
  if (cost) *cost = c;
  if (cap) *cap = (uint32_t)pol.free_capacity((int)jobs, 1, 3);
  return ARX_OK;
}

extern "C" int arx_eval_netlist_ex(const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out, int keyset,
                                   int mode, void *stream) {
  API_BEGIN
  if (mode != ARX_MODE_PLAIN && mode != ARX_MODE_GRAPH) return fail(ARX_EINVAL, "bad mode %d", mode);
  std::unique_ptr<Plan> P;
  int rc = plan_build(E, nl, keyset, mode, P);
  if (rc) return rc;
  rc = plan_exec(E, *P, ct_in, ct_out, (cudaStream_t)stream);
  if (stream) cudaStreamSynchronize((cudaStream_t)stream);  // the plan's buffers are freed below
  plan_free(*P);
  return rc;
}

extern "C" int arx_eval_netlist(const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out) {
  return arx_eval_netlist_ex(nl, ct_in, ct_out, -1, ARX_MODE_PLAIN, nullptr);
}

extern "C" int arx_plan_create(const arx_netlist *nl, int keyset, int mode) {
  API_BEGIN
  if (mode != ARX_MODE_PLAIN && mode != ARX_MODE_GRAPH) return fail(ARX_EINVAL, "bad mode %d", mode);
  std::unique_ptr<Plan> P;
  int rc = plan_build(E, nl, keyset, mode, P);
  if (rc) return rc;
  E.keysets[P->keyset].refs++;
  for (int i = 0; i < (int)E.plans.size(); ++i)
    if (!E.plans[i]) {
      E.plans[i] = std::move(P);
      return i;
    }
  E.plans.push_back(std::move(P));
  return (int)E.plans.size() - 1;
}

extern "C" int arx_plan_run(int plan, const uint32_t *ct_in, uint32_t *ct_out, void *stream) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  return plan_exec(E, *E.plans[plan], ct_in, ct_out, (cudaStream_t)stream);
}

extern "C" int arx_plan_destroy(int plan) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  cudaDeviceSynchronize();
  E.keysets[E.plans[plan]->keyset].refs--;
  plan_free(*E.plans[plan]);
  E.plans[plan].reset();
  return ARX_OK;
}

extern "C" int arx_plan_info(int plan, uint32_t *waves, uint64_t *bootstraps, uint64_t *gates) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  const Plan &P = *E.plans[plan];
  if (waves) *waves = (uint32_t)P.levels.size();
  if (bootstraps) *bootstraps = P.bootstraps;
  if (gates) *gates = P.num_gates;
  return ARX_OK;
}

extern "C" int arx_plan_shapes(int plan, uint32_t *H, uint32_t *GT, uint32_t *jobs, uint32_t cap) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  const Plan &P = *E.plans[plan];
  for (size_t w = 0; w < P.levels.size() && w < cap; ++w) {
    const Level &L = P.levels[w];
    if (H) H[w] = (uint32_t)L.shape.H;
    if (GT) GT[w] = (uint32_t)L.shape.GT;
    if (jobs) jobs[w] = (uint32_t)L.br_cnt;
  }
  return (int)P.levels.size();
}

extern "C" int arx_plan_launches(int plan, uint32_t *wave, uint32_t *H, uint32_t *GT, uint32_t *jobs, uint32_t cap) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  const Plan &P = *E.plans[plan];
  uint32_t k = 0;
  for (size_t w = 0; w < P.levels.size(); ++w) {
    const Level &L = P.levels[w];
    if (!L.br_cnt) continue;
    for (int part = 0; part < (L.br_split ? 2 : 1); ++part, ++k) {
      if (k >= cap) continue;
      const BrShape s = part ? L.shape2 : L.shape;
      if (wave) wave[k] = (uint32_t)w;
      if (H) H[k] = (uint32_t)s.H;
      if (GT) GT[k] = (uint32_t)s.GT;
      if (jobs) jobs[k] = (uint32_t)(L.br_split ? (part ? L.br_cnt - L.br_split : L.br_split) : L.br_cnt);
    }
  }
  return (int)k;
}

extern "C" int arx_plan_wires(int plan, const uint32_t *ids, size_t count, uint32_t *out) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  Plan &P = *E.plans[plan];
  if (!count) return ARX_OK;
  if (!ids || !out) return fail(ARX_EINVAL, "null argument");
  const uint64_t wires = (uint64_t)P.num_inputs + P.num_gates;
  for (size_t k = 0; k < count; ++k)
    if (ids[k] >= wires) return fail(ARX_EINVAL, "wire %u out of range", ids[k]);
  const size_t row = (size_t)P.n + 1;
  DevBuf idx, stage;
  CK(idx.reserve(count * 4));
  CK(cudaMemcpyAsync(idx.p, ids, count * 4, cudaMemcpyHostToDevice, E.stream));
  const bool dev = is_device_ptr(out);
  if (!dev) CK(stage.reserve(count * row * 4));
  CK(launch_gather(P.wires.as<uint32_t>(), idx.as<uint32_t>(), (int)count, P.n, dev ? out : stage.as<uint32_t>(),
                   (int)row, E.stream));
  if (!dev) CK(cudaMemcpyAsync(out, stage.p, count * row * 4, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaStreamSynchronize(E.stream));
  idx.release();
  stage.release();
  return ARX_OK;
}

extern "C" int arx_plan_profile(int plan, const uint32_t *ct_in, float *br_ms, float *ks_ms,
                                uint32_t *br_launches, uint32_t *ks_launches) {
  API_BEGIN
  if (plan < 0 || plan >= (int)E.plans.size() || !E.plans[plan]) return fail(ARX_EINVAL, "no plan %d", plan);
  Plan &P = *E.plans[plan];
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, P.keyset, &ks);
  if (rc) return rc;
  cudaStream_t st = E.stream;
  const size_t row = (size_t)P.n + 1;
  if (P.num_inputs) {
    if (!ct_in) return fail(ARX_EINVAL, "ct_in is null");
    CK(cudaMemcpy2DAsync(P.wires.p, kWireStride * 4, ct_in, row * 4, row * 4, P.num_inputs, cudaMemcpyDefault, st));
  }
  std::vector<cudaEvent_t> ev(4 * P.levels.size() + 1);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  uint32_t nb = 0, nk = 0;
  for (size_t l = 0; l < P.levels.size(); ++l) {
    const Level &L = P.levels[l];
    CK(cudaEventRecord(ev[4 * l], st));
    rc = launch_level_br(E, P, L, *ks, st, &nb);
    if (rc) return rc;
    CK(cudaEventRecord(ev[4 * l + 1], st));
    CK(cudaEventRecord(ev[4 * l + 2], st));
    KsArgs k{};
    k.ksk[0] = ks->ksk;
    k.br_out = P.brout.as<uint32_t>();
    k.wires = P.wires.as<uint32_t>();
    k.jobs = P.ksjobs.as<KsJob>() + L.ks_off;
    k.n = P.n;
    k.out = P.wires.as<uint32_t>();
    k.out_stride = kWireStride;
    k.splits = L.ks_splits;
    k.partial = P.kspart.as<uint32_t>();
    k.counters = P.kscnt.as<unsigned int>();
    CK(launch_ks(k, L.ks_cnt, st));
    if (L.ks_cnt) ++nk;
    CK(cudaEventRecord(ev[4 * l + 3], st));
  }
  CK(cudaStreamSynchronize(st));
  float tb = 0, tk = 0;
  for (size_t l = 0; l < P.levels.size(); ++l) {
    float x = 0, y = 0;
    CK(cudaEventElapsedTime(&x, ev[4 * l], ev[4 * l + 1]));
    CK(cudaEventElapsedTime(&y, ev[4 * l + 2], ev[4 * l + 3]));
    tb += x;
    tk += y;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (br_ms) *br_ms = tb;
  if (ks_ms) *ks_ms = tk;
  if (br_launches) *br_launches = nb;
  if (ks_launches) *ks_launches = nk;
  return read_status(E, st);
}

extern "C" int arx_set_launch_shape(int H, int GT) {
  Engine &E = eng();
  std::lock_guard<std::mutex> lk(E.mu);
  if (H == 0 && GT == 0) {
    E.policy.forced = BrShape{0, 0};
    return ARX_OK;
  }
  if (is_l2_shape(BrShape{H, GT}) || !br_shape_supported(BrShape{H, GT}))
    return fail(ARX_EINVAL, "unsupported launch shape (%d, %d)", H, GT);
  E.policy.forced = BrShape{H, GT};
  return ARX_OK;
}

extern "C" const char *arx_last_error(void) { return t_err.c_str(); }

extern "C" int arx_device_status(void) {
  API_BEGIN
  return read_status(E, E.stream);
}

extern "C" int arx_device_sms(void) { return eng().sms; }
