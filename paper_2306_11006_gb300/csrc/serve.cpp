// serve.cpp -- continuous-batching server for encrypted-circuit requests.
//
// Requests (a netlist, its encrypted inputs and a client key set) are queued by
// arx_serve_submit.  A scheduler thread admits them in arrival order while the
// device memory they need (their wires, in one wire arena) fits the HBM budget
// next to the resident keys, and then runs ticks: every tick takes the next wave
// of every admitted request and merges the waves of all requests whose key sets
// share a parameter set (LWE dimension and gadget) into one blind-rotation
// launch and one key-switch launch, whatever the key set: each job names its key
// set by an index into the launch's table of key pointers, so the gates of
// different clients run side by side on the device; in the throughput kernel a
// tile of gates (which shares every key row it streams, Sec. 5.1) is drawn from
// one key set.  A request that arrives while others run joins at the next tick;
// a finished one leaves and frees its wires for the next admission.
//
// Ticks are pipelined: the descriptors and newly admitted inputs of a tick go
// through one of two pinned staging buffers, and an event marks the tick's end;
// the host builds tick k+1 while the device runs tick k (stream order keeps
// each request's waves in order) and retires a tick -- copies out the outputs of
// the requests it finished, checks the device status word -- once its event has
// completed.  Each request's ciphertexts are computed by the same kernels the
// single-request path uses, on descriptors that differ only in wire offsets and
// key index, so its result does not depend on what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/arx.h"
#include "arx_kernels.h"
#include "engine_internal.h"

namespace arx {
namespace {

using Clock = std::chrono::steady_clock;

struct Wave {
  std::vector<BrJob> br;  // wire ids local to the request, j0/j1 local to the wave
  std::vector<KsJob> ks;
};

struct Request {
  int id = 0;
  int keyset = -1;
  int n = 0;
  int l = 3;  // gadget length of the key set
  const uint32_t *bsk = nullptr, *ksk = nullptr;  // captured at admission (key set pinned)
  uint32_t num_inputs = 0, num_gates = 0;
  std::vector<uint32_t> outputs;
  std::vector<Wave> waves;
  std::vector<uint32_t> ct_in;  // host copy of the inputs
  uint32_t *ct_out = nullptr;   // caller's host buffer
  size_t wire_base = 0;         // first wire slot in the arena
  size_t wire_count = 0;
  size_t next_wave = 0;
  int status = 0;               // 0 pending, 1 done, < 0 error
  uint64_t bootstraps = 0;
  Clock::time_point t_submit, t_admit, t_done;
};

// First-fit allocator of wire slots in the arena.
struct Arena {
  size_t slots = 0;
  std::map<size_t, size_t> free_;  // start -> length
  void reset(size_t s) {
    slots = s;
    free_.clear();
    if (s) free_[0] = s;
  }
  bool alloc(size_t len, size_t *start) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        *start = it->first;
        const size_t rest = it->second - len, at = it->first + len;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t start, size_t len) {
    auto it = free_.emplace(start, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// One tick in flight: its pinned staging, the requests it finishes, its events.
struct Tick {
  uint8_t *pinned = nullptr;  // [descriptors][admitted inputs][finished outputs]
  size_t cap = 0;
  cudaEvent_t begin = nullptr, end = nullptr;
  bool inflight = false;
  std::vector<std::shared_ptr<Request>> finishing;  // with their offsets in `pinned`
  std::vector<size_t> out_off;
  std::vector<std::shared_ptr<Request>> ran;  // requests advanced (failed together on a watchdog expiry)
  unsigned int *status_host = nullptr;        // pinned copy of the device status word
  uint64_t bootstraps = 0, gates = 0;
};

struct Server {
  std::mutex qmu;  // guards the queues, the request table and the statistics
  std::condition_variable cv;
  bool running = false, stop = false;
  std::thread th;
  size_t budget = 0;         // bytes for keys + wires + per-tick buffers
  uint32_t max_tick_bootstraps = 0;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int, std::shared_ptr<Request>> table;
  int next_id = 0;
  Arena arena;
  DevBuf wires, desc, brout, kspart, kscnt, outidx, outstage;
  Tick tick[2];
  int cur = 0;
  std::vector<double> latencies_ms;
  uint64_t done = 0, failed = 0, gates = 0, bootstraps = 0, launches = 0, ticks = 0;
  uint64_t shared_launches = 0, max_keys = 0;  // blind-rotation launches mixing key sets; most in one
  size_t peak_bytes = 0, peak_active = 0;
  double busy_s = 0;
  Clock::time_point t_start;
  cudaStream_t stream = nullptr;
  // engine state captured at start, so that ticks run without the engine lock
  ShapePolicy policy;
  TwiddleConst tc{};
  const TwiddleGlobal *tg = nullptr;
  unsigned int *status = nullptr;
  int sms = 0;
};

Server &srv() {
  static Server *s = new Server;
  return *s;
}

size_t wire_bytes(size_t slots) { return slots * kWireStride * 4; }

// Per-request device bytes: its wires.
size_t request_bytes(const Request &r) { return wire_bytes(r.wire_count); }

int build_request(Engine &E, const arx_netlist *nl, int keyset, std::shared_ptr<Request> &out) {
  Keyset *ks = nullptr;
  int rc = resolve_keyset(E, keyset, &ks);
  if (rc) return rc;
  std::vector<uint32_t> wave(nl->num_gates ? nl->num_gates : 1);
  uint32_t depth = 0;
  rc = levelize(nl, wave.data(), &depth);
  if (rc) return rc;
  auto R = std::make_shared<Request>();
  R->keyset = keyset < 0 ? E.last : keyset;
  R->n = ks->n;
  R->l = ks->l;
  R->num_inputs = nl->num_inputs;
  R->num_gates = nl->num_gates;
  R->outputs.assign(nl->outputs, nl->outputs + nl->num_outputs);
  R->wire_count = std::max<size_t>((size_t)nl->num_inputs + nl->num_gates, 1);
  R->waves.resize(depth);
  std::vector<std::vector<uint32_t>> by_wave(depth);
  for (uint32_t g = 0; g < nl->num_gates; ++g) by_wave[wave[g]].push_back(g);
  for (uint32_t w = 0; w < depth; ++w) {
    Wave &W = R->waves[w];
    for (uint32_t g : by_wave[w]) {
      const uint32_t t = nl->type[g];
      const int ar = gate_arity(t);
      emit_gate(t, ar > 0 ? nl->in0[g] : 0, ar > 1 ? nl->in1[g] : 0, ar > 2 ? nl->in2[g] : 0, nl->num_inputs + g,
                W.br, W.ks, 0);
    }
    R->bootstraps += W.br.size();
  }
  out = R;
  return ARX_OK;
}

#define SCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(ARX_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)


// Pinned staging of a tick, grown (after its last use has completed) as needed.
int reserve_pinned(Tick &T, size_t bytes) {
  if (bytes <= T.cap) return ARX_OK;
  if (T.pinned) SCK(cudaFreeHost(T.pinned));
  T.pinned = nullptr;
  T.cap = 0;
  const size_t want = std::max<size_t>(bytes + bytes / 2, 1 << 20);
  SCK(cudaMallocHost(reinterpret_cast<void **>(&T.pinned), want));
  T.cap = want;
  return ARX_OK;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The blind-rotation and key-switch jobs of one launch, over the requests of one
// parameter set, with each request's key set as an index into `keys`.
struct LaunchBuild {
  int n = 0, l = 3;
  std::vector<const uint32_t *> bsk, ksk;  // key table of the launch
  std::vector<BrJob> br;
  std::vector<KsJob> ks;
  std::vector<Request *> ran;
  BrShape shape{1, 1};
  int grid = 1;
};

// Merges the next waves of `reqs` (one parameter set, at most kMaxLaunchKeys key
// sets, at most `budget` blind rotations unless a single request needs more):
// jobs grouped by key set and, for a throughput shape with GT gates per tile,
// each group padded to a multiple of GT with copies of its first job (their
// outputs are never read), so that no tile mixes key sets.
void build_launch(Server &S, std::vector<Request *> &reqs, uint32_t budget, LaunchBuild &B) {
  std::map<int, int> kidx;
  std::vector<std::vector<Request *>> by_key;
  std::vector<Request *> rest;
  size_t jobs = 0;
  for (Request *r : reqs) {
    const Wave &W = r->waves[r->next_wave];
    if (!B.ran.empty() && jobs + W.br.size() > budget) {
      rest.push_back(r);
      continue;
    }
    auto it = kidx.find(r->keyset);
    if (it == kidx.end()) {
      if ((int)kidx.size() == kMaxLaunchKeys) {
        rest.push_back(r);
        continue;
      }
      it = kidx.emplace(r->keyset, (int)kidx.size()).first;
      B.bsk.push_back(r->bsk);
      B.ksk.push_back(r->ksk);
      by_key.emplace_back();
    }
    by_key[it->second].push_back(r);
    B.ran.push_back(r);
    jobs += W.br.size();
  }
  reqs.swap(rest);
  const Request &head = *B.ran.front();
  B.n = head.n;
  B.l = head.l;
  B.shape = S.policy.for_gadget(B.l, S.policy.pick((int)std::max<size_t>(jobs, 1), B.n), (int)jobs);
  const int gt = is_cluster_shape(B.shape) ? 1 : std::max(1, B.shape.GT);
  for (size_t k = 0; k < by_key.size(); ++k) {
    const size_t first = B.br.size();
    for (Request *r : by_key[k]) {
      const Wave &W = r->waves[r->next_wave];
      const uint32_t base = (uint32_t)r->wire_base, jb = (uint32_t)B.br.size();
      for (BrJob j : W.br) {
        j.ia += base;
        j.ib += base;
        j.key = (uint16_t)k;
        B.br.push_back(j);
      }
      for (KsJob q : W.ks) {
        q.j0 += jb;
        q.j1 += jb;
        q.ia += base;
        q.out += base;
        q.key = (uint32_t)k;
        B.ks.push_back(q);
      }
    }
    while (gt > 1 && B.br.size() > first && (B.br.size() - first) % gt) {
      const BrJob pad = B.br[first];
      B.br.push_back(pad);
    }
  }
  if (!B.br.empty()) B.grid = S.policy.grid(B.shape, (int)B.br.size());
}

// Retires tick T once its event has completed: outputs of the requests it
// finished go to the callers' buffers, the status word is checked, statistics
// and the wire arena are updated.  wait = block on the event.  Returns 1 when
// the tick was retired, 0 when it is still running.
int retire_tick(Server &S, Engine &E, Tick &T, bool wait) {
  if (!T.inflight) return 1;
  if (wait) {
    if (cudaEventSynchronize(T.end) != cudaSuccess) return fail(ARX_ECUDA, "tick event");
  } else {
    const cudaError_t q = cudaEventQuery(T.end);
    if (q == cudaErrorNotReady) return 0;
    if (q != cudaSuccess) return fail(ARX_ECUDA, "tick event: %s", cudaGetErrorString(q));
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, T.begin, T.end);
  const unsigned int st = *T.status_host;
  const auto now = Clock::now();
  for (size_t k = 0; k < T.finishing.size(); ++k) {
    Request &R = *T.finishing[k];
    const size_t bytes = R.outputs.size() * ((size_t)R.n + 1) * 4;
    if (bytes) std::memcpy(R.ct_out, T.pinned + T.out_off[k], bytes);
  }
  std::vector<std::shared_ptr<Request>> leaving = T.finishing;
  if (st) {  // a watchdog expiry inside this tick: its requests fail
    for (auto &r : T.ran)
      if (std::find(leaving.begin(), leaving.end(), r) == leaving.end()) leaving.push_back(r);
  }
  {
    std::lock_guard<std::mutex> elk(E.mu);
    std::lock_guard<std::mutex> lk(S.qmu);
    S.busy_s += ms * 1e-3;
    S.ticks++;
    S.bootstraps += T.bootstraps;
    S.gates += T.gates;
    for (auto &r : leaving) {
      if (r->status != 0) continue;
      if (!st) {
        r->t_done = now;
        r->status = 1;
        S.done++;
        S.latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      } else {
        r->status = ARX_ETIMEOUT;
        S.failed++;
      }
      S.arena.release(r->wire_base, r->wire_count);
      if (r->keyset >= 0 && r->keyset < (int)E.keysets.size()) E.keysets[r->keyset].refs--;
      S.active.erase(std::remove(S.active.begin(), S.active.end(), r), S.active.end());
    }
  }
  T.finishing.clear();
  T.out_off.clear();
  T.ran.clear();
  T.inflight = false;
  if (st) {
    cudaMemsetAsync(S.status, 0, sizeof(unsigned int), S.stream);
    cudaStreamSynchronize(S.stream);
    fail(ARX_ETIMEOUT, "device watchdog expired (status 0x%x)", st);
  }
  S.cv.notify_all();
  return 1;
}

// Enqueues one tick: the inputs of the newly admitted requests, then per
// parameter set one merged blind-rotation launch and one key-switch launch
// (more when a launch would mix more than kMaxLaunchKeys key sets or exceed the
// per-launch budget), then the outputs of the requests it finishes, the status
// word and the end event.  Nothing here waits for the device except the reuse
// of a staging buffer two ticks old.  Returns 1 when a tick was enqueued, 0
// when there was nothing to run, or an error.
int enqueue_tick(Server &S, Engine &E, const std::vector<std::shared_ptr<Request>> &admitted,
                 const std::vector<std::shared_ptr<Request>> &act) {
  Tick &T = S.tick[S.cur];
  int rc = retire_tick(S, E, T, true);  // the buffer's previous tick (two ago) must be done
  if (rc < 0) return rc;
  // group the advancing requests by parameter set
  std::map<std::pair<int, int>, std::vector<Request *>> cls;
  for (auto &r : act)
    if (r->status == 0 && r->next_wave < r->waves.size()) cls[{r->n, r->l}].push_back(r.get());
  std::vector<LaunchBuild> L;
  const uint32_t budget = S.max_tick_bootstraps ? S.max_tick_bootstraps : 0xffffffffu;
  for (auto &kv : cls) {
    std::vector<Request *> reqs = kv.second;
    while (!reqs.empty()) {
      L.emplace_back();
      build_launch(S, reqs, budget, L.back());
    }
  }
  // pinned layout: per launch [BrJob...][KsJob...] (256-byte aligned), then the admitted inputs, then outputs
  size_t off = 0, max_br = 1;
  std::vector<size_t> br_off(L.size()), ks_off(L.size());
  for (size_t k = 0; k < L.size(); ++k) {
    br_off[k] = off;
    off = align_up(off + L[k].br.size() * sizeof(BrJob), 256);
    ks_off[k] = off;
    off = align_up(off + L[k].ks.size() * sizeof(KsJob), 256);
    max_br = std::max(max_br, L[k].br.size());
  }
  const size_t desc_bytes = off;
  std::vector<size_t> in_off(admitted.size());
  for (size_t k = 0; k < admitted.size(); ++k) {
    in_off[k] = off;
    off = align_up(off + admitted[k]->ct_in.size() * 4, 256);
  }
  // the requests this tick finishes: their last wave is in one of its launches
  // (or they have no gates at all)
  std::vector<std::shared_ptr<Request>> fin;
  std::vector<size_t> out_off;
  for (auto &r : act) {
    bool in_tick = false;
    for (auto &B : L)
      if (std::find(B.ran.begin(), B.ran.end(), r.get()) != B.ran.end()) in_tick = true;
    if ((in_tick && r->next_wave + 1 == r->waves.size()) || (r->waves.empty() && r->status == 0)) fin.push_back(r);
  }
  if (L.empty() && admitted.empty() && fin.empty()) return 0;  // nothing to run (requests wait for the device)
  size_t out_rows = 0;
  for (auto &r : fin) {
    out_off.push_back(off);
    off = align_up(off + r->outputs.size() * ((size_t)r->n + 1) * 4, 256);
    out_rows += r->outputs.size();
  }
  const size_t idx_off = off;
  off = align_up(off + out_rows * 4, 256);
  off = align_up(off, 64);
  const size_t status_off = off;
  off += 64;
  rc = reserve_pinned(T, off);
  if (rc) return rc;
  T.status_host = reinterpret_cast<unsigned int *>(T.pinned + status_off);
  *T.status_host = 0;
  for (size_t k = 0; k < L.size(); ++k) {
    if (!L[k].br.empty()) std::memcpy(T.pinned + br_off[k], L[k].br.data(), L[k].br.size() * sizeof(BrJob));
    if (!L[k].ks.empty()) std::memcpy(T.pinned + ks_off[k], L[k].ks.data(), L[k].ks.size() * sizeof(KsJob));
  }
  for (size_t k = 0; k < admitted.size(); ++k)
    if (!admitted[k]->ct_in.empty())
      std::memcpy(T.pinned + in_off[k], admitted[k]->ct_in.data(), admitted[k]->ct_in.size() * 4);
  // device buffers (stream order keeps the previous tick's readers ahead of these writes)
  SCK(S.desc.reserve(std::max<size_t>(desc_bytes, 256)));
  SCK(S.brout.reserve(max_br * kOutStride * 4));
  SCK(cudaEventRecord(T.begin, S.stream));
  for (size_t k = 0; k < admitted.size(); ++k) {
    const Request &r = *admitted[k];
    const size_t row = (size_t)r.n + 1;
    if (r.num_inputs)
      SCK(cudaMemcpy2DAsync(S.wires.as<uint32_t>() + r.wire_base * kWireStride, kWireStride * 4,
                            T.pinned + in_off[k], row * 4, row * 4, r.num_inputs, cudaMemcpyHostToDevice,
                            S.stream));
  }
  if (desc_bytes) SCK(cudaMemcpyAsync(S.desc.p, T.pinned, desc_bytes, cudaMemcpyHostToDevice, S.stream));
  T.bootstraps = T.gates = 0;
  for (size_t k = 0; k < L.size(); ++k) {
    LaunchBuild &B = L[k];
    if (!B.br.empty()) {
      BrArgs a{};
      for (size_t q = 0; q < B.bsk.size(); ++q) a.bsk[q] = B.bsk[q];
      a.wires = S.wires.as<uint32_t>();
      a.jobs = reinterpret_cast<const BrJob *>(S.desc.as<uint8_t>() + br_off[k]);
      a.num_jobs = (int)B.br.size();
      a.n = B.n;
      a.out = S.brout.as<uint32_t>();
      a.tg = S.tg;
      a.status = S.status;
      a.tc = S.tc;
      SCK(launch_br(a, B.shape, B.grid, S.stream));
      S.launches++;
      if (B.bsk.size() > 1) S.shared_launches++;
      S.max_keys = std::max<uint64_t>(S.max_keys, B.bsk.size());
    }
    if (!B.ks.empty()) {
      KsArgs q{};
      for (size_t j = 0; j < B.ksk.size(); ++j) q.ksk[j] = B.ksk[j];
      q.br_out = S.brout.as<uint32_t>();
      q.wires = S.wires.as<uint32_t>();
      q.jobs = reinterpret_cast<const KsJob *>(S.desc.as<uint8_t>() + ks_off[k]);
      q.n = B.n;
      q.out = S.wires.as<uint32_t>();
      q.out_stride = kWireStride;
      q.splits = ks_splits((int)B.ks.size(), S.sms);
      rc = reserve_ks_scratch(S.kspart, S.kscnt, B.ks.size(), q.splits);
      if (rc) return rc;
      q.partial = S.kspart.as<uint32_t>();
      q.counters = S.kscnt.as<unsigned int>();
      SCK(launch_ks(q, (int)B.ks.size(), S.stream));
      S.launches++;
    }
    for (Request *r : B.ran) {
      const Wave &W = r->waves[r->next_wave];
      T.bootstraps += W.br.size();
      T.gates += W.ks.size();
      r->next_wave++;
    }
  }
  // outputs of the finishing requests: gather on the device, one copy to pinned memory
  if (out_rows) {
    uint32_t *idx = reinterpret_cast<uint32_t *>(T.pinned + idx_off);
    size_t q = 0;
    for (auto &r : fin)
      for (uint32_t o : r->outputs) idx[q++] = o + (uint32_t)r->wire_base;
    SCK(S.outidx.reserve(out_rows * 4));
    SCK(S.outstage.reserve(out_rows * kWireStride * 4));
    SCK(cudaMemcpyAsync(S.outidx.p, idx, out_rows * 4, cudaMemcpyHostToDevice, S.stream));
    size_t r0 = 0;
    for (size_t k = 0; k < fin.size(); ++k) {
      const Request &r = *fin[k];
      const size_t row = (size_t)r.n + 1, cnt = r.outputs.size();
      if (!cnt) continue;
      SCK(launch_gather(S.wires.as<uint32_t>(), S.outidx.as<uint32_t>() + r0, (int)cnt, r.n,
                        S.outstage.as<uint32_t>() + r0 * kWireStride, kWireStride, S.stream));
      SCK(cudaMemcpy2DAsync(T.pinned + out_off[k], row * 4, S.outstage.as<uint32_t>() + r0 * kWireStride,
                            kWireStride * 4, row * 4, cnt, cudaMemcpyDeviceToHost, S.stream));
      r0 += cnt;
    }
  }
  SCK(cudaMemcpyAsync(T.status_host, S.status, sizeof(unsigned int), cudaMemcpyDeviceToHost, S.stream));
  SCK(cudaEventRecord(T.end, S.stream));
  T.finishing = fin;
  T.out_off = out_off;
  T.ran.clear();
  for (auto &B : L)
    for (Request *r : B.ran)
      for (auto &a : act)
        if (a.get() == r) T.ran.push_back(a);
  T.inflight = true;
  S.cur ^= 1;
  return 1;
}

void scheduler() {
  Server &S = srv();
  Engine &E = eng();
  for (;;) {
    // retire whatever has completed without waiting
    for (Tick &T : S.tick) retire_tick(S, E, T, false);
    std::vector<std::shared_ptr<Request>> act, admitted;
    {
      std::unique_lock<std::mutex> lk(S.qmu);
      const bool inflight = S.tick[0].inflight || S.tick[1].inflight;
      bool ready_work = false;
      for (auto &r : S.active)
        if (r->status == 0 && r->next_wave < r->waves.size()) ready_work = true;
      if (!ready_work && S.pending.empty()) {
        if (S.stop && S.active.empty() && !inflight) return;
        if (inflight) {
          lk.unlock();
          for (Tick &T : S.tick)  // nothing to enqueue: wait for the device
            if (T.inflight) retire_tick(S, E, T, true);
          continue;
        }
        S.cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return S.stop || !S.pending.empty(); });
        if (S.stop && S.pending.empty() && S.active.empty()) return;
      }
    }
    {
      // admission, in arrival order, while the wires fit the budget and the arena
      std::lock_guard<std::mutex> elk(E.mu);
      std::lock_guard<std::mutex> lk(S.qmu);
      size_t used = E.resident_bytes();
      for (auto &r : S.active) used += request_bytes(*r);
      while (!S.pending.empty()) {
        auto r = S.pending.front();
        Keyset *ks = nullptr;
        if (resolve_keyset(E, r->keyset, &ks)) {
          r->status = ARX_ENOKEYS;
          S.failed++;
          S.pending.pop_front();
          continue;
        }
        const size_t need = request_bytes(*r);
        size_t base = 0;
        if (S.budget && used + need > S.budget) break;
        if (!S.arena.alloc(r->wire_count, &base)) break;
        r->wire_base = base;
        r->bsk = ks->bsk;
        r->ksk = ks->ksk;
        ks->refs++;  // the key set stays loaded while the request is admitted
        used += need;
        r->t_admit = Clock::now();
        S.pending.pop_front();
        S.active.push_back(r);
        admitted.push_back(r);
      }
      S.peak_bytes = std::max(S.peak_bytes, used);
      S.peak_active = std::max(S.peak_active, S.active.size());
      act = S.active;
    }
    if (act.empty()) continue;
    const int rc = enqueue_tick(S, E, admitted, act);  // no lock held: submissions go on meanwhile
    for (auto &r : admitted) {  // their inputs are in the staging buffer now
      r->ct_in.clear();
      r->ct_in.shrink_to_fit();
    }
    if (rc == 0) {  // every active request waits for ticks in flight
      bool waited = false;
      for (Tick &T : S.tick)
        if (T.inflight && !waited) waited = retire_tick(S, E, T, true) == 1;
      if (!waited) {
        std::unique_lock<std::mutex> lk(S.qmu);
        S.cv.wait_for(lk, std::chrono::milliseconds(2));
      }
      continue;
    }
    if (rc < 0) {  // a CUDA failure: the requests in flight fail
      for (Tick &T : S.tick) {
        if (T.inflight) cudaEventSynchronize(T.end);
        T.inflight = false;
        T.finishing.clear();
        T.ran.clear();
      }
      std::lock_guard<std::mutex> elk(E.mu);
      std::lock_guard<std::mutex> lk(S.qmu);
      for (auto &r : S.active) {
        if (r->status == 0) {
          r->status = rc;
          S.failed++;
        }
        S.arena.release(r->wire_base, r->wire_count);
        if (r->keyset >= 0 && r->keyset < (int)E.keysets.size()) E.keysets[r->keyset].refs--;
      }
      S.active.clear();
      S.cv.notify_all();
    }
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const double x = p / 100.0 * (v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace arx

using namespace arx;

extern "C" int arx_serve_start(size_t hbm_budget_bytes, size_t wire_arena_bytes, uint32_t max_tick_bootstraps) {
  Engine &E = eng();
  Server &S = srv();
  {
    std::lock_guard<std::mutex> elk(E.mu);
    int rc = ensure_init(E);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(S.qmu);
    if (S.running) return fail(ARX_EBUSY, "server already running");
    const size_t slots = std::max<size_t>(wire_arena_bytes / (kWireStride * 4), 1);
    if (hbm_budget_bytes && E.resident_bytes() >= hbm_budget_bytes)
      return fail(ARX_ENOMEM, "resident keys already exceed the HBM budget");
    cudaError_t e = S.wires.reserve(wire_bytes(slots));
    if (e != cudaSuccess) return fail(ARX_ENOMEM, "wire arena: %s", cudaGetErrorString(e));
    if (!S.stream) {
      e = cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(ARX_ECUDA, "stream: %s", cudaGetErrorString(e));
    }
    for (Tick &T : S.tick) {
      if (!T.begin) e = cudaEventCreate(&T.begin);
      if (e == cudaSuccess && !T.end) e = cudaEventCreate(&T.end);
      if (e != cudaSuccess) return fail(ARX_ECUDA, "event: %s", cudaGetErrorString(e));
      T.inflight = false;
    }
    S.cur = 0;
    // calibrate the launch shapes of every loaded dimension before serving
    for (const Keyset &k : E.keysets)
      if (k.used && E.policy.tuned_n != k.n) {
        rc = calibrate(E, k.n);
        if (rc) return rc;
      }
    S.policy = E.policy;
    S.tc = E.tc;
    S.tg = E.tg;
    S.status = E.status;
    S.sms = E.sms;
    S.arena.reset(slots);
    S.budget = hbm_budget_bytes;
    S.max_tick_bootstraps = max_tick_bootstraps;
    S.stop = false;
    S.latencies_ms.clear();
    S.done = S.failed = S.gates = S.bootstraps = S.launches = S.ticks = 0;
    S.shared_launches = S.max_keys = 0;
    S.peak_bytes = S.peak_active = 0;
    S.busy_s = 0;
    S.t_start = Clock::now();
    S.running = true;
  }
  S.th = std::thread(scheduler);
  return ARX_OK;
}

extern "C" int arx_serve_submit(int keyset, const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out) {
  Engine &E = eng();
  Server &S = srv();
  std::shared_ptr<Request> R;
  {
    std::lock_guard<std::mutex> elk(E.mu);
    if (!S.running) return fail(ARX_EINVAL, "server not running");
    if (!nl) return fail(ARX_EINVAL, "null netlist");
    int rc = build_request(E, nl, keyset, R);
    if (rc) return rc;
    if (nl->num_outputs && !ct_out) return fail(ARX_EINVAL, "ct_out is null");
    if (nl->num_inputs && !ct_in) return fail(ARX_EINVAL, "ct_in is null");
    if (S.budget && request_bytes(*R) + E.resident_bytes() > S.budget)
      return fail(ARX_ENOMEM, "request needs %zu bytes of wires, more than the budget leaves", request_bytes(*R));
    if (R->wire_count > S.arena.slots) return fail(ARX_ENOMEM, "request larger than the wire arena");
  }
  const size_t row = (size_t)R->n + 1;
  R->ct_in.assign(ct_in, ct_in + (size_t)nl->num_inputs * row);
  R->ct_out = ct_out;
  R->t_submit = Clock::now();
  int id;
  {
    std::lock_guard<std::mutex> lk(S.qmu);
    id = S.next_id++;
    R->id = id;
    S.table[id] = R;
    S.pending.push_back(R);
  }
  S.cv.notify_all();
  return id;
}

extern "C" int arx_serve_poll(int req) {
  Server &S = srv();
  std::lock_guard<std::mutex> lk(S.qmu);
  auto it = S.table.find(req);
  if (it == S.table.end()) return fail(ARX_EINVAL, "no request %d", req);
  return it->second->status;
}

extern "C" int arx_serve_wait(int req, double timeout_s) {
  Server &S = srv();
  std::unique_lock<std::mutex> lk(S.qmu);
  auto it = S.table.find(req);
  if (it == S.table.end()) return fail(ARX_EINVAL, "no request %d", req);
  auto R = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (R->status == 0) {
    if (S.cv.wait_until(lk, until) == std::cv_status::timeout && R->status == 0) return 0;
  }
  if (R->status < 0) return fail(R->status, "request %d failed", req);
  return 1;
}

extern "C" int arx_serve_stats(arx_serve_info *out) {
  Server &S = srv();
  if (!out) return fail(ARX_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S.qmu);
  out->completed = S.done;
  out->failed = S.failed;
  out->gates = S.gates;
  out->bootstraps = S.bootstraps;
  out->launches = S.launches;
  out->ticks = S.ticks;
  out->pending = S.pending.size();
  out->active = S.active.size();
  out->peak_active = S.peak_active;
  out->peak_bytes = S.peak_bytes;
  out->p50_ms = percentile(S.latencies_ms, 50);
  out->p99_ms = percentile(S.latencies_ms, 99);
  out->busy_s = S.busy_s;
  out->shared_launches = S.shared_launches;
  out->max_keys_per_launch = S.max_keys;
  out->elapsed_s = S.running ? std::chrono::duration<double>(Clock::now() - S.t_start).count() : 0.0;
  return ARX_OK;
}

extern "C" int arx_serve_stop(void) {
  Server &S = srv();
  {
    std::lock_guard<std::mutex> lk(S.qmu);
    if (!S.running) return ARX_OK;
    S.stop = true;
  }
  S.cv.notify_all();
  if (S.th.joinable()) S.th.join();
  std::lock_guard<std::mutex> lk(S.qmu);
  S.running = false;
  S.table.clear();
  return ARX_OK;
}
