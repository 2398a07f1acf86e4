// serve.cpp -- continuous-batching server for encrypted-circuit requests.
//
// Requests (a netlist, its encrypted inputs and a client key set) are queued by
// arx_serve_submit.  A scheduler thread admits them in arrival order while the
// device memory they need (their wires, in one wire arena) fits the HBM budget
// next to the resident keys, and then runs ticks: every tick takes the next wave
// of every admitted request, merges the waves of all requests that share a key
// set into one blind-rotation launch and one key-switch launch (so a key set's
// bootstrapping-key rows are reused across all of them, Sec. 5.1), and advances
// every request by one wave.  A request that arrives while others run joins at
// the next tick; a finished one leaves and frees its wires for the next
// admission.  Each request's ciphertexts are computed by exactly the kernels and
// descriptors the single-request path uses, so its result does not depend on
// what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
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
  DevBuf wires, brjobs, ksjobs, brout, kspart, kscnt, outidx, outstage;
  std::vector<double> latencies_ms;
  uint64_t done = 0, failed = 0, gates = 0, bootstraps = 0, launches = 0, ticks = 0;
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

// Copy a finished request's outputs to the caller (wires -> host buffer).
int finish_request(Server &S, Request &R) {
  const size_t row = (size_t)R.n + 1;
  const int nout = (int)R.outputs.size();
  if (nout) {
    std::vector<uint32_t> idx(R.outputs);
    for (auto &v : idx) v += (uint32_t)R.wire_base;
    SCK(S.outidx.reserve(idx.size() * 4));
    SCK(S.outstage.reserve((size_t)nout * row * 4));
    SCK(cudaMemcpyAsync(S.outidx.p, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, S.stream));
    SCK(launch_gather(S.wires.as<uint32_t>(), S.outidx.as<uint32_t>(), nout, R.n, S.outstage.as<uint32_t>(),
                      (int)row, S.stream));
    SCK(cudaMemcpyAsync(R.ct_out, S.outstage.p, (size_t)nout * row * 4, cudaMemcpyDeviceToHost, S.stream));
    SCK(cudaStreamSynchronize(S.stream));
  }
  return ARX_OK;
}

// One tick: the next wave of every active request, one launch pair per key set.
int read_server_status(Server &S) {
  unsigned int v = 0;
  SCK(cudaMemcpyAsync(&v, S.status, sizeof(v), cudaMemcpyDeviceToHost, S.stream));
  SCK(cudaStreamSynchronize(S.stream));
  if (v) {
    SCK(cudaMemsetAsync(S.status, 0, sizeof(unsigned int), S.stream));
    SCK(cudaStreamSynchronize(S.stream));
    return fail(ARX_ETIMEOUT, "device watchdog expired (status 0x%x)", v);
  }
  return ARX_OK;
}

int run_tick(Server &S, std::vector<std::shared_ptr<Request>> &act) {
  std::map<int, std::vector<Request *>> groups;
  for (auto &r : act)
    if (r->next_wave < r->waves.size()) groups[r->keyset].push_back(r.get());
  for (auto &kv : groups) {
    const Request &head = *kv.second.front();
    int rc = ARX_OK;
    std::vector<BrJob> br;
    std::vector<KsJob> ksj;
    uint32_t budget = S.max_tick_bootstraps ? S.max_tick_bootstraps : 0xffffffffu;
    std::vector<Request *> ran;
    for (Request *r : kv.second) {
      const Wave &W = r->waves[r->next_wave];
      if (!ran.empty() && br.size() + W.br.size() > budget) continue;  // waits for a later tick
      const uint32_t base = (uint32_t)r->wire_base, jb = (uint32_t)br.size();
      for (BrJob j : W.br) {
        j.ia += base;
        j.ib += base;
        br.push_back(j);
      }
      for (KsJob k : W.ks) {
        k.j0 += jb;
        k.j1 += jb;
        k.ia += base;
        k.out += base;
        ksj.push_back(k);
      }
      ran.push_back(r);
    }
    if (ran.empty()) continue;
    SCK(S.brjobs.reserve(std::max<size_t>(br.size(), 1) * sizeof(BrJob)));
    SCK(S.ksjobs.reserve(std::max<size_t>(ksj.size(), 1) * sizeof(KsJob)));
    SCK(S.brout.reserve(std::max<size_t>(br.size(), 1) * kOutStride * 4));
    if (!br.empty())
      SCK(cudaMemcpyAsync(S.brjobs.p, br.data(), br.size() * sizeof(BrJob), cudaMemcpyHostToDevice, S.stream));
    if (!ksj.empty())
      SCK(cudaMemcpyAsync(S.ksjobs.p, ksj.data(), ksj.size() * sizeof(KsJob), cudaMemcpyHostToDevice, S.stream));
    if (!br.empty()) {
      BrArgs a{};
      a.bsk = head.bsk;
      a.wires = S.wires.as<uint32_t>();
      a.jobs = S.brjobs.as<BrJob>();
      a.num_jobs = (int)br.size();
      a.n = head.n;
      a.out = S.brout.as<uint32_t>();
      a.tg = S.tg;
      a.status = S.status;
      a.tc = S.tc;
      const BrShape s = S.policy.for_gadget(head.l, S.policy.pick(a.num_jobs, head.n), a.num_jobs);
      SCK(launch_br(a, s, S.policy.grid(s, a.num_jobs), S.stream));
      S.launches++;
    }
    if (!ksj.empty()) {
      KsArgs k{};
      k.ksk = head.ksk;
      k.br_out = S.brout.as<uint32_t>();
      k.wires = S.wires.as<uint32_t>();
      k.jobs = S.ksjobs.as<KsJob>();
      k.n = head.n;
      k.out = S.wires.as<uint32_t>();
      k.out_stride = kWireStride;
      k.splits = ks_splits((int)ksj.size(), S.sms);
      rc = reserve_ks_scratch(S.kspart, S.kscnt, ksj.size(), k.splits);
      if (rc) return rc;
      k.partial = S.kspart.as<uint32_t>();
      k.counters = S.kscnt.as<unsigned int>();
      SCK(launch_ks(k, (int)ksj.size(), S.stream));
      S.launches++;
    }
    // the descriptor uploads above come from host vectors: finish before they go
    SCK(cudaStreamSynchronize(S.stream));
    for (Request *r : ran) {
      S.bootstraps += r->waves[r->next_wave].br.size();
      S.gates += r->waves[r->next_wave].ks.size();
      r->next_wave++;
    }
  }
  return read_server_status(S);
}

void scheduler() {
  Server &S = srv();
  Engine &E = eng();
  for (;;) {
    std::vector<std::shared_ptr<Request>> act;
    {
      std::unique_lock<std::mutex> lk(S.qmu);
      S.cv.wait_for(lk, std::chrono::milliseconds(20),
                    [&] { return S.stop || !S.pending.empty() || !S.active.empty(); });
      if (S.stop && S.pending.empty() && S.active.empty()) return;
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
        const size_t row = (size_t)r->n + 1;
        cudaError_t e = cudaSuccess;
        if (r->num_inputs)
          e = cudaMemcpy2DAsync(S.wires.as<uint32_t>() + base * kWireStride, kWireStride * 4, r->ct_in.data(),
                                row * 4, row * 4, r->num_inputs, cudaMemcpyHostToDevice, S.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S.stream);
        r->ct_in.clear();
        r->ct_in.shrink_to_fit();
        r->t_admit = Clock::now();
        S.pending.pop_front();
        if (e != cudaSuccess) {
          r->status = ARX_ECUDA;
          S.failed++;
          S.arena.release(base, r->wire_count);
          ks->refs--;
          continue;
        }
        S.active.push_back(r);
      }
      S.peak_bytes = std::max(S.peak_bytes, used);
      S.peak_active = std::max(S.peak_active, S.active.size());
      act = S.active;
    }
    if (act.empty()) continue;
    const auto t0 = Clock::now();
    const int rc = run_tick(S, act);  // no lock held: submissions go on meanwhile
    const auto t1 = Clock::now();
    std::vector<std::shared_ptr<Request>> leaving, still;
    for (auto &r : act) {
      if (rc) {
        r->status = rc;
        leaving.push_back(r);
      } else if (r->next_wave >= r->waves.size()) {
        const int frc = finish_request(S, *r);
        r->t_done = Clock::now();
        r->status = frc ? frc : 1;
        leaving.push_back(r);
      }
    }
    {
      std::lock_guard<std::mutex> elk(E.mu);
      std::lock_guard<std::mutex> lk(S.qmu);
      S.busy_s += std::chrono::duration<double>(t1 - t0).count();
      S.ticks++;
      for (auto &r : leaving) {
        if (r->status == 1) {
          S.done++;
          S.latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        } else {
          S.failed++;
        }
        S.arena.release(r->wire_base, r->wire_count);
        if (r->keyset >= 0 && r->keyset < (int)E.keysets.size()) E.keysets[r->keyset].refs--;
      }
      for (auto &r : S.active)
        if (std::find(leaving.begin(), leaving.end(), r) == leaving.end()) still.push_back(r);
      S.active.swap(still);
    }
    S.cv.notify_all();
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
