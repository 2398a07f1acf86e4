/*
 * arx.h -- C-ABI of libarx: CGGI gate bootstrapping over Boolean netlists on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method is that of "ArctyrEX: Accelerated Encrypted Execution of
 * General-Purpose Applications" (arXiv 2306.11006): every encrypted logic gate is
 * a linear pre-combination of LWE ciphertexts followed by a bootstrapping --
 * blind rotation through n TGSW x TLWE external products -- and a key switch
 * (Fig. 2, Sec. 2.2); a netlist is split into waves of independent gates that are
 * evaluated one wave at a time (Sec. 4.2); keys are resident on the device and
 * constant (Sec. 5.1).
 *
 * Parameters: N = 1024 (TLWE degree), k = 1, gadget Bg = 2^7 with l = 3, key
 * switch base 2^2 with t = 8, Torus32 = uint32_t arithmetic mod 2^32.  The LWE
 * dimension n is fixed per key set: 630 by default (Sec. 2.2), any 1..630
 * through arx_load_keys_ex.  Encoding: bit 1 -> +1/8 (0x20000000), bit 0 -> -1/8.
 *
 * Layouts (all little-endian uint32_t, row-major, no padding):
 *   LWE ciphertext   [n+1]: a_0 .. a_{n-1}, b  (phase = b - <a, s>)
 *   bootstrapping key [n][6][2][N]: TGSW_K(s_i); row r = c*3 + (p-1) for
 *                     c in {0: mask, 1: body}, gadget level p = 1..3; each row is
 *                     a TLWE sample (mask polynomial, body polynomial).
 *   key-switching key [N][8][4][n+1]: entry [i][j-1][v] = LWE_s(v K_i 2^(32-2j));
 *                     the v = 0 entries are never read.
 *
 * Pointers: unless stated otherwise a ciphertext or key pointer may be host or
 * device memory (classified with cudaPointerGetAttributes); it is borrowed for the
 * duration of the call (or, for the _ex variants given a stream, until the work
 * queued on that stream completes).  The library owns keys and workspace.
 *
 * Errors: every call returns ARX_OK (0) or a negative arx_status; nothing aborts
 * the process; outputs are undefined after an error; arx_last_error() gives a
 * thread-local message.  A device watchdog expiry (a bounded wait inside a kernel
 * that ran out) is reported as ARX_ETIMEOUT by the synchronous calls and by
 * arx_device_status().
 *
 * Threads and streams: calls are serialised by an internal lock.  Asynchronous
 * (_ex with a non-NULL stream) calls on the same stream share that stream's
 * workspace in stream order; calls on different streams use different
 * workspaces.
 *
 * On-chip resources: the wide-wave blind-rotation kernels take all of an SM's
 * shared memory and, in their twelve-warp shapes, all 512 columns of its tensor
 * memory (tcgen05.alloc) for as long as their block runs, and free both before
 * the block exits.  A kernel of another library that allocates tensor memory on
 * the same SM at the same time (another stream) waits until the block is done;
 * nothing here waits on such a kernel, so the two cannot deadlock.
 */
#ifndef ARX_H
#define ARX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ARX_N 1024
#define ARX_LWE_N 630
#define ARX_BSK_ROWS 6
#define ARX_KS_T 8
#define ARX_KS_BASE 4
#define ARX_MU 0x20000000u

typedef enum {
  ARX_OK = 0,
  ARX_EINVAL = -1,    /* bad argument (size, type, wire id, pointer) */
  ARX_ENOKEYS = -2,   /* no key set loaded / unknown key set id */
  ARX_ENOMEM = -3,    /* device memory or HBM budget exhausted */
  ARX_ECYCLE = -4,    /* netlist has a combinational cycle */
  ARX_ETIMEOUT = -5,  /* a device-side bounded wait expired */
  ARX_ECUDA = -6,     /* a CUDA runtime call failed */
  ARX_EBUSY = -7      /* resource in use (key set referenced by a plan) */
} arx_status;

/* Gate opcodes: the standard two-input gates, the noiseless NOT, the MUX
 * (Sec. 2.2) and the constant / copy gates of the runtime (Sec. 4.2). */
typedef enum {
  ARX_AND = 0, ARX_NAND, ARX_OR, ARX_NOR, ARX_XOR, ARX_XNOR,
  ARX_NOT, ARX_MUX, ARX_COPY, ARX_CONST0, ARX_CONST1
} arx_gate;

/* ---------------------------------------------------------------- keys ---- */

/* Copy a key pair to the device and carry the bootstrapping key into the NTT
 * domain (done once; the paper keeps keys resident, Sec. 5.1).  Layouts above,
 * n = 630.  Returns a key set id >= 0, or an error.  The most recently loaded key
 * set is the default of the calls that take no key set id.  Synchronous. */
int arx_load_keys(const uint32_t *bsk, const uint32_t *ksk);

/* As arx_load_keys for LWE dimension lwe_n (1..630); stream may be NULL. */
int arx_load_keys_ex(const uint32_t *bsk, const uint32_t *ksk, int lwe_n, void *stream);

/* As arx_load_keys_ex with the gadget given: (l, bg_bits) = (3, 7), the default
 * set, or (2, 10), the gadget of the paper's own experiments (Fig. 2 draws 4
 * forward DFTs per CMux, (k+1) l = 4; Sec. 6 uses n = 512).  The bootstrapping
 * key then has 2 l rows per index: [n][2l][2][N], row r = c*l + (p-1), gadget
 * level p scaled by 2^(32 - p bg_bits).  Key sets with l = 2 run their blind
 * rotations on kernels instantiated for 10-bit digits: the sixteen-CTA cluster
 * kernel for waves that fit its co-resident clusters, the eight-CTA one for
 * waves of up to two rounds of its clusters, else the throughput kernel with
 * l = 2 (see arx_set_launch_shape for how an override maps onto them).
 * ARX_EINVAL for any other gadget. */
int arx_load_keys_gadget(const uint32_t *bsk, const uint32_t *ksk, int lwe_n, int l, int bg_bits, void *stream);

/* LWE dimension and gadget length of a loaded key set (-1 = the default one);
 * either pointer may be NULL.  ARX_ENOKEYS for an unknown id. */
int arx_keyset_dims(int keyset, int *lwe_n, int *l);

/* Free a key set.  ARX_EBUSY while a plan references it. */
int arx_unload_keys(int keyset);

/* Make a loaded key set the default of the calls that take no key set id. */
int arx_use_keys(int keyset);

/* Device bytes held by one key set of dimension lwe_n (NTT-domain BSK + KSK). */
size_t arx_keyset_bytes(int lwe_n);
/* Device bytes held by all key sets loaded now. */
size_t arx_resident_bytes(void);

/* ------------------------------------------------------------ gates ---- */

/* count independent gates: ct_out[g] = types[g](ct_a[g], ct_b[g]) with the
 * default key set.  Each two-input gate is the gate of Fig. 2 (Sec. 2.2): its
 * linear pre-combination of the inputs, mod switch to 2N, blind rotation by n
 * CMux external products with the bootstrapping key, sample extraction and the
 * key switch; NOT / COPY / CONST are linear and not bootstrapped.  All count
 * gates run as one wave (one blind-rotation launch, one key-switch launch).
 * types: host array of arx_gate (NOT / COPY read ct_a only, CONST read
 * neither; MUX needs arx_bootstrap_gates_ex).  ct_*: [count][n+1], host or
 * device memory; ct_out may alias ct_a or ct_b (inputs are copied to the
 * device before any output is written).  count = 0 is a no-op; count > 2^24,
 * a bad type or a NULL input a gate needs: ARX_EINVAL.  Synchronous. */
int arx_bootstrap_gates(const uint8_t *types, const uint32_t *ct_a, const uint32_t *ct_b,
                        uint32_t *ct_out, size_t count);

/* As arx_bootstrap_gates with a MUX third input ct_c (MUX(a, b, c) = a ? b : c;
 * may be NULL when no gate is a MUX), a key set id (-1 = default) and a CUDA
 * stream (cudaStream_t; NULL = synchronous on the library's stream). */
int arx_bootstrap_gates_ex(const uint8_t *types, const uint32_t *ct_a, const uint32_t *ct_b,
                           const uint32_t *ct_c, uint32_t *ct_out, size_t count, int keyset,
                           void *stream);

/* ---------------------------------------------------------- netlists ---- */

/* Gate netlist (host arrays).  Wire ids 0..num_inputs-1 are the inputs,
 * num_inputs + g the output of gate g.  Gates may be listed in any order; in1 is
 * read for two-input gates and MUX, in2 for MUX only (MUX(in0, in1, in2) =
 * in0 ? in1 : in2).  outputs[o] is any wire id. */
typedef struct {
  uint32_t num_inputs, num_gates, num_outputs;
  const uint8_t *type;
  const uint32_t *in0, *in1, *in2;
  const uint32_t *outputs;
} arx_netlist;

/* Wave levelization of Sec. 4.2 (host only, no GPU needed): wave[g] = 0 for a
 * gate without gate inputs, else 1 + the largest wave of its gate inputs.
 * *depth receives the number of waves.  ARX_EINVAL / ARX_ECYCLE on bad input. */
int arx_levelize(const arx_netlist *nl, uint32_t *wave, uint32_t *depth);

/* The Sec. 4.2 levelization with launch widths evened out (host only, no GPU
 * needed); graph-mode plans use it.  The depth stays that of arx_levelize, and
 * each gate g is placed between its earliest level (arx_levelize) and its
 * latest one (the last level that still leaves one level per gate of its
 * longest chain of readers), so that every gate still runs after its inputs and
 * all results equal those of the plain levelization.  Level by level, the gates
 * whose latest level it is are taken, then more ready gates (earliest latest
 * level first) while the level's blind rotations (MUX two, NOT / COPY / CONST
 * none) stay within the free capacity of the launch: caps[0 .. ncaps-1] is an
 * increasing list of launch capacities (for a GB300, the co-resident 16-, 8-,
 * 4- and 2-CTA clusters), and a level that must run j blind rotations may be
 * filled up to the smallest cap >= j (not beyond j when j > every cap).  The
 * reason: a narrow wave runs one gate per cluster and costs the same for any
 * count up to the co-resident clusters.  wave[g], *depth as arx_levelize.
 * ARX_EINVAL / ARX_ECYCLE on bad input or non-increasing caps. */
int arx_levelize_balanced(const arx_netlist *nl, const uint32_t *caps, uint32_t ncaps, uint32_t *wave,
                          uint32_t *depth);

/* The launch plan of one wave under a table of launch shapes (host only; what
 * graph plans compute from the autotuner's measured table).  Shape s costs
 * ms[s] per round of up to gates[s] blind rotations (a persistent launch pays
 * whole rounds); cluster[s] != 0 marks a shape that takes no bulk rounds of a
 * split.  For `jobs` blind rotations: the cheapest of one launch and of two --
 * k rounds of a non-cluster shape, the rest on the best shape for them -- as
 * *bulk (shape index) for the first *bulk_jobs and *tail (shape index, -1: one
 * launch) for the rest, *cost (ms), and *cap: the widest wave that one or two
 * such launches run within *cost (graph plans fill a level up to it).  Host
 * arrays of `shapes` entries (1..64; ms > 0, gates > 0); outputs may be NULL.
 * ARX_EINVAL on bad arguments.  No counterpart in the paper: scheduling. */
int arx_split_wave(const double *ms, const uint32_t *gates, const uint8_t *cluster, uint32_t shapes, uint32_t jobs,
                   uint32_t *bulk, uint32_t *bulk_jobs, int32_t *tail, double *cost, uint32_t *cap);

/* Evaluate a netlist with the default key set (Sec. 4.2): the gates are
 * levelized into waves (arx_levelize), and every wave -- all of its ready gates,
 * of any types -- runs as one blind-rotation launch and one key-switch launch,
 * waves in order; wires stay on the device between waves.  ct_in
 * [num_inputs][n+1], ct_out [num_outputs][n+1], host or device memory.  Bad
 * wire ids or types: ARX_EINVAL; a cycle: ARX_ECYCLE; no key set: ARX_ENOKEYS.
 * Synchronous. */
int arx_eval_netlist(const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out);

/* Execution modes of a plan. */
#define ARX_MODE_PLAIN 0   /* per-wave launches, fixed heuristic shapes */
#define ARX_MODE_GRAPH 1   /* autotuned persistent shapes, launch widths balanced within slack
                              (as arx_levelize_balanced, capacities from the autotuner's
                              measured launch costs), whole plan replayed as one CUDA graph */

int arx_eval_netlist_ex(const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out, int keyset,
                        int mode, void *stream);

/* Plans: a netlist levelized and laid out on the device once, evaluated many
 * times.  arx_plan_create copies the netlist (the caller's arrays may be freed
 * afterwards) and returns a plan id >= 0.  Several netlists evaluated together
 * are simply one netlist (their disjoint union): each wave then carries the
 * ready gates of all of them in one launch. */
int arx_plan_create(const arx_netlist *nl, int keyset, int mode);
int arx_plan_run(int plan, const uint32_t *ct_in, uint32_t *ct_out, void *stream);
int arx_plan_destroy(int plan);
/* Describe a plan: waves, blind rotations, gates (any may be NULL). */
int arx_plan_info(int plan, uint32_t *waves, uint64_t *bootstraps, uint64_t *gates);
/* Launch shape of each wave of a plan (what the autotuner or the override
 * chose when the plan was created; for a wave split over two launches, see
 * arx_plan_launches, the shape of its first): for wave w < min(cap, waves), H[w] and
 * GT[w] as in arx_set_launch_shape ((96, 1) / (48, 1) / (24, 1) / (12, 1): the
 * sixteen- / eight- / four- / two-CTA cluster kernels; for key sets with
 * gadget l = 2, (80, 1) / (40, 1) their sixteen- / eight-CTA kernels and
 * (100 + H, GT) the throughput kernel with 2H warps per gate) and
 * jobs[w] = its blind rotations (0 for a wave of linear gates only, which
 * launches no blind rotation).  Host arrays; any may be NULL.  Returns the
 * number of waves.  No counterpart in the paper: introspection only. */
int arx_plan_shapes(int plan, uint32_t *H, uint32_t *GT, uint32_t *jobs, uint32_t cap);
/* Every blind-rotation launch of a plan in launch order: an autotuned (graph
 * mode, gadget l = 3) wave whose width is not a whole number of rounds of any
 * shape may run as two launches, rounds of a throughput shape and its remainder
 * on the shape that suits the remainder.  For launch k < min(cap, launches):
 * wave[k], H[k], GT[k] (as arx_plan_shapes) and jobs[k].  Host arrays; any may
 * be NULL.  Returns the number of launches.  Introspection only. */
int arx_plan_launches(int plan, uint32_t *wave, uint32_t *H, uint32_t *GT, uint32_t *jobs, uint32_t cap);
/* Copy wires of the plan's most recent evaluation: out[k] = wire ids[k]
 * ([count][n+1]; ids host array, out host or device).  Synchronous.  Lets a
 * caller inspect or checkpoint intermediate ciphertexts. */
int arx_plan_wires(int plan, const uint32_t *ids, size_t count, uint32_t *out);

/* Run the plan once, wave by wave without the graph, timing every launch with
 * CUDA events on the library's stream: br_ms / ks_ms receive the summed
 * durations of the blind-rotation and key-switch launches, br_launches /
 * ks_launches their counts (any pointer may be NULL).  Outputs stay on the
 * device.  Synchronous. */
int arx_plan_profile(int plan, const uint32_t *ct_in, float *br_ms, float *ks_ms, uint32_t *br_launches,
                     uint32_t *ks_launches);

/* Force the blind-rotation launch shape: 2H warps per gate (H in 1, 2, 3, 6)
 * and GT gates per CTA; or (12, 1), (24, 1), (48, 1), (96, 1): one gate on a
 * cluster of two, four, eight or sixteen CTAs (SMs; sixteen is a non-portable
 * cluster size).  (0, 0) restores the automatic choice.
 * Shapes: (96,1) (48,1) (24,1) (12,1) (6,1) (3,1) (3,2) (2,1) (2,3) (1,1) (1,2)
 * (1,4) (1,6).  Plans keep the shapes chosen when they were created.  Key sets
 * with gadget l = 2 run kernels of their own: the sixteen-CTA one, (80, 1),
 * for waves that fit its co-resident clusters, the eight-CTA one, (40, 1), for
 * waves of up to two rounds of its clusters, else the throughput kernel
 * (100 + H, GT) with H in 1, 2, 4 (an override (H, GT) maps to the nearest of
 * these: (96, 1) to (80, 1), the other cluster shapes to (40, 1)); none of
 * these codes is itself an override (ARX_EINVAL). */
int arx_set_launch_shape(int H, int GT);

/* ------------------------------------------------------------ serving ---- */
/* Continuous batching of encrypted-circuit requests from several clients (the
 * paper evaluates one circuit at a time; serving is this library's addition).
 * arx_serve_start launches a scheduler thread with a wire arena of
 * wire_arena_bytes of device memory and an HBM budget (bytes of resident key
 * sets + wires of admitted requests; 0 = no budget).  Requests are admitted in
 * arrival order while their wires fit the budget and the arena; every scheduler
 * tick advances each admitted request by one wave, with the waves of all
 * requests whose key sets share the LWE dimension and gadget merged into one
 * blind-rotation and one key-switch launch, whichever client's key set each
 * gate uses (up to 16 key sets per launch; at most max_tick_bootstraps blind
 * rotations per launch, 0 = no cap; a larger tick takes more launches).  Ticks
 * are pipelined: the next tick is prepared on the host while the device runs
 * the current one.  Requests arriving meanwhile join at the next tick.  A
 * request's result is bit-identical to arx_eval_netlist's on the same inputs,
 * whatever else is in flight. */
typedef struct {
  uint64_t completed, failed, gates, bootstraps, launches, ticks;
  uint64_t pending, active, peak_active, peak_bytes;
  double p50_ms, p99_ms;  /* submit-to-completion latency of completed requests */
  double busy_s, elapsed_s; /* device time of the ticks (their events), wall time since start */
  uint64_t shared_launches;      /* blind-rotation launches whose gates came from more than one key set */
  uint64_t max_keys_per_launch;  /* the most key sets one launch mixed */
} arx_serve_info;

int arx_serve_start(size_t hbm_budget_bytes, size_t wire_arena_bytes, uint32_t max_tick_bootstraps);
/* Queue a request: netlist and inputs (host memory) are copied, so the caller may
 * free them on return; ct_out (host, [num_outputs][n+1]) is written when the
 * request completes.  Returns a request id >= 0 or an error (bad netlist, no key
 * set, larger than the budget or the arena). */
int arx_serve_submit(int keyset, const arx_netlist *nl, const uint32_t *ct_in, uint32_t *ct_out);
/* 1 = done, 0 = pending, < 0 = failed. */
int arx_serve_poll(int request);
/* Wait up to timeout_s seconds: 1 = done, 0 = still pending, < 0 = failed. */
int arx_serve_wait(int request, double timeout_s);
int arx_serve_stats(arx_serve_info *out);
/* Finish every queued request, then stop the scheduler. */
int arx_serve_stop(void);

/* Key switch without allocation.  For callers that cannot allocate device
 * memory during the call -- a serving process that budgets all of its HBM up
 * front, a framework whose caching allocator must own every device buffer, or a
 * latency-critical loop in which cudaMalloc / cudaFree would synchronise the
 * device and stall other streams.  (The paper has no counterpart; this is a
 * library service.)
 *
 * Key-switches count LWE_N samples lwe_N [count][N+1] (device memory, e.g.
 * blind-rotation outputs) into LWE_n ciphertexts ct_out [count][n+1] (device
 * memory) with a loaded key set (-1 = default), exactly as the gate path does.
 * It calls no cudaMalloc, cudaFree or allocating library routine: the kernel's
 * scratch (partial sums of the split key-row gather and one counter per gate)
 * is a fixed static device array of about 2.6 MB that every GPU loading the
 * library holds until the process exits.  count <= ARX_KS_NOALLOC_MAX, else
 * ARX_EINVAL.  The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  All calls share the array and each one clears the
 * counters it uses, so calls that overlap on the GPU (different streams, or
 * concurrent host threads) race: order them on one stream.  stream NULL means
 * synchronous on the library's stream.  A key set must be loaded first. */
#define ARX_KS_NOALLOC_MAX 1024
int arx_keyswitch_noalloc(const uint32_t *lwe_N, uint32_t *ct_out, size_t count, int keyset, void *stream);

/* ------------------------------------------------------------- status ---- */

const char *arx_last_error(void);
/* Reads and clears the device watchdog status: ARX_OK or ARX_ETIMEOUT. */
int arx_device_status(void);
/* Self-test of the device watchdog (no counterpart in the paper).  One CTA of
 * four warps waits, through the same bounded wait functions as the kernels, on
 * one phase of an mbarrier that expects one arrival; post_token != 0 makes that
 * arrival before the waits, post_token == 0 withholds it, so that every wait
 * runs out after limit_cycles SM clock cycles (1000 .. 4e9; the kernels use
 * 4e9, about 2 s), sets the device status word and returns.  Synchronous, on
 * the library's stream; allocates and frees 16 bytes of device memory.
 * *waits_given_up (host pointer, may be NULL) receives how many of the four
 * warps gave up.  Returns ARX_OK (every wait completed), ARX_ETIMEOUT (the
 * status word recorded the expiry; it is cleared, and the device stays usable),
 * ARX_EINVAL (limit out of range) or ARX_ECUDA.  An expiry left over from an
 * earlier call is returned as ARX_ETIMEOUT before anything is launched. */
int arx_watchdog_selftest(int post_token, long long limit_cycles, int *waits_given_up);
/* Number of SMs of the device in use (0 before the first call that needs it). */
int arx_device_sms(void);

/* Integer-pipe throughput of the current device, the measured side of the blind
 * rotation's ALU roofline (no counterpart in the paper).  rate[i], i < count
 * (at most 7), receives lane operations per clock per SM (32 warps per SM,
 * independent dependency chains, clock64 timing) for: 0 IMAD, 1 IMAD.HI,
 * 2 IMAD.WIDE, 3 plain ALU (one unit = IADD3 + SHF + LOP), 4 Shoup butterfly
 * mod a 27-bit prime,
 * 5 Montgomery multiply-accumulate mod a 27-bit prime, 6 butterfly mod the
 * paper's 2^64 - 2^32 + 1 (Sec. 5.4).  Host array.  Synchronous, takes about a
 * second, allocates and frees a few KB of device memory.  Returns ARX_OK or
 * ARX_EINVAL / ARX_ECUDA. */
int arx_probe_alu(double *rate, int count);

/* ------------------------------------------------------- client side ---- */
/* Key generation, encryption and decryption as the client (the data owner)
 * performs them (App. D: the server only ever sees ciphertexts and public
 * keys).  All randomness is supplied by the caller; host memory only.
 *   s [n] and K [N]: binary secret keys (bytes 0/1);
 *   bsk_mask [n][6][N] uniform, bsk_noise [n][6][N] (Torus32 units);
 *   ksk_mask [N][8][3][n] uniform, ksk_noise [N][8][3];
 *   outputs in the layouts above. */
int arx_client_keygen(int lwe_n, const uint8_t *s, const uint8_t *K, const uint32_t *bsk_mask,
                      const int32_t *bsk_noise, const uint32_t *ksk_mask, const int32_t *ksk_noise,
                      uint32_t *bsk, uint32_t *ksk);
/* As arx_client_keygen with the gadget (l, bg_bits) = (3, 7) or (2, 10) (see
 * arx_load_keys_gadget): bsk_mask / bsk_noise are [n][2l][N], bsk [n][2l][2][N]. */
int arx_client_keygen_gadget(int lwe_n, int l, int bg_bits, const uint8_t *s, const uint8_t *K,
                             const uint32_t *bsk_mask, const int32_t *bsk_noise, const uint32_t *ksk_mask,
                             const int32_t *ksk_noise, uint32_t *bsk, uint32_t *ksk);
/* ct[g] = (mask[g], <mask[g], s> + noise[g] + (bits[g] ? +1/8 : -1/8)). */
int arx_client_encrypt(int lwe_n, const uint8_t *s, const uint32_t *mask, const int32_t *noise,
                       const uint8_t *bits, size_t count, uint32_t *ct);
/* bits[g] = (int32)(b - <a, s>) > 0. */
int arx_client_decrypt(int lwe_n, const uint8_t *s, const uint32_t *ct, size_t count, uint8_t *bits);

#ifdef __cplusplus
}
#endif
#endif /* ARX_H */
