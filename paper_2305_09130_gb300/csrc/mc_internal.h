// Internal declarations shared by the host side (mc_api.cu) and the kernels
// (mc_kernels.cu) of the explorer.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "mc.h"

// A counterexample or witness path returned through the C-ABI (mc_trace is
// opaque in mc.h): `words` u64 per state, states s0 .. the last one.
struct mc_trace {
  uint32_t words = 1;
  std::vector<uint64_t> keys;
};

namespace mc {

constexpr uint32_t kMaxP = 16;
constexpr uint64_t kNone = ~0ull;          // "no value" for packed minima
constexpr int kPackIdxBits = 12;           // i and j fields of a packed (time, i, j)
constexpr uint32_t kNoParent = 0xFFFFFFFFu;
constexpr uint32_t kThreads = 256;         // exploration kernel block size (maximum)
constexpr uint32_t kWarpCap = 128;         // winners staged per warp before a flush (default chunk)
constexpr uint32_t kStageCap = 192;        // exploration kernel: staging capacity per warp (largest chunk)
#ifndef MC_PROBE_DEPTH
#define MC_PROBE_DEPTH 1
#endif
constexpr uint32_t kDepth = MC_PROBE_DEPTH; // states per tile and round (probes in flight per lane)
// device-wide barrier: 128-byte lines of the arrival counter, the
// generation word and the abort flag (one more line spare)
constexpr uint32_t kBarCount = 0;
constexpr uint32_t kBarGen = 1;
constexpr uint32_t kBarAbort = 2;
constexpr size_t kBarBytes = 4 * 128;

// Packed (time, i, j) used for device-side min-reductions: time < 2^40,
// i, j < 2^12.
__host__ __device__ inline uint64_t pack_tij(uint64_t t, uint32_t i, uint32_t j) {
  return (t << (2 * kPackIdxBits)) | ((uint64_t)i << kPackIdxBits) | j;
}
__host__ __device__ inline uint64_t pack_time(uint64_t p) { return p >> (2 * kPackIdxBits); }
__host__ __device__ inline uint32_t pack_i(uint64_t p) { return (uint32_t)(p >> kPackIdxBits) & 0xFFFu; }
__host__ __device__ inline uint32_t pack_j(uint64_t p) { return (uint32_t)p & 0xFFFu; }

// Model constants every kernel needs (passed by value).
struct Params {
  uint32_t a, b, P, rule;
  uint32_t n_bits;        // bits of one n_c field
  uint32_t ts_shift;      // bit offset of j+1
  uint32_t wg_shift;      // bit offset of i+1
  uint32_t ts_mask;       // (1 << ts_bits) - 1
  uint32_t wg_mask;       // (1 << wg_bits) - 1
  uint32_t max_level;     // max N_ij + 2
  uint64_t n_mask;        // (1 << n_bits) - 1
  uint64_t swar_mask;     // low P*n_bits bits (when P*n_bits <= 64)
  uint64_t swar_mul;      // sum_t 2^(t*n_bits): the product's top field sums the n fields
  uint32_t swar_ok;       // 1 when P*n_bits <= 64
  uint32_t clk32;         // 1 when every clock (N * cost * speed) fits 32 bits
  const uint32_t* N;      // device [a*b]
  const uint32_t* cost;   // device [a*b]
  const uint32_t* speed;  // device [P]
};

// Per-pass control block header (device memory, zeroed before each pass).
struct Ctrl {
  uint32_t err;           // first error code of the pass (0 = none)
  uint32_t skipped;       // 1: a chained pass that did not run (its predecessor held or failed)
  uint32_t units_next;    // configuration engine: next configuration to take
  uint32_t units_done;    // configuration engine: configurations finished
  uint32_t levels;        // last explored level + 1
  uint32_t stop_level;    // first level holding a violating terminal (0 = none)
  uint32_t witness_level; // level the witness was taken from (0 = none)
  uint32_t trace_len;     // states in the trace buffer
  uint64_t states;        // sum of the widths of the explored levels
  uint64_t best_pack;     // min packed (time, i, j) over all violating terminals
  uint64_t wkey_lo;       // witness key
  uint64_t wkey_hi;
  uint64_t widx;          // witness index inside its level
  uint64_t wpack;         // packed (time, i, j) of the first violating level
  uint64_t T;             // threshold the pass used
  uint64_t probes;        // successors generated (PE-level explorer only)
  uint32_t stop_c;        // configuration engine, early exit: ~(least level known to hold a
                          // violating terminal), 0 while none is known
  uint32_t pad1[3];
};

// Everything one exploration pass needs.
struct ExploreArgs {
  Params p;
  void* table;            // visited set: buckets of 32 bytes
  uint64_t bucket_mask;   // buckets - 1
  uint64_t table_u64;     // table size in u64 words (for clearing)
  uint32_t max_probes;    // bucket probes before MC_ERR_TABLE_FULL
  uint32_t prune;
  uint32_t early_exit;
  uint32_t want_witness;  // find the witness of the first violating level + trace
  void* log_keys;         // frontier log: keys of every kept state, level by level
  uint32_t* log_par;      // parent index inside the previous level
  uint64_t log_cap;
  Ctrl* ctrl;
  uint64_t* levels;       // [max_level + 2] x {kept states, min packed violating terminal}
  uint64_t* off;          // [max_level + 2] first log entry of each level
  uint64_t* trace;        // [(max_level + 1) * 2] trace keys {lo, hi}
  uint64_t T;             // threshold, unless T_src is set
  const uint64_t* T_src;  // device threshold source (T = *T_src + T_delta)
  int64_t T_delta;
  uint64_t* tmin_out;     // if set: receives pack_time(best_pack) at the end
  uint32_t barrier_extra; // extra arrivals a barrier waits for (test hook)
  uint32_t stage_chunk;   // winners a warp stages before a flush (64..kStageCap)
  uint32_t* bar_lines;    // the device-wide barrier's lines (zeroed per pass)
  uint64_t timeout_ns;
  const Ctrl* prev;       // lowering chained on the device: run at (prev's counterexample
                          // time) - 1, or not at all if prev held, failed or was skipped
  uint64_t tag;           // tagged frontier log: this pass's tag (< 2^tag_bits) and the
  uint32_t tag_bits;      // bits it takes in each 64-bit word of a key (0: untagged; see
  uint32_t pad2;          // the exploration kernel)
};

// Launch helpers implemented in mc_kernels.cu.  `scheme` is the probe scheme,
// resolved (MC_PROBE_SPLIT, MC_PROBE_ONE_CALL, MC_PROBE_CAS_FIRST or
// MC_PROBE_CAS_CLEAR); the CAS-first kernels come from mc_explore_cas.cu.
const void* pick_explore_cas(int key_words, int tile, int rule, int scheme);
int explore_kernel_occupancy(int key_words, int tile, int rule, int scheme, int threads, int* blocks_per_sm);
cudaError_t launch_explore(int key_words, int tile, int rule, int scheme, int grid, int threads,
                           const ExploreArgs& args, cudaStream_t stream);
cudaError_t launch_simulate(const Params& p, uint64_t seed, uint32_t walks, uint64_t* t_out,
                            cudaStream_t stream);
cudaError_t launch_swarm(const Params& p, uint64_t seed, uint64_t w0, uint32_t walks, uint64_t bound,
                         unsigned long long* best, int grid, cudaStream_t stream);
cudaError_t launch_replay_walk(const Params& p, uint64_t seed, uint64_t w, int key_words,
                               uint64_t* trace, uint32_t* len, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Configuration engine (mc_cfg.cu).  The WG and TS selects (levels 1 and 2)
// split the state space into disjoint subtrees, one per configuration (i, j):
// every later state carries its (i, j).  A thread block explores one
// subtree level by level with its frontier and visited set in shared
// memory, so a level costs one block-wide barrier instead of a device-wide
// one.  Counts, the first violating level, the minimum and the witness are
// combined per level and per configuration, so a pass reports exactly what
// the level-synchronous kernel reports.
constexpr uint32_t kCfgMaxThreads = 512;
constexpr uint64_t kCfgMaxWidth64 = 2048;   // widest level of one configuration, 64-bit keys
constexpr uint64_t kCfgMaxWidth128 = 1024;  // 128-bit keys

// One configuration's outcome in one pass.
struct CfgRec {
  uint64_t vpack;         // min packed (time, i, j) of its violating terminals, kNone if none
  uint64_t wkey_lo;       // the smallest key among its violating terminals of that time
  uint64_t wkey_hi;
  uint32_t widx;          // log index of that key (passes that keep the log)
  uint32_t deepest;       // deepest level it reached with a nonempty width
};

// One pass over every configuration of one model.
struct CfgPass {
  Params p;
  uint64_t T;             // threshold, unless T_src or prev is set
  const uint64_t* T_src;  // device threshold source (T = *T_src + T_delta)
  int64_t T_delta;
  const Ctrl* prev;       // chained lowering: run at prev's counterexample time - 1,
                          // or not at all if prev held, failed or was skipped
  uint32_t prune;
  uint32_t early_exit;
  uint32_t want_witness;  // keep the log and find the witness and its trace
  uint32_t group;         // lanes per state: next power of two >= P
  void* log_keys;         // [seg[a*b]] keys, written only with want_witness
  uint32_t* log_par;      // parent log index of each entry
  const uint64_t* seg;    // [a*b + 1] first log entry of each configuration's segment
  uint64_t* levels;       // [max_level + 2] x {width, unused}, zeroed before the pass
  CfgRec* rec;            // [a*b]
  Ctrl* ctrl;             // header; units_next, units_done and stop_c start at 0
  uint64_t* trace;        // [(max_level + 1) * 2]
  uint64_t* tmin_out;     // if set: receives the least violating terminal time
  const uint32_t* order;  // [a*b] configurations in the order blocks take them (deepest first)
};

// A launch: one pass (`one`), or many passes of many models (`passes`, with
// `units` listing (pass index << 32 | configuration) in the order blocks
// take them).  `next` counts the units handed out.  Warp units: the
// configurations of models whose widest level fits one warp (width bound x
// lanes per state <= kCfgWarpLanes) are explored by one warp each; blocks
// [0, warp_blocks) serve them, every warp taking units from `wunits` (same
// encoding, read backwards from `wunits` when `wunits_rev` is set; a single
// pass's configurations in `one.order` when null) with `wnext`, and the
// other blocks serve `units`.
struct CfgLaunch {
  CfgPass one;
  const CfgPass* passes;
  const uint64_t* units;
  uint64_t n_units;
  const uint32_t* n_units_dev;  // if set: the unit count, read on the device
  uint32_t* next;
  uint32_t wcap;          // frontier capacity per level (states), a power of two
  uint32_t tsize;         // shared visited-set slots per level, a power of two
  const uint64_t* wunits;
  uint64_t n_wunits;
  const uint32_t* n_wunits_dev;
  uint32_t* wnext;
  uint32_t warp_blocks;
  uint32_t wunits_rev;
};
constexpr uint32_t kCfgWarpLanes = 32;  // a warp unit's widest level x lanes per state
constexpr uint32_t kCfgWarpBlockThreads = 128;  // blocks of a launch of warp units only
constexpr uint32_t kCfgMaxWarpBlocks = 1024;     // blocks serving warp units in a run's launch

size_t cfg_smem_bytes(int key_words, uint32_t wcap, uint32_t tsize);
int cfg_occupancy(int key_words, int threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_cfg(int key_words, int grid, int threads, size_t smem, const CfgLaunch& L,
                       cudaStream_t stream);

// Runs of many models on the configuration engine (batches, served jobs):
// before the passes, one launch clears every model's pass headers and level
// widths and sets its T_ini word; a second draws the T_ini simulations.
struct CfgClear {         // one model's words to clear
  uint64_t* levels;       // its passes' level-width arrays, contiguous
  uint64_t level_words;
  Ctrl* ctrl;             // its pass headers, contiguous
  uint32_t n_ctrl;
  uint32_t pad;
  uint64_t* scal;         // {T_ini = kNone, T_min = 0}
};
struct CfgSim {           // one min-time model's simulation (Section 4, Step 3)
  Params p;
  uint64_t* tini;
  uint64_t seed;
  uint32_t walks;
  uint32_t pad;
};
cudaError_t launch_cfg_clear(const CfgClear* clears, const uint32_t* n_dev, uint32_t n_max, cudaStream_t stream);
cudaError_t launch_cfg_sim(const CfgSim* sims, const uint32_t* n_dev, uint32_t n_max, uint32_t walks_max,
                           cudaStream_t stream);

// What the configuration engine needs of a model made by mc_model_create
// (host only): its constants (device pointers unset), the lanes per state,
// the closed-form widest level of one configuration, and the frontier-log
// segment starts of its configurations ([a*b + 1], owned by the model).
struct CfgModelInfo {
  Params p;
  uint32_t group;
  uint32_t key_words;
  uint64_t unit_width;
  uint64_t unit_log;
  const uint64_t* seg;
  bool eligible;
};
int cfg_model_info(mc_model* m, CfgModelInfo* out);

}  // namespace mc

// ---------------------------------------------------------------------------
// Batched exploration (mc_batch.cu): many models advance in lockstep inside
// one persistent launch.  Keys are 128-bit for every instance.
namespace mc {

constexpr uint32_t kMaxBatch = 1024;     // instances per batch launch
constexpr uint32_t kTaskUnits = 256;     // units one set-up task initialises (8 per lane)

// Phase of one instance between two device-wide barriers.
enum BPhase : uint32_t {
  B_DONE = 0,
  B_SIM = 1,      // random runs for T_ini (min-time queries)
  B_SETUP = 2,    // clear the visited set, write levels 0..2
  B_EXPAND = 3,   // expand level L into L+1
  B_WIT_HI = 4,   // witness scan of level L: smallest high key word
  B_WIT_LO = 5,   //   smallest low word among those
  B_WIT_IDX = 6,  //   its index in the level
  B_TRACE = 7,    // parent walk into the trace buffer
};

// Pass of a query: min-time runs 1 (minimum), 2 (certificate T_min - 1) and
// 3 (counterexample at T_min); a check runs 3 at its own T.
enum BPass : uint32_t { PASS_NONE = 0, PASS_MIN = 1, PASS_REFINE = 2, PASS_FINAL = 3 };

// Per instance, fixed for a launch.
struct BInst {
  Params p;
  void* table;
  uint64_t bucket_mask;
  uint64_t table_u64;
  void* log_keys;         // u128 keys
  uint32_t* log_par;
  uint64_t log_cap;
  uint64_t* levels;       // [max_level + 2] x {width, min packed violating terminal}
  uint64_t* off;          // [max_level + 2]
  uint64_t* trace;        // [(max_level + 2) * 2]
  uint32_t max_probes;
  uint32_t group;         // lanes per state: next power of two >= P
  uint32_t kind;          // MC_QUERY_*
  uint32_t pad;
  uint64_t T_query;       // threshold of a check query
};

// Per instance, rewritten by the planner at every barrier; the witness words,
// the next level's counters and err are also updated by atomics during a step.
struct BState {
  uint32_t phase;         // BPhase
  uint32_t pass;          // BPass
  uint32_t L;             // level expanded (B_EXPAND) or scanned (witness phases)
  uint32_t err;           // first error of this instance
  uint64_t W;             // width of level L
  uint64_t offL;          // log offset of level L
  uint64_t T;             // threshold of the current pass
  uint32_t prune, early_exit;
  uint32_t started;       // 0 until the first plan
  uint32_t checks;        // passes finished
  uint64_t t_ini;         // least simulated terminal time (atomicMin)
  uint64_t t_min;         // minimum of the min pass
  uint64_t states;        // unique states over finished passes
  uint64_t best_all;      // min packed violating terminal over the pass's levels
  uint32_t first_viol;    // first level of the pass with a violating terminal
  uint32_t levels;        // levels of the last finished pass
  uint32_t stop_level;    // counterexample level of the final pass (0: holds)
  uint32_t trace_len;
  uint64_t wpack;         // packed (time, i, j) of the counterexample
  uint64_t wkey_lo, wkey_hi, widx;
  uint64_t wnext;         // B_EXPAND: width of level L+1 (log reservations add to it)
  uint64_t bnext;         // B_EXPAND: min packed violating terminal of level L+1 (atomicMin)
  uint32_t seq;           // served mode: request number held by this slot
  uint32_t published;     // served mode: result written to the outbox
};

// Served mode: host-mapped request and result mailboxes, one per slot.
struct InboxEntry {
  BInst inst;             // the request (pointers into the device pool)
  uint32_t seq;           // written last by the host (release); 0 = empty
  uint32_t pad[3];
};
struct OutboxEntry {
  uint32_t seq;           // written last by the device (release)
  int32_t status;
  uint32_t holds, levels;
  uint64_t states;
  uint32_t checks, level;
  uint64_t time, t_ini, wpack;
  uint64_t key_lo, key_hi;
};
struct ServeArgs {
  InboxEntry* inbox;      // device view of host memory
  OutboxEntry* outbox;
  uint32_t* stop;         // host sets 1 to end the loop
  uint32_t* doorbell;     // host-mapped: bumped after every post
  uint32_t* seen;         // device memory: [0] last doorbell value read,
                          // [1] 1 when the inbox is to be scanned at the next plan,
                          // [2] plans so far (the doorbell is read every 8th)
  uint64_t idle_ns;       // wait for new requests this long before exiting
};

struct BatchArgs {
  BInst* inst;
  BState* state;
  uint32_t n;
  uint32_t refine;
  uint64_t* plan_prefix;  // [K + 1] task prefix over the step's active instances
  uint32_t* plan_inst;    // [K] those instances (ascending), K = *plan_count
  uint32_t* plan_count;   // K; 0 ends the launch
  uint32_t* err;          // launch-wide error word (barrier timeout)
  uint32_t* bar_lines;    // device-wide barrier lines
  uint32_t barrier_extra;
  uint32_t sim_walks;
  uint64_t sim_seed;
  uint64_t timeout_ns;
  uint32_t prune, early_exit;
  ServeArgs serve;        // inbox == nullptr: a plain batch
};

cudaError_t launch_batch(int grid, int threads, const BatchArgs& args, cudaStream_t stream);
int batch_kernel_occupancy(int threads, int* blocks_per_sm);

}  // namespace mc
