// Batched exploration: many models answered by one persistent launch.
//
// Auto-tuning asks many questions (Section 2: one check per threshold, one
// search per kernel and input size), most of them small: a single query of a
// few thousand states per BFS level leaves the GPU idle between its
// device-wide barriers.  Here every instance of a batch advances in lockstep:
// between two barriers each instance does one step of its own query program,
// and the barrier's cost is shared by all of them.
//
// Query programs (the single-model drivers of mc_api.cu, as state machines):
//   check(T)    SETUP -> EXPAND ... -> [witness scans -> TRACE] -> DONE
//   min_time    SIM -> min pass -> [certificate pass at T_min - 1] ->
//               final pass at T_min -> witness scans -> TRACE -> DONE
// The min pass keeps successors up to T_ini (with pruning) and records the
// least violating terminal of every level; a pass ends after the first level
// holding a violating terminal (early exit) or after the deepest level.
//
// Between steps, the block that completes a device-wide barrier runs the
// planner before it releases the others: it advances each instance's state
// machine from the level records the step produced and writes the prefix sum
// of the next step's tasks.  A task is one warp's unit of work: 32/group
// states of a level to expand (group = lanes per state), 32 log entries to
// scan for the witness, 256 units of set-up, 32 random runs, or the trace.
// Warps stride over the task index space; a task's instance is found by
// binary search over the prefix cached in shared memory.
//
// All instances use 128-bit keys in their own layout.  Each instance has its
// own visited set, frontier log and level records carved from one pool.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mc_cfg_jobs.h"
#include "mc_device.cuh"

namespace mc {
namespace {

using namespace mc::dev;
typedef unsigned __int128 u128;

__device__ __forceinline__ uint64_t ldcg64(const uint64_t* p) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}

// Copies of BInst / BState read from L2: in served mode a slot's request (and
// the tables it points to) can change between steps, so nothing may come
// from a stale L1 line.
// 16-byte loads, all issued before the first is used (BInst and BState are
// multiples of 16 bytes in 16-byte aligned arrays).
template <class T>
__device__ __forceinline__ void load_cg(const T* g, T& out) {
  static_assert(sizeof(T) % 16 == 0, "16-byte words");
  const ulonglong2* src = reinterpret_cast<const ulonglong2*>(g);
  ulonglong2* dst = reinterpret_cast<ulonglong2*>(&out);
#pragma unroll
  for (uint32_t k = 0; k < sizeof(T) / 16; ++k) dst[k] = __ldcg(src + k);
}

// ------------------------------------------------------------------ planner
uint64_t __host__ __device__ inline ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ uint64_t task_count(const BState& s, const BInst& I, const BatchArgs& A) {
  switch (s.phase) {
    case B_SIM: return ceil_div(A.sim_walks, 32);
    case B_SETUP: {
      uint64_t u = I.table_u64 / 2;
      u = u > (uint64_t)I.p.max_level + 2 ? u : (uint64_t)I.p.max_level + 2;
      const uint64_t init = 1 + (uint64_t)I.p.a + (uint64_t)I.p.a * I.p.b;
      u = u > init ? u : init;
      return ceil_div(u, kTaskUnits);
    }
    case B_EXPAND: return ceil_div(s.W, 32 / I.group);
    case B_WIT_HI:
    case B_WIT_LO:
    case B_WIT_IDX: return ceil_div(s.W, 32);
    case B_TRACE: return 1;
  }
  return 0;
}

__device__ void start_pass(BState& s, const BatchArgs& A, uint32_t pass, uint64_t T) {
  s.pass = pass;
  s.T = T;
  s.prune = A.prune;
  s.early_exit = pass == PASS_MIN ? 0 : A.early_exit;
  s.phase = B_SETUP;
  s.best_all = kNone;
  s.first_viol = 0;
}

__device__ void fail(BState& s, int code) {
  if (!s.err) s.err = (uint32_t)code;
  s.phase = B_DONE;
}

// The pass ends with `s.L` as its last level.
__device__ void end_pass(BState& s, const BInst& I, const BatchArgs& A) {
  s.states += s.offL + s.W;
  s.checks += 1;
  s.levels = s.L + 1;
  if (s.pass == PASS_MIN) {
    if (s.best_all == kNone) return fail(s, MC_ERR_CUDA);  // no terminal below T_ini
    s.t_min = pack_time(s.best_all);
    if (A.refine) start_pass(s, A, PASS_REFINE, s.t_min - 1);
    else start_pass(s, A, PASS_FINAL, s.t_min);
  } else if (s.pass == PASS_REFINE) {
    if (s.first_viol) return fail(s, MC_ERR_CUDA);  // certificate disagrees
    start_pass(s, A, PASS_FINAL, s.t_min);
  } else {
    s.stop_level = s.first_viol;
    if (!s.first_viol) {
      s.phase = B_DONE;
      return;
    }
    const uint32_t wl = s.first_viol;
    s.wpack = ldcg64(I.levels + 2 * wl + 1);
    s.phase = B_WIT_HI;
    s.L = wl;
    s.W = ldcg64(I.levels + 2 * wl);
    s.offL = ldcg64(I.off + wl);
    s.wkey_lo = s.wkey_hi = s.widx = kNone;
  }
}

__device__ void advance(BState& s, const BInst& I, const BatchArgs& A) {
  if (!s.started) {
    s.started = 1;
    if (I.kind == 1) {
      s.phase = B_SIM;
      s.t_ini = kNone;
    } else {
      start_pass(s, A, PASS_FINAL, I.T_query);
    }
    return;
  }
  if (s.err) {
    s.phase = B_DONE;
    return;
  }
  switch (s.phase) {
    case B_SIM:  // the min pass keeps successors up to T_ini when pruning
      start_pass(s, A, PASS_MIN, A.prune ? s.t_ini : kNone);
      break;
    case B_SETUP:
      s.phase = B_EXPAND;
      s.L = 2;
      s.W = (uint64_t)I.p.a * I.p.b;
      s.offL = 1 + (uint64_t)I.p.a;
      s.wnext = 0;
      s.bnext = kNone;
      break;
    case B_EXPAND: {
      // level L+1's counters came with the state; keep them in the level
      // records (the witness phases read them) and start the next level's
      const uint64_t Wn = s.wnext;
      const uint64_t Bn = s.bnext;
      I.levels[2 * (s.L + 1)] = Wn;
      I.levels[2 * (s.L + 1) + 1] = Bn;
      s.wnext = 0;
      s.bnext = kNone;
      if (Wn == 0) {
        end_pass(s, I, A);
        break;
      }
      if (Bn != kNone) {
        s.best_all = Bn < s.best_all ? Bn : s.best_all;
        if (!s.first_viol) s.first_viol = s.L + 1;
      }
      I.off[s.L + 1] = s.offL + s.W;
      s.offL += s.W;
      s.W = Wn;
      s.L += 1;
      if (s.L >= I.p.max_level || (s.early_exit && Bn != kNone)) end_pass(s, I, A);
      break;
    }
    case B_WIT_HI: s.phase = B_WIT_LO; break;
    case B_WIT_LO: s.phase = B_WIT_IDX; break;
    case B_WIT_IDX:
      if (s.widx >= s.W) fail(s, MC_ERR_FRONTIER);
      else s.phase = B_TRACE;
      break;
    case B_TRACE:
      s.trace_len = s.L + 1;
      s.phase = B_DONE;
      break;
    default: break;
  }
}

// Served mode: publish a finished slot's result to its host-mapped outbox
// entry (fields first, then the sequence number with release semantics).
__device__ void publish(const BatchArgs& A, uint32_t i, BState& s) {
  OutboxEntry* o = A.serve.outbox + i;
  o->status = s.err ? (int32_t)s.err : MC_OK;
  o->holds = s.stop_level == 0;
  o->levels = s.levels;
  o->states = s.states;
  o->checks = s.checks;
  o->level = s.stop_level;
  o->time = s.stop_level ? pack_time(s.wpack) : 0;
  o->t_ini = s.t_ini;
  o->wpack = s.wpack;
  o->key_lo = s.wkey_lo;
  o->key_hi = s.wkey_hi;
  __threadfence_system();
  st_release_sys_u32(&o->seq, s.seq);
  s.published = 1;
}

// Served mode: take slot i's newly posted request (if any) into the device;
// I receives its description.
__device__ void admit(const BatchArgs& A, uint32_t i, BState& s, BInst& I) {
  const InboxEntry* e = A.serve.inbox + i;
  const uint32_t seq = ld_acquire_sys_u32(&e->seq);
  if (seq == 0 || seq == s.seq) return;
  const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(&e->inst);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(A.inst + i);
  unsigned long long* loc = reinterpret_cast<unsigned long long*>(&I);
  for (uint32_t k = 0; k < sizeof(BInst) / 8; ++k) {
    const unsigned long long v = src[k];
    dst[k] = v;
    loc[k] = v;
  }
  unsigned long long* z = reinterpret_cast<unsigned long long*>(&s);
  for (uint32_t k = 0; k < sizeof(BState) / 8; ++k) z[k] = 0;
  s.seq = seq;
}

struct Planner {
  const BatchArgs* A;
  uint32_t* word;  // shared: the barrier payload describing the plan (see batch_kernel)

  // Advance every slot; returns the number of tasks of the next step and
  // writes the compact plan: the instances with tasks and their prefix.  A
  // slot with nothing to do (a finished instance; in served mode an empty or
  // published slot while the inbox is not being scanned) is recognised from
  // one word of its state and neither loaded nor written back.
  __device__ unsigned long long plan() const {
    __shared__ uint32_t s_count[kMaxBatch];
    __shared__ unsigned long long s_part[kThreads];
    __shared__ unsigned long long s_total;
    __shared__ uint32_t s_first;  // the first planned instance
    constexpr uint32_t kActShift = 48;  // (active instances << 48) + tasks, scanned together
    const bool serve = A->serve.inbox != nullptr;
    const uint32_t n = A->n;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = threadIdx.x * per, i1 = min(n, i0 + per);
    // served mode: every 8th plan reads the doorbell (host memory, a trip of
    // microseconds that would otherwise lengthen every step); the read issued
    // now is consumed at the end, so it overlaps this plan, and the inbox is
    // scanned only in a plan that follows a doorbell change.  seen[2] counts
    // plans (only planners touch it; the barriers order them).
    uint32_t db = 0;
    bool read_db = false;
    if (serve && threadIdx.x == 0) {
      const uint32_t k = __ldcg(A->serve.seen + 2);
      A->serve.seen[2] = k + 1;
      read_db = (k & 7u) == 0;
      if (read_db) db = *reinterpret_cast<const volatile uint32_t*>(A->serve.doorbell);
    }
    const bool scan_inbox = serve && __ldcg(A->serve.seen + 1) != 0;
    unsigned long long local = 0;
    for (uint32_t i = i0; i < i1; ++i) {
      // the state and the description are loaded together (one round trip
      // of L2 latency on the serial path, not three)
      BState s;
      BInst I;
      load_cg(A->state + i, s);
      load_cg(A->inst + i, I);
      const bool idle = serve ? !scan_inbox && (s.seq == 0 || s.published != 0)
                              : s.phase == B_DONE && s.started != 0;
      uint64_t c = 0;
      if (!idle) {
        if (scan_inbox) admit(*A, i, s, I);
        if (!serve || (s.seq != 0 && !s.published)) {
          advance(s, I, *A);
          c = task_count(s, I, *A);
          if (serve && s.phase == B_DONE) publish(*A, i, s);
        }
        unsigned long long* out = reinterpret_cast<unsigned long long*>(A->state + i);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&s);
        for (uint32_t k = 0; k < sizeof(BState) / 8; ++k) out[k] = src[k];
      }
      s_count[i] = (uint32_t)c;
      local += c + (c ? 1ull << kActShift : 0ull);
    }
    // block-wide exclusive scan of the per-thread (active, tasks) sums
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long incl = local;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += v;
    }
    if (lane == 31) s_part[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long run = 0;
      for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) {
        const unsigned long long v = s_part[w];
        s_part[w] = run;
        run += v;
      }
      s_total = run;
    }
    __syncthreads();
    const unsigned long long base = s_part[warp] + incl - local;
    const unsigned long long tmask = (1ull << kActShift) - 1;
    uint32_t pos = (uint32_t)(base >> kActShift);
    unsigned long long run = base & tmask;
    for (uint32_t i = i0; i < i1; ++i) {
      if (!s_count[i]) continue;
      A->plan_inst[pos] = i;
      A->plan_prefix[pos] = run;
      if (pos == 0) s_first = i;
      ++pos;
      run += s_count[i];
    }
    __syncthreads();
    const uint32_t active = (uint32_t)(s_total >> kActShift);
    const unsigned long long total = s_total & tmask;
    if (threadIdx.x == 0) {
      A->plan_prefix[active] = total;
      *A->plan_count = active;
      *word = active == 1 && s_first < 1024 && total < (1u << 21)
                  ? 1u | (s_first << 1) | ((uint32_t)total << 11)
                  : (active <= kMaxBatch ? 2u | (active << 2) : 0u);
      if (serve && read_db) {
        A->serve.seen[1] = db != __ldcg(A->serve.seen) ? 1u : 0u;
        A->serve.seen[0] = db;
      } else if (serve) {
        A->serve.seen[1] = 0;  // this plan scanned the inbox if it was asked to
      }
    }
    __syncthreads();
    return total;
  }

  // Served mode with nothing to do: wait (bounded by idle_ns) until the host
  // posts a request or asks to stop.  True when one was posted (the next
  // plan then scans the inbox).
  __device__ bool wait_for_requests() const {
    __shared__ uint32_t s_state;
    const uint64_t t0 = globaltimer();
    for (;;) {
      if (threadIdx.x == 0) {
        s_state = 0;
        if (ld_acquire_sys_u32(A->serve.stop)) {
          s_state = 2;
        } else if (__ldcg(A->serve.seen + 1) != 0) {
          s_state = 1;
        } else {
          const uint32_t db = ld_acquire_sys_u32(A->serve.doorbell);
          if (db != __ldcg(A->serve.seen)) {
            A->serve.seen[0] = db;
            A->serve.seen[1] = 1;
            s_state = 1;
          } else if (globaltimer() - t0 > A->serve.idle_ns) {
            s_state = 3;
          } else {
            __nanosleep(1000);
          }
        }
      }
      __syncthreads();
      const uint32_t st = s_state;
      __syncthreads();
      if (st == 1) return true;
      if (st >= 2) return false;
    }
  }

  __device__ void operator()() const {
    for (;;) {
      const unsigned long long total = plan();
      if (!A->serve.inbox || total > 0) {
        if (A->serve.inbox && threadIdx.x == 0 && ld_acquire_sys_u32(A->serve.stop)) {
          *A->plan_count = 0;  // the host is shutting the loop down
          *word = 2u;          // a plan of no instances
        }
        return;
      }
      if (!wait_for_requests()) return;  // total stays 0: the loop exits
    }
  }
};

// ------------------------------------------------------------------ warp staging
struct WarpBuf {
  u128 keys[kWarpCap];
  uint32_t par[kWarpCap];
};

struct Staging {
  uint32_t inst = 0xFFFFFFFFu;  // instance the buffer holds entries for
  uint32_t fill = 0;
  uint64_t offN = 0;            // log offset of the level being appended to
  uint64_t* rec = nullptr;      // {width, best} counters of that level (in the instance state)
  void* log_keys = nullptr;     // that instance's frontier log
  uint32_t* log_par = nullptr;
  uint64_t log_cap = 0;
};

__device__ void flush(const BatchArgs& A, Staging& sg, WarpBuf& wb, uint32_t lane) {
  if (sg.fill == 0) return;
  __syncwarp();
  void* log_keys = sg.log_keys;
  uint32_t* log_par = sg.log_par;
  const uint64_t log_cap = sg.log_cap;
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(reinterpret_cast<unsigned long long*>(sg.rec), (unsigned long long)sg.fill);
  b = __shfl_sync(0xffffffffu, b, 0);
  for (uint32_t x = lane; x < sg.fill; x += 32) {
    const uint64_t at = sg.offN + b + x;
    if (at < log_cap) {
      KeyOps<u128>::store(log_keys, at, wb.keys[x]);
      log_par[at] = wb.par[x];
    } else {
      set_error(&A.state[sg.inst].err, MC_ERR_FRONTIER);
    }
  }
  __syncwarp();
  sg.fill = 0;
}

// ------------------------------------------------------------------ tasks
__device__ void task_setup(const BatchArgs& A, const BInst& I, uint64_t q, uint32_t lane) {
  const Params& p = I.p;
  const uint64_t n16 = I.table_u64 / 2;
  const uint64_t nlev = (uint64_t)p.max_level + 2;
  const uint64_t ninit = 1 + (uint64_t)p.a + (uint64_t)p.a * p.b;
  ulonglong2* tb = reinterpret_cast<ulonglong2*>(I.table);
  for (uint32_t k = 0; k < kTaskUnits / 32; ++k) {
    const uint64_t u = q * kTaskUnits + k * 32 + lane;
    if (u < n16) tb[u] = make_ulonglong2(0, 0);
    if (u < nlev) {
      I.levels[2 * u] = u == 0 ? 1 : u == 1 ? p.a : u == 2 ? (uint64_t)p.a * p.b : 0;
      I.levels[2 * u + 1] = kNone;
      I.off[u] = u == 0 ? 0 : u == 1 ? 1 : u == 2 ? 1 + (uint64_t)p.a : 0;
    }
    if (u < ninit) {
      u128 key = 0;
      uint32_t par = kNoParent;
      if (u >= 1 && u <= p.a) {
        key = (u128)u << p.wg_shift;
        par = 0;
      } else if (u > p.a) {
        const uint64_t y = u - 1 - p.a;
        const uint32_t i = (uint32_t)(y / p.b), j = (uint32_t)(y % p.b);
        key = ((u128)(i + 1) << p.wg_shift) | ((u128)(j + 1) << p.ts_shift);
        par = i;
      }
      KeyOps<u128>::store(I.log_keys, u, key);
      I.log_par[u] = par;
    }
  }
}

__device__ void task_expand(const BatchArgs& A, uint32_t inst, const BInst& I, const BState& s,
                            uint64_t q, uint32_t lane, Staging& sg, WarpBuf& wb) {
  const Params& p = I.p;
  const uint32_t g = I.group;
  const uint32_t c = lane & (g - 1);
  const uint64_t sidx = q * (32 / g) + lane / g;
  const bool valid = sidx < s.W;
  const uint32_t k_cur = s.L - 2;
  const u128 key = valid ? KeyOps<u128>::load(I.log_keys, s.offL + sidx) : (u128)0;
  const uint32_t c_shift = (p.P - 1 - (c < p.P ? c : 0)) * p.n_bits;
  uint32_t i = 0, j = 0, r = 0;
  uint64_t t_c = 0, clk = 0;
  if (valid) {
    i = field(key, p.wg_shift, p.wg_mask) - 1;
    j = field(key, p.ts_shift, p.ts_mask) - 1;
    const uint32_t cfg = i * p.b + j;
    r = __ldcg(p.N + cfg) - k_cur;
    if (c < p.P) {
      t_c = (uint64_t)__ldcg(p.cost + cfg) * __ldcg(p.speed + c);
      clk = (uint64_t)field(key, c_shift, p.n_mask) * t_c;
    }
  }
  const uint64_t mx = group_max(clk, g);
  bool allowed = valid && c < p.P && r > 0;
  if (p.rule == MC_GREEDY) {
    const uint64_t mn = group_min((valid && c < p.P) ? clk : kNone, g);
    allowed = allowed && clk == mn;
  }
  const uint64_t nclk = clk + t_c;
  const uint64_t succ_time = nclk > mx ? nclk : mx;
  if (s.prune && succ_time > s.T) allowed = false;
  const u128 succ = key + ((u128)1 << c_shift);
  int won = 0;
  if (allowed) {
    const uint64_t bkt = key_hash(succ) & I.bucket_mask;
    const int rc = visited_insert<u128>(reinterpret_cast<u128*>(I.table), I.bucket_mask, I.max_probes,
                                        succ, k_cur + 1, p, bkt, nullptr);
    if (rc < 0) set_error(&A.state[inst].err, MC_ERR_TABLE_FULL);
    won = rc > 0;
  }
  const uint32_t m = __ballot_sync(0xffffffffu, won);
  if (m) {
    if (won) {
      const uint32_t at = sg.fill + __popc(m & ((1u << lane) - 1u));
      wb.keys[at] = succ;
      wb.par[at] = (uint32_t)sidx;
    }
    sg.fill += __popc(m);
    // Step 2: a terminal winner with time <= T violates G(FIN -> time > T)
    const uint64_t pk = warp_min((won && r == 1 && succ_time <= s.T) ? pack_tij(succ_time, i, j) : kNone);
    if (lane == 0 && pk != kNone)
      atomicMin(reinterpret_cast<unsigned long long*>(sg.rec + 1), (unsigned long long)pk);
  }
}

__device__ void task_witness(const BatchArgs& A, uint32_t inst, const BInst& I, const BState& s,
                             uint64_t q, uint32_t lane) {
  const Params& p = I.p;
  const uint64_t x = q * 32 + lane;
  if (x >= s.W) return;
  const u128 key = KeyOps<u128>::load(I.log_keys, s.offL + x);
  const uint64_t lo = (uint64_t)key, hi = (uint64_t)(key >> 64);
  BState* gs = A.state + inst;
  if (s.phase == B_WIT_IDX) {
    if (lo == s.wkey_lo && hi == s.wkey_hi) gs->widx = x;
    return;
  }
  const uint32_t ti = pack_i(s.wpack), tj = pack_j(s.wpack);
  if (field(key, p.wg_shift, p.wg_mask) - 1 != ti || field(key, p.ts_shift, p.ts_mask) - 1 != tj) return;
  const uint32_t cfg = ti * p.b + tj;
  if (sum_n(key, p) != __ldcg(p.N + cfg) || key_time<u128, true>(key, p, cfg) != pack_time(s.wpack))
    return;
  if (s.phase == B_WIT_HI)
    atomicMin(reinterpret_cast<unsigned long long*>(&gs->wkey_hi), (unsigned long long)hi);
  else if (hi == s.wkey_hi)
    atomicMin(reinterpret_cast<unsigned long long*>(&gs->wkey_lo), (unsigned long long)lo);
}

__device__ void task_trace(const BInst& I, const BState& s, uint32_t lane) {
  if (lane != 0) return;
  uint64_t idx = s.widx;
  uint32_t l = s.L;
  for (;;) {
    const uint64_t at = ldcg64(I.off + l) + idx;
    const u128 key = KeyOps<u128>::load(I.log_keys, at);
    I.trace[2 * l] = (uint64_t)key;
    I.trace[2 * l + 1] = (uint64_t)(key >> 64);
    if (l == 0) break;
    idx = __ldcg(I.log_par + at);
    --l;
  }
}

__device__ void task_sim(const BatchArgs& A, uint32_t inst, const BInst& I, uint64_t q, uint32_t lane) {
  const uint64_t w = q * 32 + lane;
  if (w >= A.sim_walks) return;
  const uint64_t t = simulate_walk<true>(I.p, A.sim_seed, w);
  atomicMin(reinterpret_cast<unsigned long long*>(&A.state[inst].t_ini), (unsigned long long)t);
}

// The fields of BState a task reads (written by the planner before the step).
__device__ __forceinline__ void load_state(const BState* g, BState& s) { load_cg(g, s); }

__global__ void __launch_bounds__(kThreads, 1) batch_kernel(const BatchArgs A) {
  __shared__ unsigned long long s_prefix[kMaxBatch + 1];
  __shared__ uint32_t s_inst[kMaxBatch];
  __shared__ WarpBuf s_buf[kThreads / 32];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t warp_gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const Barrier bar{A.bar_lines, A.err, A.barrier_extra, A.timeout_ns};
  // The plan's size travels in the barrier word, written by the planner: a
  // plan of one instance whole (bit 0 set, the instance in bits 1-10, its
  // task count in bits 11-31), so the blocks skip reading the plan back, and
  // a larger one as its instance count (bit 1 set, the count in bits 2-12),
  // so the blocks read the plan in one round trip instead of two.
  __shared__ uint32_t s_plan_word;
  const Planner planner{&A, &s_plan_word};
  auto plan_word = []() -> uint32_t { return s_plan_word; };
  uint32_t epoch = 0, word = 0;
  if (!grid_sync(bar, epoch, planner, plan_word, &word)) return;  // first plan
  for (;;) {
    uint32_t K;
    if (word & 1u) {
      K = 1;
      if (threadIdx.x == 0) {
        s_inst[0] = (word >> 1) & 1023u;
        s_prefix[0] = 0;
        s_prefix[1] = word >> 11;
      }
    } else {
      K = (word & 2u) ? (word >> 2) & 0x7FFu : __ldcg(A.plan_count);
      for (uint32_t i = threadIdx.x; i <= K; i += blockDim.x) {
        s_prefix[i] = __ldcg(reinterpret_cast<const unsigned long long*>(A.plan_prefix) + i);
        if (i < K) s_inst[i] = __ldcg(A.plan_inst + i);
      }
    }
    __syncthreads();
    const uint64_t total = K ? s_prefix[K] : 0;
    if (total == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) A.err[1] = epoch;  // steps of this launch
      break;
    }
    Staging sg;
    BState s;
    BInst I;
    uint32_t cur = 0xFFFFFFFFu;
    for (uint64_t t = warp_gid; t < total; t += n_warps) {
      // instance of task t: the last planned k with prefix[k] <= t (warp-uniform)
      uint32_t lo = 0, hi = K;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_prefix[mid] <= t) lo = mid;
        else hi = mid;
      }
      const uint32_t inst = s_inst[lo];
      const uint64_t q = t - s_prefix[lo];
      if (inst != cur) {
        load_state(A.state + inst, s);
        load_cg(A.inst + inst, I);
        cur = inst;
      }
      switch (s.phase) {
        case B_EXPAND:
          if (sg.inst != inst) {
            flush(A, sg, s_buf[warp], lane);
            sg.inst = inst;
            sg.offN = s.offL + s.W;
            sg.rec = &A.state[inst].wnext;  // {wnext, bnext}
            sg.log_keys = I.log_keys;
            sg.log_par = I.log_par;
            sg.log_cap = I.log_cap;
          }
          task_expand(A, inst, I, s, q, lane, sg, s_buf[warp]);
          if (sg.fill > kWarpCap - 32) flush(A, sg, s_buf[warp], lane);
          break;
        case B_SETUP: task_setup(A, I, q, lane); break;
        case B_SIM: task_sim(A, inst, I, q, lane); break;
        case B_WIT_HI:
        case B_WIT_LO:
        case B_WIT_IDX: task_witness(A, inst, I, s, q, lane); break;
        case B_TRACE: task_trace(I, s, lane); break;
        default: break;
      }
    }
    flush(A, sg, s_buf[warp], lane);
    if (!grid_sync(bar, epoch, planner, plan_word, &word)) return;
  }
}

}  // namespace

cudaError_t launch_batch(int grid, int threads, const BatchArgs& args, cudaStream_t stream) {
  void* params[] = {const_cast<BatchArgs*>(&args)};
  return cudaLaunchCooperativeKernel((const void*)batch_kernel, dim3(grid), dim3(threads), params, 0,
                                     stream);
}

int batch_kernel_occupancy(int threads, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)batch_kernel,
                                                       threads, 0) == cudaSuccess
             ? 0
             : -1;
}

}  // namespace mc

// ====================================================================== host API
namespace {

struct BatchBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

uint64_t al256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

struct mc_batch {
  uint32_t n = 0;
  mc_options opt{};
  std::vector<mc::BInst> inst;        // host copy; pointers filled at reserve
  std::vector<mc_layout> lay;
  std::vector<std::vector<uint32_t>> params;  // N, cost, speed per instance
  std::vector<std::vector<uint32_t>> wg, ts;
  std::vector<uint64_t> pool_off;     // byte offset of each instance's region
  uint64_t pool_bytes = 0;
  bool reserved = false;
  int device = -1, grid = 0, threads = 0;
  cudaStream_t stream = nullptr;
  mc_alloc_fn alloc = nullptr;
  mc_free_fn dealloc = nullptr;
  void* actx = nullptr;
  std::vector<BatchBuf> bufs;
  uint8_t* d_pool = nullptr;
  mc::BInst* d_inst = nullptr;
  mc::BState* d_state = nullptr;
  uint64_t* d_prefix = nullptr;
  uint32_t* d_ctrl = nullptr;         // err word, then the barrier lines
  // pinned staging: the instances uploaded, the states read back, and the
  // launch's {error, steps} words; a run is replayed from a CUDA graph
  mc::BInst* h_inst = nullptr;
  mc::BState* h_state = nullptr;
  uint32_t* h_ctrl2 = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;           // a refused capture leaves graph null
  cudaEvent_t ev[2] = {};
  mc_stats stats{};
  std::string last_err;
  // configuration engine (every instance one block per configuration)
  uint32_t engine = MC_ENGINE_LEVEL;
  std::vector<mc::CfgModelPrep> cm;
  mc::CfgRun run;
  uint8_t* h_run = nullptr;           // pinned mirror of the run block
  int cfg_grid = 0, cfg_threads = 0;
  uint32_t cfg_wcap = 32;
  size_t cfg_smem = 0;
  std::vector<uint32_t> trace_len;    // per instance, from the last run
};

namespace {

int bfail(mc_batch* b, cudaError_t e, const char* what) {
  b->last_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return MC_ERR_CUDA;
}

#define MCB_CUDA(b, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return bfail((b), e_, #call);   \
  } while (0)

void* balloc(mc_batch* b, size_t bytes) {
  bytes = al256(bytes ? bytes : 256);
  void* p = nullptr;
  if (b->alloc) p = b->alloc(bytes, (void*)b->stream, b->actx);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->bufs.push_back({p, bytes});
  return p;
}

void brelease(mc_batch* b) {
  if (!b->bufs.empty()) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (b->device >= 0 && prev != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    for (const BatchBuf& x : b->bufs) {
      if (b->dealloc) b->dealloc(x.ptr, x.bytes, (void*)b->stream, b->actx);
      else cudaFree(x.ptr);
    }
    b->bufs.clear();
    if (b->device >= 0 && prev >= 0 && prev != b->device) cudaSetDevice(prev);
  }
  for (cudaEvent_t& e : b->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->h_inst) cudaFreeHost(b->h_inst);
  if (b->h_state) cudaFreeHost(b->h_state);
  if (b->h_ctrl2) cudaFreeHost(b->h_ctrl2);
  if (b->h_run) cudaFreeHost(b->h_run);
  b->h_run = nullptr;
  b->graph = nullptr;
  b->graph_tried = false;
  b->cap_stream = nullptr;
  b->h_inst = nullptr;
  b->h_state = nullptr;
  b->h_ctrl2 = nullptr;
  b->reserved = false;
}

// Layout, tables and region size of one model as a batch or server instance.
int describe_instance(const mc_model_desc& d_in, const mc_options& o, mc::BInst& I, mc_layout& L,
                      std::vector<uint32_t>& pr, uint64_t& region_bytes) {
  mc_model_desc d = d_in;
  d.key_bits = 128;  // every instance uses 128-bit keys
  mc_options lo = o;
  lo.engine = MC_ENGINE_LEVEL;  // the lockstep engine's layout and buffers
  mc_model* m = nullptr;
  int rc = mc_model_create(&d, &lo, &m);
  if (rc) return rc;
  rc = mc_model_layout(m, &L);
  mc_model_destroy(m);
  if (rc) return rc;
  if (L.log_capacity == UINT64_MAX || L.table_slots == 0) return MC_ERR_NOMEM;
  const uint64_t ab = (uint64_t)d.n_wg * d.n_ts;
  pr.assign(d.n_workgroups, d.n_workgroups + ab);
  pr.insert(pr.end(), d.cost, d.cost + ab);
  for (uint32_t c = 0; c < d.P; ++c) pr.push_back(d.speed ? d.speed[c] : 1);
  std::memset(&I, 0, sizeof(I));
  mc::Params& p = I.p;
  p.a = d.n_wg;
  p.b = d.n_ts;
  p.P = d.P;
  p.rule = d.rule;
  p.n_bits = L.n_bits;
  p.ts_shift = L.ts_shift;
  p.wg_shift = L.wg_shift;
  p.ts_mask = (1u << L.ts_bits) - 1;
  p.wg_mask = (1u << L.wg_bits) - 1;
  p.max_level = L.max_level;
  p.n_mask = (1ull << L.n_bits) - 1;
  const uint32_t nf = d.P * L.n_bits;
  p.swar_ok = nf <= 64;
  p.swar_mask = nf >= 64 ? ~0ull : ((1ull << nf) - 1);
  for (uint32_t t = 0; t < d.P && t * L.n_bits < 64; ++t) p.swar_mul |= 1ull << (t * L.n_bits);
  I.bucket_mask = L.table_slots / 2 - 1;
  I.table_u64 = L.table_slots * 2;
  I.log_cap = L.log_capacity;
  I.max_probes = o.max_probes ? o.max_probes : (uint32_t)std::min<uint64_t>(L.table_slots / 2, 0xFFFFFFFFu);
  I.group = 1;
  while (I.group < d.P) I.group <<= 1;
  const uint64_t L2 = L.max_level + 2;
  region_bytes = al256(pr.size() * 4) + al256(16 * L2) + al256(8 * L2) + al256(16 * L2) +
                 al256(16 * L.table_slots) + al256(16 * L.log_capacity) + al256(4 * L.log_capacity);
  return MC_OK;
}

// Point an instance at its region: [tables][levels][off][trace][visited set][log keys][log parents].
void place_instance(mc::BInst& I, const mc_layout& L, uint8_t* q, size_t n_params) {
  const uint64_t ab = (uint64_t)I.p.a * I.p.b;
  I.p.N = (const uint32_t*)q;
  I.p.cost = (const uint32_t*)q + ab;
  I.p.speed = (const uint32_t*)q + 2 * ab;
  q += al256(n_params * 4);
  const uint64_t L2 = L.max_level + 2;
  I.levels = (uint64_t*)q;
  q += al256(16 * L2);
  I.off = (uint64_t*)q;
  q += al256(8 * L2);
  I.trace = (uint64_t*)q;
  q += al256(16 * L2);
  I.table = q;
  q += al256(16 * L.table_slots);
  I.log_keys = q;
  q += al256(16 * L.log_capacity);
  I.log_par = (uint32_t*)q;
}

// The configuration engine's batch: one pool holding every instance's region
// and the run block; the instances' tables and segment starts uploaded once.
int breserve_cfg(mc_batch* b) {
  MCB_CUDA(b, cudaGetDevice(&b->device));
  int sms = 0, bps = 0;
  MCB_CUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  uint64_t units = 0;
  b->cfg_threads = 64;
  b->cfg_wcap = 32;
  for (const mc::CfgModelPrep& M : b->cm) {
    units += M.ab;
    if (mc::cfg_warp_model(M, b->opt)) continue;  // a warp per configuration: no block shape
    b->cfg_threads = std::max<int>(b->cfg_threads, (int)M.threads);
    b->cfg_wcap = std::max(b->cfg_wcap, M.wcap);
  }
  if (b->opt.unit_threads) b->cfg_threads = (int)b->opt.unit_threads;
  b->cfg_smem = mc::cfg_smem_bytes(2, b->cfg_wcap, 2 * b->cfg_wcap);
  if (mc::cfg_occupancy(2, b->cfg_threads, b->cfg_smem, &bps) || bps < 1) {
    b->last_err = "occupancy query failed (configuration engine)";
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  if (b->opt.blocks_per_sm) bps = std::min<int>(bps, (int)b->opt.blocks_per_sm);
  b->cfg_grid = (int)std::min<uint64_t>((uint64_t)sms * bps, std::max<uint64_t>(units * 2, 1));
  b->d_pool = (uint8_t*)balloc(b, b->pool_bytes);
  if (!b->d_pool) {
    brelease(b);
    return MC_ERR_NOMEM;
  }
  const uint64_t run_bytes = mc::CfgRun::block_bytes(b->n, units);
  const uint64_t run_off = b->pool_bytes - run_bytes;
  if (cudaMallocHost((void**)&b->h_run, run_bytes) != cudaSuccess) {
    cudaGetLastError();
    brelease(b);
    return MC_ERR_NOMEM;
  }
  b->run.layout(b->n, units, b->d_pool + run_off, b->h_run);
  for (cudaEvent_t& e : b->ev) MCB_CUDA(b, cudaEventCreate(&e));
  MCB_CUDA(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  for (uint32_t i = 0; i < b->n; ++i) {
    mc::CfgModelPrep& M = b->cm[i];
    mc::cfg_place(M, b->d_pool + b->pool_off[i]);
    MCB_CUDA(b, cudaMemcpyAsync(M.base, M.params.data(), 4 * M.params.size(), cudaMemcpyHostToDevice, b->stream));
    MCB_CUDA(b, cudaMemcpyAsync(M.d_seg, M.seg.data(), 8 * M.seg.size(), cudaMemcpyHostToDevice, b->stream));
    b->stats.h2d_bytes += 4 * M.params.size() + 8 * M.seg.size();
  }
  MCB_CUDA(b, cudaStreamSynchronize(b->stream));
  b->trace_len.assign(b->n, 0);
  b->reserved = true;
  return MC_OK;
}

int breserve(mc_batch* b) {
  if (b->reserved) return MC_OK;
  if (b->engine == MC_ENGINE_CONFIG) return breserve_cfg(b);
  MCB_CUDA(b, cudaGetDevice(&b->device));
  int sms = 0, coop = 0, bps = 0;
  MCB_CUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  MCB_CUDA(b, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device));
  b->threads = (int)mc::kThreads;
  if (!coop || mc::batch_kernel_occupancy(b->threads, &bps) || bps < 1) {
    b->last_err = "cooperative launch unavailable";
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  if (b->opt.blocks_per_sm) bps = std::min<int>(bps, (int)b->opt.blocks_per_sm);
  b->grid = sms * bps;
  b->d_pool = (uint8_t*)balloc(b, b->pool_bytes);
  b->d_inst = (mc::BInst*)balloc(b, sizeof(mc::BInst) * b->n);
  b->d_state = (mc::BState*)balloc(b, sizeof(mc::BState) * b->n);
  b->d_prefix = (uint64_t*)balloc(b, 12ull * (b->n + 1));  // prefix, instance list, count
  b->d_ctrl = (uint32_t*)balloc(b, 256 + mc::kBarBytes);
  if (!b->d_pool || !b->d_inst || !b->d_state || !b->d_prefix || !b->d_ctrl) {
    brelease(b);
    return MC_ERR_NOMEM;
  }
  for (cudaEvent_t& e : b->ev) MCB_CUDA(b, cudaEventCreate(&e));
  if (cudaMallocHost((void**)&b->h_inst, sizeof(mc::BInst) * b->n) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_state, sizeof(mc::BState) * b->n) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_ctrl2, 64) != cudaSuccess) {
    cudaGetLastError();
    brelease(b);
    return MC_ERR_NOMEM;
  }
  MCB_CUDA(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  // carve each instance's region and upload its tables
  for (uint32_t i = 0; i < b->n; ++i) {
    uint8_t* q = b->d_pool + b->pool_off[i];
    const size_t np = b->params[i].size();
    MCB_CUDA(b, cudaMemcpyAsync(q, b->params[i].data(), np * 4, cudaMemcpyHostToDevice, b->stream));
    b->stats.h2d_bytes += np * 4;
    place_instance(b->inst[i], b->lay[i], q, np);
  }
  MCB_CUDA(b, cudaStreamSynchronize(b->stream));
  b->reserved = true;
  return MC_OK;
}

}  // namespace

namespace {

// One batch run on the configuration engine: the run's descriptors go to
// the pinned mirror, then the captured sequence (upload, clear, simulate,
// both pass launches, read-back) is replayed; where capture is refused the
// sequence is enqueued directly.
int batch_run_cfg(mc_batch* b, const mc_query* queries, mc_batch_result* results) {
  std::vector<mc::CfgModelPrep*> ms(b->n);
  for (uint32_t i = 0; i < b->n; ++i) ms[i] = &b->cm[i];
  b->run.prepare(ms, queries, b->opt);
  b->run.threads = b->cfg_threads;  // the launch shape of the reservation
  b->run.wcap = b->cfg_wcap;
  b->run.tsize = 2 * b->cfg_wcap;
  cudaEvent_t e0 = b->opt.timing ? b->ev[0] : nullptr, e1 = b->opt.timing ? b->ev[1] : nullptr;
  if (!b->graph_tried) {
    b->graph_tried = true;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t e1c = b->run.enqueue(b->cap_stream, b->cfg_grid, b->cfg_grid, b->cfg_smem, e0, e1, true);
      const cudaError_t e2c = cudaStreamEndCapture(b->cap_stream, &g);
      if (e1c == cudaSuccess && e2c == cudaSuccess && g && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess)
        b->graph = nullptr;
      if (e1c != cudaSuccess || e2c != cudaSuccess) b->graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a refused capture is not an error of the run
  }
  if (b->graph) {
    MCB_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->stats.graph_launches += 1;
  } else {
    MCB_CUDA(b, b->run.enqueue(b->stream, b->cfg_grid, b->cfg_grid, b->cfg_smem, e0, e1, false));
  }
  MCB_CUDA(b, cudaStreamSynchronize(b->stream));
  b->stats.h2d_bytes += b->run.upload_bytes;
  b->stats.d2h_bytes += b->run.result_bytes;
  b->stats.explore_launches += 2;
  b->stats.other_launches += 2;
  if (b->opt.timing) {
    float ms = 0.f;
    MCB_CUDA(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    b->stats.explore_ms += ms;
  }
  uint32_t deepest = 0;
  for (uint32_t i = 0; i < b->n; ++i) {
    uint64_t states = 0;
    b->run.result(b->cm[i], i, queries[i], results[i], &b->trace_len[i], &states);
    b->stats.states += states;
    deepest = std::max(deepest, results[i].levels);
  }
  b->stats.device_steps += deepest;
  return MC_OK;
}

}  // namespace

extern "C" {

int mc_batch_create(const mc_model_desc* descs, uint32_t n, const mc_options* opt, mc_batch** out) {
  if (!descs || !out || n == 0 || n > mc::kMaxBatch) return MC_ERR_INVAL;
  *out = nullptr;
  mc_options o;
  if (opt) o = *opt;
  else mc_options_default(&o);
  mc_batch* b = new (std::nothrow) mc_batch;
  if (!b) return MC_ERR_NOMEM;
  b->n = n;
  b->opt = o;
  if (o.engine != MC_ENGINE_LEVEL) {
    // the configuration engine when it takes every instance
    b->cm.resize(n);
    bool all = true;
    uint64_t off = 0, units = 0;
    b->pool_off.resize(n);
    b->wg.resize(n);
    b->ts.resize(n);
    for (uint32_t i = 0; i < n && all; ++i) {
      const int rc = mc::cfg_prepare(descs[i], o, b->cm[i]);
      if (rc == MC_ERR_INVAL && o.engine == MC_ENGINE_AUTO) {
        mc_model_desc d = descs[i];  // a malformed description stays an error
        mc_model* m = nullptr;
        const int rc2 = mc_model_create(&d, &o, &m);
        mc_model_destroy(m);
        if (rc2) {
          delete b;
          return rc2;
        }
        all = false;
        break;
      }
      if (rc) {
        delete b;
        return rc;
      }
      b->pool_off[i] = off;
      off += b->cm[i].region;
      units += b->cm[i].ab;
      b->wg[i] = b->cm[i].wg;
      b->ts[i] = b->cm[i].ts;
    }
    if (all) {
      b->engine = MC_ENGINE_CONFIG;
      b->pool_bytes = off + mc::CfgRun::block_bytes(n, units);
      *out = b;
      return MC_OK;
    }
    b->cm.clear();
  }
  b->inst.resize(n);
  b->lay.resize(n);
  b->params.resize(n);
  b->wg.resize(n);
  b->ts.resize(n);
  b->pool_off.resize(n);
  uint64_t off = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const mc_model_desc& d = descs[i];
    uint64_t bytes = 0;
    const int rc = describe_instance(d, o, b->inst[i], b->lay[i], b->params[i], bytes);
    if (rc) {
      delete b;
      return rc;
    }
    if (d.wg_values) b->wg[i].assign(d.wg_values, d.wg_values + d.n_wg);
    if (d.ts_values) b->ts[i].assign(d.ts_values, d.ts_values + d.n_ts);
    b->pool_off[i] = off;
    off += bytes;
  }
  b->pool_bytes = off;
  *out = b;
  return MC_OK;
}

void mc_batch_destroy(mc_batch* b) {
  if (!b) return;
  brelease(b);
  delete b;
}

int mc_batch_set_stream(mc_batch* b, void* stream) {
  if (!b) return MC_ERR_INVAL;
  b->stream = (cudaStream_t)stream;
  return MC_OK;
}

int mc_batch_set_allocator(mc_batch* b, mc_alloc_fn alloc, mc_free_fn free_fn, void* ctx) {
  if (!b || !alloc || !free_fn || b->reserved) return MC_ERR_INVAL;
  b->alloc = alloc;
  b->dealloc = free_fn;
  b->actx = ctx;
  return MC_OK;
}

int mc_batch_device_bytes(const mc_batch* b, uint64_t* out) {
  if (!b || !out) return MC_ERR_INVAL;
  *out = b->pool_bytes;
  return MC_OK;
}

int mc_batch_run(mc_batch* b, const mc_query* queries, mc_batch_result* results) {
  if (!b || !queries || !results) return MC_ERR_INVAL;
  for (uint32_t i = 0; i < b->n; ++i)
    if (queries[i].kind > MC_QUERY_MIN_TIME) return MC_ERR_INVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (b->device >= 0 && prev != b->device) cudaSetDevice(b->device);
  int rc = breserve(b);
  if (rc) return rc;
  if (b->engine == MC_ENGINE_CONFIG) {
    rc = batch_run_cfg(b, queries, results);
    if (b->device >= 0 && prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
  }
  for (uint32_t i = 0; i < b->n; ++i) {
    b->inst[i].kind = queries[i].kind;
    b->inst[i].T_query = queries[i].T;
  }
  mc::BatchArgs A{};
  A.inst = b->d_inst;
  A.state = b->d_state;
  A.n = b->n;
  A.refine = b->opt.refine;
  A.plan_prefix = b->d_prefix;
  A.plan_inst = reinterpret_cast<uint32_t*>(b->d_prefix + b->n + 1);
  A.plan_count = A.plan_inst + b->n;
  A.err = b->d_ctrl;
  A.bar_lines = b->d_ctrl + 64;
  A.barrier_extra = b->opt.debug_barrier_extra;
  A.sim_walks = b->opt.sim_walks;
  A.sim_seed = b->opt.sim_seed;
  A.timeout_ns = b->opt.barrier_timeout_ns ? b->opt.barrier_timeout_ns : 60ull * 1000000000ull;
  A.prune = b->opt.prune;
  A.early_exit = b->opt.early_exit;
  std::copy(b->inst.begin(), b->inst.end(), b->h_inst);
  // The run's sequence -- upload the instances, clear states and control,
  // the persistent launch, read the states and {error, steps} back -- is
  // captured once into a CUDA graph on a private stream and replayed on the
  // batch's stream; only the pinned inputs change between runs.  Where the
  // capture is refused, the sequence is enqueued directly.
  auto enqueue = [&](cudaStream_t st, bool capturing) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(mc::BInst) * b->n, cudaMemcpyHostToDevice, st)))
      return e;
    if ((e = cudaMemsetAsync(b->d_state, 0, sizeof(mc::BState) * b->n, st))) return e;
    if ((e = cudaMemsetAsync(b->d_ctrl, 0, 256 + mc::kBarBytes, st))) return e;
    if (b->opt.timing &&
        (e = capturing ? cudaEventRecordWithFlags(b->ev[0], st, cudaEventRecordExternal) : cudaEventRecord(b->ev[0], st)))
      return e;
    if ((e = mc::launch_batch(b->grid, b->threads, A, st))) return e;
    if (b->opt.timing &&
        (e = capturing ? cudaEventRecordWithFlags(b->ev[1], st, cudaEventRecordExternal) : cudaEventRecord(b->ev[1], st)))
      return e;
    if ((e = cudaMemcpyAsync(b->h_state, b->d_state, sizeof(mc::BState) * b->n, cudaMemcpyDeviceToHost, st)))
      return e;
    return cudaMemcpyAsync(b->h_ctrl2, b->d_ctrl, 8, cudaMemcpyDeviceToHost, st);
  };
  if (!b->graph_tried) {
    b->graph_tried = true;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t e1 = enqueue(b->cap_stream, true);
      const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
      if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
          cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess)
        b->graph = nullptr;
      if (e1 != cudaSuccess || e2 != cudaSuccess) b->graph = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a refused capture is not an error of the run
  }
  if (b->graph) {
    MCB_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->stats.graph_launches += 1;
  } else {
    MCB_CUDA(b, enqueue(b->stream, false));
  }
  b->stats.h2d_bytes += sizeof(mc::BInst) * b->n;
  MCB_CUDA(b, cudaStreamSynchronize(b->stream));
  const uint32_t ctrl2[2] = {b->h_ctrl2[0], b->h_ctrl2[1]};  // launch error word, steps of the launch
  b->stats.d2h_bytes += sizeof(mc::BState) * b->n + 8;
  b->stats.explore_launches += 1;
  b->stats.device_steps += ctrl2[1];
  const uint32_t err = ctrl2[0];
  if (b->opt.timing) {
    float ms = 0.f;
    MCB_CUDA(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    b->stats.explore_ms += ms;
  }
  if (b->device >= 0 && prev >= 0 && prev != b->device) cudaSetDevice(prev);
  if (err) return (int)err;
  for (uint32_t i = 0; i < b->n; ++i) {
    const mc::BState& s = b->h_state[i];
    mc_batch_result& r = results[i];
    std::memset(&r, 0, sizeof(r));
    r.status = s.err ? (int)s.err : (s.phase == mc::B_DONE ? MC_OK : MC_ERR_CUDA);
    r.kind = queries[i].kind;
    r.states = s.states;
    r.checks = s.checks;
    r.levels = s.levels;
    r.t_ini = queries[i].kind == MC_QUERY_MIN_TIME ? s.t_ini : 0;
    r.holds = s.stop_level == 0;
    b->stats.states += s.states;
    if (s.stop_level) {
      r.time = mc::pack_time(s.wpack);
      r.wg_index = mc::pack_i(s.wpack);
      r.ts_index = mc::pack_j(s.wpack);
      r.wg = b->wg[i].empty() ? r.wg_index : b->wg[i][r.wg_index];
      r.ts = b->ts[i].empty() ? r.ts_index : b->ts[i][r.ts_index];
      r.level = s.stop_level;
      r.key[0] = s.wkey_lo;
      r.key[1] = s.wkey_hi;
    }
  }
  return MC_OK;
}

int mc_batch_trace(mc_batch* b, uint32_t i, uint64_t* keys, uint32_t cap, uint32_t* len) {
  if (!b || !len || i >= b->n || (!keys && cap)) return MC_ERR_INVAL;
  if (b->engine == MC_ENGINE_CONFIG) {
    *len = b->reserved ? b->trace_len[i] : 0;
    if (!b->reserved || *len == 0 || cap == 0) return MC_OK;
    const uint32_t k = std::min(cap, *len);
    MCB_CUDA(b, cudaMemcpyAsync(keys, b->cm[i].d_trace, 16ull * k, cudaMemcpyDeviceToHost, b->stream));
    MCB_CUDA(b, cudaStreamSynchronize(b->stream));
    b->stats.d2h_bytes += 16ull * k;
    return MC_OK;
  }
  const mc::BState& s = b->h_state[i];
  *len = s.trace_len;
  if (!b->reserved || s.trace_len == 0 || cap == 0) return MC_OK;
  const uint32_t k = std::min(cap, s.trace_len);
  MCB_CUDA(b, cudaMemcpyAsync(keys, b->inst[i].trace, 16ull * k, cudaMemcpyDeviceToHost, b->stream));
  MCB_CUDA(b, cudaStreamSynchronize(b->stream));
  b->stats.d2h_bytes += 16ull * k;
  return MC_OK;
}

int mc_batch_get_stats(const mc_batch* b, mc_stats* out) {
  if (!b || !out) return MC_ERR_INVAL;
  *out = b->stats;
  return MC_OK;
}

const char* mc_batch_last_error(const mc_batch* b) { return b ? b->last_err.c_str() : ""; }

}  // extern "C"

// ====================================================================== served queries
// A request loop over the batched engine: the device runs the persistent
// lockstep loop with slots; its planner admits requests the host posts into
// host-mapped inbox entries at every barrier and publishes finished results
// to host-mapped outbox entries, so requests that arrive while others are
// on the GPU join them at the next step.  A host thread (the pump) admits
// queued requests when a slot and enough of the device pool are free
// (first fit over the pool, by each request's closed-form bound), harvests
// results, and relaunches the device loop when it has exited after being
// idle.  Visited sets, frontier logs and tables stay resident in the pool.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First fit over [0, size), offsets and sizes multiples of 256 bytes.
struct RegionAlloc {
  std::map<uint64_t, uint64_t> free_;  // offset -> bytes
  void init(uint64_t size) {
    free_.clear();
    free_[0] = size;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes, o2 = it->first + bytes;
      free_.erase(it);
      if (rest) free_[o2] = rest;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    auto it = free_.emplace(off, bytes).first;
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

struct Request {
  uint64_t ticket = 0;
  mc_query q{};
  mc::BInst inst{};
  mc_layout lay{};
  std::vector<uint32_t> params, wg, ts;
  uint64_t bytes = 0;
  double t_submit = 0;
  bool cfg = false;         // runs in a configuration-engine job
  mc::CfgModelPrep cm;      // its layout there (tables travel with the job)
};

// A configuration-engine job: requests admitted together, answered by one
// run on the job's own stream; jobs on different streams overlap on the
// device.
struct CfgJob {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t* d_block = nullptr;
  uint8_t* h_block = nullptr;
  mc::CfgRun run;
  std::vector<Request> reqs;
  std::vector<uint64_t> offs;
  std::vector<mc_query> qs;
  bool busy = false;
  double t_admit = 0;
};

constexpr uint32_t kJobs = 8;             // job streams
constexpr uint32_t kJobModels = 256;      // requests per job at most
constexpr uint64_t kJobUnits = 1u << 16;  // configurations per job at most
constexpr uint64_t kJobTables = 8ull << 20;  // bytes of model tables per job

struct SlotInfo {
  bool busy = false;
  uint32_t seq = 0;
  uint64_t off = 0;
  double t_admit = 0;
  Request req;
};

}  // namespace

struct mc_server {
  mc_server_config cfg{};
  mc_options opt{};
  int device = -1, grid = 0, threads = 0;
  cudaStream_t stream = nullptr, copy = nullptr;
  uint8_t* d_pool = nullptr;
  mc::BInst* d_inst = nullptr;
  mc::BState* d_state = nullptr;
  uint64_t* d_prefix = nullptr;
  uint32_t* d_ctrl = nullptr;
  mc::InboxEntry *h_inbox = nullptr, *d_inbox = nullptr;
  mc::OutboxEntry *h_outbox = nullptr, *d_outbox = nullptr;
  uint32_t *h_stop = nullptr, *d_stop = nullptr;
  uint32_t *h_doorbell = nullptr, *d_doorbell = nullptr;  // inside the h_stop allocation
  uint32_t* d_seen = nullptr;
  cudaEvent_t kdone = nullptr;
  bool kernel_running = false;
  uint64_t launches = 0;
  uint64_t solo_states = 0;  // requests at most this large may run alone
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<Request> queue;
  std::vector<SlotInfo> slots;
  RegionAlloc pool;
  std::deque<mc_server_result> done;
  uint64_t next_ticket = 1;
  uint32_t next_seq = 1;
  std::vector<CfgJob> jobs;
  std::map<uint64_t, int> cfg_grid;  // (threads << 32 | frontier capacity) -> blocks of a launch
  int sms = 0;
  uint32_t jobs_running = 0;
  std::thread pump;
  std::atomic<bool> shutdown{false};
  int fatal = 0;
  std::string last_err;
};

namespace {

void finish_slot(mc_server* S, uint32_t i, const mc::OutboxEntry& o, int status_override) {
  SlotInfo& sl = S->slots[i];
  mc_server_result res;
  std::memset(&res, 0, sizeof(res));
  res.ticket = sl.req.ticket;
  mc_batch_result& r = res.result;
  r.status = status_override ? status_override : o.status;
  r.kind = sl.req.q.kind;
  r.holds = o.holds;
  r.levels = o.levels;
  r.states = o.states;
  r.checks = o.checks;
  r.level = o.level;
  r.time = o.time;
  r.t_ini = sl.req.q.kind == MC_QUERY_MIN_TIME ? o.t_ini : 0;
  if (o.level) {
    r.wg_index = mc::pack_i(o.wpack);
    r.ts_index = mc::pack_j(o.wpack);
    r.wg = sl.req.wg.empty() ? r.wg_index : sl.req.wg[r.wg_index];
    r.ts = sl.req.ts.empty() ? r.ts_index : sl.req.ts[r.ts_index];
    r.key[0] = o.key_lo;
    r.key[1] = o.key_hi;
  }
  res.submit_s = sl.req.t_submit;
  res.admit_s = sl.t_admit;
  res.done_s = now_s();
  S->done.push_back(res);
  S->pool.release(sl.off, sl.req.bytes);
  sl.busy = false;
}

int launch_server(mc_server* S) {
  mc::BatchArgs A{};
  A.inst = S->d_inst;
  A.state = S->d_state;
  A.n = S->cfg.slots;
  A.refine = S->opt.refine;
  A.plan_prefix = S->d_prefix;
  A.plan_inst = reinterpret_cast<uint32_t*>(S->d_prefix + S->cfg.slots + 1);
  A.plan_count = A.plan_inst + S->cfg.slots;
  A.err = S->d_ctrl;
  A.bar_lines = S->d_ctrl + 64;
  A.barrier_extra = 0;
  A.sim_walks = S->opt.sim_walks;
  A.sim_seed = S->opt.sim_seed;
  A.timeout_ns = S->opt.barrier_timeout_ns ? S->opt.barrier_timeout_ns : 60ull * 1000000000ull;
  A.prune = S->opt.prune;
  A.early_exit = S->opt.early_exit;
  A.serve.inbox = S->d_inbox;
  A.serve.outbox = S->d_outbox;
  A.serve.stop = S->d_stop;
  A.serve.doorbell = S->d_doorbell;
  A.serve.seen = S->d_seen;
  A.serve.idle_ns = S->cfg.idle_ns ? S->cfg.idle_ns : 200000ull;
  if (cudaMemsetAsync(S->d_ctrl, 0, 256 + mc::kBarBytes, S->stream) != cudaSuccess ||
      mc::launch_batch(S->grid, S->threads, A, S->stream) != cudaSuccess ||
      cudaEventRecord(S->kdone, S->stream) != cudaSuccess) {
    S->last_err = cudaGetErrorString(cudaGetLastError());
    return MC_ERR_CUDA;
  }
  S->kernel_running = true;
  S->launches += 1;
  return MC_OK;
}

// Latency path: one request on an idle server runs on the single-model
// explorer (mc_api.cu), whose BFS level costs about half a lockstep step.
// Its buffers come from the server's pool through a bump allocator; options
// are the server's with search SINGLE, so every field of the result equals
// what the device loop would report.  Returns false (request untouched) when
// the pool has no room, and the request then takes the device loop.
struct Bump {
  uint8_t* base;
  uint64_t size, used;
};
void* bump_alloc(size_t bytes, void*, void* ctx) {
  Bump* b = static_cast<Bump*>(ctx);
  const uint64_t at = (b->used + 255) & ~255ull;
  if (at + bytes > b->size) return nullptr;
  b->used = at + bytes;
  return b->base + at;
}
void bump_free(void*, size_t, void*, void*) {}

bool run_alone(mc_server* S, Request& req, mc_server_result& res) {
  const uint64_t ab = (uint64_t)req.inst.p.a * req.inst.p.b;
  mc_model_desc d{};
  d.n_wg = req.inst.p.a;
  d.n_ts = req.inst.p.b;
  d.P = req.inst.p.P;
  d.wg_values = req.wg.empty() ? nullptr : req.wg.data();
  d.ts_values = req.ts.empty() ? nullptr : req.ts.data();
  d.n_workgroups = req.params.data();
  d.cost = req.params.data() + ab;
  d.speed = req.params.data() + 2 * ab;
  d.rule = req.inst.p.rule;
  d.key_bits = 128;
  mc_options o = S->opt;
  o.search = MC_SEARCH_SINGLE;
  o.timing = 0;
  mc_model* m = nullptr;
  if (mc_model_create(&d, &o, &m) != MC_OK) return false;
  mc_layout L;
  mc_model_layout(m, &L);
  const uint64_t bytes = L.device_bytes + 16 * 256;
  uint64_t off = 0;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (!S->pool.alloc(bytes, &off)) {
      mc_model_destroy(m);
      return false;
    }
  }
  Bump bump{S->d_pool + off, bytes, 0};
  mc_set_allocator(m, bump_alloc, bump_free, &bump);
  mc_set_stream(m, S->stream);
  std::memset(&res, 0, sizeof(res));
  res.ticket = req.ticket;
  res.submit_s = req.t_submit;
  res.admit_s = now_s();
  res.path = 1;
  mc_batch_result& r = res.result;
  r.kind = req.q.kind;
  if (req.q.kind == MC_QUERY_MIN_TIME) {
    mc_min_result mr;
    r.status = mc_min_time(m, &mr, nullptr);
    if (r.status == MC_OK) {
      uint32_t levels = 0;
      mc_last_widths(m, nullptr, 0, &levels);
      r.holds = 0;
      r.levels = levels;
      r.states = mr.states;
      r.checks = mr.checks;
      r.level = mr.level;
      r.time = mr.t_min;
      r.t_ini = mr.t_ini;
      r.wg_index = mr.wg_index;
      r.ts_index = mr.ts_index;
      r.wg = mr.wg;
      r.ts = mr.ts;
      r.key[0] = mr.witness_key[0];
      r.key[1] = mr.witness_key[1];
    }
  } else {
    mc_check_result cr;
    r.status = mc_check(m, req.q.T, &cr, nullptr);
    if (r.status == MC_OK) {
      r.holds = cr.holds;
      r.levels = cr.levels;
      r.states = cr.states;
      r.checks = 1;
      if (!cr.holds) {
        r.level = cr.cex_level;
        r.time = cr.cex_time;
        r.wg_index = cr.cex_wg_index;
        r.ts_index = cr.cex_ts_index;
        r.wg = cr.cex_wg;
        r.ts = cr.cex_ts;
        r.key[0] = cr.cex_key[0];
        r.key[1] = cr.cex_key[1];
      }
    }
  }
  mc_model_destroy(m);  // waits for the model's work on the server stream
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->pool.release(off, bytes);
  }
  res.done_s = now_s();
  return true;
}

// Blocks of a configuration-engine launch for a job's launch shape (the
// occupancy maximum, cached per shape).
int job_grid(mc_server* S, uint32_t threads, uint32_t wcap, size_t* smem) {
  *smem = mc::cfg_smem_bytes(2, wcap, 2 * wcap);
  const uint64_t key = ((uint64_t)threads << 32) | wcap;
  auto it = S->cfg_grid.find(key);
  if (it != S->cfg_grid.end()) return it->second;
  int bps = 0;
  if (mc::cfg_occupancy(2, (int)threads, *smem, &bps) || bps < 1) {
    cudaGetLastError();
    return 0;
  }
  if (S->opt.blocks_per_sm) bps = std::min<int>(bps, (int)S->opt.blocks_per_sm);
  const int g = S->sms * bps;
  S->cfg_grid[key] = g;
  return g;
}

// Harvest finished jobs (caller holds S->mu).  Returns true on progress.
bool harvest_jobs(mc_server* S) {
  bool progress = false;
  for (CfgJob& j : S->jobs) {
    if (!j.busy) continue;
    const cudaError_t q = cudaEventQuery(j.done);
    if (q == cudaErrorNotReady) continue;
    const double t = now_s();
    for (size_t k = 0; k < j.reqs.size(); ++k) {
      Request& req = j.reqs[k];
      mc_server_result res;
      std::memset(&res, 0, sizeof(res));
      res.ticket = req.ticket;
      if (q == cudaSuccess) {
        j.run.result(req.cm, (uint32_t)k, j.qs[k], res.result, nullptr, nullptr);
      } else {
        res.result.status = MC_ERR_CUDA;
        res.result.kind = req.q.kind;
      }
      res.submit_s = req.t_submit;
      res.admit_s = j.t_admit;
      res.done_s = t;
      res.path = 2;
      S->done.push_back(res);
      S->pool.release(j.offs[k], req.bytes);
    }
    if (q != cudaSuccess) {
      S->fatal = MC_ERR_CUDA;
      S->last_err = cudaGetErrorString(q);
      cudaGetLastError();
    }
    j.reqs.clear();
    j.offs.clear();
    j.qs.clear();
    j.busy = false;
    S->jobs_running -= 1;
    progress = true;
  }
  return progress;
}

// Admit queued configuration-engine requests (from the front of the queue,
// in arrival order) into free jobs while the pool has room for their
// regions; each job is launched at once.  Caller holds S->mu.
bool admit_jobs(mc_server* S) {
  bool progress = false;
  for (CfgJob& j : S->jobs) {
    if (S->queue.empty() || !S->queue.front().cfg || S->fatal) break;
    if (j.busy) continue;
    j.run.tables_used = 0;
    uint64_t units = 0;
    while (!S->queue.empty() && S->queue.front().cfg && j.reqs.size() < kJobModels) {
      Request& req = S->queue.front();
      if (units + req.cm.ab > kJobUnits && !j.reqs.empty()) break;
      uint64_t off = 0;
      if (!S->pool.alloc(req.bytes, &off)) break;
      if (!j.run.place_tables(req.cm)) {
        S->pool.release(off, req.bytes);
        break;
      }
      mc::cfg_place_state(req.cm, S->d_pool + off);
      units += req.cm.ab;
      j.offs.push_back(off);
      j.qs.push_back(req.q);
      j.reqs.push_back(std::move(req));
      S->queue.pop_front();
    }
    if (j.reqs.empty()) break;  // the front request waits for pool room
    std::vector<mc::CfgModelPrep*> ms(j.reqs.size());
    for (size_t k = 0; k < j.reqs.size(); ++k) ms[k] = &j.reqs[k].cm;
    j.run.prepare(ms, j.qs.data(), S->opt);
    size_t smem = 0;
    const int grid = job_grid(S, j.run.threads, j.run.wcap, &smem);
    const int ga = (int)std::min<uint64_t>((uint64_t)grid, std::max<uint64_t>(j.run.n_units_a, 1));
    const int gb = (int)std::min<uint64_t>((uint64_t)grid, std::max<uint64_t>(j.run.n_units_b, 1));
    j.t_admit = now_s();
    if (!grid || j.run.enqueue(j.stream, ga, gb, smem, nullptr, nullptr, false) != cudaSuccess ||
        cudaEventRecord(j.done, j.stream) != cudaSuccess) {
      S->fatal = MC_ERR_CUDA;
      S->last_err = cudaGetErrorString(cudaGetLastError());
    }
    j.busy = true;
    S->jobs_running += 1;
    S->launches += 1;
    progress = true;
  }
  return progress;
}

// Requests waiting on an idle server that still take the latency path one
// after another (FIFO); a longer queue goes to the device loop, where the
// requests share its steps.
constexpr size_t kSoloQueue = 2;

void pump_loop(mc_server* S) {
  cudaSetDevice(S->device);
  const uint32_t n = S->cfg.slots;
  while (!S->shutdown.load()) {
    bool progress = false;
    {  // configuration-engine jobs: harvest finished ones, launch new ones
      std::lock_guard<std::mutex> g(S->mu);
      progress |= harvest_jobs(S);
      progress |= admit_jobs(S);
    }
    if (progress) S->cv_done.notify_all();
    {  // latency path for a lone request on an idle server
      std::unique_lock<std::mutex> g(S->mu);
      bool idle = !S->fatal && !S->kernel_running && !S->queue.empty() && S->queue.size() <= kSoloQueue &&
                  !S->queue.front().cfg && S->queue.front().lay.state_bound <= S->solo_states;
      for (uint32_t i = 0; i < n && idle; ++i) idle = !S->slots[i].busy;
      if (idle) {
        Request req = std::move(S->queue.front());
        S->queue.pop_front();
        g.unlock();
        mc_server_result res;
        const bool ran = run_alone(S, req, res);
        g.lock();
        if (ran) {
          S->done.push_back(res);
          g.unlock();
          S->cv_done.notify_all();
          continue;
        }
        S->queue.push_front(std::move(req));  // no pool room: take the device loop
      }
    }
    {
      std::lock_guard<std::mutex> g(S->mu);
      // harvest published results
      for (uint32_t i = 0; i < n; ++i) {
        SlotInfo& sl = S->slots[i];
        if (!sl.busy) continue;
        if (__atomic_load_n(&S->h_outbox[i].seq, __ATOMIC_ACQUIRE) != sl.seq) continue;
        mc::OutboxEntry o = S->h_outbox[i];
        finish_slot(S, i, o, 0);
        progress = true;
      }
      // admit queued requests in arrival order while a slot and pool room are free
      uint32_t scan = 0;
      while (!S->queue.empty() && !S->fatal && !S->queue.front().cfg) {
        while (scan < n && S->slots[scan].busy) ++scan;
        if (scan == n) break;
        Request& req = S->queue.front();
        uint64_t off = 0;
        if (!S->pool.alloc(req.bytes, &off)) break;
        uint8_t* base = S->d_pool + off;
        place_instance(req.inst, req.lay, base, req.params.size());
        req.inst.kind = req.q.kind;
        req.inst.T_query = req.q.T;
        if (cudaMemcpyAsync(base, req.params.data(), req.params.size() * 4, cudaMemcpyHostToDevice,
                            S->copy) != cudaSuccess ||
            cudaStreamSynchronize(S->copy) != cudaSuccess) {
          S->fatal = MC_ERR_CUDA;
          S->last_err = cudaGetErrorString(cudaGetLastError());
          S->pool.release(off, req.bytes);
          break;
        }
        mc::InboxEntry& e = S->h_inbox[scan];
        std::memcpy((void*)&e.inst, &req.inst, sizeof(mc::BInst));
        const uint32_t seq = S->next_seq++;
        if (S->next_seq == 0) S->next_seq = 1;
        __atomic_store_n(&e.seq, seq, __ATOMIC_RELEASE);
        __atomic_add_fetch(S->h_doorbell, 1u, __ATOMIC_RELEASE);
        SlotInfo& sl = S->slots[scan];
        sl.busy = true;
        sl.seq = seq;
        sl.off = off;
        sl.t_admit = now_s();
        sl.req = std::move(req);
        S->queue.pop_front();
        progress = true;
      }
      // keep the device loop running while a slot is busy
      bool any_busy = false;
      for (uint32_t i = 0; i < n && !any_busy; ++i) any_busy = S->slots[i].busy;
      if (S->kernel_running) {
        const cudaError_t q = cudaEventQuery(S->kdone);
        if (q == cudaSuccess) {
          S->kernel_running = false;
          uint32_t err = 0;
          if (cudaMemcpyAsync(&err, S->d_ctrl, 4, cudaMemcpyDeviceToHost, S->copy) == cudaSuccess &&
              cudaStreamSynchronize(S->copy) == cudaSuccess && err)
            S->fatal = (int)err;
        } else if (q != cudaErrorNotReady) {
          S->fatal = MC_ERR_CUDA;
          S->last_err = cudaGetErrorString(q);
          S->kernel_running = false;
        }
      }
      if (S->fatal) {  // fail every request in flight or queued
        mc::OutboxEntry none{};
        for (uint32_t i = 0; i < n; ++i)
          if (S->slots[i].busy) finish_slot(S, i, none, S->fatal);
        for (CfgJob& j : S->jobs)
          if (j.busy) cudaStreamSynchronize(j.stream);
        harvest_jobs(S);
        while (!S->queue.empty()) {
          mc_server_result res;
          std::memset(&res, 0, sizeof(res));
          res.ticket = S->queue.front().ticket;
          res.result.status = S->fatal;
          res.result.kind = S->queue.front().q.kind;
          res.submit_s = S->queue.front().t_submit;
          res.done_s = now_s();
          S->done.push_back(res);
          S->queue.pop_front();
        }
        progress = true;
      } else if (any_busy && !S->kernel_running) {
        if (launch_server(S)) S->fatal = MC_ERR_CUDA;
      }
    }
    if (progress) S->cv_done.notify_all();
    else if (S->jobs_running) std::this_thread::sleep_for(std::chrono::microseconds(2));  // a job is due soon
    else std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void server_free(mc_server* S) {
  if (S->h_stop) __atomic_store_n(S->h_stop, 1u, __ATOMIC_RELEASE);
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (CfgJob& j : S->jobs) {
    if (j.stream) cudaStreamSynchronize(j.stream);
    if (j.d_block) cudaFree(j.d_block);
    if (j.h_block) cudaFreeHost(j.h_block);
    if (j.done) cudaEventDestroy(j.done);
    if (j.stream) cudaStreamDestroy(j.stream);
  }
  S->jobs.clear();
  if (S->d_pool) cudaFree(S->d_pool);
  if (S->d_inst) cudaFree(S->d_inst);
  if (S->d_state) cudaFree(S->d_state);
  if (S->d_prefix) cudaFree(S->d_prefix);
  if (S->d_ctrl) cudaFree(S->d_ctrl);
  if (S->d_seen) cudaFree(S->d_seen);
  if (S->h_inbox) cudaFreeHost(S->h_inbox);
  if (S->h_outbox) cudaFreeHost(S->h_outbox);
  if (S->h_stop) cudaFreeHost(S->h_stop);
  if (S->kdone) cudaEventDestroy(S->kdone);
  if (S->stream) cudaStreamDestroy(S->stream);
  if (S->copy) cudaStreamDestroy(S->copy);
}

}  // namespace

extern "C" {

int mc_server_create(const mc_server_config* cfg, const mc_options* opt, mc_server** out) {
  if (!cfg || !out || cfg->slots == 0 || cfg->slots > mc::kMaxBatch || cfg->pool_bytes < (1u << 20))
    return MC_ERR_INVAL;
  *out = nullptr;
  mc_server* S = new (std::nothrow) mc_server;
  if (!S) return MC_ERR_NOMEM;
  S->cfg = *cfg;
  if (opt) S->opt = *opt;
  else mc_options_default(&S->opt);
  S->solo_states = cfg->solo_states ? cfg->solo_states : (1ull << 22);
  const uint32_t n = cfg->slots;
  S->slots.resize(n);
  S->pool.init(cfg->pool_bytes);
  int sms = 0, coop = 0, bps = 0;
  auto bad = [&](int code) {
    cudaGetLastError();
    server_free(S);
    delete S;
    return code;
  };
  if (cudaGetDevice(&S->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, S->device) != cudaSuccess || !coop)
    return bad(MC_ERR_CUDA);
  S->sms = sms;
  if (S->opt.engine != MC_ENGINE_LEVEL) {
    // configuration-engine jobs: a stream, an event, a run block and its
    // pinned mirror each
    S->jobs.resize(kJobs);
    const uint64_t jb = mc::CfgRun::block_bytes(kJobModels, kJobUnits, kJobTables);
    for (CfgJob& j : S->jobs) {
      if (cudaStreamCreateWithFlags(&j.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming) != cudaSuccess)
        return bad(MC_ERR_CUDA);
      if (cudaMalloc((void**)&j.d_block, jb) != cudaSuccess || cudaMallocHost((void**)&j.h_block, jb) != cudaSuccess)
        return bad(MC_ERR_NOMEM);
      j.run.layout(kJobModels, kJobUnits, j.d_block, j.h_block, kJobTables);
    }
  }
  S->threads = (int)mc::kThreads;
  if (mc::batch_kernel_occupancy(S->threads, &bps) || bps < 1) return bad(MC_ERR_CUDA);
  // the served loop's steps are short and latency-bound: one block per SM
  // (the cheapest device-wide barrier) unless the options ask otherwise
  bps = S->opt.blocks_per_sm ? std::min<int>(bps, (int)S->opt.blocks_per_sm) : 1;
  S->grid = sms * bps;
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming) != cudaSuccess)
    return bad(MC_ERR_CUDA);
  if (cudaMalloc(&S->d_pool, cfg->pool_bytes) != cudaSuccess ||
      cudaMalloc(&S->d_inst, sizeof(mc::BInst) * n) != cudaSuccess ||
      cudaMalloc(&S->d_state, sizeof(mc::BState) * n) != cudaSuccess ||
      cudaMalloc(&S->d_prefix, 12ull * (n + 1)) != cudaSuccess ||
      cudaMalloc(&S->d_ctrl, 256 + mc::kBarBytes) != cudaSuccess ||
      cudaMalloc(&S->d_seen, 256) != cudaSuccess)
    return bad(MC_ERR_NOMEM);
  if (cudaHostAlloc((void**)&S->h_inbox, sizeof(mc::InboxEntry) * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_outbox, sizeof(mc::OutboxEntry) * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_stop, 64, cudaHostAllocMapped) != cudaSuccess)
    return bad(MC_ERR_NOMEM);
  std::memset(S->h_inbox, 0, sizeof(mc::InboxEntry) * n);
  std::memset(S->h_outbox, 0, sizeof(mc::OutboxEntry) * n);
  std::memset(S->h_stop, 0, 64);
  S->h_doorbell = S->h_stop + 8;  // its own 32 bytes of the same mapped allocation
  if (cudaHostGetDevicePointer((void**)&S->d_inbox, S->h_inbox, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&S->d_outbox, S->h_outbox, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&S->d_stop, S->h_stop, 0) != cudaSuccess ||
      !(S->d_doorbell = S->d_stop + 8) ||
      cudaMemsetAsync(S->d_seen, 0, 256, S->stream) != cudaSuccess ||
      cudaMemsetAsync(S->d_state, 0, sizeof(mc::BState) * n, S->stream) != cudaSuccess ||
      cudaStreamSynchronize(S->stream) != cudaSuccess)
    return bad(MC_ERR_CUDA);
  S->pump = std::thread(pump_loop, S);
  *out = S;
  return MC_OK;
}

int mc_server_submit(mc_server* S, const mc_model_desc* desc, const mc_query* q, uint64_t* ticket) {
  if (!S || !desc || !q || q->kind > MC_QUERY_MIN_TIME) return MC_ERR_INVAL;
  Request req;
  req.t_submit = now_s();
  req.q = *q;
  int rc = MC_ERR_INVAL;
  if (S->opt.engine != MC_ENGINE_LEVEL) {
    // the configuration engine when it takes the model and it fits a job
    rc = mc::cfg_prepare(*desc, S->opt, req.cm);
    if (rc == MC_OK && (req.cm.ab > kJobUnits || mc::cfg_tables_bytes(req.cm) > kJobTables)) rc = MC_ERR_INVAL;
    if (rc == MC_OK) {
      req.cfg = true;
      req.bytes = req.cm.region - mc::cfg_tables_bytes(req.cm);
    } else if (rc != MC_ERR_INVAL || S->opt.engine == MC_ENGINE_CONFIG) {
      return rc;
    }
  }
  if (!req.cfg) {
    rc = describe_instance(*desc, S->opt, req.inst, req.lay, req.params, req.bytes);
    if (rc) return rc;
  }
  if (req.bytes > S->cfg.pool_bytes) return MC_ERR_NOMEM;
  if (desc->wg_values) req.wg.assign(desc->wg_values, desc->wg_values + desc->n_wg);
  if (desc->ts_values) req.ts.assign(desc->ts_values, desc->ts_values + desc->n_ts);
  std::lock_guard<std::mutex> g(S->mu);
  if (S->fatal) return S->fatal;
  req.ticket = S->next_ticket++;
  if (ticket) *ticket = req.ticket;
  S->queue.push_back(std::move(req));
  return MC_OK;
}

int mc_server_poll(mc_server* S, mc_server_result* out, uint32_t cap, uint32_t* n, uint32_t wait_ms) {
  if (!S || !n || (!out && cap)) return MC_ERR_INVAL;
  std::unique_lock<std::mutex> g(S->mu);
  if (S->done.empty() && wait_ms)
    S->cv_done.wait_for(g, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  uint32_t k = 0;
  while (k < cap && !S->done.empty()) {
    out[k++] = S->done.front();
    S->done.pop_front();
  }
  *n = k;
  return MC_OK;
}

int mc_server_status(mc_server* S, uint32_t* queued, uint32_t* running, uint64_t* launches) {
  if (!S) return MC_ERR_INVAL;
  std::lock_guard<std::mutex> g(S->mu);
  if (queued) *queued = (uint32_t)S->queue.size();
  if (running) {
    uint32_t r = 0;
    for (const SlotInfo& sl : S->slots) r += sl.busy;
    for (const CfgJob& j : S->jobs) r += (uint32_t)j.reqs.size();
    *running = r;
  }
  if (launches) *launches = S->launches;
  return S->fatal;
}

void mc_server_destroy(mc_server* S) {
  if (!S) return;
  S->shutdown.store(true);
  if (S->pump.joinable()) S->pump.join();
  server_free(S);
  delete S;
}

}  // extern "C"
