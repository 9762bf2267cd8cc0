// The exploration pass of the level-synchronous engine, shared by the
// translation units that instantiate it (mc_kernels.cu: the split and
// one-call inserts; mc_explore_cas.cu: the CAS-first inserts).
//
// Device side of the explorer: one persistent, cooperatively launched kernel
// per exploration pass, plus the simulation kernel that gives T_ini.
//
// Layout in HBM (one model):
//   frontier log   keys (u64 or 2 x u64) and u32 parent indices of every kept
//                  state, level after level; a state's parent index points
//                  into the previous level, so the log doubles as the BFS tree
//                  the counterexample trace is read from (Section 4, Step 4).
//   visited set    open addressing, 32-byte buckets (4 u64 keys or 2 u128
//                  keys), linear probing over buckets, lock-free atomicCAS
//                  insert.  The key 0 (s0) marks an empty slot.
//   control block  per-level widths, log offsets, minima of packed
//                  (time, i, j) over violating terminals, the trace buffer.
//
// Tagged frontier log (keys with at least 8 spare top bits per 64-bit word):
// every pass stores its log keys with its own tag in the top bits of each
// word (a 128-bit key is split into two halves of 64 - tag_bits bits), and at the end of
// a level a block arrives at the barrier and reserves the log space for its
// warps' remaining winners in one atomic, then writes them.  Readers of the
// next level therefore check the tag of every entry they load and, if the
// entry is not yet this pass's, load it again (bounded by the barrier
// timeout).  A position is written once per pass, so a matching tag means
// the entry is the one this pass wrote; each 8-byte word is written and read
// whole, so a 16-byte entry whose two tags match is whole too.  The host
// clears the log when a model reserves its buffers and whenever the tag
// counter wraps.  Without spare bits the blocks reserve first, write, and
// arrive with a release reduction, so the barrier alone orders the entries.
//
// Why a per-pass table that is never cleared between levels: every
// transition raises sum(n) by one (the WG/TS selects sit at levels 1 and 2
// and are written directly), so a state can only be generated again within
// its own BFS level.  A slot holding a key of an earlier level is therefore
// as good as empty: insertion treats it as free and overwrites it with CAS.
// Keys of one level never leave the table during that level, so two threads
// inserting the same key walk the same probe sequence and meet at the same
// slot.  The table only has to hold one level (sized from the widest level),
// and nothing is cleared between levels.  (The CAS-first-with-clearing probe
// scheme empties a key's first slot when its state is expanded, one level
// after it was inserted: the table then holds about two levels' keys, and a
// first probe meets an empty slot far more often in deep searches over small
// tables; the rule above is unchanged.)
#pragma once
#include <cstdint>

#include "mc_device.cuh"

namespace mc {
namespace {

using namespace mc::dev;


// The frontier log is streamed: a level's entries are written once and read
// once, by the next level.  Its loads and stores ask L2 to evict their lines
// first, so the visited set's lines, where a successor proposed again soon
// finds its key, stay longer (measured: C3 at G=36 259.4 -> 258.0 ms, at
// G=24 12.36 -> 12.25 ms; C2 at G=80, whose table and log share L2, the same).
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
template <class K>
struct LogIO;
template <>
struct LogIO<uint64_t> {
  __device__ static uint64_t load(const void* base, uint64_t i, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v)
                 : "l"(reinterpret_cast<const uint64_t*>(base) + i), "l"(pol));
    return v;
  }
  __device__ static void store(void* base, uint64_t i, uint64_t k, uint64_t pol) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.u64 [%0], %1, %2;" ::
                 "l"(reinterpret_cast<uint64_t*>(base) + i), "l"(k), "l"(pol) : "memory");
  }
};
template <>
struct LogIO<u128> {
  __device__ static u128 load(const void* base, uint64_t i, uint64_t pol) {
    uint64_t lo, hi;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(lo), "=l"(hi)
                 : "l"(reinterpret_cast<const ulonglong2*>(base) + i), "l"(pol));
    return ((u128)hi << 64) | lo;
  }
  __device__ static void store(void* base, uint64_t i, u128 k, uint64_t pol) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::
                 "l"(reinterpret_cast<ulonglong2*>(base) + i), "l"((uint64_t)k), "l"((uint64_t)(k >> 64)), "l"(pol)
                 : "memory");
  }
};
__device__ __forceinline__ void st_u32_ef(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.u32 [%0], %1, %2;" :: "l"(p), "r"(v), "l"(pol) : "memory");
}

// How a key is stored in a tagged frontier log (see the top of this file).
template <class K>
struct LogTag;

template <>
struct LogTag<uint64_t> {  // payload in the low 64 - tb bits, the tag above
  __device__ static uint64_t pack(uint64_t k, uint32_t tb, uint64_t tag) { return tb ? k | (tag << (64 - tb)) : k; }
  __device__ static bool unpack(uint64_t& k, uint32_t tb, uint64_t tag) {
    if ((k >> (64 - tb)) != tag) return false;
    k &= ~0ull >> tb;
    return true;
  }
};

template <>
struct LogTag<u128> {  // each 64-bit word: 64 - tb payload bits, then the tag
  __device__ static u128 pack(u128 k, uint32_t tb, uint64_t tag) {
    if (!tb) return k;
    const uint32_t pb = 64 - tb;
    const uint64_t m = ~0ull >> tb;
    const uint64_t lo = ((uint64_t)k & m) | (tag << pb);
    const uint64_t hi = ((uint64_t)(k >> pb) & m) | (tag << pb);
    return ((u128)hi << 64) | lo;
  }
  __device__ static bool unpack(u128& k, uint32_t tb, uint64_t tag) {
    const uint32_t pb = 64 - tb;
    const uint64_t lo = (uint64_t)k, hi = (uint64_t)(k >> 64);
    if ((lo >> pb) != tag || (hi >> pb) != tag) return false;
    const uint64_t m = ~0ull >> tb;
    k = ((u128)(hi & m) << pb) | (lo & m);
    return true;
  }
};

// ------------------------------------------------------------------ expansion of one level
// Winners are staged per warp in shared memory.  A warp whose buffer is
// nearly full reserves log slots with one global atomicAdd and copies the
// buffer out coalesced; at the end of the level the block reserves one range
// for the remainders of all its warps.  Within a level no block-wide
// synchronisation happens, so warps run their rounds independently.
template <class K>
struct Stage {
  K keys[kThreads / 32][kStageCap];
  uint32_t par[kThreads / 32][kStageCap];
  uint32_t fill[kThreads / 32];
  unsigned long long base;
  uint32_t flags;  // this level: kFlagError | kFlagViolation
};

constexpr uint32_t kFlagError = 1;
constexpr uint32_t kFlagViolation = 2;

template <class K>
__device__ __forceinline__ void copy_out(const ExploreArgs& A, const K* keys, const uint32_t* par,
                                         uint32_t n, uint64_t at0, uint32_t lane, uint32_t* flags) {
  const uint64_t pol = evict_first_policy();
  for (uint32_t x = lane; x < n; x += 32) {
    const uint64_t at = at0 + x;
    if (at < A.log_cap) {
      LogIO<K>::store(A.log_keys, at, LogTag<K>::pack(keys[x], A.tag_bits, A.tag), pol);
      st_u32_ef(A.log_par + at, par[x], pol);
    } else {
      set_error(A.ctrl, MC_ERR_FRONTIER);
      atomicOr(flags, kFlagError);
    }
  }
}

// The key of log entry `pos` of this pass from a first load `key`: in a
// tagged log, loaded again until it carries this pass's tag, then stripped.
// False (and MC_ERR_TIMEOUT) when it does not appear within the barrier
// timeout.
template <class K>
__device__ __forceinline__ bool log_entry(const ExploreArgs& A, uint64_t pos, K& key) {
  if (!A.tag_bits || LogTag<K>::unpack(key, A.tag_bits, A.tag)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    __nanosleep(64);
    key = KeyOps<K>::load(A.log_keys, pos);
    if (LogTag<K>::unpack(key, A.tag_bits, A.tag)) return true;
    if (globaltimer() - t0 > A.timeout_ns) {
      set_error(A.ctrl, MC_ERR_TIMEOUT);
      return false;
    }
  }
}

// A tile of TILE >= P lanes handles kDepth states per round; lane c proposes,
// for each of them, the successor in which unit c takes the next work-group
// (Listings 4-5): FREE allows every unit, GREEDY only the units with the
// smallest clock.  With the split and one-call schemes the first
// visited-set bucket of every proposal is fetched with cp.async into this
// thread's slice of shared memory, all kDepth at once, so the probes are in
// flight together without holding registers; then each is resolved (a hit
// is a duplicate; otherwise CAS into the first free slot).  The CAS-first
// scheme skips the fetch (see the insert below).  Winners are staged and
// appended to the next level of the frontier log, and a winner that is
// terminal (FIN, Listing 4) with time <= T updates the level's minimum
// packed (time, i, j) -- the property G(FIN -> time > T) of Step 2.  The
// keys of the next round are loaded before the current round's probes.
// SCHEME is the probe scheme (mc_probe_scheme, resolved).
template <class K, int TILE, int RULE, int SCHEME>
__device__ __forceinline__ void expand_level(const ExploreArgs& A, Stage<K>& st, uint64_t T,
                                             uint32_t L, uint64_t offL, uint64_t W, uint64_t offN,
                                             const K (&first)[kDepth], bool have_first, uint32_t stop_mask) {
  constexpr int S = KeyOps<K>::kSlots;
  constexpr uint32_t D = kDepth;
  constexpr bool kCas = SCHEME == MC_PROBE_CAS_FIRST || SCHEME == MC_PROBE_CAS_CLEAR;
  __shared__ __align__(16) K probe[kThreads][D][S];
  const Params& p = A.p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t c = lane & (TILE - 1);
  constexpr uint32_t kTilesPerWarp = 32 / TILE;
  const uint64_t warp_gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * kTilesPerWarp * D;
  const uint32_t k_cur = L - 2;  // sum of n at level L
  const uint32_t c_shift = (p.P - 1 - (c < p.P ? c : 0)) * p.n_bits;
  const uint64_t speed_c = c < p.P ? __ldg(p.speed + c) : 0;
  K* table = reinterpret_cast<K*>(A.table);
  K* wkeys = st.keys[warp];
  uint32_t* wpar = st.par[warp];
  uint64_t* lvl_next = A.levels + 2 * (L + 1);  // {width, best} of level L+1
  uint64_t cached_best = kNone;
  uint32_t fill = 0;  // warp-uniform
  auto level_of = [&p](K k) { return sum_n(k, p); };

  uint64_t base = warp_gid * kTilesPerWarp * D;
  const uint64_t my = lane / TILE;
  const uint64_t lpol = evict_first_policy();
  K key_next[D];
#pragma unroll
  for (uint32_t d = 0; d < D; ++d) {
    const uint64_t s = base + d * kTilesPerWarp + my;
    key_next[d] = s < W ? (have_first ? first[d] : LogIO<K>::load(A.log_keys, offL + s, lpol)) : (K)0;
  }
  for (; base < W; base += stride) {
    K succ[D];
    uint64_t succ_time[D], bkt[D];
    uint32_t ij[D];
    bool allowed[D], terminal[D];
#pragma unroll
    for (uint32_t d = 0; d < D; ++d) {
      const uint64_t s = base + d * kTilesPerWarp + my;
      bool valid = s < W;
      K key = key_next[d];
      if (s + stride < W) key_next[d] = LogIO<K>::load(A.log_keys, offL + s + stride, lpol);
      if (valid && !log_entry<K>(A, offL + s, key)) {
        valid = false;
        atomicOr(&st.flags, kFlagError);
      }
      uint32_t i = 0, j = 0, r = 0;
      uint64_t t_c = 0, clk = 0;
      // CAS-first with clearing: this state's key (inserted during the
      // previous level) leaves its first slot, so the slot is empty for the
      // next level's keys; the compare-and-swap only removes this very key,
      // never a key of the level being built, and its result is not used
      if (SCHEME == MC_PROBE_CAS_CLEAR && valid && c == 0)
        (void)slot_cas(table + (key_hash(key) & A.bucket_mask) * S, key, (K)0);
      if (valid) {
        i = field(key, p.wg_shift, p.wg_mask) - 1;
        j = field(key, p.ts_shift, p.ts_mask) - 1;
        const uint32_t cfg = i * p.b + j;
        r = __ldg(p.N + cfg) - k_cur;
        if (c < p.P) {
          t_c = (uint64_t)__ldg(p.cost + cfg) * speed_c;
          clk = (uint64_t)field(key, c_shift, p.n_mask) * t_c;
        }
      }
      const uint64_t mx = tile_max<TILE>(clk);
      bool ok = valid && c < p.P && r > 0;
      if (RULE == MC_GREEDY) {
        const uint64_t mn = tile_min<TILE>((valid && c < p.P) ? clk : kNone);
        ok = ok && clk == mn;
      }
      const uint64_t nclk = clk + t_c;
      succ_time[d] = nclk > mx ? nclk : mx;
      if (A.prune && succ_time[d] > T) ok = false;
      allowed[d] = ok;
      terminal[d] = r == 1;
      ij[d] = (i << 16) | j;
      succ[d] = key + ((K)1 << c_shift);
      bkt[d] = key_hash(succ[d]) & A.bucket_mask;
      if (ok && !kCas) {
        const K* src = table + bkt[d] * S;
        cp_async16(&probe[threadIdx.x][d][0], src);
        cp_async16(reinterpret_cast<char*>(&probe[threadIdx.x][d][0]) + 16,
                   reinterpret_cast<const char*>(src) + 16);
      }
    }
    if (!kCas) cp_async_wait_all();
    // Split: pick a slot for every proposal from the fetched bucket, issue
    // all of their CAS, and only then look at the results, with the general
    // insert (rereading the bucket) when the slot went to another key or the
    // bucket is full.  One call: each proposal takes the general insert from
    // the fetched bucket directly.  (Measured: the split form is 8% faster
    // on C2 at G=80 with 64-bit keys and 2-3% slower per level with 128-bit
    // keys, which is why the default follows the key width.)  CAS-first: the
    // CAS from empty on the first slot of the first bucket, unfetched.  If
    // it succeeds the key was nowhere in its probe sequence (a key placed
    // further along means the slots before it held keys of this level when
    // it was placed, and those stay for the whole level); if it returns the
    // key, a duplicate; a key of an earlier level, one more compare-and-swap
    // from it (below); anything else takes the general insert, which
    // rereads the bucket.
    constexpr bool kPicked = SCHEME == MC_PROBE_SPLIT || kCas;
    uint32_t pick[D];
    K cur[D], old[D];
#pragma unroll
    for (uint32_t d = 0; d < D; ++d) {
      pick[d] = allowed[d] ? kPickFull : kPickDup;
      if (SCHEME == MC_PROBE_SPLIT && allowed[d])
        pick[d] = bucket_pick<K>(probe[threadIdx.x][d], succ[d], k_cur + 1, level_of, cur[d]);
      if (kCas && allowed[d]) {
        pick[d] = 0;
        cur[d] = (K)0;
      }
    }
#pragma unroll
    for (uint32_t d = 0; d < D; ++d)
      if (kPicked && pick[d] < (uint32_t)S) old[d] = slot_cas(table + bkt[d] * S + pick[d], cur[d], succ[d]);
    // CAS-first, when the first slot returned a key of an earlier level: the
    // slot is free, and the key is in no slot of this level (a slot taken
    // this level keeps its key until the level ends, so an earlier insert of
    // the key would have stopped at this one), so compare-and-swap once more
    // from the value returned instead of rereading the bucket
    if (kCas) {
#pragma unroll
      for (uint32_t d = 0; d < D; ++d)
        if (pick[d] == 0 && old[d] != cur[d] && old[d] != succ[d] && level_of(old[d]) <= k_cur) {
          cur[d] = old[d];
          old[d] = slot_cas(table + bkt[d] * S, cur[d], succ[d]);
        }
    }
#pragma unroll
    for (uint32_t d = 0; d < D; ++d) {
      const uint64_t s = base + d * kTilesPerWarp + my;
      int won = 0;
      if (kPicked && pick[d] < (uint32_t)S) {
        if (old[d] == cur[d]) won = 1;
        else if (old[d] != succ[d]) pick[d] = kPickFull;  // the slot went to another key
      }
      if (pick[d] == kPickFull) {
        const int rc = visited_insert<K>(table, A.bucket_mask, A.max_probes, succ[d], k_cur + 1, p, bkt[d],
                                         kPicked ? nullptr : probe[threadIdx.x][d]);
        if (rc < 0) {
          set_error(A.ctrl, MC_ERR_TABLE_FULL);
          atomicOr(&st.flags, kFlagError);
        }
        won = rc > 0;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, won);
      if (m) {
        if (won) {
          const uint32_t at = fill + __popc(m & ((1u << lane) - 1u));
          wkeys[at] = succ[d];
          wpar[at] = (uint32_t)s;
        }
        fill += __popc(m);
        // Step 2: a terminal winner with time <= T violates G(FIN -> time > T)
        const uint64_t pk = warp_min((won && terminal[d] && succ_time[d] <= T)
                                         ? pack_tij(succ_time[d], ij[d] >> 16, ij[d] & 0xFFFFu)
                                         : kNone);
        if (lane == 0 && pk != kNone) atomicOr(&st.flags, kFlagViolation);
        if (lane == 0 && pk < cached_best) {
          cached_best = ld_relaxed_u64(lvl_next + 1);
          if (pk < cached_best) {
            atomicMin(reinterpret_cast<unsigned long long*>(lvl_next + 1), (unsigned long long)pk);
            cached_best = pk;
          }
        }
      }
    }
    // each round adds at most 32 * D winners to the warp's buffer, which
    // is flushed once it holds more than stage_chunk - 32 * D of them
    if (fill > A.stage_chunk - 32 * D) {
      __syncwarp();
      unsigned long long b = 0;
      if (lane == 0)
        b = level_reserve(lvl_next, fill);
      b = __shfl_sync(0xffffffffu, b, 0);
      copy_out<K>(A, wkeys, wpar, fill, offN + b, lane, &st.flags);
      __syncwarp();
      fill = 0;
    }
  }
  // end of level: one reservation per block for the warps' remainders; in a
  // tagged log the same atomic is the block's arrival at the level barrier
  if (lane == 0) st.fill[warp] = fill;
  __syncthreads();
  const uint32_t nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    uint32_t total = 0;
    for (uint32_t w = 0; w < nw; ++w) total += st.fill[w];
    if (A.tag_bits) st.base = level_arrive_reserve(lvl_next, &st.flags, stop_mask, total);
    else st.base = total ? level_reserve(lvl_next, total) : 0ull;
  }
  __syncthreads();
  if (fill) {
    uint64_t at0 = offN + st.base;
    for (uint32_t w = 0; w < warp; ++w) at0 += st.fill[w];
    copy_out<K>(A, wkeys, wpar, fill, at0, lane, &st.flags);
  }
}

// ------------------------------------------------------------------ the exploration pass
template <class K, int TILE, int RULE, int SCHEME>
__global__ void __launch_bounds__(kThreads, 4) explore_kernel(const ExploreArgs A) {
  const Params& p = A.p;
  Ctrl* ctrl = A.ctrl;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  __shared__ Stage<K> stage;
  uint32_t epoch = 0;  // device-wide barriers passed in this pass
  const Barrier bar{A.bar_lines, &A.ctrl->err, A.barrier_extra, A.timeout_ns};

  // The threshold: given, read from the device (T_src + T_delta), or --
  // Step 3's lowering chained on the device -- one below the predecessor's
  // counterexample time, with no run at all once a predecessor held (or
  // failed).  One thread per block reads those words (thousands of warps
  // polling one line would queue at its L2 slice) and shares them.
  __shared__ unsigned long long s_T;
  __shared__ uint32_t s_skip;
  if (threadIdx.x == 0) {
    uint64_t t = A.T;
    uint32_t skip = 0;
    if (A.T_src) t = ld_relaxed_u64(A.T_src) + (uint64_t)A.T_delta;
    if (A.prev) {
      const Ctrl* q = A.prev;
      if (ld_relaxed_u32(&q->err) || ld_relaxed_u32(&q->skipped) || ld_relaxed_u32(&q->stop_level) == 0) skip = 1;
      else t = pack_time(ld_relaxed_u64(&q->wpack)) - 1;
    }
    s_T = t;
    s_skip = skip;
  }
  __syncthreads();
  if (s_skip) {
    if (gtid == 0) ctrl->skipped = 1;
    return;
  }
  const uint64_t T = s_T;

  // prologue: empty visited set, level arrays, levels 0..2 (the selects of
  // WG and TS, Listing 3) written directly: they are distinct by construction
  {
    ulonglong2* tb = reinterpret_cast<ulonglong2*>(A.table);
    const uint64_t n16 = A.table_u64 / 2;
    for (uint64_t x = gtid; x < n16; x += nthreads) tb[x] = make_ulonglong2(0, 0);
    for (uint64_t l = gtid; l < (uint64_t)p.max_level + 2; l += nthreads) {
      A.levels[2 * l] = l == 0 ? 1 : l == 1 ? p.a : l == 2 ? (uint64_t)p.a * p.b : 0;
      A.levels[2 * l + 1] = kNone;
      A.off[l] = l == 0 ? 0 : l == 1 ? 1 : l == 2 ? 1 + (uint64_t)p.a : 0;
    }
    const uint64_t n_init = 1 + (uint64_t)p.a + (uint64_t)p.a * p.b;
    for (uint64_t x = gtid; x < n_init; x += nthreads) {
      K key = 0;
      uint32_t par = kNoParent;
      if (x >= 1 && x <= p.a) {
        key = (K)x << p.wg_shift;
        par = 0;
      } else if (x > p.a) {
        const uint64_t y = x - 1 - p.a;
        const uint32_t i = (uint32_t)(y / p.b), j = (uint32_t)(y % p.b);
        key = ((K)(i + 1) << p.wg_shift) | ((K)(j + 1) << p.ts_shift);
        par = i;
      }
      KeyOps<K>::store(A.log_keys, x, LogTag<K>::pack(key, A.tag_bits, A.tag));
      A.log_par[x] = par;
    }
    if (threadIdx.x == 0) stage.flags = 0;
    if (gtid == 0) {
      ctrl->T = T;
      ctrl->best_pack = kNone;
      ctrl->wkey_lo = kNone;
      ctrl->wkey_hi = kNone;
      ctrl->widx = kNone;
    }
  }
  if (!grid_sync(bar, epoch)) return;

  // level loop (one device-wide barrier per level)
  uint32_t last = 2;
  uint64_t off_last = 1 + (uint64_t)p.a;
  uint64_t W = (uint64_t)p.a * p.b;
  // this thread's first keys of a level sit at fixed positions from the
  // level's start, so after each barrier they are loaded together with the
  // level's record rather than after it (positions past the level's end
  // read stale log entries that are never used; they stay inside the log)
  const uint64_t first_pos = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 *
                             (32 / TILE) * kDepth + (threadIdx.x & 31u) / TILE;
  K first[kDepth];
  bool have_first = false;
  for (;;) {
    const uint32_t L = last;
    if (L >= p.max_level) break;  // the deepest level holds only terminals
    const uint64_t offN = off_last + W;
    if (gtid == 0) A.off[L + 1] = offN;
    const uint32_t stop_mask = kFlagError | (A.early_exit ? kFlagViolation : 0u);
    expand_level<K, TILE, RULE, SCHEME>(A, stage, T, L, off_last, W, offN, first, have_first, stop_mask);
    // level L+1's width word doubles as the barrier: it ends with the width
    // and the number of blocks that saw an error or (with early exit) a
    // violating terminal (a tagged log's blocks arrived in expand_level)
    uint64_t word = 0;
    if (!(A.tag_bits ? level_wait(bar, A.levels + 2 * (L + 1), &word)
                     : level_sync(bar, A.levels + 2 * (L + 1), &stage.flags, stop_mask, &word)))
      return;
#pragma unroll
    for (uint32_t d = 0; d < kDepth; ++d) {
      const uint64_t at = offN + first_pos + d * (32 / TILE);
      first[d] = LogIO<K>::load(A.log_keys, at < A.log_cap ? at : A.log_cap - 1, evict_first_policy());
    }
    have_first = true;
    const uint64_t Wn = word & kLevelWidthMask;
    if (offN + Wn > A.log_cap) {  // the same decision in every block (one final word)
      set_error(ctrl, MC_ERR_FRONTIER);
      break;
    }
    if ((word >> kLevelStopShift) & 0xFFFFu) {  // an error, or level L+1 holds a violating terminal
      if (ld_relaxed_u32(&ctrl->err)) break;
      last = L + 1;
      off_last = offN;
      W = Wn;
      break;
    }
    if (Wn == 0) break;
    last = L + 1;
    off_last = offN;
    W = Wn;
  }
  if (ld_relaxed_u32(&ctrl->err)) return;

  // first level holding a violating terminal, and the minimum over all
  // levels.  With early exit only the last level can hold one; otherwise
  // every block scans the per-level minima (a few thousand words at most).
  uint32_t wl = 0;
  uint64_t best_all = kNone;
  if (A.early_exit) {
    best_all = ld_relaxed_u64(A.levels + 2 * last + 1);
    wl = best_all != kNone ? last : 0;
  } else {
    __shared__ unsigned long long s_best;
    __shared__ unsigned int s_wl;
    if (threadIdx.x == 0) {
      s_best = kNone;
      s_wl = 0xFFFFFFFFu;
    }
    __syncthreads();
    for (uint32_t l = 3 + threadIdx.x; l <= last; l += blockDim.x) {
      const uint64_t b = ld_relaxed_u64(A.levels + 2 * l + 1);
      if (b != kNone) {
        atomicMin(&s_best, (unsigned long long)b);
        atomicMin(&s_wl, l);
      }
    }
    __syncthreads();
    best_all = s_best;
    wl = s_wl == 0xFFFFFFFFu ? 0 : s_wl;
  }
  if (gtid == 0) {
    ctrl->levels = last + 1;
    ctrl->states = off_last + W;
    ctrl->stop_level = wl;
    ctrl->best_pack = best_all;
    ctrl->wpack = wl ? ld_relaxed_u64(A.levels + 2 * wl + 1) : kNone;
    if (A.tmin_out && best_all != kNone) *A.tmin_out = pack_time(best_all);
  }
  if (!A.want_witness || wl == 0) return;

  // witness: the violating terminal of level wl with the smallest key among
  // those with the level's minimum (time, i, j)
  const uint64_t target = ld_relaxed_u64(A.levels + 2 * wl + 1);
  const uint64_t offW = ld_relaxed_u64(&A.off[wl]);
  const uint64_t Ww = ld_relaxed_u64(A.levels + 2 * wl) & kLevelWidthMask;
  const uint32_t ti = pack_i(target), tj = pack_j(target);
  const uint64_t tt = pack_time(target);
  const uint32_t cfg_t = ti * p.b + tj;
  const uint32_t n_t = __ldg(p.N + cfg_t);
  for (uint64_t x = gtid; x < Ww; x += nthreads) {
    K key = KeyOps<K>::load(A.log_keys, offW + x);
    if (!log_entry<K>(A, offW + x, key)) break;
    if (field(key, p.wg_shift, p.wg_mask) - 1 != ti || field(key, p.ts_shift, p.ts_mask) - 1 != tj)
      continue;
    if (sum_n(key, p) != n_t || key_time(key, p, cfg_t) != tt) continue;
    if (sizeof(K) == 8)
      atomicMin(reinterpret_cast<unsigned long long*>(&ctrl->wkey_lo),
                (unsigned long long)KeyOps<K>::lo(key));
    else
      atomicMin(reinterpret_cast<unsigned long long*>(&ctrl->wkey_hi),
                (unsigned long long)KeyOps<K>::hi(key));
  }
  if (!grid_sync(bar, epoch)) return;
  if (sizeof(K) == 16) {
    const uint64_t whi = ld_relaxed_u64(&ctrl->wkey_hi);
    for (uint64_t x = gtid; x < Ww; x += nthreads) {
      K key = KeyOps<K>::load(A.log_keys, offW + x);
      if (!log_entry<K>(A, offW + x, key)) break;
      if (KeyOps<K>::hi(key) != whi) continue;
      if (field(key, p.wg_shift, p.wg_mask) - 1 != ti || field(key, p.ts_shift, p.ts_mask) - 1 != tj)
        continue;
      if (sum_n(key, p) != n_t || key_time(key, p, cfg_t) != tt) continue;
      atomicMin(reinterpret_cast<unsigned long long*>(&ctrl->wkey_lo),
                (unsigned long long)KeyOps<K>::lo(key));
    }
    if (!grid_sync(bar, epoch)) return;
  } else if (gtid == 0) {
    ctrl->wkey_hi = 0;
  }
  {
    const uint64_t wlo = ld_relaxed_u64(&ctrl->wkey_lo);
    const uint64_t whi = sizeof(K) == 16 ? ld_relaxed_u64(&ctrl->wkey_hi) : 0;
    for (uint64_t x = gtid; x < Ww; x += nthreads) {
      K key = KeyOps<K>::load(A.log_keys, offW + x);
      if (!log_entry<K>(A, offW + x, key)) break;
      if (KeyOps<K>::lo(key) == wlo && KeyOps<K>::hi(key) == whi) ctrl->widx = x;
    }
  }
  if (!grid_sync(bar, epoch)) return;
  // trace: follow parent indices from the witness back to s0
  if (gtid == 0) {
    uint64_t idx = ld_relaxed_u64(&ctrl->widx);
    if (idx >= Ww) {  // cannot happen when the level is intact; never walk from it
      set_error(ctrl, MC_ERR_FRONTIER);
      return;
    }
    uint32_t l = wl;
    for (;;) {
      const uint64_t at = ld_relaxed_u64(&A.off[l]) + idx;
      K key = KeyOps<K>::load(A.log_keys, at);
      if (!log_entry<K>(A, at, key)) return;
      A.trace[2 * l] = KeyOps<K>::lo(key);
      A.trace[2 * l + 1] = KeyOps<K>::hi(key);
      if (l == 0) break;
      idx = __ldcg(A.log_par + at);
      --l;
    }
    ctrl->witness_level = wl;
    ctrl->trace_len = wl + 1;
  }
}

// ------------------------------------------------------------------ dispatch tables
template <class K, int RULE, int SCHEME>
const void* pick_tile(int tile) {
  switch (tile) {
    case 1: return (const void*)explore_kernel<K, 1, RULE, SCHEME>;
    case 2: return (const void*)explore_kernel<K, 2, RULE, SCHEME>;
    case 4: return (const void*)explore_kernel<K, 4, RULE, SCHEME>;
    case 8: return (const void*)explore_kernel<K, 8, RULE, SCHEME>;
    case 16: return (const void*)explore_kernel<K, 16, RULE, SCHEME>;
  }
  return nullptr;
}

template <class K, int SCHEME>
const void* pick_rule(int tile, int rule) {
  return rule == MC_FREE ? pick_tile<K, MC_FREE, SCHEME>(tile) : pick_tile<K, MC_GREEDY, SCHEME>(tile);
}

}  // namespace
}  // namespace mc
