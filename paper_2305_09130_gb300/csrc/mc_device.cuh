// Device helpers shared by the exploration kernels (mc_kernels.cu: one model
// per launch; mc_batch.cu: many models in lockstep).  Internal; included by
// CUDA translation units only.
#pragma once

#include <cstdint>
#include <type_traits>

#include "mc.h"
#include "mc_internal.h"

namespace mc {
namespace dev {

typedef unsigned __int128 u128;

// ------------------------------------------------------------------ memory
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void ld_relaxed_v2u64(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_sys_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  return *reinterpret_cast<const volatile uint64_t*>(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 16-byte global -> shared copy that bypasses L1 (the visited set is written
// by atomics at L2), then wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void set_error(uint32_t* err, int code) {
  atomicCAS(err, 0u, (uint32_t)code);
}
__device__ __forceinline__ void set_error(Ctrl* ctrl, int code) { set_error(&ctrl->err, code); }

// ------------------------------------------------------------------ keys
template <class K>
struct KeyOps;

template <>
struct KeyOps<uint64_t> {
  static constexpr int kSlots = 4;  // keys per 32-byte bucket
  __device__ static uint64_t load(const void* base, uint64_t i) {
    return __ldcg(reinterpret_cast<const unsigned long long*>(base) + i);
  }
  __device__ static void store(void* base, uint64_t i, uint64_t k) {
    reinterpret_cast<unsigned long long*>(base)[i] = k;
  }
  __device__ static uint64_t lo(uint64_t k) { return k; }
  __device__ static uint64_t hi(uint64_t) { return 0; }
};

template <>
struct KeyOps<u128> {
  static constexpr int kSlots = 2;
  __device__ static u128 load(const void* base, uint64_t i) {
    ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(base) + i);
    return ((u128)v.y << 64) | v.x;
  }
  __device__ static void store(void* base, uint64_t i, u128 k) {
    reinterpret_cast<ulonglong2*>(base)[i] = make_ulonglong2((uint64_t)k, (uint64_t)(k >> 64));
  }
  __device__ static uint64_t lo(u128 k) { return (uint64_t)k; }
  __device__ static uint64_t hi(u128 k) { return (uint64_t)(k >> 64); }
};

// splitmix64 output function (Steele, Lea, Flood 2014)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t key_hash(uint64_t k) { return mix64(k); }
__device__ __forceinline__ uint64_t key_hash(u128 k) {
  return mix64((uint64_t)k ^ mix64((uint64_t)(k >> 64) + 0x9E3779B97F4A7C15ull));
}

template <class K>
__device__ __forceinline__ uint32_t field(K key, uint32_t shift, uint64_t mask) {
  return (uint32_t)((uint64_t)(key >> shift) & mask);
}

// sum of the n_c fields of a key = its BFS level - 2
template <class K>
__device__ __forceinline__ uint32_t sum_n(K key, const Params& p) {
  if (p.swar_ok) {
    uint64_t x = (uint64_t)key & p.swar_mask;
    return (uint32_t)(((x * p.swar_mul) >> ((p.P - 1) * p.n_bits)) & p.n_mask);
  }
  uint32_t s = 0;
  for (uint32_t c = 0; c < p.P; ++c) s += field(key, (p.P - 1 - c) * p.n_bits, p.n_mask);
  return s;
}

// Model-table load: through the read-only cache when the tables are fixed for
// the launch (CG = false), from L2 when a persistent loop may swap them (CG).
template <bool CG>
__device__ __forceinline__ uint32_t ldp(const uint32_t* p) {
  return CG ? __ldcg(p) : __ldg(p);
}

// model time of a key (max over units of n_c * cost * speed_c)
template <class K, bool CG = false>
__device__ __forceinline__ uint64_t key_time(K key, const Params& p, uint32_t cfg) {
  uint64_t c0 = ldp<CG>(p.cost + cfg);
  uint64_t mx = 0;
  for (uint32_t c = 0; c < p.P; ++c) {
    uint64_t t = (uint64_t)field(key, (p.P - 1 - c) * p.n_bits, p.n_mask) * c0 * ldp<CG>(p.speed + c);
    mx = t > mx ? t : mx;
  }
  return mx;
}

// ------------------------------------------------------------------ visited set
__device__ __forceinline__ u128 cas128(u128* addr, u128 cmp, u128 val) {
  uint64_t olo, ohi;
  asm volatile(
      "{\n\t.reg .b128 c, v, o;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.relaxed.gpu.global.cas.b128 o, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, o;\n\t}"
      : "=l"(olo), "=l"(ohi)
      : "l"((uint64_t)cmp), "l"((uint64_t)(cmp >> 64)), "l"((uint64_t)val),
        "l"((uint64_t)(val >> 64)), "l"(addr)
      : "memory");
  return ((u128)ohi << 64) | olo;
}

__device__ __forceinline__ uint64_t slot_cas(uint64_t* addr, uint64_t cmp, uint64_t val) {
  return atomicCAS(reinterpret_cast<unsigned long long*>(addr), cmp, val);
}
__device__ __forceinline__ u128 slot_cas(u128* addr, u128 cmp, u128 val) { return cas128(addr, cmp, val); }

template <class K>
__device__ __forceinline__ void load_bucket(const K* b, K (&v)[KeyOps<K>::kSlots]);

template <>
__device__ __forceinline__ void load_bucket<uint64_t>(const uint64_t* b, uint64_t (&v)[4]) {
  ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(b));
  ulonglong2 y = __ldcg(reinterpret_cast<const ulonglong2*>(b) + 1);
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
template <>
__device__ __forceinline__ void load_bucket<u128>(const u128* b, u128 (&v)[2]) {
  ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(b));
  ulonglong2 y = __ldcg(reinterpret_cast<const ulonglong2*>(b) + 1);
  v[0] = ((u128)x.y << 64) | x.x;
  v[1] = ((u128)y.y << 64) | y.x;
}

// Insert `key` (BFS level lvl, as level_of reports it for any key) into the
// visited set, starting at bucket `bkt`, whose 32 bytes are already in
// `first` (shared memory) unless `first` is null.
// Returns 1 if this thread inserted it, 0 if it was already there, -1 when
// the probe limit was reached.  A slot is free when it holds 0 or a key of an
// earlier level; the first free slot of the probe sequence is taken.
template <class K, class LevelOf>
__device__ int visited_insert_lv(K* table, uint64_t bucket_mask, uint32_t max_probes, K key,
                                 uint32_t lvl, const LevelOf& level_of, uint64_t bkt, const K* first) {
  constexpr int S = KeyOps<K>::kSlots;
  for (uint32_t probe = 0; probe < max_probes; ++probe) {
    K* slot = table + bkt * S;
    K v[S];
    if (probe == 0 && first) {
#pragma unroll
      for (int s = 0; s < S; ++s) v[s] = first[s];
    } else {
      load_bucket<K>(slot, v);
    }
    bool hit = false;
#pragma unroll
    for (int s = 0; s < S; ++s) hit |= (v[s] == key);
    if (hit) return 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      K cur = v[s];
      // a slot changes at most once per level (free -> a key of this
      // level), so two CAS attempts settle it; the bound is defensive
      for (int tries = 0; tries < 3; ++tries) {
        if (cur == key) return 0;
        if (cur != (K)0 && level_of(cur) >= lvl) break;  // taken this level
        K old = slot_cas(slot + s, cur, key);
        if (old == cur) return 1;
        cur = old;
      }
    }
    bkt = (bkt + 1) & bucket_mask;
  }
  return -1;
}

// The first step of an insert whose first bucket is already in shared
// memory, split off so that a thread can issue the CAS of several inserts
// before it waits for any: kPickDup when the key is in the bucket, kPickFull
// when every slot holds a key of this level, else the first free slot (its
// content in cur).  After the CAS on that slot, an old value equal to cur
// means the insert won, equal to the key a duplicate, and anything else (the
// slot went to another key) sends the insert to visited_insert_lv from the
// same bucket, which rereads it.
constexpr uint32_t kPickDup = 0xFFu;
constexpr uint32_t kPickFull = 0xFEu;
template <class K, class LevelOf>
__device__ __forceinline__ uint32_t bucket_pick(const K* first, K key, uint32_t lvl, const LevelOf& level_of,
                                                K& cur) {
  constexpr int S = KeyOps<K>::kSlots;
  K v[S];
#pragma unroll
  for (int s = 0; s < S; ++s) v[s] = first[s];
  bool hit = false;
#pragma unroll
  for (int s = 0; s < S; ++s) hit |= (v[s] == key);
  if (hit) return kPickDup;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (v[s] == (K)0 || level_of(v[s]) < lvl) {
      cur = v[s];
      return (uint32_t)s;
    }
  }
  return kPickFull;
}

// The cost-table model's keys: the level is 2 + sum(n), so `lvl` here is the
// sum of the n fields.
template <class K>
__device__ __forceinline__ int visited_insert(K* table, uint64_t bucket_mask, uint32_t max_probes, K key,
                                              uint32_t lvl, const Params& p, uint64_t bkt, const K* first) {
  return visited_insert_lv<K>(table, bucket_mask, max_probes, key, lvl,
                              [&p](K k) { return sum_n(k, p); }, bkt, first);
}

// ------------------------------------------------------------------ device-wide barrier
// All blocks are co-resident (cooperative launch).  Each block's thread 0
// counts its arrival with one acquire-release atomic on a single counter in
// its own 128-byte line.  (A two-level tree of 16 group counters and a top
// counter puts a second dependent atomic on the last arriver's path; one
// counter for all blocks measured 12% faster per level on deep, narrow
// searches and 3% on the widest ones.)  The counter only grows: the k-th
// barrier of a launch (k = 1, 2, ...) completes when it reaches k * blocks.
// The last arriver publishes a 64-bit word: generation k in the high half and
// a 32-bit payload in the low half, with a release store; the waiters poll it
// with acquire loads, so the payload reaches every block with the load that
// ends its wait.  (A value every block needs after the barrier -- the next
// level's width -- is read once by the releaser instead of by hundreds of
// blocks at once from a line the step just updated with atomics, which
// doubled the barrier's cost.)  Every block passes the same sequence of
// barriers, so each tracks k itself.  With a serial section, the releasing
// block runs it (all its threads) before publishing.  Each wait is bounded by
// timeout_ns of %globaltimer; on expiry the block records MC_ERR_TIMEOUT in
// *err, raises the abort flag so the other waiters leave too, and returns
// false.
struct Barrier {
  uint32_t* lines;      // kBarBytes / 128 lines of 128 bytes, zeroed per launch
  uint32_t* err;        // error word of the launch
  uint32_t extra;       // extra arrivals to wait for (test hook)
  uint64_t timeout_ns;
};

struct NoSerial {
  __device__ void operator()() const {}
};
struct NoPayload {
  __device__ uint32_t operator()() const { return 0; }
};

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Returns false on timeout/abort; *payload (if given) receives the releaser's
// payload of this barrier.
template <class Serial = NoSerial, class Payload = NoPayload>
__device__ bool grid_sync(const Barrier& B, uint32_t& epoch, const Serial& serial = Serial(),
                          const Payload& payload_fn = Payload(), uint32_t* payload = nullptr) {
  constexpr bool kSerial = !std::is_same<Serial, NoSerial>::value;
  __shared__ uint32_t s_ok, s_release, s_payload;
  __syncthreads();
  const uint32_t target = ++epoch;
  uint64_t* gen = reinterpret_cast<uint64_t*>(B.lines + kBarGen * 32);
  if (threadIdx.x == 0) {
    s_release = 0;
    if (atom_add_acq_rel(B.lines + kBarCount * 32, 1u) + 1 == gridDim.x * target && B.extra == 0) {
      if (kSerial) s_release = 1;
      else st_release_u64(gen, ((uint64_t)target << 32) | payload_fn());
    }
  }
  if (kSerial) {
    __syncthreads();
    if (s_release) {
      serial();
      __syncthreads();
      // the block's writes are ordered before thread 0's release by the
      // barrier above (release is cumulative)
      if (threadIdx.x == 0) st_release_u64(gen, ((uint64_t)target << 32) | payload_fn());
    }
  }
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    uint32_t* abort_flag = B.lines + kBarAbort * 32;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    uint64_t w;
    // one load per spin; the abort flag and the clock every 16th
    while (((w = ld_acquire_u64(gen)) >> 32) < target) {
      if ((++spins & 15u) == 0) {
        if (ld_relaxed_u32(abort_flag)) { ok = 0; break; }
        if (globaltimer() - t0 > B.timeout_ns) {
          set_error(B.err, MC_ERR_TIMEOUT);
          atomicExch(abort_flag, 1u);
          ok = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    s_payload = (uint32_t)w;
    s_ok = ok;
  }
  __syncthreads();
  if (payload) *payload = s_payload;
  return s_ok != 0;
}

// ------------------------------------------------------------------ level barrier
// The device-wide barrier at the end of a BFS level, fused with the level's
// width counter.  The 64-bit word of the next level is, from the top,
// [blocks arrived : 16][blocks that ask to stop : 16][width : 32].  During
// the level, warps reserve frontier-log ranges by adding to the width field;
// at the end each block (after its last reservation and log writes) adds one
// arrival, plus one stop when its shared `flags` word has a bit of
// stop_mask set (an error, or what ends the search; the word is cleared for
// the next level), with a release reduction, and polls the word with acquire loads
// until every block has arrived.  The value that ends the wait carries the
// final width and the stop count, and every arrival is in the release
// sequence it reads from, so each block's log writes are visible after the
// wait.  No block releases the others: one dependent L2 round trip fewer for
// the record read and one for the release store, per level.  Widths stay
// below 2^31 (checked on the host), so the width field never carries.  The
// wait is bounded like grid_sync's; `extra` adds arrivals to wait for (test
// hook).  Returns false on timeout/abort; *value receives the final word.
__device__ __forceinline__ void red_add_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
constexpr uint32_t kLevelArriveShift = 48;
constexpr uint32_t kLevelStopShift = 32;
constexpr uint64_t kLevelWidthMask = 0xFFFFFFFFull;

// Reserve n frontier-log entries of the level whose word this is; returns
// the offset of the first (blocks that already arrived have raised the high
// fields, which the offset leaves out).
__device__ __forceinline__ uint64_t level_reserve(uint64_t* word, uint32_t n) {
  return atomicAdd(reinterpret_cast<unsigned long long*>(word), (unsigned long long)n) & kLevelWidthMask;
}

__device__ __forceinline__ uint64_t atom_add_release_u64(uint64_t* p, uint64_t v) {
  uint64_t old;
  asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// Thread 0 only: the arrival of this block (with its stop vote from `flags`,
// which is cleared) plus `n` frontier-log entries reserved in the same
// atomic; returns the offset of the first.  A block that arrives this way
// writes those entries after its arrival, so readers of the next level check
// each entry's tag (see the exploration kernel) instead of relying on the
// barrier for them.  Wait with level_wait.
__device__ __forceinline__ uint64_t level_arrive_reserve(uint64_t* word, uint32_t* flags, uint32_t stop_mask,
                                                         uint32_t n) {
  const bool stop = (*flags & stop_mask) != 0;
  *flags = 0;
  return atom_add_release_u64(word, (1ull << kLevelArriveShift) | (stop ? 1ull << kLevelStopShift : 0ull) | n) &
         kLevelWidthMask;
}

// The waiting half of level_sync for blocks that arrived with
// level_arrive_reserve: every thread of the block calls it.
__device__ __forceinline__ bool level_wait(const Barrier& B, uint64_t* word, uint64_t* value);

__device__ __forceinline__ bool level_sync(const Barrier& B, uint64_t* word, uint32_t* flags,
                                           uint32_t stop_mask, uint64_t* value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool stop = (*flags & stop_mask) != 0;
    *flags = 0;
    red_add_release_u64(word, (1ull << kLevelArriveShift) | (stop ? 1ull << kLevelStopShift : 0ull));
  }
  return level_wait(B, word, value);
}

__device__ __forceinline__ bool level_wait(const Barrier& B, uint64_t* word, uint64_t* value) {
  __shared__ uint32_t s_ok;
  __shared__ unsigned long long s_v;
  if (threadIdx.x == 0) {
    const uint64_t target = (uint64_t)gridDim.x + B.extra;
    uint32_t* abort_flag = B.lines + kBarAbort * 32;
    const uint64_t t0 = globaltimer();
    uint32_t ok = 1, spins = 0;
    uint64_t v;
    while (((v = ld_acquire_u64(word)) >> kLevelArriveShift) < target) {
      if ((++spins & 15u) == 0) {
        if (ld_relaxed_u32(abort_flag)) { ok = 0; break; }
        if (globaltimer() - t0 > B.timeout_ns) {
          set_error(B.err, MC_ERR_TIMEOUT);
          atomicExch(abort_flag, 1u);
          ok = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    s_v = v;
    s_ok = ok;
  }
  __syncthreads();
  *value = s_v;
  return s_ok != 0;
}

// ------------------------------------------------------------------ tile reductions
template <int TILE>
__device__ __forceinline__ uint64_t tile_max(uint64_t v) {
#pragma unroll
  for (int o = TILE / 2; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
template <int TILE>
__device__ __forceinline__ uint64_t tile_min(uint64_t v) {
#pragma unroll
  for (int o = TILE / 2; o > 0; o >>= 1) {
    uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// reductions over aligned groups of g lanes (g a power of two, warp-uniform)
__device__ __forceinline__ uint64_t group_max(uint64_t v, uint32_t g) {
  for (uint32_t o = 1; o < g; o <<= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ uint64_t group_min(uint64_t v, uint32_t g) {
  for (uint32_t o = 1; o < g; o <<= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
// Minimum over the warp; most calls have no lane with a value (kNone), and
// one vote settles those.
__device__ __forceinline__ uint64_t warp_min(uint64_t v) {
  if (!__any_sync(0xffffffffu, v != kNone)) return kNone;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// ------------------------------------------------------------------ splitmix64
// Output number ctr of the splitmix64 stream started at seed (Steele, Lea,
// Flood 2014), as a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  return mix64(seed + (ctr + 1) * 0x9E3779B97F4A7C15ull);
}

// One random run of the model (Section 4, Step 3: SPIN's simulation mode
// gives T_ini; Section 5: a swarm is many such runs).  Walk w draws
// splitmix64 outputs number (w << 32) + 0, 1, ...: the WG index, the TS index,
// then per work-group the unit among the allowed ones in index order.
// Returns the terminal's model time, or kNone when some clock passes `bound`
// first (the run cannot end at or below it).  *cfg receives i * b + j.
template <bool CG = false>
__device__ inline uint64_t walk_time(const Params& p, uint64_t seed, uint64_t w, uint64_t bound,
                                     uint32_t* cfg_out = nullptr) {
  uint64_t ctr = w << 32;
  const uint32_t i = (uint32_t)(splitmix64_at(seed, ctr++) % p.a);
  const uint32_t j = (uint32_t)(splitmix64_at(seed, ctr++) % p.b);
  const uint32_t cfg = i * p.b + j;
  if (cfg_out) *cfg_out = cfg;
  const uint32_t N = ldp<CG>(p.N + cfg);
  const uint64_t cost = ldp<CG>(p.cost + cfg);
  uint64_t clk[kMaxP], t[kMaxP];
  for (uint32_t c = 0; c < p.P; ++c) {
    t[c] = cost * ldp<CG>(p.speed + c);
    clk[c] = 0;
  }
  for (uint32_t k = 0; k < N; ++k) {
    uint32_t c = 0;
    if (p.rule == MC_FREE) {
      c = (uint32_t)(splitmix64_at(seed, ctr++) % p.P);
    } else {
      uint64_t mn = kNone;
      for (uint32_t u = 0; u < p.P; ++u) mn = clk[u] < mn ? clk[u] : mn;
      uint32_t cnt = 0;
      for (uint32_t u = 0; u < p.P; ++u) cnt += clk[u] == mn;
      uint32_t pick = (uint32_t)(splitmix64_at(seed, ctr++) % cnt);
      for (uint32_t u = 0; u < p.P; ++u) {
        if (clk[u] == mn) {
          if (pick == 0) { c = u; break; }
          --pick;
        }
      }
    }
    clk[c] += t[c];
    if (clk[c] > bound) return kNone;
  }
  uint64_t mx = 0;
  for (uint32_t c = 0; c < p.P; ++c) mx = clk[c] > mx ? clk[c] : mx;
  return mx;
}

template <bool CG = false>
__device__ inline uint64_t simulate_walk(const Params& p, uint64_t seed, uint64_t w) {
  return walk_time<CG>(p, seed, w, kNone);
}

}  // namespace dev
}  // namespace mc
