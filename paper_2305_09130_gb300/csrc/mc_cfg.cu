// Configuration engine: one thread block per (WG, TS) configuration.
//
// After the two selects of `main` (Listing 3) every state carries the
// configuration (i, j) it was selected with, and no transition changes it
// (`host` and `device` only hand out work-groups, Listings 4-5).  The state
// space below level 2 is therefore a forest of disjoint subtrees, one per
// configuration, and a BFS level of the whole space is the union of the
// same level of every subtree.  Here one thread block explores one subtree:
// its frontier and its visited set live in shared memory, a level ends with
// one __syncthreads, and nothing waits for other blocks.  Narrow searches
// (the GREEDY rule keeps at most C(P, P/2) states per configuration and
// level; small FREE models keep C(k+P-1, P-1)) then cost a block barrier per
// level instead of a device-wide one.
//
// Exactness.  The pass reports what the level-synchronous kernel reports:
//   * every block adds its level widths into the pass's per-level array,
//     so the count of levels 0..L is the sum over configurations;
//   * all terminals (FIN, Listing 4) of configuration (i, j) sit at level
//     2 + N_ij, so the first level holding a violating terminal is the least
//     2 + N_ij over configurations with one, and its minimum packed
//     (time, i, j) is the least over those configurations; the witness (the
//     smallest key of that time in that configuration) is found by the block
//     that owns the configuration;
//   * with early exit a block stops expanding once a level at or below its
//     current one is known to hold a violating terminal (it has already
//     added every width up to that level; deeper widths are not counted);
//   * the block that finishes the pass's last configuration combines the
//     per-configuration records and the widths into the pass header, walks
//     the witness's parents through the frontier log into the trace, and
//     publishes the least violating time for a chained pass.
//
// Shared memory of a block: two frontiers (the level being expanded and the
// next) of `wcap` keys and two open-addressing tables of `tsize` slots (the
// next level's, and the one cleared for the level after it).  A slot is
// claimed with a compare-and-swap from 0 (128-bit keys: atom.shared.cas.b128)
// so two lanes inserting the same key meet at the same slot; a key is never
// 0 (the WG index field is at least 1).
#include <cstdint>

#include "mc_device.cuh"

namespace mc {
namespace {

using namespace mc::dev;

__device__ __forceinline__ uint64_t smem_cas(uint64_t* p, uint64_t cmp, uint64_t val) {
  return atomicCAS(reinterpret_cast<unsigned long long*>(p), cmp, val);
}

__device__ __forceinline__ u128 smem_cas(u128* p, u128 cmp, u128 val) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(p);
  uint64_t olo, ohi;
  asm volatile(
      "{\n\t.reg .b128 c, v, o;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.relaxed.cta.shared::cta.cas.b128 o, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, o;\n\t}"
      : "=l"(olo), "=l"(ohi)
      : "l"((uint64_t)cmp), "l"((uint64_t)(cmp >> 64)), "l"((uint64_t)val), "l"((uint64_t)(val >> 64)),
        "r"(sa)
      : "memory");
  return ((u128)ohi << 64) | olo;
}

// Slot of a key in a shared table: the top bits of a multiplicative hash
// (the keys of one configuration differ only in their work-group counts).
__device__ __forceinline__ uint32_t slot_hash(uint64_t k) {
  return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 40);
}
__device__ __forceinline__ uint32_t slot_hash(u128 k) {
  const uint64_t x = (uint64_t)k ^ ((uint64_t)(k >> 64) * 0xC2B2AE3D27D4EB4Full);
  return (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> 40);
}

// Insert into a shared table of mask + 1 slots by linear probing.  Every
// probe is a compare-and-swap from 0, so no thread reads a slot another is
// writing.  1: inserted by this thread, 0: already there, -1: table full.
template <class K>
__device__ __forceinline__ int shared_insert(K* tab, uint32_t mask, K key) {
  uint32_t h = slot_hash(key) & mask;
  for (uint32_t n = 0; n <= mask; ++n) {
    const K old = smem_cas(tab + h, (K)0, key);
    if (old == (K)0) return 1;
    if (old == key) return 0;
    h = (h + 1) & mask;
  }
  return -1;
}

template <class K>
__device__ __forceinline__ void log_store(void* base, uint64_t i, K k) {
  KeyOps<K>::store(base, i, k);
}

// Block state kept in static shared memory.
struct CfgShared {
  CfgPass Q;                     // the pass of the current unit
  unsigned long long vmin;       // least violating terminal time of the unit
  unsigned long long whi, wlo;   // witness key of the unit
  uint64_t T;
  uint32_t cnt[3];               // level widths, rotating: level L+1 counts into cnt[(L+1) % 3]
  uint32_t cut[2];               // early exit: least level known to violate (read per level)
  uint32_t unit;
  uint32_t widx;
  uint32_t skip;                 // chained pass that does not run
  uint32_t last;                 // this block finished the pass's last unit
  uint32_t err;                  // an error of this unit (uniform after a barrier)
  // epilogue
  unsigned long long e_best, e_wpack, e_sum;
  uint32_t e_stop, e_deep;
};

constexpr uint32_t kNoLevel = 0xFFFFFFFFu;

// Maximum (and, for GREEDY, minimum) of a value over the aligned group of
// g lanes that holds one state: butterfly steps below g, unrolled, the two
// reductions interleaved (g is uniform across the block).
template <bool MIN, class C>
__device__ __forceinline__ void group_minmax(C& mx, C& mn, uint32_t g) {
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    if (o < g) {
      const C a = __shfl_xor_sync(0xffffffffu, mx, o);
      C b = 0;
      if (MIN) b = __shfl_xor_sync(0xffffffffu, mn, o);
      mx = a > mx ? a : mx;
      if (MIN) mn = b < mn ? b : mn;
    }
  }
}

// Explore configuration `cfg` of pass Q at threshold T.  Clocks are kept in
// C: 32 bits when every clock of the model fits (one shuffle per reduction
// step instead of two), else 64.
template <class K, class C>
__device__ void explore_unit(const CfgPass& Q, uint32_t cfg, uint64_t T, K* front0, K* front1, K* tab0,
                             K* tab1, uint32_t wcap, uint32_t tsize, CfgShared& S) {
  // the pass's fields in registers (Q lives in shared memory, which the
  // level's stores could alias)
  const uint32_t P = Q.p.P, n_bits = Q.p.n_bits, b = Q.p.b;
  const uint64_t n_mask = Q.p.n_mask;
  const bool greedy = Q.p.rule == MC_GREEDY, prune = Q.prune != 0, early = Q.early_exit != 0;
  const uint32_t* Np = Q.p.N;
  const uint32_t* costp = Q.p.cost;
  const uint32_t* speedp = Q.p.speed;
  void* const log_keys = Q.log_keys;
  uint32_t* const log_par = Q.log_par;
  uint64_t* const levels = Q.levels;
  Ctrl* const ctrl = Q.ctrl;
  const uint32_t tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31u;
  const uint32_t g = Q.group;
  const uint32_t spr = nthr / g;  // states per round
  const uint32_t c = tid & (g - 1);
  const uint32_t my = tid / g;
  const uint32_t warp_my = (tid & ~31u) / g;  // the warp's first state in a round
  const uint32_t i = cfg / b, j = cfg % b;
  const uint32_t N = __ldg(Np + cfg);
  const bool unit_ok = c < P;
  const C t_c = unit_ok ? (C)((uint64_t)__ldg(costp + cfg) * __ldg(speedp + c)) : (C)0;
  const C Tc = T < (uint64_t)(C)~(C)0 ? (C)T : (C)~(C)0;  // T, saturated at the clock type's maximum
  constexpr C kNoneC = (C)~(C)0;
  const uint32_t c_shift = (P - 1 - (unit_ok ? c : 0)) * n_bits;
  const K one_c = (K)1 << c_shift;
  const bool log_on = Q.want_witness != 0;
  const uint64_t seg0 = log_on ? Q.seg[cfg] : 0, seg1 = log_on ? Q.seg[cfg + 1] : 0;
  const uint32_t tmask = tsize - 1;
  const K key2 = ((K)(i + 1) << Q.p.wg_shift) | ((K)(j + 1) << Q.p.ts_shift);

  if (tid == 0) {
    front0[0] = key2;  // level 2: (i+1, j+1, 0...0)
    if (log_on) {
      log_store<K>(log_keys, seg0, key2);
      log_par[seg0] = kNoParent;
    }
  }
  __syncthreads();
  uint64_t lvl_base = seg0;  // log index of the current level's first entry
  uint32_t W = 1, L = 2, deepest = 2;
  while (L < 2 + N) {
    if (early && S.cut[L & 1u] <= L) break;  // deeper widths are not counted
    K* cur = (L & 1u) ? front1 : front0;
    K* nxt = (L & 1u) ? front0 : front1;
    K* tnx = (L & 1u) ? tab0 : tab1;  // receives level L+1
    K* tcl = (L & 1u) ? tab1 : tab0;  // held level L: cleared for level L+2
    uint32_t* cnx = &S.cnt[(L + 1) % 3];
    // the least level known to violate, for the cut at the next level: the
    // load is issued here and its value stored after the level's rounds, so
    // its latency overlaps them
    uint32_t sc = 0;
    if (tid == 0) {
      S.cnt[(L + 2) % 3] = 0;
      if (early) sc = ld_relaxed_u32(&ctrl->stop_c);
    }
    if (L > 2)
      for (uint32_t x = tid; x < tsize; x += nthr) tcl[x] = (K)0;
    const bool to_terminal = L + 1 == 2 + N;
    for (uint32_t base = 0; base < W; base += spr) {
      if (base + warp_my >= W) continue;  // no state for this warp in this round
      const uint32_t s = base + my;
      const bool valid = s < W;
      const K key = valid ? cur[s] : (K)0;
      C clk = 0;
      if (valid && unit_ok) clk = (C)field(key, c_shift, n_mask) * t_c;
      C mx = clk, mn = (valid && unit_ok) ? clk : kNoneC;
      bool ok = valid && unit_ok;
      if (greedy) {
        group_minmax<true>(mx, mn, g);
        ok = ok && clk == mn;
      } else {
        group_minmax<false>(mx, mn, g);
      }
      const C nclk = clk + t_c;
      const C st = nclk > mx ? nclk : mx;  // model time of the successor
      if (prune && st > Tc) ok = false;
      const K succ = key + one_c;
      int won = 0;
      if (ok) {
        const int rc = shared_insert<K>(tnx, tmask, succ);
        if (rc < 0) S.err = (uint32_t)MC_ERR_TABLE_FULL;
        won = rc > 0;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, won);
      if (m) {
        const uint32_t leader = __ffs(m) - 1;
        uint32_t pos0 = 0;
        if (lane == leader) pos0 = atomicAdd(cnx, (uint32_t)__popc(m));
        pos0 = __shfl_sync(0xffffffffu, pos0, leader);
        if (won) {
          const uint32_t pos = pos0 + __popc(m & ((1u << lane) - 1u));
          if (pos < wcap) nxt[pos] = succ;
          else S.err = (uint32_t)MC_ERR_FRONTIER;
          if (log_on) {
            const uint64_t at = lvl_base + W + pos;
            if (at < seg1) {
              log_store<K>(log_keys, at, succ);
              log_par[at] = (uint32_t)(lvl_base + s);
            } else {
              S.err = (uint32_t)MC_ERR_FRONTIER;
            }
          }
          // Step 2: a terminal winner with time <= T violates G(FIN -> time > T)
          if (to_terminal && (uint64_t)st <= T) atomicMin(&S.vmin, (unsigned long long)st);
        }
      }
    }
    if (tid == 0) S.cut[(L + 1) & 1u] = sc ? ~sc : kNoLevel;
    __syncthreads();
    const uint32_t Wn = S.cnt[(L + 1) % 3];
    if (S.err) return;
    if (tid == 0 && Wn) atomicAdd(reinterpret_cast<unsigned long long*>(levels + 2 * (L + 1)), (unsigned long long)Wn);
    lvl_base += W;
    W = Wn;
    ++L;
    if (W == 0) break;
    deepest = L;
  }

  // this configuration's violating terminals (all at level 2 + N): the
  // smallest key of the least time, and its log index
  const uint64_t tv = S.vmin;
  if (tv != kNone) {
    K* fr = (L & 1u) ? front1 : front0;  // level 2 + N
    auto time_of = [&](K k) {
      const uint64_t c0 = __ldg(costp + cfg);
      uint64_t mx = 0;
      for (uint32_t u = 0; u < P; ++u) {
        const uint64_t t = (uint64_t)field(k, (P - 1 - u) * n_bits, n_mask) * c0 * __ldg(speedp + u);
        mx = t > mx ? t : mx;
      }
      return mx;
    };
    if (tid == 0 && early) atomicMax(&ctrl->stop_c, ~(2u + N));
    for (uint32_t x = tid; x < W; x += nthr)
      if (time_of(fr[x]) == tv) atomicMin(&S.whi, (unsigned long long)KeyOps<K>::hi(fr[x]));
    __syncthreads();
    for (uint32_t x = tid; x < W; x += nthr)
      if (KeyOps<K>::hi(fr[x]) == S.whi && time_of(fr[x]) == tv)
        atomicMin(&S.wlo, (unsigned long long)KeyOps<K>::lo(fr[x]));
    __syncthreads();
    for (uint32_t x = tid; x < W; x += nthr)
      if (KeyOps<K>::hi(fr[x]) == S.whi && KeyOps<K>::lo(fr[x]) == S.wlo) S.widx = (uint32_t)(lvl_base + x);
    __syncthreads();
  }
  if (tid == 0) {
    CfgRec r;
    r.vpack = tv != kNone ? pack_tij(tv, i, j) : kNone;
    r.wkey_lo = tv != kNone ? S.wlo : kNone;
    r.wkey_hi = tv != kNone ? S.whi : kNone;
    r.widx = tv != kNone ? S.widx : 0u;
    r.deepest = deepest;
    Q.rec[cfg] = r;
  }
}

// ------------------------------------------------------------------ warp units
// A configuration whose widest level fits one warp (width bound x lanes per
// state <= 32) is explored by a single warp, its level in registers: state
// s of the level is held by lanes [s*g, s*g + g), every proposal of the level
// is in the warp, so duplicates are found exactly by matching the proposed
// keys across the warp (the lowest lane of equal keys wins), and the winners,
// ranked by a ballot, become the next level.  No table, no shared counter, no
// block barrier; the same counts, records, log entries and early exit as
// explore_unit.

// Position of set bit number k (from 0) of m; k < popc(m).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t k) {
  uint32_t pos = 0, c;
  c = __popc(m & 0xFFFFu);
  if (k >= c) { k -= c; pos += 16; m >>= 16; }
  c = __popc(m & 0xFFu);
  if (k >= c) { k -= c; pos += 8; m >>= 8; }
  c = __popc(m & 0xFu);
  if (k >= c) { k -= c; pos += 4; m >>= 4; }
  c = __popc(m & 0x3u);
  if (k >= c) { k -= c; pos += 2; m >>= 2; }
  c = m & 1u;
  if (k >= c) pos += 1;
  return pos;
}

template <class K>
__device__ __forceinline__ K shfl_key(K k, uint32_t src) {
  if (sizeof(K) == 8) return (K)__shfl_sync(0xffffffffu, (unsigned long long)k, src);
  const uint64_t lo = __shfl_sync(0xffffffffu, (unsigned long long)KeyOps<K>::lo(k), src);
  const uint64_t hi = __shfl_sync(0xffffffffu, (unsigned long long)KeyOps<K>::hi(k), src);
  return (K)(((u128)hi << 64) | lo);
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class K, class C>
__device__ uint32_t explore_unit_warp(const CfgPass& Q, uint32_t cfg, uint64_t T) {
  const uint32_t P = Q.p.P, n_bits = Q.p.n_bits, b = Q.p.b;
  const uint64_t n_mask = Q.p.n_mask;
  const bool greedy = Q.p.rule == MC_GREEDY, prune = Q.prune != 0, early = Q.early_exit != 0;
  const uint32_t* costp = Q.p.cost;
  const uint32_t* speedp = Q.p.speed;
  void* const log_keys = Q.log_keys;
  uint32_t* const log_par = Q.log_par;
  uint64_t* const levels = Q.levels;
  Ctrl* const ctrl = Q.ctrl;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = Q.group;
  const uint32_t spw = 32u / g;  // states the warp holds
  const uint32_t c = lane & (g - 1);
  const uint32_t my = lane / g;
  const uint32_t i = cfg / b, j = cfg % b;
  const uint32_t N = __ldg(Q.p.N + cfg);
  const bool unit_ok = c < P;
  const C t_c = unit_ok ? (C)((uint64_t)__ldg(costp + cfg) * __ldg(speedp + c)) : (C)0;
  const C Tc = T < (uint64_t)(C)~(C)0 ? (C)T : (C)~(C)0;
  constexpr C kNoneC = (C)~(C)0;
  const uint32_t c_shift = (P - 1 - (unit_ok ? c : 0)) * n_bits;
  const K one_c = (K)1 << c_shift;
  const bool log_on = Q.want_witness != 0;
  const uint64_t seg0 = log_on ? Q.seg[cfg] : 0, seg1 = log_on ? Q.seg[cfg + 1] : 0;
  const K key2 = ((K)(i + 1) << Q.p.wg_shift) | ((K)(j + 1) << Q.p.ts_shift);
  if (log_on && lane == 0) {
    log_store<K>(log_keys, seg0, key2);
    log_par[seg0] = kNoParent;
  }
  K key = key2;  // the state of this lane's group (valid for my < W)
  uint64_t lvl_base = seg0;
  uint32_t W = 1, L = 2, deepest = 2, err = 0;
  uint32_t cut = kNoLevel;  // least level known to violate, read one level before it is used
  uint64_t vmin = kNone;
  while (L < 2 + N) {
    if (early && cut <= L) break;  // deeper widths are not counted
    const uint32_t sc = early ? ld_relaxed_u32(&ctrl->stop_c) : 0u;
    const bool valid = my < W;
    C clk = 0;
    if (valid && unit_ok) clk = (C)field(key, c_shift, n_mask) * t_c;
    C mx = clk, mn = (valid && unit_ok) ? clk : kNoneC;
    bool ok = valid && unit_ok;
    if (greedy) {
      group_minmax<true>(mx, mn, g);
      ok = ok && clk == mn;
    } else {
      group_minmax<false>(mx, mn, g);
    }
    const C nclk = clk + t_c;
    const C st = nclk > mx ? nclk : mx;  // model time of the successor
    if (prune && st > Tc) ok = false;
    const K succ = key + one_c;
    // every proposal of the level is in the warp: of equal keys the lowest
    // lane wins, the others are its duplicates
    const uint32_t am = __ballot_sync(0xffffffffu, ok);
    bool won = false;
    if (ok) {
      uint32_t peers = __match_any_sync(am, (unsigned long long)KeyOps<K>::lo(succ));
      if (sizeof(K) == 16) peers &= __match_any_sync(am, (unsigned long long)KeyOps<K>::hi(succ));
      won = lane == (uint32_t)(__ffs(peers) - 1);
    }
    const uint32_t wm = __ballot_sync(0xffffffffu, won);
    const uint32_t Wn = __popc(wm);
    if (won && log_on) {
      const uint64_t at = lvl_base + W + __popc(wm & ((1u << lane) - 1u));
      if (at < seg1) {
        log_store<K>(log_keys, at, succ);
        log_par[at] = (uint32_t)(lvl_base + my);
      } else {
        err = (uint32_t)MC_ERR_FRONTIER;
      }
    }
    // Step 2: a terminal winner with time <= T violates G(FIN -> time > T)
    if (L + 1 == 2 + N) vmin = warp_min_u64((won && (uint64_t)st <= T) ? (uint64_t)st : kNone);
    if (Wn > spw) {  // cannot happen when the width bound holds
      err = (uint32_t)MC_ERR_FRONTIER;
      break;
    }
    if (lane == 0 && Wn) atomicAdd(reinterpret_cast<unsigned long long*>(levels + 2 * (L + 1)), (unsigned long long)Wn);
    // the next level: state r from winner number r
    const uint32_t r = my < Wn ? my : 0u;
    key = shfl_key<K>(succ, Wn ? nth_set_bit(wm, r) : 0u);
    cut = sc ? ~sc : kNoLevel;
    lvl_base += W;
    W = Wn;
    ++L;
    if (W == 0) break;
    deepest = L;
  }
  // (uniform: the break above and a lane's log overflow)
  const uint32_t errs = __ballot_sync(0xffffffffu, err != 0);
  if (errs) return __shfl_sync(0xffffffffu, err, __ffs(errs) - 1);
  // this configuration's violating terminals (all at level 2 + N, held by
  // the warp): the smallest key of the least time, and its log index
  uint64_t whi = kNone, wlo = kNone;
  uint32_t widx = 0;
  if (vmin != kNone) {
    if (lane == 0 && early) atomicMax(&ctrl->stop_c, ~(2u + N));
    const bool mine = my < W && c == 0;
    uint64_t t = kNone;
    if (mine) {
      const uint64_t c0 = __ldg(costp + cfg);
      t = 0;
      for (uint32_t u = 0; u < P; ++u) {
        const uint64_t tu = (uint64_t)field(key, (P - 1 - u) * n_bits, n_mask) * c0 * __ldg(speedp + u);
        t = tu > t ? tu : t;
      }
    }
    const bool cand = mine && t == vmin;
    whi = warp_min_u64(cand ? (uint64_t)KeyOps<K>::hi(key) : kNone);
    const bool cand_hi = cand && (uint64_t)KeyOps<K>::hi(key) == whi;
    wlo = warp_min_u64(cand_hi ? (uint64_t)KeyOps<K>::lo(key) : kNone);
    const uint32_t wl = __ballot_sync(0xffffffffu, cand_hi && (uint64_t)KeyOps<K>::lo(key) == wlo);
    widx = (uint32_t)(lvl_base + (uint32_t)(__ffs(wl) - 1) / g);
  }
  if (lane == 0) {
    CfgRec rec;
    rec.vpack = vmin != kNone ? pack_tij(vmin, i, j) : kNone;
    rec.wkey_lo = vmin != kNone ? wlo : kNone;
    rec.wkey_hi = vmin != kNone ? whi : kNone;
    rec.widx = vmin != kNone ? widx : 0u;
    rec.deepest = deepest;
    Q.rec[cfg] = rec;
  }
  return 0;
}

// The pass header from the combined records (one thread): counts, first
// violating level, minima, the witness's trace, the published minimum.
template <class K>
__device__ void epilogue_publish(const CfgPass& Q, uint64_t T, uint32_t stop, uint32_t last, uint64_t e_best,
                                 uint64_t e_wpack, uint64_t e_sum) {
  const Params& p = Q.p;
  const uint32_t ab = p.a * p.b;
  Ctrl* ctrl = Q.ctrl;
  const uint64_t wpack = stop != kNoLevel ? e_wpack : kNone;
  const uint64_t best = Q.early_exit ? wpack : e_best;
  Q.levels[0] = 1;
  Q.levels[2] = p.a;
  Q.levels[4] = (uint64_t)ab;
  ctrl->T = T;
  ctrl->levels = last + 1;
  ctrl->states = 1 + (uint64_t)p.a + ab + e_sum;
  ctrl->stop_level = stop != kNoLevel ? stop : 0u;
  ctrl->best_pack = best;
  ctrl->wpack = wpack;
  if (Q.tmin_out && best != kNone) *Q.tmin_out = pack_time(best);
  if (!Q.want_witness || stop == kNoLevel) return;
  // witness: the smallest key of the least (time, i, j) at the first
  // violating level, found by its configuration's block; trace s0 -> it
  const uint32_t wi = pack_i(wpack), wj = pack_j(wpack);
  const uint32_t wcfg = wi * p.b + wj;
  const uint64_t klo = __ldcg(&Q.rec[wcfg].wkey_lo), khi = __ldcg(&Q.rec[wcfg].wkey_hi);
  uint64_t idx = __ldcg(&Q.rec[wcfg].widx);
  ctrl->wkey_lo = klo;
  ctrl->wkey_hi = sizeof(K) == 16 ? khi : 0;
  ctrl->widx = idx;
  for (uint32_t l = stop; l >= 2; --l) {
    const K key = KeyOps<K>::load(Q.log_keys, idx);
    Q.trace[2 * l] = KeyOps<K>::lo(key);
    Q.trace[2 * l + 1] = KeyOps<K>::hi(key);
    if (l == 2) break;
    idx = __ldcg(Q.log_par + idx);
    if (idx >= Q.seg[wcfg + 1] || idx < Q.seg[wcfg]) {  // cannot happen when the log is intact
      set_error(ctrl, MC_ERR_FRONTIER);
      return;
    }
  }
  const K k1 = (K)(wi + 1) << p.wg_shift;  // level 1: (i+1, 0, 0...0); level 0: s0
  Q.trace[2] = KeyOps<K>::lo(k1);
  Q.trace[3] = KeyOps<K>::hi(k1);
  Q.trace[0] = 0;
  Q.trace[1] = 0;
  ctrl->witness_level = stop;
  ctrl->trace_len = stop + 1;
}

// The block that finished a pass's last configuration: combine the
// configurations' records and the level widths into the pass header, write
// the trace of the witness, publish the minimum for a chained pass.
template <class K>
__device__ void cfg_epilogue(const CfgPass& Q, uint64_t T, CfgShared& S) {
  const Params& p = Q.p;
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  const uint32_t ab = p.a * p.b;
  Ctrl* ctrl = Q.ctrl;
  if (tid == 0) {
    S.e_best = kNone;
    S.e_wpack = kNone;
    S.e_sum = 0;
    S.e_stop = kNoLevel;
    S.e_deep = 2;
    S.err = ld_relaxed_u32(&ctrl->err);
  }
  __syncthreads();
  if (S.err) return;
  for (uint32_t cfg = tid; cfg < ab; cfg += nthr) {
    const uint64_t v = __ldcg(&Q.rec[cfg].vpack);
    const uint32_t d = __ldcg(&Q.rec[cfg].deepest);
    atomicMax(&S.e_deep, d);
    if (v != kNone) {
      atomicMin(&S.e_stop, 2u + __ldg(p.N + cfg));
      atomicMin(&S.e_best, (unsigned long long)v);
    }
  }
  __syncthreads();
  const uint32_t stop = S.e_stop;
  if (stop != kNoLevel)
    for (uint32_t cfg = tid; cfg < ab; cfg += nthr) {
      const uint64_t v = __ldcg(&Q.rec[cfg].vpack);
      if (v != kNone && 2u + __ldg(p.N + cfg) == stop) atomicMin(&S.e_wpack, (unsigned long long)v);
    }
  const uint32_t last = (Q.early_exit && stop != kNoLevel) ? stop : S.e_deep;
  uint64_t part = 0;
  for (uint32_t l = 3 + tid; l <= last; l += nthr) part += __ldcg(Q.levels + 2 * l);
  atomicAdd(&S.e_sum, (unsigned long long)part);
  __syncthreads();
  if (tid != 0) return;
  epilogue_publish<K>(Q, T, stop, last, (uint64_t)S.e_best, (uint64_t)S.e_wpack, (uint64_t)S.e_sum);
}

// The warp that finished a pass's last configuration, when it is a warp
// unit: the same combination as cfg_epilogue, reduced across the warp.
template <class K>
__device__ void cfg_epilogue_warp(const CfgPass& Q, uint64_t T) {
  const Params& p = Q.p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t ab = p.a * p.b;
  if (ld_relaxed_u32(&Q.ctrl->err)) return;
  uint64_t best = kNone;
  uint32_t stop = kNoLevel, deep = 2;
  for (uint32_t cfg = lane; cfg < ab; cfg += 32) {
    const uint64_t v = __ldcg(&Q.rec[cfg].vpack);
    const uint32_t d = __ldcg(&Q.rec[cfg].deepest);
    deep = d > deep ? d : deep;
    if (v != kNone) {
      const uint32_t s = 2u + __ldg(p.N + cfg);
      stop = s < stop ? s : stop;
      best = v < best ? v : best;
    }
  }
  deep = __reduce_max_sync(0xffffffffu, deep);
  stop = __reduce_min_sync(0xffffffffu, stop);
  best = warp_min_u64(best);
  uint64_t wpack = kNone;
  if (stop != kNoLevel) {
    for (uint32_t cfg = lane; cfg < ab; cfg += 32) {
      const uint64_t v = __ldcg(&Q.rec[cfg].vpack);
      if (v != kNone && 2u + __ldg(p.N + cfg) == stop) wpack = v < wpack ? v : wpack;
    }
    wpack = warp_min_u64(wpack);
  }
  const uint32_t last = (Q.early_exit && stop != kNoLevel) ? stop : deep;
  uint64_t part = 0;
  for (uint32_t l = 3 + lane; l <= last; l += 32) part += __ldcg(Q.levels + 2 * l);
  const uint64_t sum = warp_sum_u64(part);
  if (lane == 0) epilogue_publish<K>(Q, T, stop, last, best, wpack, sum);
}

// Blocks [0, warp_blocks) of a launch: every warp takes warp units until
// none is left (no block barrier: the warps of a block run independently).
// (Measured: inlined, the block units' code runs 0.8% slower than without
// the warp path; kept out of line, 3.7%.)
template <class K>
__device__ void warp_role(const CfgLaunch& A) {
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(A.wnext, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    const uint64_t n = A.n_wunits_dev ? (uint64_t)*A.n_wunits_dev : A.n_wunits;
    if (u >= n) return;
    const uint64_t code = A.wunits ? __ldg(A.wunits_rev ? A.wunits - u : A.wunits + u) : 0ull;
    const CfgPass& Q = A.wunits ? A.passes[code >> 32] : A.one;
    const uint32_t cfg = A.wunits ? (uint32_t)code : __ldg(Q.order + u);
    // the threshold, as for a block unit
    unsigned long long t = 0;
    uint32_t skip = 0;
    if (lane == 0) {
      t = Q.T;
      if (Q.T_src) t = ld_relaxed_u64(Q.T_src) + (uint64_t)Q.T_delta;
      if (Q.prev) {
        const Ctrl* q = Q.prev;
        if (ld_relaxed_u32(&q->err) || ld_relaxed_u32(&q->skipped) || ld_relaxed_u32(&q->stop_level) == 0) skip = 1;
        else t = pack_time(ld_relaxed_u64(&q->wpack)) - 1;
      }
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    skip = __shfl_sync(0xffffffffu, skip, 0);
    if (!skip) {
      const uint32_t err = Q.p.clk32 ? explore_unit_warp<K, uint32_t>(Q, cfg, t)
                                     : explore_unit_warp<K, uint64_t>(Q, cfg, t);
      if (lane == 0 && err) set_error(Q.ctrl, (int)err);
    }
    // completion, as for a block unit: the warp that finishes the pass's
    // last configuration combines the pass
    uint32_t last = 0;
    if (lane == 0) {
      __threadfence();
      const uint32_t done = atomicAdd(&Q.ctrl->units_done, 1u) + 1;
      last = done == Q.p.a * Q.p.b;
      if (last) __threadfence();
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      if (skip) {
        if (lane == 0) Q.ctrl->skipped = 1;
      } else {
        cfg_epilogue_warp<K>(Q, t);
      }
    }
    __syncwarp();
  }
}

template <class K>
__global__ void __launch_bounds__(kCfgMaxThreads) cfg_kernel(const __grid_constant__ CfgLaunch A) {
  extern __shared__ __align__(16) unsigned char cfg_dyn[];
  __shared__ CfgShared S;
  K* front0 = reinterpret_cast<K*>(cfg_dyn);
  K* front1 = front0 + A.wcap;
  K* tab0 = front1 + A.wcap;
  K* tab1 = tab0 + A.tsize;
  if (blockIdx.x < A.warp_blocks) {  // a block of warp units (no block barrier below)
    warp_role<K>(A);
    return;
  }
  const uint32_t tid = threadIdx.x, nthr = blockDim.x;
  constexpr uint32_t kWords = sizeof(CfgPass) / 8;
  static_assert(sizeof(CfgPass) % 8 == 0, "CfgPass is copied in 8-byte words");
  for (;;) {
    // the next unit: a pass and one of its configurations
    if (tid == 0) S.unit = atomicAdd(A.next, 1u);
    __syncthreads();
    const uint32_t u = S.unit;
    const uint64_t n_units = A.n_units_dev ? (uint64_t)*A.n_units_dev : A.n_units;
    if (u >= n_units) return;
    const uint64_t code = A.units ? __ldg(A.units + u) : 0ull;
    const CfgPass* src = A.units ? A.passes + (code >> 32) : &A.one;
    for (uint32_t w = tid; w < kWords; w += nthr)
      reinterpret_cast<uint64_t*>(&S.Q)[w] = reinterpret_cast<const uint64_t*>(src)[w];
    __syncthreads();
    const CfgPass& Q = S.Q;
    const uint32_t cfg = A.units ? (uint32_t)code : __ldg(Q.order + u);
    if (tid == 0) {
      // the threshold: given, read from the device, or one below the
      // chained predecessor's counterexample time (no run once it held)
      uint64_t t = Q.T;
      uint32_t skip = 0;
      if (Q.T_src) t = ld_relaxed_u64(Q.T_src) + (uint64_t)Q.T_delta;
      if (Q.prev) {
        const Ctrl* q = Q.prev;
        if (ld_relaxed_u32(&q->err) || ld_relaxed_u32(&q->skipped) || ld_relaxed_u32(&q->stop_level) == 0) skip = 1;
        else t = pack_time(ld_relaxed_u64(&q->wpack)) - 1;
      }
      S.T = t;
      S.skip = skip;
      S.vmin = kNone;
      S.whi = kNone;
      S.wlo = kNone;
      S.widx = 0;
      S.err = 0;
      S.cnt[0] = 0;  // level 3 counts into cnt[3 % 3]; level 2 (the configuration's
      S.cnt[1] = 0;  // select state alone) is not counted here
      S.cnt[2] = 0;
      S.cut[0] = kNoLevel;
      S.cut[1] = kNoLevel;
    }
    for (uint32_t x = tid; x < 2 * A.tsize; x += nthr) tab0[x] = (K)0;
    __syncthreads();
    const uint64_t T = S.T;
    if (!S.skip) {
      if (Q.p.clk32) explore_unit<K, uint32_t>(Q, cfg, T, front0, front1, tab0, tab1, A.wcap, A.tsize, S);
      else explore_unit<K, uint64_t>(Q, cfg, T, front0, front1, tab0, tab1, A.wcap, A.tsize, S);
      __syncthreads();
      if (tid == 0 && S.err) set_error(Q.ctrl, (int)S.err);
    }
    // completion: the block that finishes the pass's last configuration
    // combines the pass (its own and every other block's writes are ordered
    // before the count by the fences)
    if (tid == 0) {
      __threadfence();
      const uint32_t done = atomicAdd(&Q.ctrl->units_done, 1u) + 1;
      S.last = done == Q.p.a * Q.p.b;
      if (S.last) __threadfence();
    }
    __syncthreads();
    if (S.last) {
      if (S.skip) {
        if (tid == 0) Q.ctrl->skipped = 1;
      } else {
        cfg_epilogue<K>(Q, T, S);
      }
    }
    __syncthreads();
  }
}

// Clear the pass headers and level widths of every model of a run and set
// its {T_ini, T_min} words; one block per model.
__global__ void cfg_clear_kernel(const CfgClear* clears, const uint32_t* n_dev) {
  const uint32_t n = *n_dev;
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    const CfgClear c = clears[k];
    for (uint64_t x = threadIdx.x; x < c.level_words; x += blockDim.x) c.levels[x] = 0;
    uint64_t* h = reinterpret_cast<uint64_t*>(c.ctrl);
    const uint64_t hw = (uint64_t)c.n_ctrl * sizeof(Ctrl) / 8;
    for (uint64_t x = threadIdx.x; x < hw; x += blockDim.x) h[x] = 0;
    if (threadIdx.x == 0) {
      c.scal[0] = kNone;
      c.scal[1] = 0;
    }
  }
}

// T_ini of every min-time model of a run: walk w of model k is random run
// number w of its seed (as mc_simulate), the least terminal time wins.
__global__ void cfg_sim_kernel(const CfgSim* sims, const uint32_t* n_dev, uint32_t walks_max) {
  const uint32_t n = *n_dev;
  const uint64_t total = (uint64_t)n * walks_max;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(x / walks_max), w = (uint32_t)(x % walks_max);
    const CfgSim& s = sims[k];
    if (w >= s.walks) continue;
    atomicMin(reinterpret_cast<unsigned long long*>(s.tini), (unsigned long long)simulate_walk(s.p, s.seed, w));
  }
}

}  // namespace

cudaError_t launch_cfg_clear(const CfgClear* clears, const uint32_t* n_dev, uint32_t n_max, cudaStream_t stream) {
  if (n_max == 0) return cudaSuccess;
  const int grid = (int)(n_max < 4096 ? n_max : 4096);
  cfg_clear_kernel<<<grid, 256, 0, stream>>>(clears, n_dev);
  return cudaGetLastError();
}

cudaError_t launch_cfg_sim(const CfgSim* sims, const uint32_t* n_dev, uint32_t n_max, uint32_t walks_max,
                           cudaStream_t stream) {
  if (n_max == 0 || walks_max == 0) return cudaSuccess;
  const uint64_t total = (uint64_t)n_max * walks_max;
  int grid = (int)((total + 127) / 128);
  if (grid > 4096) grid = 4096;
  cfg_sim_kernel<<<grid, 128, 0, stream>>>(sims, n_dev, walks_max);
  return cudaGetLastError();
}

size_t cfg_smem_bytes(int key_words, uint32_t wcap, uint32_t tsize) {
  return (size_t)8 * key_words * (2ull * wcap + 2ull * tsize);
}

// The kernels' dynamic shared memory limit is a property of the function,
// shared by every model: it is raised once to the device's opt-in maximum
// (a model's own size would lower it under a larger one reserved earlier).
int cfg_occupancy(int key_words, int threads, size_t smem, int* blocks_per_sm) {
  const void* f = key_words == 1 ? (const void*)cfg_kernel<uint64_t> : (const void*)cfg_kernel<u128>;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return -1;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return -1;
  const int static_bytes = (int)fa.sharedSizeBytes;
  if ((int)smem > optin - static_bytes) return -1;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - static_bytes) != cudaSuccess)
    return -1;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem) == cudaSuccess ? 0 : -1;
}

cudaError_t launch_cfg(int key_words, int grid, int threads, size_t smem, const CfgLaunch& L,
                       cudaStream_t stream) {
  if (key_words == 1) cfg_kernel<uint64_t><<<grid, threads, smem, stream>>>(L);
  else cfg_kernel<u128><<<grid, threads, smem, stream>>>(L);
  return cudaGetLastError();
}

}  // namespace mc
