// Processing-element level model (include/mc_pe.h): device explorer and its
// host driver.
//
// The state keeps, per compute unit, the work-groups it has taken, whether it
// is busy, its program step and the set of its PEs that marked the step
// (reported a clock tick or arrived at the local barrier).  One tile of lanes
// handles one state: lane (c, e) for c < P, e < M proposes "PE e of unit c
// marks", lane P*M + c proposes "unit c passes its barrier" or "unit c takes
// the next work-group", and lane P*M + P proposes the clock tick (Listings
// 5-9).  The rest of a pass is the level-synchronous BFS of the cost-table
// explorer (mc_kernels.cu): lock-free visited set with CAS on 128-bit keys,
// frontier log with parent indices, a device-wide barrier per level, the
// minimum packed (time, i, j) over violating FIN states per level, witness and
// trace.  The BFS level is a field of the key (every path to a state has the
// same length), so a slot holding a key of an earlier level counts as free.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mc.h"
#include "mc_device.cuh"
#include "mc_host.h"
#include "mc_internal.h"
#include "mc_pe.h"

namespace mc {
namespace {

using namespace mc::dev;

constexpr uint32_t kPeMaxUnits = 8;
constexpr uint32_t kPeMaxPes = 8;
constexpr uint32_t kBarrierBit = 1u << 16;  // step info: barrier flag | participating PEs
// successors per lane a tile of `tile` lanes can propose: one for a whole
// warp, two for half a warp, three for smaller tiles
__host__ __device__ constexpr uint32_t slots_for(uint32_t tile) { return tile >= 32 ? 1 : tile == 16 ? 2 : 3; }

struct PeParams {
  uint32_t a, b, P, M;          // M: mask bits per unit (largest NWE)
  uint32_t n_bits, pc_bits, unit_bits, lvl_bits;
  uint32_t wg_shift, ts_shift, lvl_shift, max_level;
  uint32_t wg_mask, ts_mask;
  uint64_t unit_mask, lvl_mask;
  const uint32_t* N;       // [a*b] work-groups
  const uint32_t* tau;     // [a*b] ticks of one program
  const uint32_t* nsteps;  // [a*b] steps of one program
  const uint32_t* soff;    // [a*b] first step of each program
  const uint2* step;       // [steps] {barrier bit | pes, ticks before the step}
};

struct PeArgs {
  PeParams p;
  void* table;
  uint64_t bucket_mask;
  uint64_t table_u64;
  uint32_t max_probes;
  uint32_t prune;
  uint32_t early_exit;
  uint32_t want_witness;
  void* log_keys;
  uint32_t* log_par;
  uint64_t log_cap;
  Ctrl* ctrl;
  uint64_t* levels;  // [max_level + 2] x {width, min packed violating FIN}
  uint64_t* off;
  uint64_t* trace;
  uint64_t T;
  const uint64_t* T_src;
  int64_t T_delta;
  uint64_t* tmin_out;
  uint32_t* bar;
  uint64_t timeout_ns;
  uint32_t slots;    // successors per lane: ceil(lanes / TILE) <= slots_for(TILE)
  uint32_t pad;
};

struct Unit {
  uint32_t n, busy, pc, mask;
};

__device__ __forceinline__ uint64_t unit_field(u128 key, const PeParams& p, uint32_t c) {
  return (uint64_t)(key >> ((p.P - 1 - c) * p.unit_bits)) & p.unit_mask;
}
__device__ __forceinline__ uint32_t pe_level(u128 key, const PeParams& p) {
  return (uint32_t)((uint64_t)(key >> p.lvl_shift) & p.lvl_mask);
}
__device__ __forceinline__ Unit unpack(uint64_t f, const PeParams& p) {
  Unit u;
  u.mask = (uint32_t)(f & ((1u << p.M) - 1));
  u.pc = (uint32_t)((f >> p.M) & ((1ull << p.pc_bits) - 1));
  u.busy = (uint32_t)((f >> (p.M + p.pc_bits)) & 1u);
  u.n = (uint32_t)(f >> (p.M + p.pc_bits + 1));
  return u;
}
__device__ __forceinline__ uint64_t pack(const Unit& u, const PeParams& p) {
  return ((uint64_t)u.n << (p.M + p.pc_bits + 1)) | ((uint64_t)u.busy << (p.M + p.pc_bits)) |
         ((uint64_t)u.pc << p.M) | u.mask;
}

// What every lane of a tile needs about its state, in scalars (the loops over
// units are unrolled to kPeMaxUnits with a guard, so nothing is indexed at run
// time and nothing goes to local memory).
struct Decoded {
  uint32_t i, j, cfg, left, S, so;
  uint32_t busy_mask;  // bit c: unit c is busy
  uint32_t mark_floor; // 1 + the highest marked (unit, PE) index c * M + e, 0 when nothing is marked
  uint64_t tau, time;
  bool ready;          // every busy unit is at a tick step with all participants marked
};

template <bool CG = false>
__device__ __forceinline__ void decode(u128 key, const PeParams& p, Decoded& d) {
  d.i = (uint32_t)((uint64_t)(key >> p.wg_shift) & p.wg_mask) - 1;
  d.j = (uint32_t)((uint64_t)(key >> p.ts_shift) & p.ts_mask) - 1;
  d.cfg = d.i * p.b + d.j;
  d.tau = ldp<CG>(p.tau + d.cfg);
  d.S = ldp<CG>(p.nsteps + d.cfg);
  d.so = ldp<CG>(p.soff + d.cfg);
  uint32_t taken = 0;
  d.busy_mask = 0;
  d.mark_floor = 0;
  d.ready = true;
  d.time = 0;
#pragma unroll
  for (uint32_t c = 0; c < kPeMaxUnits; ++c) {
    if (c >= p.P) break;
    const Unit u = unpack(unit_field(key, p, c), p);
    taken += u.n;
    uint64_t clk;
    if (u.busy) {
      const uint2 st = __ldg(p.step + d.so + u.pc);
      d.busy_mask |= 1u << c;
      const uint32_t pes = st.x & 0xFFFFu;
      if ((st.x & kBarrierBit) || u.mask != (1u << pes) - 1u) d.ready = false;
      if (u.mask) d.mark_floor = c * p.M + (32u - __clz(u.mask));
      clk = (uint64_t)(u.n - 1) * d.tau + st.y;
    } else {
      clk = (uint64_t)u.n * d.tau;
    }
    d.time = clk > d.time ? clk : d.time;
  }
  d.left = ldp<CG>(p.N + d.cfg) - taken;
}

__device__ __forceinline__ bool is_fin(const Decoded& d) { return d.left == 0 && d.busy_mask == 0; }
__device__ __forceinline__ bool any_idle(const Decoded& d, const PeParams& p) {
  return d.busy_mask != (1u << p.P) - 1u;
}

// next program step of a busy unit (idle at the program's end)
__device__ __forceinline__ Unit step_on(Unit u, uint32_t S) {
  u.pc += 1;
  u.mask = 0;
  if (u.pc == S) {
    u.busy = 0;
    u.pc = 0;
  }
  return u;
}

template <int TILE>
struct PeStage {
  u128 keys[kThreads / 32][kWarpCap];
  uint32_t par[kThreads / 32][kWarpCap];
  uint32_t fill[kThreads / 32];
  unsigned long long base;
  uint32_t flags;  // this level: kPeFlagError | kPeFlagViolation
};

constexpr uint32_t kPeFlagError = 1;
constexpr uint32_t kPeFlagViolation = 2;

__device__ __forceinline__ void pe_copy_out(const PeArgs& A, const u128* keys, const uint32_t* par,
                                            uint32_t n, uint64_t at0, uint32_t lane, uint32_t* flags) {
  for (uint32_t x = lane; x < n; x += 32) {
    const uint64_t at = at0 + x;
    if (at < A.log_cap) {
      KeyOps<u128>::store(A.log_keys, at, keys[x]);
      A.log_par[at] = par[x];
    } else {
      set_error(A.ctrl, MC_ERR_FRONTIER);
      atomicOr(flags, kPeFlagError);
    }
  }
}

// Successor number `slot` of a decoded state (the lane roles above).  Sets
// ok when the transition is enabled, with the successor's key (level field
// not yet raised), its model time and whether it is FIN.
__device__ __forceinline__ void propose(const PeParams& p, const Decoded& d, u128 key, uint32_t slot,
                                        bool& ok, u128& succ, uint64_t& t, bool& term) {
  const uint32_t PM = p.P * p.M;
  ok = false;
  term = false;
  succ = key;
  t = d.time;
  if (slot < PM + p.P) {  // a mark of PE e of unit c, or unit c's release / dispatch
    const uint32_t c = slot < PM ? slot / p.M : slot - PM;
    const uint32_t shift = (p.P - 1 - c) * p.unit_bits;
    const Unit u = unpack(unit_field(key, p, c), p);
    const uint32_t info = u.busy ? __ldg(&p.step[d.so + u.pc].x) : 0u;
    const uint32_t pes = info & 0xFFFFu;
    if (slot < PM) {
      // marks are proposed only above the highest marked (unit, PE) index:
      // a state whose highest mark is (c, e) is still reached from the state
      // without that mark, and the other orders of the same marks only
      // generated it again
      const uint32_t e = slot - c * p.M;
      if (u.busy && e < pes && !((u.mask >> e) & 1u) && slot >= d.mark_floor) {
        ok = true;
        succ = key ^ ((u128)(1u << e) << shift);
      }
    } else {
      Unit v = u;
      if (u.busy) {
        if ((info & kBarrierBit) && u.mask == (1u << pes) - 1u) {
          ok = true;
          v = step_on(u, d.S);
          term = d.left == 0 && !v.busy && (d.busy_mask & ~(1u << c)) == 0;
        }
      } else if (d.left > 0) {
        ok = true;
        v.n = u.n + 1;
        v.busy = 1;
        v.pc = 0;
        v.mask = 0;
      }
      if (ok) succ = key ^ ((u128)(pack(u, p) ^ pack(v, p)) << shift);
    }
  } else if (slot == PM + p.P && d.busy_mask && d.ready && !(d.left > 0 && any_idle(d, p))) {
    ok = true;  // the clock ticks; every busy unit moves on
    bool all_idle = true;
#pragma unroll
    for (uint32_t c = 0; c < kPeMaxUnits; ++c) {
      if (c >= p.P) break;
      if (!((d.busy_mask >> c) & 1u)) continue;
      const Unit u = unpack(unit_field(key, p, c), p);
      const Unit v = step_on(u, d.S);
      if (v.busy) all_idle = false;
      succ ^= (u128)(pack(u, p) ^ pack(v, p)) << ((p.P - 1 - c) * p.unit_bits);
    }
    t = d.time + 1;
    term = d.left == 0 && all_idle;
  }
}

// Expand level L (states offL .. offL+W-1 of the log) into level L+1.  A tile
// of TILE lanes owns one state; lane l proposes successors l, l + TILE, ...
// (A.slots of them), fetches the first bucket of each with cp.async so that
// all of its probes are in flight together, then inserts them in turn.
// `probes` (lane 0 of each warp) accumulates the successors the warp made.
template <int TILE>
__device__ void pe_expand_level(const PeArgs& A, PeStage<TILE>& st, uint64_t T, uint32_t L,
                                uint64_t offL, uint64_t W, uint64_t offN, uint64_t& probes) {
  constexpr uint32_t SL = slots_for(TILE);
  __shared__ __align__(16) u128 probe[kThreads][SL][2];
  const PeParams& p = A.p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t l = lane & (TILE - 1);
  constexpr uint32_t kTilesPerWarp = 32 / TILE;
  const uint64_t warp_gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * kTilesPerWarp;
  const uint32_t slots = A.slots;
  u128* table = reinterpret_cast<u128*>(A.table);
  u128* wkeys = st.keys[warp];
  uint32_t* wpar = st.par[warp];
  uint64_t* lvl_next = A.levels + 2 * (L + 1);
  uint64_t cached_best = kNone;
  uint32_t fill = 0;
  const u128 lvl_one = (u128)1 << p.lvl_shift;
  auto level_of = [&p](u128 k) { return pe_level(k, p); };

  uint64_t base = warp_gid * kTilesPerWarp;
  u128 key_next = base + lane / TILE < W ? KeyOps<u128>::load(A.log_keys, offL + base + lane / TILE) : (u128)0;
  for (; base < W; base += stride) {
    const uint64_t s = base + lane / TILE;
    const bool valid = s < W;
    const u128 key = key_next;
    if (s + stride < W) key_next = KeyOps<u128>::load(A.log_keys, offL + s + stride);
    bool ok[SL], term[SL];
    u128 succ[SL];
    uint64_t st_time[SL], bkt[SL];
    uint32_t ci = 0, cj = 0;
    Decoded d;
    if (valid) {
      decode(key, p, d);
      ci = d.i;
      cj = d.j;
    }
#pragma unroll
    for (uint32_t k = 0; k < SL; ++k) {
      ok[k] = false;
      term[k] = false;
      bkt[k] = 0;
      st_time[k] = 0;
      succ[k] = 0;
      if (valid && k < slots) {
        propose(p, d, key, l + k * TILE, ok[k], succ[k], st_time[k], term[k]);
        if (ok[k] && A.prune && st_time[k] > T) ok[k] = false;
        succ[k] += lvl_one;
      }
      probes += __popc(__ballot_sync(0xffffffffu, ok[k]));
      if (ok[k]) {
        bkt[k] = key_hash(succ[k]) & A.bucket_mask;
        const u128* src = table + bkt[k] * 2;
        cp_async16(&probe[threadIdx.x][k][0], src);
        cp_async16(&probe[threadIdx.x][k][1], src + 1);
      }
    }
    cp_async_wait_all();
#pragma unroll
    for (uint32_t k = 0; k < SL; ++k) {
      int won = 0;
      if (ok[k]) {
        const int rc = visited_insert_lv<u128>(table, A.bucket_mask, A.max_probes, succ[k], L + 1, level_of,
                                               bkt[k], probe[threadIdx.x][k]);
        if (rc < 0) {
          set_error(A.ctrl, MC_ERR_TABLE_FULL);
          atomicOr(&st.flags, kPeFlagError);
        }
        won = rc > 0;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, won);
      if (m) {
        if (won) {
          const uint32_t at = fill + __popc(m & ((1u << lane) - 1u));
          wkeys[at] = succ[k];
          wpar[at] = (uint32_t)s;
        }
        fill += __popc(m);
        uint64_t pk = (won && term[k] && st_time[k] <= T) ? pack_tij(st_time[k], ci, cj) : kNone;
        pk = warp_min(pk);
        if (lane == 0 && pk != kNone) atomicOr(&st.flags, kPeFlagViolation);
        if (lane == 0 && pk < cached_best) {
          cached_best = ld_relaxed_u64(lvl_next + 1);
          if (pk < cached_best) {
            atomicMin(reinterpret_cast<unsigned long long*>(lvl_next + 1), (unsigned long long)pk);
            cached_best = pk;
          }
        }
      }
      // each slot adds at most 32 winners to the warp's buffer
      if (fill > kWarpCap - 32) {
        __syncwarp();
        unsigned long long b = 0;
        if (lane == 0) b = level_reserve(lvl_next, fill);
        b = __shfl_sync(0xffffffffu, b, 0);
        pe_copy_out(A, wkeys, wpar, fill, offN + b, lane, &st.flags);
        __syncwarp();
        fill = 0;
      }
    }
  }
  if (lane == 0) st.fill[warp] = fill;
  __syncthreads();
  const uint32_t nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    uint32_t total = 0;
    for (uint32_t w = 0; w < nw; ++w) total += st.fill[w];
    st.base = total ? level_reserve(lvl_next, total) : 0ull;
  }
  __syncthreads();
  if (fill) {
    uint64_t at0 = offN + st.base;
    for (uint32_t w = 0; w < warp; ++w) at0 += st.fill[w];
    pe_copy_out(A, wkeys, wpar, fill, at0, lane, &st.flags);
  }
}

// Register budgets: 64 per thread (4 blocks of 256 per SM) for warp-wide
// tiles (one successor per lane), 85 (3 blocks) for the narrower tiles, whose
// lanes propose two or three successors and spill at 64 (the Minimum model
// measured 4% faster at 16 lanes without the spill).
template <int TILE>
__global__ void __launch_bounds__(kThreads, TILE >= 32 ? 4 : 3) pe_explore_kernel(const PeArgs A) {
  const PeParams& p = A.p;
  Ctrl* ctrl = A.ctrl;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  __shared__ PeStage<TILE> stage;
  uint32_t epoch = 0;
  const Barrier bar{A.bar, &A.ctrl->err, 0, A.timeout_ns};

  // threshold from the device when chained (one read per block: thousands of
  // warps polling one line would queue at its L2 slice)
  __shared__ unsigned long long s_T;
  if (threadIdx.x == 0) s_T = A.T_src ? ld_relaxed_u64(A.T_src) + (uint64_t)A.T_delta : A.T;
  __syncthreads();
  const uint64_t T = s_T;

  // prologue: empty visited set; levels 0..2 (the selects of Listing 3)
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
      u128 key = 0;
      uint32_t par = kNoParent;
      if (x >= 1 && x <= p.a) {
        key = ((u128)x << p.wg_shift) | ((u128)1 << p.lvl_shift);
        par = 0;
      } else if (x > p.a) {
        const uint64_t y = x - 1 - p.a;
        const uint32_t i = (uint32_t)(y / p.b), j = (uint32_t)(y % p.b);
        key = ((u128)(i + 1) << p.wg_shift) | ((u128)(j + 1) << p.ts_shift) | ((u128)2 << p.lvl_shift);
        par = i;
      }
      KeyOps<u128>::store(A.log_keys, x, key);
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

  uint32_t last = 2;
  uint64_t off_last = 1 + (uint64_t)p.a;
  uint64_t W = (uint64_t)p.a * p.b;
  uint64_t probes = 0;
  for (;;) {
    const uint32_t L = last;
    if (L >= p.max_level) break;
    const uint64_t offN = off_last + W;
    if (gtid == 0) A.off[L + 1] = offN;
    pe_expand_level<TILE>(A, stage, T, L, off_last, W, offN, probes);
    // level L+1's width word is the barrier (level_sync)
    uint64_t word = 0;
    if (!level_sync(bar, A.levels + 2 * (L + 1), &stage.flags,
                    kPeFlagError | (A.early_exit ? kPeFlagViolation : 0u), &word))
      return;
    const uint64_t Wn = word & kLevelWidthMask;
    if ((word >> kLevelStopShift) & 0xFFFFu) {
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
  if ((threadIdx.x & 31u) == 0 && probes)
    atomicAdd(reinterpret_cast<unsigned long long*>(&ctrl->probes), (unsigned long long)probes);
  if (ld_relaxed_u32(&ctrl->err)) return;

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

  // witness: among the FIN states of level wl with the level's minimum
  // (time, i, j), the smallest key (high word first, then low word)
  const uint64_t target = ld_relaxed_u64(A.levels + 2 * wl + 1);
  const uint64_t offW = ld_relaxed_u64(&A.off[wl]);
  const uint64_t Ww = ld_relaxed_u64(A.levels + 2 * wl) & kLevelWidthMask;
  auto matches = [&](u128 key) {
    Decoded d;
    decode(key, p, d);
    return is_fin(d) && pack_tij(d.time, d.i, d.j) == target;
  };
  for (uint64_t x = gtid; x < Ww; x += nthreads) {
    const u128 key = KeyOps<u128>::load(A.log_keys, offW + x);
    if (matches(key))
      atomicMin(reinterpret_cast<unsigned long long*>(&ctrl->wkey_hi), (unsigned long long)(key >> 64));
  }
  if (!grid_sync(bar, epoch)) return;
  const uint64_t whi = ld_relaxed_u64(&ctrl->wkey_hi);
  for (uint64_t x = gtid; x < Ww; x += nthreads) {
    const u128 key = KeyOps<u128>::load(A.log_keys, offW + x);
    if ((uint64_t)(key >> 64) == whi && matches(key))
      atomicMin(reinterpret_cast<unsigned long long*>(&ctrl->wkey_lo), (unsigned long long)key);
  }
  if (!grid_sync(bar, epoch)) return;
  {
    const uint64_t wlo = ld_relaxed_u64(&ctrl->wkey_lo);
    for (uint64_t x = gtid; x < Ww; x += nthreads) {
      const u128 key = KeyOps<u128>::load(A.log_keys, offW + x);
      if ((uint64_t)key == wlo && (uint64_t)(key >> 64) == whi) ctrl->widx = x;
    }
  }
  if (!grid_sync(bar, epoch)) return;
  if (gtid == 0) {
    uint64_t idx = ld_relaxed_u64(&ctrl->widx);
    if (idx >= Ww) {
      set_error(ctrl, MC_ERR_FRONTIER);
      return;
    }
    uint32_t l = wl;
    for (;;) {
      const uint64_t at = ld_relaxed_u64(&A.off[l]) + idx;
      const u128 key = KeyOps<u128>::load(A.log_keys, at);
      A.trace[2 * l] = (uint64_t)key;
      A.trace[2 * l + 1] = (uint64_t)(key >> 64);
      if (l == 0) break;
      idx = __ldcg(A.log_par + at);
      --l;
    }
    ctrl->witness_level = wl;
    ctrl->trace_len = wl + 1;
  }
}

const void* pe_pick(uint32_t tile) {
  switch (tile) {
    case 4: return (const void*)pe_explore_kernel<4>;
    case 8: return (const void*)pe_explore_kernel<8>;
    case 16: return (const void*)pe_explore_kernel<16>;
    case 32: return (const void*)pe_explore_kernel<32>;
  }
  return nullptr;
}

uint32_t bits_for(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace
}  // namespace mc

// ------------------------------------------------------------------ host side
struct mc_pe_model {
  uint32_t a = 0, b = 0, P = 0, M = 0;
  std::vector<uint32_t> wg, ts, N, tau, nsteps, soff;
  std::vector<uint2> steps;
  mc_options opt{};
  mc_pe_layout lay{};
  mc::PeParams params{};
  uint64_t table_slots = 0, log_cap = 0;
  uint32_t max_probes = 64;
  // device state
  int device = -1, grid = 0, threads = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> bufs;
  void* d_table = nullptr;
  void* d_log_keys = nullptr;
  uint32_t* d_log_par = nullptr;
  mc::Ctrl* d_ctrl = nullptr;
  uint32_t* d_bar = nullptr;
  uint64_t *d_levels = nullptr, *d_off = nullptr, *d_trace = nullptr, *d_tmin = nullptr;
  uint8_t* h_block = nullptr;    // pinned host staging (pooled), carved into:
  size_t h_block_bytes = 0;
  mc::Ctrl* h_ctrl = nullptr;    // [3]
  uint64_t* h_trace = nullptr;   // [(max_level + 2) * 2]
  cudaEvent_t ev[6] = {};
  bool ev_pending[3] = {};
  bool reserved = false;
  uint32_t last_levels = 0;
  mc_stats stats{};
  std::string last_err;
};

namespace {

using mc::Ctrl;
using mc::kNone;

int pe_cuda_fail(mc_pe_model* m, cudaError_t e, const char* what) {
  m->last_err = std::string(what) + ": " + cudaGetErrorString(e);
  return MC_ERR_CUDA;
}

#define PE_CUDA(m, call)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return pe_cuda_fail((m), e_, #call); \
  } while (0)

#define PE_TRY(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

void pe_release(mc_pe_model* m) {
  if (!m->bufs.empty()) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (m->device >= 0 && prev != m->device) cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    for (void* b : m->bufs) cudaFree(b);
    m->bufs.clear();
    if (prev >= 0 && prev != m->device) cudaSetDevice(prev);
  }
  if (m->h_block) mc::pinned_free(m->h_block, m->h_block_bytes);
  m->h_block = nullptr;
  for (cudaEvent_t& e : m->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  m->h_ctrl = nullptr;
  m->h_trace = nullptr;
  m->reserved = false;
}

void* pe_alloc(mc_pe_model* m, size_t bytes) {
  bytes = (std::max<size_t>(bytes, 256) + 255) & ~(size_t)255;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  m->bufs.push_back(p);
  return p;
}

uint64_t pe_device_bytes(const mc_pe_model* m) {
  const uint64_t L2 = m->lay.max_level + 2;
  return m->table_slots * 16 + m->log_cap * 20 + 256 + mc::kBarBytes + 40 * L2 + 64 +
         4ull * (4 * (uint64_t)m->a * m->b) + 8ull * m->steps.size();
}

int pe_reserve(mc_pe_model* m) {
  if (m->reserved) return MC_OK;
  int dev = 0;
  PE_CUDA(m, cudaGetDevice(&dev));
  m->device = dev;
  int sms = 0, coop = 0;
  PE_CUDA(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PE_CUDA(m, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    m->last_err = "device lacks cooperative launch";
    return MC_ERR_CUDA;
  }
  m->threads = m->opt.threads_per_block ? (int)m->opt.threads_per_block : (int)mc::kThreads;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mc::pe_pick(m->lay.tile), m->threads, 0) !=
          cudaSuccess ||
      bps < 1) {
    cudaGetLastError();
    m->last_err = "occupancy query failed";
    return MC_ERR_CUDA;
  }
  if (m->opt.blocks_per_sm) bps = std::min<int>(bps, (int)m->opt.blocks_per_sm);
  m->grid = sms * bps;

  const size_t ab = (size_t)m->a * m->b;
  const size_t L2 = m->lay.max_level + 2;
  uint32_t* d_cfg = (uint32_t*)pe_alloc(m, 4 * 4 * ab);
  uint2* d_steps = (uint2*)pe_alloc(m, 8 * m->steps.size());
  m->d_table = pe_alloc(m, m->table_slots * 16);
  m->d_log_keys = pe_alloc(m, m->log_cap * 16);
  m->d_log_par = (uint32_t*)pe_alloc(m, m->log_cap * 4);
  uint8_t* q = (uint8_t*)pe_alloc(m, 256 + mc::kBarBytes + 40 * L2 + 64);
  if (!d_cfg || !d_steps || !m->d_table || !m->d_log_keys || !m->d_log_par || !q) {
    pe_release(m);
    return MC_ERR_NOMEM;
  }
  m->d_ctrl = (Ctrl*)q;
  q += 256;
  m->d_bar = (uint32_t*)q;
  q += mc::kBarBytes;
  m->d_levels = (uint64_t*)q;
  q += 16 * L2;
  m->d_off = (uint64_t*)q;
  q += 8 * L2;
  m->d_trace = (uint64_t*)q;
  q += 16 * L2;
  m->d_tmin = (uint64_t*)q;
  const size_t o_trace = (sizeof(Ctrl) * 3 + 63) / 64 * 64;
  m->h_block_bytes = o_trace + 16 * L2;
  m->h_block = (uint8_t*)mc::pinned_alloc(m->h_block_bytes);
  if (!m->h_block) {
    pe_release(m);
    return MC_ERR_NOMEM;
  }
  m->h_ctrl = (Ctrl*)m->h_block;
  m->h_trace = (uint64_t*)(m->h_block + o_trace);
  if (m->opt.timing && !m->ev[0])
    for (cudaEvent_t& e : m->ev) PE_CUDA(m, cudaEventCreate(&e));
  std::vector<uint32_t> cfg(4 * ab);
  std::copy(m->N.begin(), m->N.end(), cfg.begin());
  std::copy(m->tau.begin(), m->tau.end(), cfg.begin() + ab);
  std::copy(m->nsteps.begin(), m->nsteps.end(), cfg.begin() + 2 * ab);
  std::copy(m->soff.begin(), m->soff.end(), cfg.begin() + 3 * ab);
  // pageable sources: these copies complete before the calls return
  PE_CUDA(m, cudaMemcpy(d_cfg, cfg.data(), 4 * cfg.size(), cudaMemcpyHostToDevice));
  PE_CUDA(m, cudaMemcpy(d_steps, m->steps.data(), 8 * m->steps.size(), cudaMemcpyHostToDevice));
  m->stats.h2d_bytes += 4 * cfg.size() + 8 * m->steps.size();
  mc::PeParams& p = m->params;
  p.N = d_cfg;
  p.tau = d_cfg + ab;
  p.nsteps = d_cfg + 2 * ab;
  p.soff = d_cfg + 3 * ab;
  p.step = d_steps;
  m->lay.table_slots = m->table_slots;
  m->lay.log_capacity = m->log_cap;
  m->lay.device_bytes = pe_device_bytes(m);
  m->reserved = true;
  return MC_OK;
}

int pe_enqueue(mc_pe_model* m, uint64_t T, const uint64_t* T_src, int64_t delta, bool prune, bool early,
               bool witness, uint64_t* tmin_out, int slot) {
  mc::PeArgs A{};
  A.p = m->params;
  A.table = m->d_table;
  A.bucket_mask = m->table_slots / 2 - 1;
  A.table_u64 = m->table_slots * 2;
  A.max_probes = m->max_probes;
  A.prune = prune;
  A.early_exit = early;
  A.want_witness = witness;
  A.log_keys = m->d_log_keys;
  A.log_par = m->d_log_par;
  A.log_cap = m->log_cap;
  A.ctrl = m->d_ctrl;
  A.levels = m->d_levels;
  A.off = m->d_off;
  A.trace = m->d_trace;
  A.T = T;
  A.T_src = T_src;
  A.T_delta = delta;
  A.tmin_out = tmin_out;
  A.bar = m->d_bar;
  A.timeout_ns = m->opt.barrier_timeout_ns ? m->opt.barrier_timeout_ns : 60ull * 1000000000ull;
  const uint32_t lanes = m->P * m->M + m->P + 1;
  A.slots = (lanes + m->lay.tile - 1) / m->lay.tile;
  static_assert(sizeof(Ctrl) <= 256, "control block header");
  PE_CUDA(m, cudaMemsetAsync(m->d_ctrl, 0, 256 + mc::kBarBytes, m->stream));
  if (m->opt.timing && !m->ev[0])
    for (cudaEvent_t& e : m->ev) PE_CUDA(m, cudaEventCreate(&e));
  if (m->opt.timing) PE_CUDA(m, cudaEventRecord(m->ev[2 * slot], m->stream));
  void* args[] = {&A};
  PE_CUDA(m, cudaLaunchCooperativeKernel(mc::pe_pick(m->lay.tile), dim3(m->grid), dim3(m->threads), args, 0,
                                         m->stream));
  if (m->opt.timing) {
    PE_CUDA(m, cudaEventRecord(m->ev[2 * slot + 1], m->stream));
    m->ev_pending[slot] = true;
  }
  PE_CUDA(m, cudaMemcpyAsync(&m->h_ctrl[slot], m->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, m->stream));
  m->stats.d2h_bytes += sizeof(Ctrl);
  m->stats.explore_launches += 1;
  return MC_OK;
}

int pe_sync(mc_pe_model* m) {
  PE_CUDA(m, cudaStreamSynchronize(m->stream));
  for (int s = 0; s < 3; ++s) {
    if (!m->ev_pending[s]) continue;
    float ms = 0.f;
    PE_CUDA(m, cudaEventElapsedTime(&ms, m->ev[2 * s], m->ev[2 * s + 1]));
    m->stats.explore_ms += ms;
    m->ev_pending[s] = false;
  }
  return MC_OK;
}

int pe_pass_error(mc_pe_model* m, int slot) {
  const Ctrl& c = m->h_ctrl[slot];
  m->last_levels = c.levels;
  m->stats.states += c.states;
  m->stats.device_steps += c.levels;
  m->stats.probes += c.probes;
  return c.err ? (int)c.err : MC_OK;
}

int pe_trace(mc_pe_model* m, const Ctrl& c, mc_trace** out) {
  if (!out) return MC_OK;
  *out = nullptr;
  if (c.trace_len == 0) return MC_OK;
  PE_CUDA(m, cudaMemcpyAsync(m->h_trace, m->d_trace, 16ull * c.trace_len, cudaMemcpyDeviceToHost, m->stream));
  PE_CUDA(m, cudaStreamSynchronize(m->stream));
  m->stats.d2h_bytes += 16ull * c.trace_len;
  mc_trace* t = new (std::nothrow) mc_trace;
  if (!t) return MC_ERR_NOMEM;
  t->words = 2;
  t->keys.assign(m->h_trace, m->h_trace + 2ull * c.trace_len);
  *out = t;
  return MC_OK;
}

void pe_fill_check(const mc_pe_model* m, const Ctrl& c, mc_check_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->holds = c.stop_level == 0;
  out->levels = c.levels;
  out->states = c.states;
  out->key_words = 2;
  if (!out->holds) {
    out->cex_time = mc::pack_time(c.wpack);
    out->cex_wg_index = mc::pack_i(c.wpack);
    out->cex_ts_index = mc::pack_j(c.wpack);
    out->cex_wg = m->wg.empty() ? out->cex_wg_index : m->wg[out->cex_wg_index];
    out->cex_ts = m->ts.empty() ? out->cex_ts_index : m->ts[out->cex_ts_index];
    out->cex_level = c.stop_level;
    out->cex_key[0] = c.wkey_lo;
    out->cex_key[1] = c.wkey_hi;
  }
}

// Runs `query`; when it ends in TABLE_FULL or FRONTIER the failing buffer
// grows fourfold (while the device has room for it) and the query reruns.
template <class Query>
int with_growth(mc_pe_model* m, Query query) {
  for (;;) {
    PE_TRY(pe_reserve(m));
    const int rc = query();
    if (rc != MC_ERR_TABLE_FULL && rc != MC_ERR_FRONTIER) return rc;
    if (m->opt.table_log2 && rc == MC_ERR_TABLE_FULL) return rc;
    // a level's width is counted in 32 bits of its barrier word and cannot
    // exceed the visited set's slots, which stay at or below 2^31
    if (rc == MC_ERR_TABLE_FULL && m->table_slots * 4 > (1ull << 31)) return rc;
    if (m->opt.log_capacity && rc == MC_ERR_FRONTIER) return rc;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      return rc;
    }
    const uint64_t have = pe_device_bytes(m);
    const uint64_t extra = rc == MC_ERR_TABLE_FULL ? 3 * m->table_slots * 16 : 3 * m->log_cap * 20;
    if (have + extra > ((uint64_t)free_b + have) / 2) return rc;
    pe_release(m);
    if (rc == MC_ERR_TABLE_FULL) m->table_slots *= 4;
    else m->log_cap *= 4;
  }
}

}  // namespace

extern "C" {

int mc_pe_model_create(const mc_pe_model_desc* d, const mc_options* opt, mc_pe_model** out) {
  if (!d || !out) return MC_ERR_INVAL;
  *out = nullptr;
  if (d->n_wg == 0 || d->n_ts == 0 || d->P == 0 || d->P > mc::kPeMaxUnits) return MC_ERR_INVAL;
  if (!d->n_workgroups || !d->pes || !d->prog_off || !d->seg_ticks || !d->seg_pes) return MC_ERR_INVAL;
  if (d->n_wg > 255 || d->n_ts > 255) return MC_ERR_OVERFLOW;
  mc_options o;
  if (opt) o = *opt;
  else mc_options_default(&o);
  if (o.load_factor_pct < 10 || o.load_factor_pct > 90) return MC_ERR_INVAL;
  if (o.threads_per_block &&
      (o.threads_per_block < 64 || o.threads_per_block > mc::kThreads || o.threads_per_block % 32))
    return MC_ERR_INVAL;
  if (o.table_log2 && (o.table_log2 < 3 || o.table_log2 > 40)) return MC_ERR_INVAL;

  mc_pe_model* m = new (std::nothrow) mc_pe_model;
  if (!m) return MC_ERR_NOMEM;
  auto fail = [m](int rc) {
    delete m;
    return rc;
  };
  m->a = d->n_wg;
  m->b = d->n_ts;
  m->P = d->P;
  m->opt = o;
  const size_t ab = (size_t)m->a * m->b;
  if (d->wg_values) m->wg.assign(d->wg_values, d->wg_values + m->a);
  if (d->ts_values) m->ts.assign(d->ts_values, d->ts_values + m->b);
  m->N.assign(d->n_workgroups, d->n_workgroups + ab);
  uint32_t n_max = 0, M = 0;
  uint64_t s_max = 0, lvl_max = 0;
  if (d->prog_off[0] != 0) return fail(MC_ERR_INVAL);
  for (size_t k = 0; k < ab; ++k) {
    const uint32_t nwe = d->pes[k];
    if (m->N[k] == 0 || nwe == 0 || nwe > mc::kPeMaxPes) return fail(MC_ERR_INVAL);
    if (d->prog_off[k + 1] <= d->prog_off[k]) return fail(MC_ERR_INVAL);
    n_max = std::max(n_max, m->N[k]);
    M = std::max(M, nwe);
    uint64_t ticks = 0, marks = 0, barriers = 0, S = 0;
    m->soff.push_back((uint32_t)m->steps.size());
    for (uint32_t s = d->prog_off[k]; s < d->prog_off[k + 1]; ++s) {
      const uint32_t t = d->seg_ticks[s], pe = d->seg_pes[s];
      if (pe == 0 || pe > nwe || t > 65535) return fail(MC_ERR_INVAL);
      if (t == 0) {
        m->steps.push_back(make_uint2(mc::kBarrierBit | pe, (uint32_t)ticks));
        marks += pe;
        barriers += 1;
        S += 1;
      } else {
        for (uint32_t x = 0; x < t; ++x) m->steps.push_back(make_uint2(pe, (uint32_t)(ticks + x)));
        ticks += t;
        marks += (uint64_t)t * pe;
        S += t;
      }
      if (m->steps.size() > (1ull << 26)) return fail(MC_ERR_OVERFLOW);
    }
    m->tau.push_back((uint32_t)ticks);
    m->nsteps.push_back((uint32_t)S);
    s_max = std::max(s_max, S);
    // level of FIN: two selects, then per work-group a dispatch, the marks
    // and releases of its program, plus one step per clock tick
    const uint64_t waves = (m->N[k] + m->P - 1) / m->P;
    const uint64_t t_fin = waves * ticks;
    if (t_fin >= (1ull << 40)) return fail(MC_ERR_OVERFLOW);
    lvl_max = std::max<uint64_t>(lvl_max, 2 + (uint64_t)m->N[k] * (1 + marks + barriers) + t_fin);
  }
  if (m->P * M + m->P + 1 > 32) return fail(MC_ERR_INVAL);
  if (lvl_max >= (1ull << 30)) return fail(MC_ERR_OVERFLOW);
  m->M = M;
  mc_pe_layout& L = m->lay;
  L.P = m->P;
  L.mask_bits = M;
  L.n_bits = mc::bits_for(n_max);
  L.pc_bits = std::max<uint32_t>(1, mc::bits_for(s_max - 1));
  L.unit_bits = L.n_bits + 1 + L.pc_bits + M;
  L.level_bits = mc::bits_for(lvl_max);
  L.ts_bits = mc::bits_for(m->b);
  L.wg_bits = mc::bits_for(m->a);
  L.used_bits = L.wg_bits + L.ts_bits + L.level_bits + m->P * L.unit_bits;
  if (L.used_bits > 128 || L.unit_bits > 64) return fail(MC_ERR_OVERFLOW);
  L.level_shift = m->P * L.unit_bits;
  L.ts_shift = L.level_shift + L.level_bits;
  L.wg_shift = L.ts_shift + L.ts_bits;
  for (uint32_t c = 0; c < m->P; ++c) L.unit_shift[c] = (m->P - 1 - c) * L.unit_bits;
  L.max_level = (uint32_t)lvl_max;
  L.max_steps = s_max;
  const uint32_t lanes = m->P * M + m->P + 1;
  if (o.lanes_per_state) {
    const uint32_t t = o.lanes_per_state;
    if ((t != 4 && t != 8 && t != 16 && t != 32) || (lanes + t - 1) / t > mc::slots_for(t))
      return fail(MC_ERR_INVAL);
    L.tile = t;
  } else {
    L.tile = 4;
    while ((lanes + L.tile - 1) / L.tile > mc::slots_for(L.tile)) L.tile <<= 1;
  }
  mc::PeParams& p = m->params;
  p.a = m->a;
  p.b = m->b;
  p.P = m->P;
  p.M = M;
  p.n_bits = L.n_bits;
  p.pc_bits = L.pc_bits;
  p.unit_bits = L.unit_bits;
  p.lvl_bits = L.level_bits;
  p.wg_shift = L.wg_shift;
  p.ts_shift = L.ts_shift;
  p.lvl_shift = L.level_shift;
  p.max_level = L.max_level;
  p.wg_mask = (1u << L.wg_bits) - 1;
  p.ts_mask = (1u << L.ts_bits) - 1;
  p.unit_mask = L.unit_bits >= 64 ? ~0ull : (1ull << L.unit_bits) - 1;
  p.lvl_mask = (1ull << L.level_bits) - 1;
  if (o.table_log2 > 31) return fail(MC_ERR_OVERFLOW);
  m->table_slots = o.table_log2 ? (1ull << o.table_log2) : (1ull << 20);
  if (m->table_slots < 2) m->table_slots = 2;
  const uint64_t n_init = 1 + (uint64_t)m->a + ab;
  m->log_cap = std::max<uint64_t>(o.log_capacity ? o.log_capacity : (1ull << 22), n_init);
  m->max_probes = o.max_probes ? o.max_probes : 64;
  L.table_slots = m->table_slots;
  L.log_capacity = m->log_cap;
  L.device_bytes = pe_device_bytes(m);
  *out = m;
  return MC_OK;
}

void mc_pe_model_destroy(mc_pe_model* m) {
  if (!m) return;
  pe_release(m);
  delete m;
}

int mc_pe_set_stream(mc_pe_model* m, void* stream) {
  if (!m) return MC_ERR_INVAL;
  m->stream = (cudaStream_t)stream;
  return MC_OK;
}

int mc_pe_model_layout(const mc_pe_model* m, mc_pe_layout* out) {
  if (!m || !out) return MC_ERR_INVAL;
  *out = m->lay;
  out->table_slots = m->table_slots;
  out->log_capacity = m->log_cap;
  out->device_bytes = pe_device_bytes(m);
  return MC_OK;
}

int mc_pe_check(mc_pe_model* m, uint64_t T, mc_check_result* out, mc_trace** cex) {
  if (!m || !out) return MC_ERR_INVAL;
  if (cex) *cex = nullptr;
  PE_TRY(with_growth(m, [&]() -> int {
    PE_TRY(pe_enqueue(m, T, nullptr, 0, m->opt.prune != 0, m->opt.early_exit != 0, true, nullptr, 0));
    PE_TRY(pe_sync(m));
    return pe_pass_error(m, 0);
  }));
  pe_fill_check(m, m->h_ctrl[0], out);
  return pe_trace(m, m->h_ctrl[0], cex);
}

int mc_pe_count_states(mc_pe_model* m, uint64_t* out) {
  if (!m || !out) return MC_ERR_INVAL;
  PE_TRY(with_growth(m, [&]() -> int {
    PE_TRY(pe_enqueue(m, kNone, nullptr, 0, false, false, false, nullptr, 0));
    PE_TRY(pe_sync(m));
    return pe_pass_error(m, 0);
  }));
  *out = m->h_ctrl[0].states;
  return MC_OK;
}

int mc_pe_min_time(mc_pe_model* m, mc_min_result* out, mc_trace** trace) {
  if (!m || !out) return MC_ERR_INVAL;
  if (trace) *trace = nullptr;
  std::memset(out, 0, sizeof(*out));
  const bool refine = m->opt.refine != 0;
  const int final_slot = refine ? 2 : 1;
  PE_TRY(with_growth(m, [&]() -> int {
    // pass 0: every FIN state is "violating" at T = infinity, so the minimum
    // packed (time, i, j) over all levels is T_min; passes 1 (certificate at
    // T_min - 1) and 2 (counterexample at T_min) read T from the device
    PE_TRY(pe_enqueue(m, kNone, nullptr, 0, false, false, false, m->d_tmin, 0));
    if (refine)
      PE_TRY(pe_enqueue(m, 0, m->d_tmin, -1, m->opt.prune != 0, m->opt.early_exit != 0, false, nullptr, 1));
    PE_TRY(pe_enqueue(m, 0, m->d_tmin, 0, m->opt.prune != 0, m->opt.early_exit != 0, true, nullptr,
                      final_slot));
    PE_TRY(pe_sync(m));
    for (int s = 0; s <= final_slot; ++s) PE_TRY(pe_pass_error(m, s));
    return MC_OK;
  }));
  const Ctrl& c0 = m->h_ctrl[0];
  const Ctrl& cf = m->h_ctrl[final_slot];
  if (c0.best_pack == kNone || cf.stop_level == 0 || (refine && m->h_ctrl[1].stop_level != 0)) {
    m->last_err = "inconsistent passes";
    return MC_ERR_CUDA;
  }
  out->t_min = mc::pack_time(cf.wpack);
  out->t_ini = 0;
  out->wg_index = mc::pack_i(cf.wpack);
  out->ts_index = mc::pack_j(cf.wpack);
  out->wg = m->wg.empty() ? out->wg_index : m->wg[out->wg_index];
  out->ts = m->ts.empty() ? out->ts_index : m->ts[out->ts_index];
  for (int s = 0; s <= final_slot; ++s) out->states += m->h_ctrl[s].states;
  out->checks = final_slot + 1;
  out->level = cf.stop_level;
  out->witness_key[0] = cf.wkey_lo;
  out->witness_key[1] = cf.wkey_hi;
  return pe_trace(m, cf, trace);
}

int mc_pe_last_widths(mc_pe_model* m, uint64_t* out, uint32_t cap, uint32_t* n) {
  if (!m || !n) return MC_ERR_INVAL;
  *n = m->last_levels;
  if (!m->reserved || !out || cap == 0) return MC_OK;
  const uint32_t k = std::min(cap, m->last_levels);
  std::vector<uint64_t> rec(2ull * k);
  PE_CUDA(m, cudaMemcpyAsync(rec.data(), m->d_levels, 16ull * k, cudaMemcpyDeviceToHost, m->stream));
  PE_CUDA(m, cudaStreamSynchronize(m->stream));
  m->stats.d2h_bytes += 16ull * k;
  for (uint32_t l = 0; l < k; ++l) out[l] = rec[2 * l] & 0xFFFFFFFFull;  // width field of the word
  return MC_OK;
}

int mc_pe_get_stats(const mc_pe_model* m, mc_stats* out) {
  if (!m || !out) return MC_ERR_INVAL;
  *out = m->stats;
  return MC_OK;
}

int mc_pe_reset_stats(mc_pe_model* m) {
  if (!m) return MC_ERR_INVAL;
  m->stats = mc_stats{};
  return MC_OK;
}

const char* mc_pe_last_error(const mc_pe_model* m) { return m ? m->last_err.c_str() : "null model"; }

}  // extern "C"
