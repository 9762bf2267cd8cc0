// Plain CPU oracle for the processing-element level model (test
// infrastructure only).
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg load
// this library.  It shares no code with the CUDA path: its own state struct
// (every field unpacked, the model time kept as a counter of clock ticks),
// its own successor function, a breadth-first search over one
// std::unordered_set of serialised states.  It is deliberately slow and
// obvious.
//
// The model keeps the processes the cost-table model folds away (Section 4,
// Step 1, Listings 3-9): every compute unit runs a work-group as NWE
// processing elements `pex`, each of which reports every tick of its
// `long_work` to the `clock`, and the unit's `barrier` waits for all of them.
// Per configuration (i, j) the input gives N work-groups and one program:
// segments that are either `ticks` clock ticks in which `pes` PEs report, or a
// local barrier (ticks = 0) that `pes` PEs arrive at.  A program step is one
// tick of a work segment or one barrier.
//   * s0 -> (WG i) -> (WG i, TS j, every unit idle, N work-groups left):
//     the selects of `main` (Listing 3).
//   * dispatch: a unit that is idle while work-groups are left takes the next
//     one (the device's `dev_u ! go` reaches any waiting unit, Listing 5); it
//     starts at program step 0 with no PE marked.
//   * mark: a participating PE of a busy unit that has not marked itself in
//     the current step does so -- in a tick step it reports NRP_work++
//     (Listing 8), at a barrier it sends `done` to the barrier (Listing 7).
//   * release: a busy unit at a barrier step with every participant marked
//     moves to its next step (the barrier's `b_pex ! go`).
//   * tick: when every busy unit is at a tick step with every participant
//     marked, and no unit is idle while work-groups are left, `time` grows by
//     one (Listing 9) and every busy unit moves to its next step.
//   * a unit whose program ends becomes idle; FIN holds when no work-group is
//     left and every unit is idle, and the model time is the tick count.
// Property (Step 2): G(FIN -> time > T).
//
// Counting rules: the level of a state is its breadth-first depth; with
// pruning a successor whose time exceeds T is not kept; with early exit the
// search stops after the first level holding a violating terminal, and the
// count covers the kept states of the levels up to that one; the
// counterexample is the smallest (time, i, j) among that level's violating
// terminals.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

extern "C" {

typedef struct {
  uint32_t a, b, P;           // |D_WG|, |D_TS|, compute units (1..8)
  const uint32_t* N;          // [a*b] work-groups
  const uint32_t* pes;        // [a*b] PEs per unit (1..8)
  const uint32_t* prog_off;   // [a*b + 1] first segment of each program
  const uint32_t* seg_ticks;  // [segments] ticks, 0 = barrier
  const uint32_t* seg_pes;    // [segments] participating PEs
} or_pe_model;

typedef struct {
  uint32_t holds, levels;
  uint64_t states;
  uint64_t cex_time;
  uint32_t cex_i, cex_j, cex_level, pad;
} or_pe_check_result;

typedef struct {
  uint64_t t_min, states;
  uint32_t checks, i, j, level;
} or_pe_min_result;

}  // extern "C"

namespace {

constexpr uint64_t kNoLimit = ~0ull;
constexpr uint32_t kMaxUnits = 8;

struct Step {
  bool barrier;
  uint32_t pes;
};

struct Model {
  uint32_t a = 0, b = 0, P = 0;
  std::vector<uint32_t> N;
  std::vector<std::vector<Step>> steps;  // per configuration
};

// phase: 0 = s0, 1 = WG selected, 2 = running
struct State {
  uint32_t phase = 0, i = 0, j = 0;
  uint64_t time = 0;
  uint32_t n[kMaxUnits] = {}, busy[kMaxUnits] = {}, pc[kMaxUnits] = {}, mask[kMaxUnits] = {};
};

std::string serial(const State& s, uint32_t P) {
  std::string k;
  auto put = [&k](uint64_t v) { k.append(reinterpret_cast<const char*>(&v), sizeof(v)); };
  put(s.phase);
  put(s.i);
  put(s.j);
  put(s.time);
  for (uint32_t c = 0; c < P; ++c) {
    put(s.n[c]);
    put(s.busy[c]);
    put(s.pc[c]);
    put(s.mask[c]);
  }
  return k;
}

bool load(const or_pe_model* mm, Model& m) {
  if (!mm || mm->a == 0 || mm->b == 0 || mm->P == 0 || mm->P > kMaxUnits) return false;
  m.a = mm->a;
  m.b = mm->b;
  m.P = mm->P;
  const uint32_t cfgs = m.a * m.b;
  m.N.assign(mm->N, mm->N + cfgs);
  m.steps.resize(cfgs);
  for (uint32_t c = 0; c < cfgs; ++c) {
    for (uint32_t s = mm->prog_off[c]; s < mm->prog_off[c + 1]; ++s) {
      if (mm->seg_ticks[s] == 0) {
        m.steps[c].push_back({true, mm->seg_pes[s]});
      } else {
        for (uint32_t t = 0; t < mm->seg_ticks[s]; ++t) m.steps[c].push_back({false, mm->seg_pes[s]});
      }
    }
    if (m.steps[c].empty()) return false;
  }
  return true;
}

uint32_t full(uint32_t pes) { return (1u << pes) - 1u; }

bool is_fin(const Model& m, const State& s) {
  if (s.phase != 2) return false;
  uint32_t sum = 0;
  for (uint32_t c = 0; c < m.P; ++c) {
    if (s.busy[c]) return false;
    sum += s.n[c];
  }
  return sum == m.N[s.i * m.b + s.j];
}

void advance(const std::vector<Step>& steps, State& s, uint32_t c) {
  s.pc[c] += 1;
  s.mask[c] = 0;
  if (s.pc[c] == steps.size()) {
    s.busy[c] = 0;
    s.pc[c] = 0;
  }
}

void successors(const Model& m, const State& s, std::vector<State>& out) {
  out.clear();
  if (s.phase == 0) {
    for (uint32_t i = 0; i < m.a; ++i) {
      State u;
      u.phase = 1;
      u.i = i;
      out.push_back(u);
    }
    return;
  }
  if (s.phase == 1) {
    for (uint32_t j = 0; j < m.b; ++j) {
      State u;
      u.phase = 2;
      u.i = s.i;
      u.j = j;
      out.push_back(u);
    }
    return;
  }
  const uint32_t cfg = s.i * m.b + s.j;
  const std::vector<Step>& steps = m.steps[cfg];
  uint32_t dispatched = 0;
  for (uint32_t c = 0; c < m.P; ++c) dispatched += s.n[c];
  const bool left = dispatched < m.N[cfg];
  bool any_busy = false, any_idle = false, ready = true;
  for (uint32_t c = 0; c < m.P; ++c) {
    if (!s.busy[c]) {
      any_idle = true;
      if (left) {  // dispatch
        State u = s;
        u.n[c] += 1;
        u.busy[c] = 1;
        u.pc[c] = 0;
        u.mask[c] = 0;
        out.push_back(u);
      }
      continue;
    }
    any_busy = true;
    const Step& st = steps[s.pc[c]];
    for (uint32_t e = 0; e < st.pes; ++e) {  // mark
      if (s.mask[c] & (1u << e)) continue;
      State u = s;
      u.mask[c] |= 1u << e;
      out.push_back(u);
    }
    const bool all_marked = s.mask[c] == full(st.pes);
    if (st.barrier && all_marked) {  // release
      State u = s;
      advance(steps, u, c);
      out.push_back(u);
    }
    if (st.barrier || !all_marked) ready = false;
  }
  if (any_busy && ready && !(left && any_idle)) {  // tick
    State u = s;
    u.time += 1;
    for (uint32_t c = 0; c < m.P; ++c)
      if (s.busy[c]) advance(steps, u, c);
    out.push_back(u);
  }
}

struct Result {
  bool holds = true;
  uint32_t levels = 1, cex_level = 0;
  uint64_t states = 1;
  uint64_t cex_time = 0;
  uint32_t cex_i = 0, cex_j = 0;
  uint64_t min_fin = kNoLimit;  // least FIN time over every kept level
};

// Level-synchronous exploration with the counting rules above.
Result explore(const Model& m, uint64_t T, bool prune, bool early_exit, std::vector<uint64_t>* widths) {
  Result r;
  std::unordered_set<std::string> seen;
  std::vector<State> frontier(1), next, succ;
  seen.insert(serial(frontier[0], m.P));
  if (widths) widths->push_back(1);
  uint32_t level = 0;
  while (!frontier.empty()) {
    next.clear();
    bool viol = false;
    uint64_t vt = 0;
    uint32_t vi = 0, vj = 0;
    for (const State& s : frontier) {
      successors(m, s, succ);
      for (const State& u : succ) {
        if (prune && u.time > T) continue;
        if (!seen.insert(serial(u, m.P)).second) continue;
        next.push_back(u);
        if (is_fin(m, u)) {
          r.min_fin = std::min(r.min_fin, u.time);
          if (u.time <= T) {
            const bool better = !viol || u.time < vt || (u.time == vt && (u.i < vi || (u.i == vi && u.j < vj)));
            if (better) {
              viol = true;
              vt = u.time;
              vi = u.i;
              vj = u.j;
            }
          }
        }
      }
    }
    if (next.empty()) break;
    ++level;
    r.states += next.size();
    r.levels = level + 1;
    if (widths) widths->push_back(next.size());
    if (viol && r.holds) {
      r.holds = false;
      r.cex_time = vt;
      r.cex_i = vi;
      r.cex_j = vj;
      r.cex_level = level;
      if (early_exit) break;
    }
    frontier.swap(next);
  }
  return r;
}

}  // namespace

extern "C" {

int oracle_pe_check(const or_pe_model* mm, uint64_t T, int prune, int early_exit,
                    or_pe_check_result* out, uint64_t* widths, uint32_t wcap) {
  Model m;
  if (!out || !load(mm, m)) return -1;
  std::vector<uint64_t> w;
  const Result r = explore(m, T, prune != 0, early_exit != 0, widths ? &w : nullptr);
  std::memset(out, 0, sizeof(*out));
  out->holds = r.holds;
  out->levels = r.levels;
  out->states = r.states;
  if (!r.holds) {
    out->cex_time = r.cex_time;
    out->cex_i = r.cex_i;
    out->cex_j = r.cex_j;
    out->cex_level = r.cex_level;
  }
  if (widths)
    for (size_t l = 0; l < w.size() && l < wcap; ++l) widths[l] = w[l];
  return 0;
}

int oracle_pe_count(const or_pe_model* mm, uint64_t* out) {
  Model m;
  if (!out || !load(mm, m)) return -1;
  *out = explore(m, kNoLimit, false, false, nullptr).states;
  return 0;
}

// Section 4, Steps 3-4: one full exploration gives T_min (the least FIN
// time); check(T_min - 1) must hold (refine) and check(T_min) gives the
// counterexample whose (WG, TS) is the answer.
int oracle_pe_min_time(const or_pe_model* mm, int prune, int early_exit, int refine,
                       or_pe_min_result* out) {
  Model m;
  if (!out || !load(mm, m)) return -1;
  std::memset(out, 0, sizeof(*out));
  const Result all = explore(m, kNoLimit, false, false, nullptr);
  out->states += all.states;
  out->checks += 1;
  const uint64_t t_min = all.min_fin;
  if (t_min == kNoLimit) return -1;
  if (refine) {
    const Result r = explore(m, t_min - 1, prune != 0, early_exit != 0, nullptr);
    out->states += r.states;
    out->checks += 1;
    if (!r.holds) return -1;
  }
  const Result r = explore(m, t_min, prune != 0, early_exit != 0, nullptr);
  out->states += r.states;
  out->checks += 1;
  if (r.holds) return -1;
  out->t_min = r.cex_time;
  out->i = r.cex_i;
  out->j = r.cex_j;
  out->level = r.cex_level;
  return 0;
}

}  // extern "C"
