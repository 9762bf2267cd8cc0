// Plain CPU oracle for the explicit-state exploration of the OpenCL-launch
// model (test infrastructure only).
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg load
// this library.  It shares no code with the CUDA path: its own state struct,
// its own successor function, a depth-first search over std::unordered_set.
// It is deliberately slow and obvious.
//
// The model (Section 4, Step 1; Listings 3-9) reduced to its scheduling
// semantics:
//   * s0 = (i=0, j=0, n=0^P) -- nothing selected yet.
//   * `select` of WG (Listing 3): s0 -> (i, 0, 0^P) for every WG index i
//     (stored 1-based, 0 = not selected).
//   * `select` of TS (Listing 3): (i, 0, 0^P) -> (i, j, 0^P) for every j.
//   * dispatch (Listings 4-5, `host` and `device` handing work-groups to
//     compute units): from a selected state with r = N_ij - sum(n) > 0
//       FREE   -- any compute unit c takes the next work-group: n + e_c;
//       GREEDY -- only units whose clock n_c * t_c is minimal (the unit that
//                 reported `done` first is re-dispatched), ties in every order.
//     t_c = cost[i][j] * speed[c] is the time one work-group takes on unit c
//     (the `unit`/`pex`/`clock` processes, Listings 6-9, folded into a cost).
//   * r = 0 is the terminal state where `host` sets FIN (Listing 4); its model
//     time is max_c n_c * t_c (the value of `time` when `clock`, Listing 9,
//     stops).
// Property (Step 2): Phi = G(FIN -> time > T).  A terminal with time <= T
// violates it; such a terminal is a counterexample.
//
// Counting rules (shared definition with the CUDA path, not shared code):
//   * the level of a state is 0 for s0, 1 after the WG select, and
//     2 + sum(n) after the TS select; every path to a state has that length.
//   * with pruning, a successor whose max clock exceeds T is not kept (clocks
//     only grow, so it cannot reach a violating terminal).
//   * with early exit, the search stops at the end of the first level that
//     holds a violating terminal; the count is the number of kept states of
//     levels up to and including that level.
//   * the counterexample is, within that first violating level, the
//     violating terminal with the smallest (time, i, j, n_0, ..., n_{P-1}).
//
// Parity notes: every function here is pinned by tests (brute force over all
// schedules on tiny models, closed forms, invariants); see tests/.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <limits>
#include <unordered_set>
#include <vector>

extern "C" {

typedef struct {
  uint32_t a, b, P, rule;   // |D_WG|, |D_TS|, compute units, 0 FREE / 1 GREEDY
  const uint32_t* N;        // [a*b] work-groups of configuration (i, j)
  const uint32_t* cost;     // [a*b] time of one work-group, speed 1
  const uint32_t* speed;    // [P]   speed factor of each compute unit
} or_model;

typedef struct {
  uint32_t holds;       // 1: no kept terminal has time <= T
  uint32_t levels;      // levels counted (last level + 1)
  uint64_t states;      // kept unique states of the counted levels
  uint64_t cex_time;    // counterexample (holds == 0)
  uint32_t cex_i, cex_j, cex_level, pad;
  uint32_t cex_n[16];
} or_check_result;

typedef struct {
  uint64_t t_min;
  uint64_t t_ini;
  uint64_t states;      // sum of counted states over every exploration pass
  uint32_t checks;      // exploration passes run
  uint32_t i, j, level;
  uint32_t n[16];
} or_min_result;

}  // extern "C"

namespace {

const uint64_t kNoLimit = std::numeric_limits<uint64_t>::max();

struct State {
  uint32_t i = 0, j = 0;        // 1-based once selected, 0 = not selected
  std::vector<uint32_t> n;      // work-groups taken by each compute unit
  bool operator==(const State& o) const { return i == o.i && j == o.j && n == o.n; }
};

struct StateHash {
  size_t operator()(const State& s) const {
    uint64_t h = 1469598103934665603ull;
    auto add = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    add(s.i);
    add(s.j);
    for (uint32_t x : s.n) add(x);
    return (size_t)h;
  }
};

struct Model {
  uint32_t a, b, P, rule;
  std::vector<uint32_t> N, cost, speed;
};

Model load(const or_model* m) {
  Model r;
  r.a = m->a; r.b = m->b; r.P = m->P; r.rule = m->rule;
  r.N.assign(m->N, m->N + m->a * m->b);
  r.cost.assign(m->cost, m->cost + m->a * m->b);
  r.speed.assign(m->speed, m->speed + m->P);
  return r;
}

uint32_t sum_n(const State& s) {
  uint32_t t = 0;
  for (uint32_t x : s.n) t += x;
  return t;
}

uint32_t level_of(const State& s) {
  if (s.i == 0) return 0;
  if (s.j == 0) return 1;
  return 2 + sum_n(s);
}

bool selected(const State& s) { return s.i != 0 && s.j != 0; }

// time one work-group takes on unit c under the selected configuration
uint64_t unit_time(const Model& m, const State& s, uint32_t c) {
  uint32_t cfg = (s.i - 1) * m.b + (s.j - 1);
  return (uint64_t)m.cost[cfg] * m.speed[c];
}

// clock of unit c: the end of its last work-group
uint64_t clock_of(const Model& m, const State& s, uint32_t c) {
  if (!selected(s)) return 0;
  return (uint64_t)s.n[c] * unit_time(m, s, c);
}

// model time of a state: the latest unit clock
uint64_t time_of(const Model& m, const State& s) {
  uint64_t t = 0;
  for (uint32_t c = 0; c < m.P; ++c) t = std::max(t, clock_of(m, s, c));
  return t;
}

uint32_t remaining(const Model& m, const State& s) {
  uint32_t cfg = (s.i - 1) * m.b + (s.j - 1);
  return m.N[cfg] - sum_n(s);
}

bool terminal(const Model& m, const State& s) { return selected(s) && remaining(m, s) == 0; }

// units allowed to take the next work-group (index order)
std::vector<uint32_t> allowed_units(const Model& m, const State& s) {
  std::vector<uint32_t> out;
  if (m.rule == 0) {
    for (uint32_t c = 0; c < m.P; ++c) out.push_back(c);
    return out;
  }
  uint64_t mn = kNoLimit;
  for (uint32_t c = 0; c < m.P; ++c) mn = std::min(mn, clock_of(m, s, c));
  for (uint32_t c = 0; c < m.P; ++c)
    if (clock_of(m, s, c) == mn) out.push_back(c);
  return out;
}

std::vector<State> successors(const Model& m, const State& s) {
  std::vector<State> out;
  if (s.i == 0) {                       // select WG
    for (uint32_t i = 0; i < m.a; ++i) {
      State t = s;
      t.i = i + 1;
      out.push_back(t);
    }
  } else if (s.j == 0) {                // select TS
    for (uint32_t j = 0; j < m.b; ++j) {
      State t = s;
      t.j = j + 1;
      out.push_back(t);
    }
  } else if (remaining(m, s) > 0) {     // dispatch one work-group
    for (uint32_t c : allowed_units(m, s)) {
      State t = s;
      t.n[c] += 1;
      out.push_back(t);
    }
  }                                     // terminal (FIN): no successor
  return out;
}

// (time, i, j, n_0, ..., n_{P-1}) with 0-based i, j; compared lexicographically
std::vector<uint64_t> order_tuple(const Model& m, const State& s) {
  std::vector<uint64_t> t;
  t.push_back(time_of(m, s));
  t.push_back(s.i - 1);
  t.push_back(s.j - 1);
  for (uint32_t x : s.n) t.push_back(x);
  return t;
}

struct Exploration {
  std::vector<uint64_t> width;                       // kept states per level
  std::vector<bool> has_violation;                   // level holds a terminal with time <= T
  std::vector<std::vector<uint64_t>> best;           // smallest violating tuple per level
};

// Depth-first search over every kept reachable state.
Exploration explore(const Model& m, uint64_t T, bool prune) {
  Exploration ex;
  std::unordered_set<State, StateHash> visited;
  std::vector<State> stack;
  State s0;
  s0.n.assign(m.P, 0);
  visited.insert(s0);
  stack.push_back(s0);
  while (!stack.empty()) {
    State s = stack.back();
    stack.pop_back();
    uint32_t lv = level_of(s);
    if (ex.width.size() <= lv) {
      ex.width.resize(lv + 1, 0);
      ex.has_violation.resize(lv + 1, false);
      ex.best.resize(lv + 1);
    }
    ex.width[lv] += 1;
    if (terminal(m, s) && time_of(m, s) <= T) {
      std::vector<uint64_t> t = order_tuple(m, s);
      if (!ex.has_violation[lv] || t < ex.best[lv]) ex.best[lv] = t;
      ex.has_violation[lv] = true;
    }
    for (const State& t : successors(m, s)) {
      if (prune && time_of(m, t) > T) continue;
      if (visited.insert(t).second) stack.push_back(t);
    }
  }
  return ex;
}

void fill_check(const Model& m, const Exploration& ex, bool early_exit, or_check_result* out) {
  std::memset(out, 0, sizeof(*out));
  int64_t first = -1;
  for (size_t l = 0; l < ex.width.size(); ++l)
    if (ex.has_violation[l]) { first = (int64_t)l; break; }
  size_t last = ex.width.size() - 1;
  if (first >= 0 && early_exit) last = (size_t)first;
  uint64_t states = 0;
  for (size_t l = 0; l <= last; ++l) states += ex.width[l];
  out->states = states;
  out->levels = (uint32_t)(last + 1);
  out->holds = first < 0 ? 1 : 0;
  if (first >= 0) {
    const std::vector<uint64_t>& t = ex.best[first];
    out->cex_time = t[0];
    out->cex_i = (uint32_t)t[1];
    out->cex_j = (uint32_t)t[2];
    out->cex_level = (uint32_t)first;
    for (uint32_t c = 0; c < m.P && c < 16; ++c) out->cex_n[c] = (uint32_t)t[3 + c];
  }
}

const uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// splitmix64 (Steele, Lea, Flood 2014): output number ctr of the stream
// started at `seed`, as a counter-based generator.
uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One random run of the model (Step 3: SPIN's simulation mode gives T_ini).
// Walk w draws from counters (w << 32) + 0, 1, 2, ...: the WG index, the TS
// index, then one draw per dispatched work-group picking among the allowed
// units in index order.
uint64_t simulate_walk(const Model& m, uint64_t seed, uint64_t w) {
  uint64_t ctr = (uint64_t)w << 32;
  State s;
  s.n.assign(m.P, 0);
  s.i = (uint32_t)(splitmix64_at(seed, ctr++) % m.a) + 1;
  s.j = (uint32_t)(splitmix64_at(seed, ctr++) % m.b) + 1;
  while (remaining(m, s) > 0) {
    std::vector<uint32_t> al = allowed_units(m, s);
    uint32_t c = al[splitmix64_at(seed, ctr++) % al.size()];
    s.n[c] += 1;
  }
  return time_of(m, s);
}

}  // namespace

extern "C" {

int oracle_check(const or_model* mm, uint64_t T, int prune, int early_exit, or_check_result* out,
                 uint64_t* widths, uint32_t widths_cap) {
  if (!mm || !out || mm->a == 0 || mm->b == 0 || mm->P == 0 || mm->P > 16) return -1;
  Model m = load(mm);
  Exploration ex = explore(m, T, prune != 0);
  fill_check(m, ex, early_exit != 0, out);
  if (widths)
    for (uint32_t l = 0; l < widths_cap; ++l) widths[l] = l < out->levels ? ex.width[l] : 0;
  return 0;
}

int oracle_count(const or_model* mm, uint64_t* out) {
  or_check_result r;
  int rc = oracle_check(mm, kNoLimit, 0, 0, &r, nullptr, 0);
  if (rc == 0) *out = r.states;
  return rc;
}

// One random run (walk number w of `seed`): its terminal time and (i, j).
int oracle_walk(const or_model* mm, uint64_t seed, uint64_t w, uint64_t* time, uint32_t* i,
                uint32_t* j) {
  if (!mm || !time || !i || !j) return -1;
  Model m = load(mm);
  uint64_t ctr = w << 32;
  *i = (uint32_t)(splitmix64_at(seed, ctr++) % m.a);
  *j = (uint32_t)(splitmix64_at(seed, ctr++) % m.b);
  *time = simulate_walk(m, seed, w);
  return 0;
}

int oracle_simulate(const or_model* mm, uint64_t seed, uint32_t walks, uint64_t* t_ini) {
  if (!mm || !t_ini || walks == 0) return -1;
  Model m = load(mm);
  uint64_t best = kNoLimit;
  for (uint32_t w = 0; w < walks; ++w) best = std::min(best, simulate_walk(m, seed, w));
  *t_ini = best;
  return 0;
}

// Step 3 (find T_min) and Step 4 (read the configuration from the last
// counterexample).  search: 0 = single pass (one exploration pruned at T_ini
// gives the minimum terminal time, then check(T_min-1) and check(T_min)),
// 1 = lower T to (counterexample time - 1) until the property holds,
// 2 = bisection between 0 (never violated: every time is >= 1) and T_ini.
// In every mode the configuration is the counterexample of check(T_min).
int oracle_min_time(const or_model* mm, int search, int prune, int early_exit, int refine,
                    uint64_t seed, uint32_t walks, or_min_result* out) {
  if (!mm || !out) return -1;
  std::memset(out, 0, sizeof(*out));
  uint64_t t_ini = 0;
  if (oracle_simulate(mm, seed, walks, &t_ini) != 0) return -1;
  out->t_ini = t_ini;
  or_check_result r;
  or_check_result last;
  bool have_last = false;
  auto run = [&](uint64_t T, int ee) {
    oracle_check(mm, T, prune, ee, &r, nullptr, 0);
    out->states += r.states;
    out->checks += 1;
  };
  if (search == 0) {
    // single pass: minimum over every kept terminal
    Model m = load(mm);
    Exploration ex = explore(m, prune ? t_ini : kNoLimit, prune != 0);
    uint64_t states = 0;
    for (uint64_t w : ex.width) states += w;
    out->states += states;
    out->checks += 1;
    uint64_t t_min = kNoLimit;
    for (size_t l = 0; l < ex.width.size(); ++l)
      if (ex.has_violation[l]) t_min = std::min(t_min, ex.best[l][0]);
    if (refine) run(t_min - 1, early_exit);      // must hold
    run(t_min, early_exit);                      // must be violated
    last = r;
    have_last = true;
  } else if (search == 1) {
    uint64_t T = t_ini;
    for (;;) {
      run(T, early_exit);
      if (r.holds) break;
      last = r;
      have_last = true;
      T = r.cex_time - 1;
    }
  } else if (search == 2) {
    uint64_t lo = 0, hi = t_ini;
    while (hi - lo > 1) {
      uint64_t mid = lo + (hi - lo) / 2;
      run(mid, early_exit);
      if (r.holds) {
        lo = mid;
      } else {
        hi = r.cex_time;
        last = r;
        have_last = true;
      }
    }
    if (!have_last || last.cex_time != hi) {
      run(hi, early_exit);
      last = r;
      have_last = true;
    }
  } else {
    return -1;
  }
  if (!have_last || last.holds) return -1;
  out->t_min = last.cex_time;
  out->i = last.cex_i;
  out->j = last.cex_j;
  out->level = last.cex_level;
  for (int c = 0; c < 16; ++c) out->n[c] = last.cex_n[c];
  return 0;
}

}  // extern "C"
