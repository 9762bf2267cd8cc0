/*
 * mc_pe.h -- C-ABI of the processing-element level model: the same queries
 * as mc.h (check, min-time, count) on a finer transition system that keeps
 * the processes the cost-table model folds into one number per work-group.
 *
 * Model (Section 4, Step 1, Listings 3-9; the Minimum model of Section 6,
 * Listings 10-15, is an instance with another program).  Each of P compute
 * units (`unit`) runs the work-group it was given as NWE processing elements
 * (`pex`) with one local `barrier`; the `clock` counts global time.  Per
 * configuration (WG index i, TS index j) the caller gives N_ij work-groups,
 * NWE_ij and a *program*: the segments every PE of a unit executes for one
 * work-group, each either `ticks` clock ticks of `long_work` in which `pes`
 * PEs take part, or a local barrier (ticks = 0) that `pes` PEs arrive at.
 * A program step is one tick of a work segment or one barrier.  Transitions:
 *
 *   select    s0 -> (i) -> (i, j, every unit idle): `select` in `main`
 *             (Listing 3);
 *   dispatch  a unit that is idle while work-groups are left takes the next
 *             one and starts its program (the device's `go`, Listing 5);
 *   mark      a participating PE of a busy unit that has not yet marked the
 *             current step marks it: at a tick step it reports NRP_work++
 *             and waits for the clock (`long_work`, Listing 8), at a barrier
 *             step it sends `done` to the barrier (Listing 7);
 *   release   a unit at a barrier step whose participants have all marked
 *             moves on (the barrier's `go`);
 *   tick      when every busy unit is at a tick step with all participants
 *             marked and no unit is idle while work-groups are left, time
 *             grows by one (Listing 9) and every busy unit moves on;
 *   FIN       no work-group left and every unit idle (Listing 4); the model
 *             time is the number of ticks.
 *
 * Every transition order is explored: the marks of one step interleave in
 * every order (2^pes states per unit and step), as in SPIN without partial
 * order reduction.  Every path to a state has the same length, so the graph
 * is layered and explored one BFS level per device-wide step.
 *
 * Conventions are those of mc.h: MC_OK or a negative MC_ERR_* code; host
 * pointers in the description are copied; the library owns the model, its
 * buffers and the traces; a model is not thread-safe; work runs on the
 * model's stream; there is no CPU fallback.
 */
#ifndef MC_PE_H
#define MC_PE_H

#include <stdint.h>

#include "mc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mc_pe_model mc_pe_model;

/* PE-level model description.  Per-configuration arrays are row-major
 * [i][j]; the segments of configuration k are seg_*[prog_off[k] ..
 * prog_off[k+1]-1].  Limits: a, b 1..255, P 1..8, NWE 1..8 with
 * P*max(NWE) + P + 1 <= 32 (the successors of one state), at least one
 * segment per program, seg_pes 1..NWE of its configuration, seg_ticks <=
 * 65535, the packed state within 128 bits. */
typedef struct {
  uint32_t n_wg;                /* a = |D_WG|                                */
  uint32_t n_ts;                /* b = |D_TS|                                */
  uint32_t P;                   /* compute units                             */
  const uint32_t* wg_values;    /* [a] echoed in results; NULL ok           */
  const uint32_t* ts_values;    /* [b] echoed in results; NULL ok           */
  const uint32_t* n_workgroups; /* [a*b] N_ij >= 1                           */
  const uint32_t* pes;          /* [a*b] NWE_ij: PEs per unit                */
  const uint32_t* prog_off;     /* [a*b + 1] first segment of each program   */
  const uint32_t* seg_ticks;    /* [prog_off[a*b]] ticks; 0 = local barrier */
  const uint32_t* seg_pes;      /* [prog_off[a*b]] PEs taking part           */
} mc_pe_model_desc;

/* Packed-state layout, for decoding trace keys (always two u64 words, {lo,
 * hi}).  Bits from the top of the used width: [i+1 : wg_bits][j+1 : ts_bits]
 * [level : level_bits] then one field of unit_bits per unit, unit c at bit
 * unit_shift[c] = (P-1-c) * unit_bits; inside a unit field, from the top:
 * [n : n_bits] work-groups taken, [busy : 1], [pc : pc_bits] program step,
 * [mask : mask_bits] PEs that marked the step (bit e = PE e).  s0 is the
 * all-zero key; the level field holds the state's BFS level. */
typedef struct {
  uint32_t used_bits, P;
  uint32_t wg_bits, ts_bits, level_bits, unit_bits;
  uint32_t n_bits, pc_bits, mask_bits, tile;  /* tile: lanes expanding one state */
  uint32_t wg_shift, ts_shift, level_shift, max_level;
  uint32_t unit_shift[8];
  uint64_t max_steps;    /* longest program in steps                        */
  uint64_t table_slots;  /* visited-set slots                               */
  uint64_t log_capacity; /* frontier-log entries                            */
  uint64_t device_bytes; /* device memory of the current buffers            */
} mc_pe_layout;

/* Validate and copy the description, compute the key layout.  No device
 * memory is touched.  opt may be NULL (mc_options_default); search modes
 * other than SINGLE, sim_* and key options are ignored.  The visited set and
 * the frontier log start at table_log2 / log_capacity when given, else at
 * 2^20 slots and 2^22 entries, and grow fourfold (up to half the device's
 * free memory, and the visited set up to 2^31 slots) whenever a query ends
 * in TABLE_FULL or FRONTIER, which then reruns; max_probes 0 means 64 bucket
 * probes.  Errors: INVAL, OVERFLOW (also table_log2 > 31). */
int mc_pe_model_create(const mc_pe_model_desc* desc, const mc_options* opt, mc_pe_model** out);
void mc_pe_model_destroy(mc_pe_model* m);
int mc_pe_set_stream(mc_pe_model* m, void* stream);
int mc_pe_model_layout(const mc_pe_model* m, mc_pe_layout* out);

/* G(FIN -> time > T) (Section 4, Step 2): level-synchronous BFS; prune drops
 * successors whose time exceeds T, early_exit stops after the first level
 * holding a FIN state of time <= T.  The counterexample is, in that level,
 * the violating FIN state with the smallest (time, i, j, key); *cex (NULL ok)
 * receives the path s0 -> counterexample (two words per state).  out uses
 * mc_check_result with key_words = 2.  Errors: INVAL, NOMEM, TABLE_FULL,
 * FRONTIER, TIMEOUT, CUDA (after growth stopped). */
int mc_pe_check(mc_pe_model* m, uint64_t T, mc_check_result* out, mc_trace** cex);

/* T_min and its configuration (Section 4, Steps 3-4): one full exploration
 * takes the least FIN time; check(T_min - 1) must hold (with refine) and the
 * counterexample of check(T_min) gives (WG, TS) and *trace.  t_ini in the
 * result is 0.  Errors: as mc_pe_check. */
int mc_pe_min_time(mc_pe_model* m, mc_min_result* out, mc_trace** trace);

/* Every reachable state (no pruning, no early exit).  Errors: as above. */
int mc_pe_count_states(mc_pe_model* m, uint64_t* out);

/* Per-level widths of the last exploration (up to cap). Errors: INVAL, CUDA. */
int mc_pe_last_widths(mc_pe_model* m, uint64_t* out, uint32_t cap, uint32_t* n);

int mc_pe_get_stats(const mc_pe_model* m, mc_stats* out);
int mc_pe_reset_stats(mc_pe_model* m);
const char* mc_pe_last_error(const mc_pe_model* m);

#ifdef __cplusplus
}
#endif

#endif /* MC_PE_H */
