/*
 * mc.h -- C-ABI of the GB300 explicit-state explorer for auto-tuning by
 * model checking (Garanina, Staroletov, Gorlatch: "Auto-Tuning
 * High-Performance Programs Using Model Checking in Promela").
 *
 * The library explores, on one GPU, the transition system of an OpenCL
 * kernel launch (Section 4, Step 1, processes `main`, `host`, `device`,
 * `unit`, `pex`, `clock`, Listings 3-9) with its scheduling semantics kept
 * and the per-processing-element ticking folded into a cost table:
 *
 *   state  (i, j, n_0..n_{P-1}): WG index i and TS index j chosen by the
 *          nondeterministic `select` of `main` (Listing 3), and n_c, the
 *          work-groups compute unit c has taken (`host`/`device`,
 *          Listings 4-5);
 *   clock  clk_c = n_c * t_c with t_c = cost[i][j] * speed[c] -- the time
 *          the unit has worked; the model time of a state is max_c clk_c
 *          (`clock`, Listing 9);
 *   FIN    a state whose N_ij work-groups are all dispatched (Listing 4).
 *
 * Dispatch rules: MC_FREE lets any unit take the next work-group (every
 * interleaving); MC_GREEDY lets only the units whose clock is minimal take it
 * (the unit that reported `done` first is re-dispatched, Listing 5), ties in
 * every order.
 *
 * Queries follow the counterexample method (Section 2, Section 4 Steps 2-4):
 * mc_check decides the over-time property  G(FIN -> time > T)  and returns a
 * counterexample trace when it fails; mc_min_time finds the minimal T for
 * which a counterexample exists and the (WG, TS) of that counterexample.
 *
 * Conventions
 *   - Every function returns MC_OK (0) or a negative MC_ERR_* code; nothing
 *     throws across the ABI.  mc_strerror() names the code.
 *   - All pointers in mc_model_desc are HOST pointers owned by the caller;
 *     mc_model_create copies them.  The library owns the model, its device
 *     buffers and every mc_trace it returns.
 *   - A model is not thread-safe.  Queries run on the model's CUDA stream
 *     (default: the legacy default stream; see mc_set_stream) and return
 *     after that stream has finished the query's work.
 *   - Device memory comes from the allocator set by mc_set_allocator
 *     (default: the library's stream-ordered pool on the model's device,
 *     which keeps up to 1 GiB of freed blocks for later models), allocated
 *     on the first query or by mc_reserve, and released by
 *     mc_model_destroy.  Pinned host staging is pooled the same way.
 *   - There is no CPU fallback: without a usable CUDA device, queries return
 *     MC_ERR_CUDA.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define MC_OK 0
#define MC_ERR_INVAL (-1)      /* bad argument or model description         */
#define MC_ERR_NOMEM (-2)      /* device or host allocation failed          */
#define MC_ERR_TABLE_FULL (-3) /* visited-set probe limit reached           */
#define MC_ERR_FRONTIER (-4)   /* frontier log capacity exceeded            */
#define MC_ERR_TIMEOUT (-5)    /* a device-side wait exceeded its limit     */
#define MC_ERR_CUDA (-6)       /* CUDA runtime error (see mc_last_error)    */
#define MC_ERR_OVERFLOW (-7)   /* key wider than 128 bits, clock >= 2^40,
                                  a level wider than 2^31, or a, b > 4095   */

typedef enum { MC_FREE = 0, MC_GREEDY = 1 } mc_rule;

/* How mc_min_time searches for T_min (Section 2, Fig. 1; Section 4 Step 3). */
typedef enum {
  MC_SEARCH_SINGLE = 0, /* one exploration, min-reduction over terminal times,
                           then the certificate checks at T_min-1 and T_min  */
  MC_SEARCH_LOWER = 1,  /* check(T), then T := counterexample time - 1, until
                           the property holds                                */
  MC_SEARCH_BISECT = 2  /* bisection between 0 and T_ini (Fig. 1)            */
} mc_search;

/* How the exploration kernel inserts a successor into the visited set
 * (mc_options.probe_scheme).  SPLIT and ONE_CALL fetch the successor's first
 * 32-byte bucket into shared memory first; CAS_FIRST starts with the
 * compare-and-swap.  The results are identical, only the speed differs. */
typedef enum {
  MC_PROBE_AUTO = 0,     /* SPLIT with 64-bit keys, CAS_FIRST with 128-bit
                            (the fastest on C2 at G=80, whose table stays in
                            L2, and on C3 at G=36, whose probes go to DRAM) */
  MC_PROBE_SPLIT = 1,    /* pick the slot from the fetched bucket, issue the
                            CAS of every proposal of the round, then resolve
                            (a lost slot or a full bucket falls back to the
                            general insert from the same bucket)              */
  MC_PROBE_ONE_CALL = 2, /* the general insert (scan, CAS, next bucket) from
                            the fetched bucket, one proposal at a time        */
  MC_PROBE_CAS_FIRST = 3, /* compare-and-swap from empty on the first slot
                            of the first bucket, no fetch: an empty slot is
                            a win and the key itself a duplicate in one
                            round trip; a key of an earlier level (a free
                            slot) gets a second compare-and-swap from that
                            key; another key of the level falls back to
                            the general insert                             */
  MC_PROBE_CAS_CLEAR = 4 /* CAS_FIRST, and every expanded state empties its
                            own first slot (compare-and-swap from its key),
                            so the table holds about two levels' keys and
                            most first slots are empty when probed: faster
                            in deep searches over tables that stay in L2,
                            slower where the extra atomic goes to DRAM    */
} mc_probe_scheme;

/* Which kernel explores a pass (mc_options.engine).  Both report identical
 * results; only the speed differs. */
typedef enum {
  MC_ENGINE_AUTO = 0,    /* CONFIG when one configuration's widest level fits
                            the shared memory of a thread block (closed-form
                            bound: at most 2048 states with 64-bit keys, 1024
                            with 128-bit keys), else LEVEL                    */
  MC_ENGINE_LEVEL = 1,   /* level-synchronous BFS over the whole state space:
                            one persistent cooperative launch per pass, a
                            device-wide barrier per level, the visited set in
                            device memory (any model)                         */
  MC_ENGINE_CONFIG = 2   /* one thread block per (WG, TS) configuration: the
                            selects of Listing 3 split the states below level 2
                            into disjoint subtrees, and a block explores one
                            subtree with its frontier and visited set in shared
                            memory and a block-wide barrier per level (models
                            whose per-configuration levels fit, see AUTO)     */
} mc_engine;

typedef struct mc_model mc_model;
typedef struct mc_trace mc_trace;

/* Model description (Section 4, Step 1).  All arrays are host memory owned
 * by the caller and copied by mc_model_create.  Row-major [i][j] arrays are
 * indexed by i < n_wg (work-group size index) and j < n_ts (tile size index). */
typedef struct {
  uint32_t n_wg;                /* a = |D_WG|, 1..4095                       */
  uint32_t n_ts;                /* b = |D_TS|, 1..4095                       */
  uint32_t P;                   /* compute units, 1..16                      */
  const uint32_t* wg_values;    /* [a] WG values, echoed in results; NULL ok */
  const uint32_t* ts_values;    /* [b] TS values, echoed in results; NULL ok */
  const uint32_t* n_workgroups; /* [a*b] N_ij >= 1 work-groups               */
  const uint32_t* cost;         /* [a*b] time of one work-group, >= 1        */
  const uint32_t* speed;        /* [P] speed factor per unit, >= 1; NULL = 1 */
  uint32_t rule;                /* mc_rule                                   */
  uint32_t key_bits;            /* packed state width: 0 = auto (64 when the
                                   state fits in 64 bits, else 128), 64, 128 */
} mc_model_desc;

/* Query options.  Start from mc_options_default(). */
typedef struct {
  uint32_t prune;               /* 1: drop successors whose clock exceeds T
                                   (they cannot reach a violating terminal)  */
  uint32_t early_exit;          /* 1: mc_check stops after the first BFS level
                                   that holds a violating terminal           */
  uint32_t search;              /* mc_search used by mc_min_time             */
  uint32_t refine;              /* SINGLE: also run check(T_min - 1)         */
  uint64_t sim_seed;            /* seed of the T_ini simulation              */
  uint32_t sim_walks;           /* random runs taken for T_ini (>= 1)        */
  uint32_t load_factor_pct;     /* visited-set load-factor cap, 10..90       */
  uint32_t table_log2;          /* 0: size the visited set from the bound;
                                   else 2^table_log2 slots                   */
  uint32_t threads_per_block;   /* 0: 256; else 64..256, multiple of 32      */
  uint32_t blocks_per_sm;       /* 0: occupancy maximum                      */
  uint32_t max_probes;          /* 0: whole table; else bucket probe limit   */
  uint64_t log_capacity;        /* 0: closed-form bound; else states kept in
                                   the frontier log (MC_ERR_FRONTIER beyond) */
  uint64_t barrier_timeout_ns;  /* 0: 60 s.  Limit of each device-wide wait  */
  uint32_t debug_barrier_extra; /* test hook: >0 makes every device-wide wait
                                   expect that many extra arrivals, so it
                                   times out and the query returns
                                   MC_ERR_TIMEOUT.  Keep 0.                 */
  uint32_t timing;              /* 1: time the exploration kernels with CUDA
                                   events on the model's stream (mc_get_stats):
                                   one pair around each run of launches a
                                   query enqueues back to back (PE-level
                                   model, mc_pe.h: one pair per launch)     */
  uint32_t lanes_per_state;     /* lanes of the warp tile that expands one
                                   state.  Cost-table model: a power of two
                                   from P (rounded up) to 16, one unit per
                                   lane; PE-level model (mc_pe.h): 4 or 8 (up
                                   to 3 successors per lane), 16 (up to 2) or
                                   32 (1).  0 = the smallest that fits      */
  uint32_t probe_scheme;        /* mc_probe_scheme of the single-model
                                   explorer (mc_check, mc_min_time,
                                   mc_count_states); batches and the PE-level
                                   model keep their own                      */
  uint32_t no_log_tags;         /* 1: never tag the frontier log (every block
                                   writes its entries before it arrives at the
                                   level barrier); 0: tag it where the keys
                                   have room (mc_layout.log_tag_bits)        */
  uint32_t engine;              /* mc_engine of the single-model queries    */
  uint32_t unit_threads;        /* CONFIG engine: threads of the block that
                                   explores one configuration, 64..512, a
                                   multiple of 32; 0 = from the model's
                                   widest configuration level, and one warp
                                   per configuration when that level's lanes
                                   fit a warp (P <= 4 under GREEDY)          */
  uint32_t stage_chunk;         /* LEVEL engine: winners a warp stages in
                                   shared memory before it reserves frontier-
                                   log space and copies them out: 64 to 192,
                                   a multiple of 32; 0 = 128                 */
} mc_options;

/* Result of mc_check (Section 4, Step 2: Phi = G(FIN -> time > T)). */
typedef struct {
  uint32_t holds;        /* 1: every kept terminal has time > T            */
  uint32_t levels;       /* BFS levels explored (last level + 1)           */
  uint64_t states;       /* unique states kept in those levels             */
  uint64_t cex_time;     /* counterexample model time (holds == 0)         */
  uint32_t cex_wg_index; /* i of the counterexample                        */
  uint32_t cex_ts_index; /* j of the counterexample                        */
  uint32_t cex_wg;       /* wg_values[i] (or i when wg_values was NULL)    */
  uint32_t cex_ts;       /* ts_values[j] (or j)                            */
  uint32_t cex_level;    /* BFS level of the counterexample terminal       */
  uint32_t key_words;    /* 1 or 2: u64 words per packed state             */
  uint64_t cex_key[2];   /* packed counterexample state, {lo, hi}          */
} mc_check_result;

/* Result of mc_min_time (Section 4, Steps 3 and 4). */
typedef struct {
  uint64_t t_min;        /* minimal model time of any terminal             */
  uint64_t t_ini;        /* initial bound from the simulation              */
  uint32_t wg_index;     /* configuration of the counterexample of check(T_min) */
  uint32_t ts_index;
  uint32_t wg;           /* wg_values[wg_index] (or the index)             */
  uint32_t ts;           /* ts_values[ts_index] (or the index)             */
  uint64_t states;       /* unique states summed over every exploration    */
  uint32_t checks;       /* explorations run                               */
  uint32_t level;        /* BFS level of the witness terminal              */
  uint64_t witness_key[2];
} mc_min_result;

/* Packed-state layout, for decoding trace keys.  Bits from the top of the
 * used width: [i+1 : wg_bits][j+1 : ts_bits][n_0 : n_bits]...[n_{P-1}];
 * n_c sits at bit offset n_shift[c] = (P-1-c) * n_bits, j+1 at ts_shift,
 * i+1 at wg_shift.  s0 (nothing selected) is the all-zero key.             */
typedef struct {
  uint32_t key_bits;     /* 64 or 128                                      */
  uint32_t key_words;    /* 1 or 2                                         */
  uint32_t used_bits;    /* wg_bits + ts_bits + P * n_bits                 */
  uint32_t P, n_bits, ts_bits, wg_bits, ts_shift, wg_shift;
  uint32_t max_level;    /* deepest BFS level: max N_ij + 2                */
  uint32_t n_shift[16];
  uint64_t table_slots;  /* visited-set slots                              */
  uint64_t log_capacity; /* frontier-log entries                           */
  uint64_t max_width;    /* bound on one level's width                     */
  uint64_t state_bound;  /* bound on all reachable states (saturates)      */
  uint64_t device_bytes; /* device memory the model needs                  */
  uint32_t probe_scheme; /* the insert its explorations use (mc_probe_scheme,
                            AUTO resolved)                                 */
  uint32_t log_tag_bits; /* bits per 64-bit word of a frontier-log entry
                            that tag it with its pass, so a block can arrive
                            at a level's barrier before writing its last
                            entries: 8 to 16 where the key leaves that many
                            spare (a 128-bit key is stored as two words of
                            64 - log_tag_bits payload bits), else 0        */
  uint32_t engine;       /* MC_ENGINE_LEVEL or MC_ENGINE_CONFIG (AUTO
                            resolved); with CONFIG, table_slots is the
                            shared-memory table of one block and the log
                            holds one segment per configuration           */
  uint32_t unit_threads; /* CONFIG: threads that explore one configuration:
                            32 when one warp does (its widest level x lanes
                            per state fits a warp and mc_options.
                            unit_threads is 0), else the block's threads;
                            0 with LEVEL                                  */
  uint64_t unit_width;   /* bound on one configuration's widest level      */
} mc_layout;

/* Counters accumulated over the model's queries (reset by mc_reset_stats). */
typedef struct {
  uint64_t explore_launches; /* exploration kernel launches                  */
  uint64_t other_launches;   /* simulation kernel launches                   */
  uint64_t states;           /* unique states summed over those launches     */
  uint64_t h2d_bytes;        /* host -> device bytes copied                  */
  uint64_t d2h_bytes;        /* device -> host bytes copied                  */
  double explore_ms;         /* summed CUDA-event time of the exploration
                                kernels (only with mc_options.timing = 1):
                                a query's chained checks are timed as one
                                window, gaps between their launches included
                                (PE-level model: each launch alone)          */
  uint64_t device_steps;     /* device-wide barrier steps: BFS levels of the
                                passes, or lockstep steps of a batch launch  */
  uint64_t probes;           /* successors generated, each one visited-set
                                probe (PE-level model, mc_pe.h, only)        */
  uint64_t graph_launches;   /* batch runs replayed from the captured CUDA
                                graph of mc_batch_run (batches only)         */
} mc_stats;

typedef void* (*mc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*mc_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* Fill *opt with the defaults: prune 1, early_exit 1, search SINGLE,
 * refine 1, sim_seed 2305091300, sim_walks 1, load_factor_pct 25, the rest 0. */
void mc_options_default(mc_options* opt);

/* The model of Section 4, Step 1 (the problem statement of the method):
 * the domains of the tuning parameters that `main` selects from (Listing 3),
 * the work-groups of each configuration and the time one of them takes on
 * a compute unit (the abstract kernel of Listing 2 folded into a cost per
 * (WG, TS) and a speed per unit), and the unit count of the abstract
 * platform (Section 3.1).  Validate and copy the description; compute the
 * key layout and the closed-form bounds that size the device buffers.  No
 * device memory is touched.  opt may be NULL (defaults).  Errors: INVAL
 * (NULL or zero sizes, P > 16, N/cost/speed of 0, unknown rule or
 * key_bits), OVERFLOW. */
int mc_model_create(const mc_model_desc* desc, const mc_options* opt, mc_model** out);

/* Free the model, its device buffers (through the allocator that made them)
 * and its pinned host buffers.  NULL is ignored. */
void mc_model_destroy(mc_model* m);

/* Replace the options of later queries.  Options that size buffers or the
 * launch (load_factor_pct, table_log2, log_capacity, threads_per_block,
 * blocks_per_sm, probe_scheme, no_log_tags, engine, unit_threads,
 * lanes_per_state) only act before the buffers exist.  Errors: INVAL. */
int mc_set_options(mc_model* m, const mc_options* opt);

/* CUDA stream (a cudaStream_t, NULL = legacy default stream) for every later
 * query.  Errors: INVAL. */
int mc_set_stream(mc_model* m, void* stream);

/* Device allocator for the model's buffers; call before the first query or
 * mc_reserve.  alloc returns NULL on failure.  Errors: INVAL (NULL function,
 * or buffers already allocated). */
int mc_set_allocator(mc_model* m, mc_alloc_fn alloc, mc_free_fn free_fn, void* ctx);

/* Allocate the device buffers now.  Errors: NOMEM, CUDA, OVERFLOW. */
int mc_reserve(mc_model* m);

/* Key layout and buffer sizes of the model.  Errors: INVAL. */
int mc_model_layout(const mc_model* m, mc_layout* out);

/* Decide G(FIN -> time > T) (Section 4, Step 2) by level-synchronous BFS.
 * With prune, successors whose max clock exceeds T are dropped; with
 * early_exit, the search ends after the first level holding a terminal of
 * time <= T.  The counterexample is, in that first level, the violating
 * terminal with the smallest (time, key); *cex (NULL ok) receives the path
 * s0 -> counterexample when the property fails, else NULL.  Errors: INVAL,
 * NOMEM, TABLE_FULL, FRONTIER, TIMEOUT, CUDA. */
int mc_check(mc_model* m, uint64_t T, mc_check_result* out, mc_trace** cex);

/* Find T_min, the least T for which check(T) fails, and its configuration
 * (Section 4, Steps 3 and 4) with the options' search mode.  T_ini comes from
 * sim_walks random runs (Step 3's simulation).  In every mode the reported
 * configuration and witness are the counterexample of check(T_min), so all
 * modes agree.  *trace (NULL ok) receives the witness path.  Errors: as
 * mc_check. */
int mc_min_time(mc_model* m, mc_min_result* out, mc_trace** trace);

/* The reachable-state count of exhaustive verification (Section 6, Table 1
 * reports the memory such a search takes): every state reachable from s0
 * under the model's dispatch rule, explored without pruning and without
 * early exit.  Errors: as mc_check. */
int mc_count_states(mc_model* m, uint64_t* out);

/* T_ini: the least terminal time over `walks` random runs (Section 4,
 * Step 3).  Walk w draws splitmix64 outputs number (w << 32) + 0, 1, ...
 * of the stream seeded with `seed`: the WG index (x % a), the TS index
 * (x % b), then per work-group the unit among the allowed ones in index
 * order (x % count).  Errors: INVAL, NOMEM, CUDA. */
int mc_simulate(mc_model* m, uint64_t seed, uint32_t walks, uint64_t* t_ini);

/* Swarm search (Section 5): a first round of `walks_per_round` random runs
 * (the swarm checking G(!FIN): every run that terminates is a counterexample)
 * gives the first trail; each further round runs as many fresh random runs
 * cut as soon as a clock passes T-1, T the best time so far (the swarm
 * checking the over-time property at T-1).  The search stops after the first
 * round that finds nothing -- the paper's stopping criterion -- or after
 * max_rounds.  Runs are the walks of mc_simulate: round r uses walks
 * r*walks_per_round .. (r+1)*walks_per_round-1 of `seed`.  Not a proof of
 * optimality: compare with mc_min_time.  *trace (NULL ok) receives the best
 * run.  Errors: INVAL (walks_per_round 0 or above 2^24), NOMEM, CUDA. */
typedef struct {
  uint64_t best_time;     /* least terminal time found                      */
  uint64_t first_time;    /* least time of the first round                  */
  uint32_t wg_index, ts_index, wg, ts;   /* configuration of the best run   */
  uint32_t rounds;        /* rounds run (the last one found nothing unless
                             max_rounds stopped the search)                 */
  uint32_t key_words;
  uint64_t walks;         /* random runs made                               */
  uint64_t best_walk;     /* walk index of the best run                     */
  double first_trail_ms;  /* host time from the call to the first round's end */
  double total_ms;        /* host time of the whole search                  */
} mc_swarm_result;
int mc_swarm(mc_model* m, uint64_t seed, uint32_t walks_per_round, uint32_t max_rounds,
             mc_swarm_result* out, mc_trace** trace);

/* Per-level widths of the model's last exploration; *n receives the level
 * count and up to cap widths are copied.  Errors: INVAL, CUDA. */
int mc_last_widths(mc_model* m, uint64_t* out, uint32_t cap, uint32_t* n);

/* Copy the model's counters into *out.  Errors: INVAL. */
int mc_get_stats(const mc_model* m, mc_stats* out);

/* Zero the model's counters.  Errors: INVAL. */
int mc_reset_stats(mc_model* m);

/* Trace accessors: states s0 .. witness, each key_words u64 ({lo, hi}). */
int mc_trace_length(const mc_trace* t);
uint32_t mc_trace_key_words(const mc_trace* t);
const uint64_t* mc_trace_states(const mc_trace* t);
void mc_trace_free(mc_trace* t);

/* ------------------------------------------------------------ batched queries
 * Many models answered by one persistent launch (auto-tuning issues many
 * queries, Section 2): every instance runs its own query program (mc_check or
 * mc_min_time in SINGLE mode) and all of them advance in lockstep, so each
 * device-wide barrier serves the whole batch.  Every instance uses 128-bit
 * keys; results equal those of mc_check / mc_min_time on the same model and
 * options (search mode SINGLE; lowering and bisection are single-model only). */
typedef struct mc_batch mc_batch;
typedef enum { MC_QUERY_CHECK = 0, MC_QUERY_MIN_TIME = 1 } mc_query_kind;
typedef struct {
  uint32_t kind;         /* mc_query_kind                                   */
  uint32_t reserved;
  uint64_t T;            /* threshold of MC_QUERY_CHECK                     */
} mc_query;
typedef struct {
  int32_t status;        /* MC_OK or this instance's MC_ERR_*               */
  uint32_t kind;
  uint32_t holds;        /* check: 1 when the property holds                */
  uint32_t levels;       /* levels of the last pass                         */
  uint64_t states;       /* unique states over every pass                   */
  uint32_t checks;       /* passes run                                      */
  uint32_t level;        /* counterexample level (0 when it holds)          */
  uint64_t time;         /* counterexample time; T_min for min-time         */
  uint64_t t_ini;        /* min-time: the simulated bound                   */
  uint32_t wg_index, ts_index, wg, ts;
  uint64_t key[2];       /* packed counterexample / witness state {lo, hi}  */
} mc_batch_result;

/* Validate and lay out `n` (1..1024) models with one set of options.  Host
 * only; device memory is taken at the first run.  Errors: as
 * mc_model_create, INVAL, NOMEM (a model's bound does not fit). */
int mc_batch_create(const mc_model_desc* descs, uint32_t n, const mc_options* opt, mc_batch** out);
void mc_batch_destroy(mc_batch* b);
int mc_batch_set_stream(mc_batch* b, void* stream);
int mc_batch_set_allocator(mc_batch* b, mc_alloc_fn alloc, mc_free_fn free_fn, void* ctx);
/* Device bytes of the batch's pool (visited sets, logs, level records). */
int mc_batch_device_bytes(const mc_batch* b, uint64_t* out);
/* Run queries[i] on model i for every i, in one launch; fills results[n].
 * The first run captures its work (uploads, clears, the persistent launch,
 * read-backs) into a CUDA graph, which later runs replay with new queries;
 * where capture is not possible the work is enqueued directly.
 * Errors: INVAL, NOMEM, TIMEOUT, CUDA; per-instance errors in status. */
int mc_batch_run(mc_batch* b, const mc_query* queries, mc_batch_result* results);
/* Trace of instance i's counterexample from the last run: *len states of two
 * u64 words ({lo, hi}); up to cap states are copied.  Errors: INVAL, CUDA. */
int mc_batch_trace(mc_batch* b, uint32_t i, uint64_t* keys, uint32_t cap, uint32_t* len);
int mc_batch_get_stats(const mc_batch* b, mc_stats* out);
const char* mc_batch_last_error(const mc_batch* b);

/* ------------------------------------------------------------ served queries
 * A request loop (no counterpart in the paper's tooling, which runs one SPIN
 * verification per process): queries for models of different sizes are
 * submitted as they arrive and answered by a persistent device loop that
 * keeps up to `slots` of them on the GPU at once.  A request is admitted when
 * a slot is free and the device pool has room for its visited set, frontier
 * log and tables (closed-form bound); requests admitted while others run
 * join the device loop at its next step, so their work overlaps.  Results
 * equal those of mc_batch_run / mc_check / mc_min_time for the same model.
 * A host thread of the library admits, harvests and relaunches; the device
 * loop exits after `idle_ns` without work and is relaunched on demand.  The
 * loop runs one block per SM unless mc_options.blocks_per_sm says otherwise. */
typedef struct mc_server mc_server;
typedef struct {
  uint32_t slots;        /* requests on the device at once, 1..1024        */
  uint32_t reserved0;
  uint64_t pool_bytes;   /* device memory for the requests' buffers        */
  uint64_t idle_ns;      /* device loop's wait for new work (0: 0.2 ms)    */
  uint64_t solo_states;  /* latency path: a request that finds the server
                            idle (nothing on the device, nothing else
                            queued) and whose closed-form state bound is at
                            most this runs alone on the single-model
                            explorer, whose BFS levels cost half a lockstep
                            step; requests arriving meanwhile wait for it.
                            0: 2^22 states; 1: never                        */
  uint64_t reserved[3];
} mc_server_config;
typedef struct {
  uint64_t ticket;
  mc_batch_result result;
  double submit_s;       /* host steady-clock seconds: submitted,          */
  double admit_s;        /*   posted to the device (or started alone),     */
  double done_s;         /*   result harvested                             */
  uint32_t path;         /* 0: the lockstep device loop, 1: alone
                            (solo_states), 2: a configuration-engine job  */
  uint32_t reserved;
} mc_server_result;

/* Allocate the pool and mailboxes, start the host thread.  Errors: INVAL,
 * NOMEM, CUDA. */
int mc_server_create(const mc_server_config* cfg, const mc_options* opt, mc_server** out);
/* Queue one query on a model (copied).  Errors: INVAL, OVERFLOW, NOMEM (the
 * model does not fit the pool at all), or the server's fatal error. */
int mc_server_submit(mc_server* s, const mc_model_desc* desc, const mc_query* q, uint64_t* ticket);
/* Take up to cap finished results, waiting up to wait_ms for the first. */
int mc_server_poll(mc_server* s, mc_server_result* out, uint32_t cap, uint32_t* n, uint32_t wait_ms);
/* Queued and running requests, device-loop launches; returns the server's
 * fatal error (0 if none). */
int mc_server_status(mc_server* s, uint32_t* queued, uint32_t* running, uint64_t* launches);
/* Stop the device loop (requests in flight are abandoned) and free all. */
void mc_server_destroy(mc_server* s);

/* Random-access roofline of the current device (a measurement utility, not a
 * step of the method): times `accesses` independent random 32-byte sector
 * reads (op 0), reads followed by an atomicCAS on the sector (op 1), or an
 * atomicCAS from 0 alone (op 2) over a freshly allocated buffer of
 * `buffer_bytes` (use one far larger than L2), and writes the sustained
 * sectors per second.  The visited set of an exploration larger than L2 is
 * accessed this way (ops 0 and 1: the split and one-call inserts; op 2: the
 * CAS-first inserts), so these rates bound its HBM regime.
 * Allocates and frees its buffer.  Errors: INVAL, NOMEM, CUDA. */
int mc_measure_random_access(uint64_t buffer_bytes, uint64_t accesses, int op,
                             double* sectors_per_s, double* ms);

/* ------------------------------------------------- no-allocation variant
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a host framework that owns the device's
 * memory budget and offers no allocator, a serving path where an allocation
 * could block or fail, a plugin that may only launch on a stream it is
 * given.  It answers the same question as mc_check(T) for the model
 * described by `desc` (host memory, read during the call; options: `prune`,
 * `early_exit`, load factor 25%) and writes *out (host memory); no trace.
 *
 * Every scratch buffer comes from one static device array of
 * MC_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that
 * loads the library holds until exit.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  Its first call on
 * a device looks the array's device address up (cudaGetSymbolAddress, with
 * that device current), so make that first call before any stream capture.
 * Work runs on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * the call returns after it finished.  Calls share the array: calls that
 * overlap on the GPU race.  Errors: INVAL, OVERFLOW (as mc_model_create),
 * NOMEM when the model's visited set, frontier log and tables need more than
 * MC_NOALLOC_SCRATCH_BYTES, TABLE_FULL, FRONTIER, TIMEOUT, CUDA. */
#define MC_NOALLOC_SCRATCH_BYTES (32ull << 20)
int mc_check_noalloc(const mc_model_desc* desc, uint64_t T, uint32_t prune, uint32_t early_exit,
                     void* stream, mc_check_result* out);

/* Give the library's cached memory back: the freed device blocks kept in its
 * stream-ordered pools (up to the retention below, per device) and the
 * pinned host blocks kept for reuse (up to 64 MiB).  Models in use keep
 * theirs.  Safe at any time, also without a device.  Returns MC_OK. */
int mc_release_cached(void);

/* How many bytes of freed device memory each of the library's pools keeps
 * for later models instead of giving them back to the driver at the next
 * synchronisation (cudaMemPoolAttrReleaseThreshold): 1 GiB by default.  A
 * caller that creates and destroys large models in a loop (a server) raises
 * it so that a model's buffers are not unmapped and mapped again each time.
 * Applies to the pools that exist and to those made later; memory above the
 * new value is given back at the pool's next synchronisation.  Not a step of
 * the method.  Errors: CUDA when a pool refuses the value. */
int mc_set_pool_retention(uint64_t bytes);

/* Static name of an error code. */
const char* mc_strerror(int code);

/* Detail of the model's last MC_ERR_CUDA (a static or model-owned string). */
const char* mc_last_error(const mc_model* m);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
