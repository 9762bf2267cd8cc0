// Host side of the C-ABI declared in include/mc.h: model validation, key
// layout, closed-form sizing of the device buffers, and the query drivers of
// the counterexample method (Section 2; Section 4, Steps 2-4).  Every step of
// a query runs in the kernels of mc_kernels.cu; this file only enqueues them
// on the model's stream and reads back a few words of results.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mc.h"
#include "mc_host.h"
#include "mc_internal.h"

using mc::Ctrl;
using mc::ExploreArgs;
using mc::kNone;
using mc::Params;

namespace mc {

// Pinned host blocks, kept for reuse across models: pinning and unpinning
// pages (cudaMallocHost / cudaFreeHost) cost tens of microseconds each, which
// a create-query-destroy cycle would otherwise pay every time.  Blocks come
// in power-of-two classes from 4 KiB; at most 64 MiB stay cached.
namespace {
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;
size_t g_pinned_cached = 0;
constexpr size_t kPinnedCacheMax = 64ull << 20;

size_t pinned_class(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  return c;
}
}  // namespace

void* pinned_alloc(size_t bytes) {
  const size_t c = pinned_class(bytes);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    auto it = g_pinned_free.find(c);
    if (it != g_pinned_free.end()) {
      void* p = it->second;
      g_pinned_free.erase(it);
      g_pinned_cached -= c;
      return p;
    }
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, c, cudaHostAllocPortable) != cudaSuccess) {  // pinned for every device
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

// The library's stream-ordered device pool of each device, made on first
// use; freed blocks stay in it for reuse up to the retention (1 GiB unless
// mc_set_pool_retention changed it; the process's other allocations and
// pools are left alone).
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
uint64_t g_pool_keep = 1ull << 30;  // guarded by g_pool_mu
}  // namespace

cudaMemPool_t device_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = g_pool_keep;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

int set_pool_retention(uint64_t bytes) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  g_pool_keep = bytes;
  int rc = MC_OK;
  for (cudaMemPool_t pool : g_pools) {
    if (!pool) continue;
    uint64_t keep = bytes;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      rc = MC_ERR_CUDA;
    }
  }
  return rc;
}

void release_cached() {
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (cudaMemPool_t pool : g_pools)
      if (pool) cudaMemPoolTrimTo(pool, 0);
  }
  std::multimap<size_t, void*> blocks;
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    blocks.swap(g_pinned_free);
    g_pinned_cached = 0;
  }
  for (auto& b : blocks) cudaFreeHost(b.second);
  cudaGetLastError();
}

void pinned_free(void* p, size_t bytes) {
  const size_t c = pinned_class(bytes);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (g_pinned_cached + c <= kPinnedCacheMax) {
      g_pinned_free.emplace(c, p);
      g_pinned_cached += c;
      return;
    }
  }
  cudaFreeHost(p);
}

}  // namespace mc

namespace {

constexpr int kSlots = 4;  // per-pass result slots (device header + pinned copy)
constexpr int kTimingRing = 64;  // event pairs of timed launches (their times are read lazily)
// Device control block, in this order:
//   barrier lines  kSlots x kBarBytes (one device-wide barrier per slot)
//   headers        kSlots x Ctrl      (one pass result per slot)
//   scalars        kScalarBytes       (T_ini, T_min, spare)
//   trace          16 x (max_level + 2)
//   levels         16 x (max_level + 2), then off 8 x (max_level + 2)
// The headers, scalars and trace are contiguous and mirrored in pinned host
// memory with the same layout, so one copy reads a whole query's results
// back, and the barrier lines and headers are cleared by one memset.
constexpr size_t kScalarBytes = 64;
static_assert(sizeof(Ctrl) % 16 == 0, "headers keep 16-byte alignment");

struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool pooled = false;  // from the library's stream-ordered pool
};

uint32_t bits_for(uint64_t x) {  // bits to store values 0..x
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// C(n, k) saturating at 2^64 - 1
uint64_t binom_sat(uint64_t n, uint64_t k) {
  if (k > n) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (uint64_t i = 0; i < k; ++i) {
    r = r * (n - i) / (i + 1);
    if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
  }
  return (uint64_t)r;
}

uint64_t add_sat(uint64_t a, uint64_t b) { return a > UINT64_MAX - b ? UINT64_MAX : a + b; }
uint64_t mul_sat(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  return a > UINT64_MAX / b ? UINT64_MAX : a * b;
}

}  // namespace

struct mc_model {
  // description
  uint32_t a = 0, b = 0, P = 0, rule = 0;
  std::vector<uint32_t> wg, ts, N, cost, speed;
  mc_options opt{};
  // layout and bounds
  uint32_t key_bits = 64, key_words = 1, n_bits = 0, ts_bits = 0, wg_bits = 0;
  uint32_t ts_shift = 0, wg_shift = 0, used_bits = 0, max_level = 0, tile = 1;
  uint64_t max_width = 0, state_bound = 0;
  uint64_t log_cap = 0, table_slots = 0, device_bytes = 0;
  // configuration engine: closed-form widest level of one configuration,
  // and each configuration's frontier-log segment (its states' bound)
  uint64_t unit_width = 0, unit_log = 0;
  std::vector<uint64_t> seg;       // [a*b + 1] segment starts
  std::vector<uint32_t> order;     // [a*b] configurations, deepest first
  uint32_t engine = MC_ENGINE_LEVEL;
  uint32_t cfg_wcap = 0, cfg_tsize = 0;
  int cfg_threads = 0, cfg_grid = 0, cfg_grid_max = 0;
  size_t cfg_smem = 0;
  bool cfg_warp = false;  // one warp per configuration (widest level x lanes per state <= 32)
  // device state
  bool reserved = false;
  int device = -1;
  int grid = 0, threads = 0;
  int scheme = MC_PROBE_SPLIT;  // probe scheme of the exploration kernel (resolved at reserve)
  uint32_t tag_bits = 0;  // spare top key bits tagging the frontier log (0: untagged)
  uint32_t tag = 0;       // the last pass's tag
  cudaStream_t stream = nullptr;
  mc_alloc_fn alloc = nullptr;
  mc_free_fn dealloc = nullptr;
  void* actx = nullptr;
  std::vector<Buf> bufs;
  uint32_t* d_params = nullptr;
  void* d_table = nullptr;
  void* d_log_keys = nullptr;
  uint32_t* d_log_par = nullptr;
  uint8_t* d_ctrl_block = nullptr;
  Ctrl* d_ctrl = nullptr;
  uint64_t *d_levels = nullptr, *d_off = nullptr, *d_trace = nullptr;
  uint64_t *d_tini = nullptr, *d_tmin = nullptr;
  uint64_t* d_seg = nullptr;         // configuration engine: segment starts, records, order,
  mc::CfgRec* d_rec = nullptr;       // and one level-width array per result slot (a skipped
  uint32_t* d_order = nullptr;       // chained pass must not clear the last pass's widths)
  uint64_t* d_cfg_levels = nullptr;
  int last_slot = 0;                 // slot of the last pass that ran
  // min-time's certificate and counterexample checks in one launch: their
  // pass descriptors (slots 1 and 2, T_min read on the device) and the units
  // [(check, configuration) deepest first; with and without the certificate]
  mc::CfgPass* d_pair_pass = nullptr;
  uint64_t* d_pair_units = nullptr;
  uint8_t* h_block = nullptr;   // pinned host staging (from the pool), carved into:
  size_t h_block_bytes = 0;
  Ctrl* h_ctrl = nullptr;       // [kSlots]  } the device's headers, scalars and trace,
  uint64_t* h_scalar = nullptr; // [8]       } contiguous, read back by one copy
  uint64_t* h_trace = nullptr;  // [(max_level + 2) * 2]
  size_t mirror_bytes = 0;
  uint32_t* h_params = nullptr; // staging of N, cost, speed (then seg and order)
  cudaEvent_t ev[2 * kTimingRing] = {};  // [2p] start, [2p + 1] end of timed launch pair p
  uint64_t ev_pending = 0;               // bit p: pair p recorded, its time not yet in stats
  uint32_t ev_next = 0;                  // the pair the next timed run takes
  bool chain_open = false;               // a timed run of exploration launches is open
  uint32_t chain_pair = 0;               // its pair
  mc_stats stats{};
  std::string last_err;
  uint32_t last_levels = 0;
  Params params{};
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int cuda_fail(mc_model* m, cudaError_t e, const char* what) {
  m->last_err = std::string(what) + ": " + cudaGetErrorString(e);
  return MC_ERR_CUDA;
}

#define MC_CUDA(m, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail((m), e_, #call); \
  } while (0)

// The timing events, made when a query first asks for timing.
int make_events(mc_model* m) {
  if (m->ev[0]) return MC_OK;
  for (cudaEvent_t& e : m->ev) MC_CUDA(m, cudaEventCreate(&e));
  return MC_OK;
}

// Timing: the exploration launches a query enqueues back to back (the
// chained checks of a search) are bracketed by one pair of events taken from
// a ring; the window includes the short gaps between the launches.  An event
// between two dependent kernels delays the second (about 2 us on a GB300),
// so a pair per launch would lengthen the query it measures.  A pair's
// elapsed time is added to the statistics when they are read (mc_get_stats)
// or when the pair comes round again.  Every query waits for its stream
// before returning, so a pending pair has completed by then.
int settle_pair(mc_model* m, uint32_t p) {
  float ms = 0.f;
  MC_CUDA(m, cudaEventSynchronize(m->ev[2 * p + 1]));
  MC_CUDA(m, cudaEventElapsedTime(&ms, m->ev[2 * p], m->ev[2 * p + 1]));
  m->stats.explore_ms += ms;
  m->ev_pending &= ~(1ull << p);
  return MC_OK;
}

int settle_timing(mc_model* m) {
  while (m->ev_pending) {
    const int rc_ = settle_pair(m, (uint32_t)__builtin_ctzll(m->ev_pending));
    if (rc_) return rc_;
  }
  return MC_OK;
}

// Records the start of a timed launch on the model's stream; *pair is the
// ring index to pass to time_end after the launch.
int time_begin(mc_model* m, uint32_t* pair) {
  int rc_ = make_events(m);
  if (rc_) return rc_;
  const uint32_t p = m->ev_next;
  m->ev_next = (p + 1) % kTimingRing;
  if ((m->ev_pending >> p) & 1u) {
    rc_ = settle_pair(m, p);
    if (rc_) return rc_;
  }
  MC_CUDA(m, cudaEventRecord(m->ev[2 * p], m->stream));
  *pair = p;
  return MC_OK;
}

int time_end(mc_model* m, uint32_t p) {
  MC_CUDA(m, cudaEventRecord(m->ev[2 * p + 1], m->stream));
  m->ev_pending |= 1ull << p;
  return MC_OK;
}

// Before an exploration launch: opens the timed run unless one is open.
int timed_launch(mc_model* m) {
  if (!m->opt.timing || m->chain_open) return MC_OK;
  const int rc_ = time_begin(m, &m->chain_pair);
  if (rc_) return rc_;
  m->chain_open = true;
  return MC_OK;
}

// Closes the open timed run (fetch_ctrl and sync call it).
int close_chain(mc_model* m) {
  if (!m->chain_open) return MC_OK;
  m->chain_open = false;
  return time_end(m, m->chain_pair);
}

// Makes the model's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  int target = -1;
  explicit DeviceGuard(int dev) : target(dev) {
    if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (target >= 0 && prev >= 0 && prev != target) cudaSetDevice(prev);
  }
};

// Device buffers: through the caller's allocator when one is set, else
// stream-ordered from the library's pool on the model's device.
void* dev_alloc(mc_model* m, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  bool pooled = false;
  if (m->alloc) {
    p = m->alloc(bytes, (void*)m->stream, m->actx);
  } else {
    cudaMemPool_t pool = mc::device_pool(m->device);
    if (pool && cudaMallocFromPoolAsync(&p, bytes, pool, m->stream) == cudaSuccess) {
      pooled = true;
    } else {
      cudaGetLastError();
      p = nullptr;
      if (!pool && cudaMalloc(&p, bytes) != cudaSuccess) {  // no pool on this device: plain allocation
        cudaGetLastError();
        p = nullptr;
      }
    }
  }
  if (p) m->bufs.push_back({p, bytes, pooled});
  return p;
}

void release(mc_model* m) {
  if (!m->bufs.empty()) {
    DeviceGuard g(m->device);
    cudaStreamSynchronize(m->stream);
    for (const Buf& b : m->bufs) {
      if (b.pooled) cudaFreeAsync(b.ptr, m->stream);
      else if (m->dealloc) m->dealloc(b.ptr, b.bytes, (void*)m->stream, m->actx);
      else cudaFree(b.ptr);
    }
    m->bufs.clear();
  }
  if (m->h_block) mc::pinned_free(m->h_block, m->h_block_bytes);
  m->h_block = nullptr;
  m->chain_open = false;
  if (m->ev_pending && settle_timing(m) != MC_OK) m->ev_pending = 0;  // keep the times of launches already run
  m->ev_next = 0;
  for (cudaEvent_t& e : m->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  m->h_ctrl = nullptr;
  m->h_trace = nullptr;
  m->h_scalar = nullptr;
  m->h_params = nullptr;
  m->reserved = false;
}

bool valid_options(const mc_options* o) {
  if (o->load_factor_pct < 10 || o->load_factor_pct > 90) return false;
  if (o->sim_walks == 0) return false;
  if (o->search > MC_SEARCH_BISECT) return false;
  if (o->threads_per_block && (o->threads_per_block < 64 || o->threads_per_block > mc::kThreads ||
                               o->threads_per_block % 32))
    return false;
  if (o->table_log2 && (o->table_log2 < 3 || o->table_log2 > 40)) return false;
  if (o->probe_scheme > MC_PROBE_CAS_CLEAR) return false;
  if (o->no_log_tags > 1) return false;
  if (o->engine > MC_ENGINE_CONFIG) return false;
  if (o->stage_chunk && (o->stage_chunk < 64 || o->stage_chunk > mc::kStageCap || o->stage_chunk % 32)) return false;
  if (o->unit_threads && (o->unit_threads < 64 || o->unit_threads > mc::kCfgMaxThreads || o->unit_threads % 32))
    return false;
  return true;
}

// Lanes per state: the options' lanes_per_state (a power of two from P
// rounded up to 16), else P rounded up to a power of two.
int resolve_tile(mc_model* m) {
  uint32_t t = 1;
  while (t < m->P) t <<= 1;
  const uint32_t want = m->opt.lanes_per_state;
  if (want) {
    if (want < t || want > 16 || (want & (want - 1))) return MC_ERR_INVAL;
    t = want;
  }
  m->tile = t;
  return MC_OK;
}

// the configuration engine takes a model whose per-configuration levels fit
// a block's shared memory and whose log indices fit 32 bits
bool cfg_eligible(const mc_model* m) {
  const uint64_t cap = m->key_words == 1 ? mc::kCfgMaxWidth64 : mc::kCfgMaxWidth128;
  return m->unit_width <= cap && m->unit_log < (1ull << 32) && (uint64_t)m->a * m->b < (1ull << 31);
}

uint32_t resolve_engine(const mc_model* m) {
  if (m->opt.engine == MC_ENGINE_AUTO) return cfg_eligible(m) ? MC_ENGINE_CONFIG : MC_ENGINE_LEVEL;
  return m->opt.engine;
}

// spare top bits per 64-bit word of a key that tag the frontier log (8 to
// 16), or 0: a 128-bit key is stored as two words of 64 - t payload bits
uint32_t log_tag_bits(const mc_model* m) {
  if (m->opt.no_log_tags) return 0;
  const uint32_t spare = m->key_words == 1 ? 64 - m->used_bits : (128 - m->used_bits) / 2;
  return spare >= 8 ? std::min<uint32_t>(spare, 16) : 0;
}

// the probe scheme of the exploration kernel: AUTO follows the key width
// (measured: with 64-bit keys the split insert is fastest on C2 at G=80,
// whose table stays in L2; with 128-bit keys the CAS-first insert without
// clearing is fastest on C3 at G=36 and G=24, whose probes go to DRAM)
int resolve_scheme(uint32_t scheme, uint32_t key_words) {
  if (scheme == MC_PROBE_AUTO) return key_words == 1 ? MC_PROBE_SPLIT : MC_PROBE_CAS_FIRST;
  return (int)scheme;
}

// sizes of the frontier log and the visited set
int size_buffers(mc_model* m) {
  if (resolve_tile(m)) return MC_ERR_INVAL;
  m->engine = resolve_engine(m);
  if (m->engine == MC_ENGINE_CONFIG) {
    if (!cfg_eligible(m)) return MC_ERR_INVAL;
    // a segment of the log per configuration, shared-memory tables per block
    const uint64_t ab = (uint64_t)m->a * m->b;
    m->log_cap = m->unit_log;
    uint32_t w = 32;
    while (w < m->unit_width) w <<= 1;
    m->cfg_wcap = w;
    m->cfg_tsize = 2 * w;  // at most half full
    m->table_slots = m->cfg_tsize;
    // a warp per configuration when its widest level's lanes fit one warp
    // (unless the caller asks for blocks of unit_threads); else enough
    // threads for the widest level's lanes in one round, 64..512
    m->cfg_warp = !m->opt.unit_threads && m->unit_width * m->tile <= mc::kCfgWarpLanes;
    if (m->cfg_warp) {
      m->cfg_threads = (int)mc::kCfgWarpBlockThreads;
    } else if (m->opt.unit_threads) {
      m->cfg_threads = (int)m->opt.unit_threads;
    } else {
      const uint64_t want = m->unit_width * m->tile;
      int t = 64;
      while ((uint64_t)t < want && t < (int)mc::kCfgMaxThreads) t <<= 1;
      m->cfg_threads = t;
    }
    const uint64_t key_bytes = 8ull * m->key_words;
    const uint64_t ctrl_bytes = (mc::kBarBytes + sizeof(Ctrl)) * kSlots + kScalarBytes + 8ull * (m->max_level + 2) * 5;
    uint64_t total = mul_sat(m->log_cap, key_bytes + 4);
    total = add_sat(total, ctrl_bytes + 4ull * (2 * ab + m->P));
    total = add_sat(total, 8 * (ab + 1) + 2 * sizeof(mc::CfgRec) * ab + 4 * ab + 24 * ab + 8 * sizeof(mc::CfgPass));
    total = add_sat(total, 16ull * (m->max_level + 2) * kSlots);  // level widths per result slot
    m->device_bytes = total;
    return MC_OK;
  }
  const uint64_t n_init = 1 + (uint64_t)m->a + (uint64_t)m->a * m->b;
  m->log_cap = m->opt.log_capacity ? std::max(m->opt.log_capacity, n_init) : m->state_bound;
  if (m->log_cap == UINT64_MAX) return MC_ERR_NOMEM;
  // a level's width is counted in the low 32 bits of its barrier word: the
  // winners of a level number at most its width bound and at most the
  // visited set's slots, and at most the log's capacity reach the next level
  if (std::min(m->max_width, m->log_cap) >= (1ull << 31)) return MC_ERR_OVERFLOW;
  const uint64_t per_bucket = m->key_words == 1 ? 4 : 2;
  uint64_t slots;
  if (m->opt.table_log2) {
    slots = 1ull << m->opt.table_log2;
  } else {
    const uint64_t want = mul_sat(std::max<uint64_t>(m->max_width, 1), 100) / m->opt.load_factor_pct + 1;
    slots = 64;
    while (slots < want && slots < (1ull << 40)) slots <<= 1;
    if (slots < want) return MC_ERR_NOMEM;
  }
  if (slots < per_bucket) slots = per_bucket;
  if (m->max_width >= (1ull << 31) && slots > (1ull << 31)) return MC_ERR_OVERFLOW;
  m->table_slots = slots;
  const uint64_t key_bytes = 8ull * m->key_words;
  const uint64_t ctrl_bytes = (mc::kBarBytes + sizeof(Ctrl)) * kSlots + kScalarBytes + 8ull * (m->max_level + 2) * 5;
  uint64_t total = mul_sat(slots, key_bytes);
  total = add_sat(total, mul_sat(m->log_cap, key_bytes + 4));
  total = add_sat(total, ctrl_bytes + 4ull * (2ull * m->a * m->b + m->P));
  m->device_bytes = total;
  return MC_OK;
}

Ctrl* ctrl_at(mc_model* m, int slot) { return m->d_ctrl + slot; }
uint64_t* cfg_levels_at(mc_model* m, int slot) { return m->d_cfg_levels + 2ull * (m->max_level + 2) * slot; }

// The model's constants every kernel takes (device table pointers unset).
void fill_params(const mc_model* m, Params& p) {
  p = Params{};
  p.a = m->a;
  p.b = m->b;
  p.P = m->P;
  p.rule = m->rule;
  p.n_bits = m->n_bits;
  p.ts_shift = m->ts_shift;
  p.wg_shift = m->wg_shift;
  p.ts_mask = (1u << m->ts_bits) - 1;
  p.wg_mask = (1u << m->wg_bits) - 1;
  p.max_level = m->max_level;
  p.n_mask = (1ull << m->n_bits) - 1;
  const uint32_t nf = m->P * m->n_bits;
  p.swar_ok = nf <= 64;
  p.swar_mask = nf >= 64 ? ~0ull : ((1ull << nf) - 1);
  p.swar_mul = 0;
  for (uint32_t t = 0; t < m->P && t * m->n_bits < 64; ++t) p.swar_mul |= 1ull << (t * m->n_bits);
  uint64_t s_max = 0, clk_max = 0;
  for (uint32_t c = 0; c < m->P; ++c) s_max = std::max<uint64_t>(s_max, m->speed[c]);
  for (size_t k = 0; k < m->N.size(); ++k) clk_max = std::max<uint64_t>(clk_max, (uint64_t)m->N[k] * m->cost[k] * s_max);
  p.clk32 = clk_max < (1ull << 32);
}

int reserve(mc_model* m) {
  m->chain_open = false;  // every query starts here; a run left open by a failed query is dropped
  if (m->reserved) return MC_OK;
  int rc = size_buffers(m);
  if (rc) return rc;
  int dev = 0;
  MC_CUDA(m, cudaGetDevice(&dev));
  m->device = dev;
  int sms = 0;
  MC_CUDA(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool cfg = m->engine == MC_ENGINE_CONFIG;
  const uint64_t ab = (uint64_t)m->a * m->b;
  int bps = 0;
  if (!cfg) {
    int coop = 0;
    MC_CUDA(m, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) {
      m->last_err = "device lacks cooperative launch";
      return MC_ERR_CUDA;
    }
    m->threads = m->opt.threads_per_block ? (int)m->opt.threads_per_block : (int)mc::kThreads;
    m->scheme = resolve_scheme(m->opt.probe_scheme, m->key_words);
    if (mc::explore_kernel_occupancy(m->key_words, m->tile, m->rule, m->scheme, m->threads, &bps) || bps < 1) {
      m->last_err = "occupancy query failed";
      cudaGetLastError();
      return MC_ERR_CUDA;
    }
    if (m->opt.blocks_per_sm) bps = std::min<int>(bps, (int)m->opt.blocks_per_sm);
    m->grid = sms * bps;
  } else {
    // a block per configuration (threads from size_buffers), shared memory
    // for two frontiers and two tables; as many blocks as fit, at most one
    // per configuration
    // (warp units use no dynamic shared memory: a launch of warp units only
    // is sized by its threads, a warp per configuration)
    m->cfg_smem = m->cfg_warp ? 0 : mc::cfg_smem_bytes((int)m->key_words, m->cfg_wcap, m->cfg_tsize);
    if (mc::cfg_occupancy((int)m->key_words, m->cfg_threads, m->cfg_smem, &bps) || bps < 1) {
      m->last_err = "occupancy query failed (configuration engine)";
      cudaGetLastError();
      return MC_ERR_CUDA;
    }
    if (m->opt.blocks_per_sm) bps = std::min<int>(bps, (int)m->opt.blocks_per_sm);
    m->cfg_grid_max = sms * bps;
    const uint64_t per_block = m->cfg_warp ? (uint64_t)m->cfg_threads / 32 : 1;
    m->cfg_grid = (int)std::min<uint64_t>((ab + per_block - 1) / per_block, (uint64_t)sms * bps);
  }

  const uint64_t key_bytes = 8ull * m->key_words;
  const size_t np = 2ull * m->a * m->b + m->P;
  m->d_params = (uint32_t*)dev_alloc(m, np * 4);
  if (!cfg) m->d_table = dev_alloc(m, m->table_slots * key_bytes);
  m->d_log_keys = dev_alloc(m, m->log_cap * key_bytes);
  m->d_log_par = (uint32_t*)dev_alloc(m, m->log_cap * 4);
  const size_t L2 = m->max_level + 2;
  const size_t mirror_bytes = sizeof(Ctrl) * kSlots + kScalarBytes + 16 * L2;  // headers, scalars, trace
  const size_t ctrl_bytes = mc::kBarBytes * kSlots + mirror_bytes + 16 * L2 + 8 * L2;
  m->d_ctrl_block = (uint8_t*)dev_alloc(m, ctrl_bytes);
  if (cfg) {
    m->d_seg = (uint64_t*)dev_alloc(m, 8 * (ab + 1));
    m->d_rec = (mc::CfgRec*)dev_alloc(m, 2 * sizeof(mc::CfgRec) * ab);  // two passes at once
    m->d_order = (uint32_t*)dev_alloc(m, 4 * ab);
    m->d_cfg_levels = (uint64_t*)dev_alloc(m, 16 * L2 * kSlots);
    m->d_pair_pass = (mc::CfgPass*)dev_alloc(m, 8 * sizeof(mc::CfgPass));
    m->d_pair_units = (uint64_t*)dev_alloc(m, 8 * 3 * ab);
  }
  if (!m->d_params || (!cfg && !m->d_table) || !m->d_log_keys || !m->d_log_par || !m->d_ctrl_block ||
      (cfg && (!m->d_seg || !m->d_rec || !m->d_order || !m->d_cfg_levels || !m->d_pair_pass ||
               !m->d_pair_units))) {
    release(m);
    return MC_ERR_NOMEM;
  }
  uint8_t* q = m->d_ctrl_block + mc::kBarBytes * kSlots;  // after the barrier lines
  m->d_ctrl = (Ctrl*)q;
  q += sizeof(Ctrl) * kSlots;
  m->d_tini = (uint64_t*)q;
  m->d_tmin = (uint64_t*)q + 1;
  q += kScalarBytes;
  m->d_trace = (uint64_t*)q;
  q += 16 * L2;
  m->d_levels = (uint64_t*)q;
  q += 16 * L2;
  m->d_off = (uint64_t*)q;
  m->mirror_bytes = mirror_bytes;
  // tagged frontier log for 64-bit keys with 8 or more spare top bits: the
  // log starts cleared, so no entry of freed memory carries a tag
  m->tag_bits = cfg ? 0 : log_tag_bits(m);  // the configuration engine's log is read only after its pass
  m->tag = 0;
  if (m->tag_bits) MC_CUDA(m, cudaMemsetAsync(m->d_log_keys, 0, m->log_cap * key_bytes, m->stream));

  // host staging: one pinned block (from the process-wide pool): the mirror
  // of headers, scalars and trace, then the model arrays (and, for the
  // configuration engine, the segment starts and the order)
  const size_t o_params = align_up(mirror_bytes, 64);
  const size_t o_seg = align_up(o_params + np * 4, 8);
  const size_t o_order = o_seg + (cfg ? 8 * (ab + 1) : 0);
  const size_t o_pair = align_up(o_order + (cfg ? 4 * ab : 0), 64);
  const size_t o_pair_units = o_pair + (cfg ? 8 * sizeof(mc::CfgPass) : 0);
  m->h_block_bytes = o_pair_units + (cfg ? 8 * 3 * ab : 0);
  m->h_block = (uint8_t*)mc::pinned_alloc(m->h_block_bytes);
  if (!m->h_block) {
    release(m);
    return MC_ERR_NOMEM;
  }
  m->h_ctrl = (Ctrl*)m->h_block;
  m->h_scalar = (uint64_t*)(m->h_block + sizeof(Ctrl) * kSlots);
  m->h_trace = (uint64_t*)(m->h_block + sizeof(Ctrl) * kSlots + kScalarBytes);
  m->h_params = (uint32_t*)(m->h_block + o_params);
  if (m->opt.timing) {
    const int rc_ = make_events(m);
    if (rc_) return rc_;
  }
  std::copy(m->N.begin(), m->N.end(), m->h_params);
  std::copy(m->cost.begin(), m->cost.end(), m->h_params + (size_t)m->a * m->b);
  std::copy(m->speed.begin(), m->speed.end(), m->h_params + 2ull * m->a * m->b);
  // stream-ordered before every query's kernels; the pinned staging is not
  // written again, so the host need not wait for the copy
  MC_CUDA(m, cudaMemcpyAsync(m->d_params, m->h_params, np * 4, cudaMemcpyHostToDevice, m->stream));
  m->stats.h2d_bytes += np * 4;
  if (cfg) {
    uint64_t* h_seg = (uint64_t*)(m->h_block + o_seg);
    uint32_t* h_order = (uint32_t*)(m->h_block + o_order);
    std::copy(m->seg.begin(), m->seg.end(), h_seg);
    std::copy(m->order.begin(), m->order.end(), h_order);
    MC_CUDA(m, cudaMemcpyAsync(m->d_seg, h_seg, 8 * (ab + 1), cudaMemcpyHostToDevice, m->stream));
    MC_CUDA(m, cudaMemcpyAsync(m->d_order, h_order, 4 * ab, cudaMemcpyHostToDevice, m->stream));
    m->stats.h2d_bytes += 12 * ab + 8;
  }

  Params& p = m->params;
  fill_params(m, p);
  p.N = m->d_params;
  p.cost = m->d_params + (size_t)m->a * m->b;
  p.speed = m->d_params + 2ull * m->a * m->b;
  if (cfg) {
    // the certificate check (T_min - 1) and the counterexample check (T_min)
    // of a single-pass min-time query, launched together
    mc::CfgPass* hp = (mc::CfgPass*)(m->h_block + o_pair);
    for (int k = 0; k < 8; ++k) {  // (prune, early exit) x (certificate, counterexample)
      mc::CfgPass& Q = hp[k];
      std::memset(&Q, 0, sizeof(Q));
      Q.prune = (k >> 2) & 1;
      Q.early_exit = (k >> 1) & 1;
      Q.p = p;
      const int c = k & 1;  // 0: certificate at T_min - 1, 1: counterexample at T_min
      Q.T_src = m->d_tmin;
      Q.T_delta = c == 0 ? -1 : 0;
      Q.group = m->tile;
      Q.log_keys = m->d_log_keys;
      Q.log_par = m->d_log_par;
      Q.seg = m->d_seg;
      Q.levels = cfg_levels_at(m, 1 + c);
      Q.rec = m->d_rec + ab * c;  // the min pass's records are not read after its pass
      Q.ctrl = ctrl_at(m, 1 + c);
      Q.trace = m->d_trace;
      Q.want_witness = c == 1;
    }
    uint64_t* hu = (uint64_t*)(m->h_block + o_pair_units);
    for (uint64_t x = 0; x < ab; ++x) {
      hu[2 * x] = m->order[x];                        // certificate
      hu[2 * x + 1] = (1ull << 32) | m->order[x];     // counterexample
      hu[2 * ab + x] = (1ull << 32) | m->order[x];    // counterexample alone
    }
    MC_CUDA(m, cudaMemcpyAsync(m->d_pair_pass, hp, 8 * sizeof(mc::CfgPass), cudaMemcpyHostToDevice, m->stream));
    MC_CUDA(m, cudaMemcpyAsync(m->d_pair_units, hu, 8 * 3 * ab, cudaMemcpyHostToDevice, m->stream));
    m->stats.h2d_bytes += 8 * sizeof(mc::CfgPass) + 24 * ab;
  }
  m->reserved = true;
  return MC_OK;
}


uint32_t* bar_lines_at(mc_model* m, int slot) {
  return reinterpret_cast<uint32_t*>(m->d_ctrl_block + mc::kBarBytes * slot);
}

// One memset: every slot's barrier lines and the headers of slots 0 ..
// n_headers - 1 (with n_headers == kSlots + 1 also the scalars, T_min = 0).
int clear_ctrl(mc_model* m, int n_headers) {
  const size_t n = mc::kBarBytes * kSlots +
                   (n_headers > kSlots ? sizeof(Ctrl) * kSlots + kScalarBytes : sizeof(Ctrl) * n_headers);
  MC_CUDA(m, cudaMemsetAsync(m->d_ctrl_block, 0, n, m->stream));
  return MC_OK;
}

// One copy: every header, the scalars and the trace buffer into the mirror.
int fetch_ctrl(mc_model* m) {
  {
    const int rc_ = close_chain(m);
    if (rc_) return rc_;
  }
  MC_CUDA(m, cudaMemcpyAsync(m->h_ctrl, m->d_ctrl, m->mirror_bytes, cudaMemcpyDeviceToHost, m->stream));
  m->stats.d2h_bytes += m->mirror_bytes;
  return MC_OK;
}

// Enqueue one exploration pass into `slot`, whose header and barrier lines
// the caller has cleared (clear_ctrl); fetch_ctrl reads the header back.
// With `prev`, the pass takes its threshold from that slot's counterexample
// (see ExploreArgs::prev).

// The configuration engine's pass: the level widths start at zero, the
// header's unit counters and stop word are cleared with it (clear_ctrl).
int enqueue_cfg_pass(mc_model* m, uint64_t T, const uint64_t* T_src, int64_t delta, bool prune,
                     bool early_exit, bool witness, uint64_t* tmin_out, int slot, int prev) {
  mc::CfgLaunch L{};
  mc::CfgPass& Q = L.one;
  Q.p = m->params;
  Q.T = T;
  Q.T_src = T_src;
  Q.T_delta = delta;
  Q.prev = prev >= 0 ? ctrl_at(m, prev) : nullptr;
  Q.prune = prune;
  Q.early_exit = early_exit;
  Q.want_witness = witness;
  Q.group = m->tile;
  Q.log_keys = m->d_log_keys;
  Q.log_par = m->d_log_par;
  Q.seg = m->d_seg;
  Q.levels = cfg_levels_at(m, slot);
  Q.rec = m->d_rec;
  Q.ctrl = ctrl_at(m, slot);
  Q.trace = m->d_trace;
  Q.tmin_out = tmin_out;
  Q.order = m->d_order;
  L.wcap = m->cfg_wcap;
  L.tsize = m->cfg_tsize;
  if (m->cfg_warp) {  // every block serves warp units
    L.n_wunits = (uint64_t)m->a * m->b;
    L.wnext = &Q.ctrl->units_next;
    L.warp_blocks = (uint32_t)m->cfg_grid;
  } else {
    L.n_units = (uint64_t)m->a * m->b;
    L.next = &Q.ctrl->units_next;
  }
  MC_CUDA(m, cudaMemsetAsync(Q.levels, 0, 16ull * (m->max_level + 2), m->stream));
  {
    const int rc_ = timed_launch(m);
    if (rc_) return rc_;
  }
  MC_CUDA(m, mc::launch_cfg((int)m->key_words, m->cfg_grid, m->cfg_threads, m->cfg_smem, L, m->stream));
  m->stats.explore_launches += 1;
  return MC_OK;
}

// Configuration engine, min-time: the certificate check at T_min - 1 (slot
// 1, unless refine is off) and the counterexample check at T_min (slot 2)
// in one launch; T_min is read on the device from the min pass.
int enqueue_cfg_pair(mc_model* m, bool prune, bool early_exit, bool refine) {
  const uint64_t ab = (uint64_t)m->a * m->b;
  MC_CUDA(m, cudaMemsetAsync(cfg_levels_at(m, 1), 0, 2 * 16ull * (m->max_level + 2), m->stream));
  mc::CfgLaunch L{};
  L.passes = m->d_pair_pass + 2 * ((prune ? 2 : 0) + (early_exit ? 1 : 0));  // descriptors per option pair
  const uint64_t* units = refine ? m->d_pair_units : m->d_pair_units + 2 * ab;
  const uint64_t n_units = refine ? 2 * ab : ab;
  uint32_t* next = &ctrl_at(m, 2)->units_next;  // the launch's unit counter (the header starts at zero)
  L.wcap = m->cfg_wcap;
  L.tsize = m->cfg_tsize;
  const uint64_t per_block = m->cfg_warp ? (uint64_t)m->cfg_threads / 32 : 1;
  const int grid = (int)std::min<uint64_t>((uint64_t)m->cfg_grid_max, (n_units + per_block - 1) / per_block);
  if (m->cfg_warp) {
    L.wunits = units;
    L.n_wunits = n_units;
    L.wnext = next;
    L.warp_blocks = (uint32_t)grid;
  } else {
    L.units = units;
    L.n_units = n_units;
    L.next = next;
  }
  {
    const int rc_ = timed_launch(m);
    if (rc_) return rc_;
  }
  MC_CUDA(m, mc::launch_cfg((int)m->key_words, grid, m->cfg_threads, m->cfg_smem, L, m->stream));
  m->stats.explore_launches += 1;
  return MC_OK;
}

int enqueue_pass(mc_model* m, uint64_t T, const uint64_t* T_src, int64_t delta, bool prune,
                 bool early_exit, bool witness, uint64_t* tmin_out, int slot, int prev = -1) {
  if (m->engine == MC_ENGINE_CONFIG)
    return enqueue_cfg_pass(m, T, T_src, delta, prune, early_exit, witness, tmin_out, slot, prev);
  ExploreArgs A{};
  A.p = m->params;
  A.table = m->d_table;
  const uint64_t per_bucket = m->key_words == 1 ? 4 : 2;
  A.bucket_mask = m->table_slots / per_bucket - 1;
  A.table_u64 = m->table_slots * m->key_words;
  A.max_probes = m->opt.max_probes ? m->opt.max_probes
                                   : (uint32_t)std::min<uint64_t>(m->table_slots / per_bucket, 0xFFFFFFFFu);
  A.prune = prune;
  A.early_exit = early_exit;
  A.want_witness = witness;
  A.log_keys = m->d_log_keys;
  A.log_par = m->d_log_par;
  A.log_cap = m->log_cap;
  A.ctrl = ctrl_at(m, slot);
  A.prev = prev >= 0 ? ctrl_at(m, prev) : nullptr;
  A.levels = m->d_levels;
  A.off = m->d_off;
  A.trace = m->d_trace;
  A.T = T;
  A.T_src = T_src;
  A.T_delta = delta;
  A.tmin_out = tmin_out;
  A.barrier_extra = m->opt.debug_barrier_extra;
  A.stage_chunk = m->opt.stage_chunk ? m->opt.stage_chunk : mc::kWarpCap;
  A.bar_lines = bar_lines_at(m, slot);
  A.timeout_ns = m->opt.barrier_timeout_ns ? m->opt.barrier_timeout_ns : 60ull * 1000000000ull;
  if (m->tag_bits) {  // a new tag per pass; the log is cleared when the tags wrap
    if (++m->tag >= (1u << m->tag_bits)) {
      MC_CUDA(m, cudaMemsetAsync(m->d_log_keys, 0, m->log_cap * 8ull * m->key_words, m->stream));
      m->tag = 1;
    }
    A.tag_bits = m->tag_bits;
    A.tag = m->tag;
  }
  {
    const int rc_ = timed_launch(m);
    if (rc_) return rc_;
  }
  MC_CUDA(m, mc::launch_explore(m->key_words, m->tile, m->rule, m->scheme, m->grid, m->threads, A, m->stream));
  m->stats.explore_launches += 1;
  return MC_OK;
}

int sync(mc_model* m) {
  {
    const int rc_ = close_chain(m);
    if (rc_) return rc_;
  }
  MC_CUDA(m, cudaStreamSynchronize(m->stream));
  return MC_OK;
}

int pass_error(mc_model* m, int slot) {
  const Ctrl& c = m->h_ctrl[slot];
  m->last_levels = c.levels;
  m->last_slot = slot;
  m->stats.states += c.states;
  m->stats.device_steps += c.levels;
  return c.err ? (int)c.err : MC_OK;  // the kernel stores the negative MC_ERR_* code
}

uint32_t wg_value(const mc_model* m, uint32_t i) { return m->wg.empty() ? i : m->wg[i]; }
uint32_t ts_value(const mc_model* m, uint32_t j) { return m->ts.empty() ? j : m->ts[j]; }

int make_trace(mc_model* m, const Ctrl& c, mc_trace** out) {
  if (!out) return MC_OK;
  *out = nullptr;
  if (c.trace_len == 0) return MC_OK;
  mc_trace* t = new (std::nothrow) mc_trace;
  if (!t) return MC_ERR_NOMEM;
  t->words = m->key_words;
  t->keys.resize((size_t)c.trace_len * m->key_words);
  for (uint32_t l = 0; l < c.trace_len; ++l) {
    t->keys[(size_t)l * m->key_words] = m->h_trace[2 * l];
    if (m->key_words == 2) t->keys[(size_t)l * 2 + 1] = m->h_trace[2 * l + 1];
  }
  *out = t;
  return MC_OK;
}

void fill_check(const mc_model* m, const Ctrl& c, mc_check_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->holds = c.stop_level == 0;
  out->levels = c.levels;
  out->states = c.states;
  out->key_words = m->key_words;
  if (!out->holds) {
    out->cex_time = mc::pack_time(c.wpack);
    out->cex_wg_index = mc::pack_i(c.wpack);
    out->cex_ts_index = mc::pack_j(c.wpack);
    out->cex_wg = wg_value(m, out->cex_wg_index);
    out->cex_ts = ts_value(m, out->cex_ts_index);
    out->cex_level = c.stop_level;
    out->cex_key[0] = c.wkey_lo;
    out->cex_key[1] = m->key_words == 2 ? c.wkey_hi : 0;
  }
}

int run_simulation(mc_model* m, uint64_t seed, uint32_t walks, uint64_t* dst) {
  MC_CUDA(m, cudaMemsetAsync(dst, 0xFF, 8, m->stream));
  MC_CUDA(m, mc::launch_simulate(m->params, seed, walks, dst, m->stream));
  m->stats.other_launches += 1;
  return MC_OK;
}

#define MC_TRY(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

}  // namespace

namespace mc {

int cfg_model_info(mc_model* m, CfgModelInfo* out) {
  if (!m || !out) return MC_ERR_INVAL;
  fill_params(m, out->p);
  out->group = m->tile;
  out->key_words = m->key_words;
  out->unit_width = m->unit_width;
  out->unit_log = m->unit_log;
  out->seg = m->seg.data();
  out->eligible = cfg_eligible(m);
  return MC_OK;
}

}  // namespace mc

extern "C" {

void mc_options_default(mc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->prune = 1;
  o->early_exit = 1;
  o->search = MC_SEARCH_SINGLE;
  o->refine = 1;
  o->sim_seed = 2305091300ull;
  o->sim_walks = 1;
  o->load_factor_pct = 25;
}

int mc_model_create(const mc_model_desc* d, const mc_options* opt, mc_model** out) {
  if (!d || !out) return MC_ERR_INVAL;
  *out = nullptr;
  if (d->n_wg == 0 || d->n_ts == 0 || d->P == 0 || d->P > mc::kMaxP) return MC_ERR_INVAL;
  if (!d->n_workgroups || !d->cost) return MC_ERR_INVAL;
  if (d->rule > MC_GREEDY) return MC_ERR_INVAL;
  if (d->key_bits != 0 && d->key_bits != 64 && d->key_bits != 128) return MC_ERR_INVAL;
  if (d->n_wg > 4095 || d->n_ts > 4095) return MC_ERR_OVERFLOW;
  mc_options o;
  if (opt) o = *opt;
  else mc_options_default(&o);
  if (!valid_options(&o)) return MC_ERR_INVAL;

  mc_model* m = new (std::nothrow) mc_model;
  if (!m) return MC_ERR_NOMEM;
  m->a = d->n_wg;
  m->b = d->n_ts;
  m->P = d->P;
  m->rule = d->rule;
  m->opt = o;
  const size_t ab = (size_t)m->a * m->b;
  m->N.assign(d->n_workgroups, d->n_workgroups + ab);
  m->cost.assign(d->cost, d->cost + ab);
  if (d->speed) m->speed.assign(d->speed, d->speed + m->P);
  else m->speed.assign(m->P, 1);
  if (d->wg_values) m->wg.assign(d->wg_values, d->wg_values + m->a);
  if (d->ts_values) m->ts.assign(d->ts_values, d->ts_values + m->b);
  uint32_t n_max = 0, s_max = 0;
  for (size_t k = 0; k < ab; ++k) {
    if (m->N[k] == 0 || m->cost[k] == 0) {
      delete m;
      return MC_ERR_INVAL;
    }
    n_max = std::max(n_max, m->N[k]);
  }
  for (uint32_t s : m->speed) {
    if (s == 0) {
      delete m;
      return MC_ERR_INVAL;
    }
    s_max = std::max(s_max, s);
  }
  // every clock stays below 2^40 (packed (time, i, j) reductions)
  for (size_t k = 0; k < ab; ++k) {
    if ((unsigned __int128)m->N[k] * m->cost[k] * s_max >= ((unsigned __int128)1 << 40)) {
      delete m;
      return MC_ERR_OVERFLOW;
    }
  }
  // key layout: [i+1][j+1][n_0]...[n_{P-1}] from the top of the used bits
  m->n_bits = bits_for(n_max);
  m->ts_bits = bits_for(m->b);
  m->wg_bits = bits_for(m->a);
  m->used_bits = m->wg_bits + m->ts_bits + m->P * m->n_bits;
  m->ts_shift = m->P * m->n_bits;
  m->wg_shift = m->ts_shift + m->ts_bits;
  if (d->key_bits == 0) m->key_bits = m->used_bits <= 64 ? 64 : 128;
  else m->key_bits = d->key_bits;
  if (m->used_bits > m->key_bits) {
    delete m;
    return MC_ERR_OVERFLOW;
  }
  m->key_words = m->key_bits / 64;
  m->max_level = n_max + 2;
  if (resolve_tile(m)) {
    delete m;
    return MC_ERR_INVAL;
  }

  // closed-form bounds on the widths of the levels (sizing only):
  //   FREE:   C(k+P-1, P-1) states of sum(n) = k per configuration;
  //   GREEDY: at most C(P, floor(P/2)) per configuration and level, since
  //           after k dispatches only the units tied at the next start time
  //           can differ.
  const uint64_t greedy_cap = binom_sat(m->P, m->P / 2);
  // configurations with N_ij >= k, for every k (suffix sums of a histogram)
  std::vector<uint64_t> at_least(n_max + 2, 0);
  for (size_t k = 0; k < ab; ++k) at_least[m->N[k]] += 1;
  for (int64_t k = (int64_t)n_max - 1; k >= 0; --k) at_least[k] += at_least[k + 1];
  uint64_t total = add_sat(1 + (uint64_t)m->a, ab);
  uint64_t widest = 0;
  uint64_t per_free = 1;  // C(k+P-1, P-1), updated incrementally (saturating)
  for (uint32_t k = 1; k <= n_max; ++k) {
    if (per_free != UINT64_MAX) {
      const unsigned __int128 nx = (unsigned __int128)per_free * (k + m->P - 1) / k;
      per_free = nx > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)nx;
    }
    uint64_t per = per_free;
    if (m->rule == MC_GREEDY) per = std::min(per, greedy_cap);
    const uint64_t w = mul_sat(per, at_least[k]);
    widest = std::max(widest, w);
    total = add_sat(total, w);
  }
  m->max_width = widest;
  m->state_bound = total;
  // the configuration engine's bounds: the widest level of one
  // configuration is w(n_max) (w grows with k), and configuration c's
  // states number at most sum_{k <= N_c} w(k); its frontier-log segment
  // has that size.  Configurations are taken deepest first.
  {
    std::vector<uint64_t> upto(n_max + 1);  // sum_{k' <= k} w(k')
    uint64_t pf = 1, acc = 0;
    for (uint32_t k = 0; k <= n_max; ++k) {
      if (k > 0 && pf != UINT64_MAX) {
        const unsigned __int128 nx = (unsigned __int128)pf * (k + m->P - 1) / k;
        pf = nx > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)nx;
      }
      const uint64_t w = m->rule == MC_GREEDY ? std::min(pf, greedy_cap) : pf;
      acc = add_sat(acc, w);
      upto[k] = acc;
      if (k == n_max) m->unit_width = w;
    }
    m->seg.assign(ab + 1, 0);
    for (size_t k = 0; k < ab; ++k) m->seg[k + 1] = add_sat(m->seg[k], upto[m->N[k]]);
    m->unit_log = m->seg[ab];
    m->order.resize(ab);
    for (size_t k = 0; k < ab; ++k) m->order[k] = (uint32_t)k;
    std::stable_sort(m->order.begin(), m->order.end(),
                     [m](uint32_t x, uint32_t y) { return m->N[x] > m->N[y]; });
  }
  *out = m;
  return MC_OK;
}

void mc_model_destroy(mc_model* m) {
  if (!m) return;
  release(m);
  delete m;
}

int mc_set_options(mc_model* m, const mc_options* o) {
  if (!m || !o || !valid_options(o)) return MC_ERR_INVAL;
  mc_options keep = m->opt;
  m->opt = *o;
  if (m->reserved) {  // buffer sizes are fixed once allocated
    m->opt.load_factor_pct = keep.load_factor_pct;
    m->opt.table_log2 = keep.table_log2;
    m->opt.log_capacity = keep.log_capacity;
    m->opt.threads_per_block = keep.threads_per_block;
    m->opt.blocks_per_sm = keep.blocks_per_sm;
    m->opt.probe_scheme = keep.probe_scheme;  // the grid was sized for its kernel
    m->opt.no_log_tags = keep.no_log_tags;    // the log was cleared (or not) for it
    m->opt.engine = keep.engine;              // the buffers were made for one engine
    m->opt.unit_threads = keep.unit_threads;
    m->opt.lanes_per_state = keep.lanes_per_state;  // the grid was sized for its tile
  }
  return MC_OK;
}

int mc_set_stream(mc_model* m, void* stream) {
  if (!m) return MC_ERR_INVAL;
  m->stream = (cudaStream_t)stream;
  return MC_OK;
}

int mc_set_allocator(mc_model* m, mc_alloc_fn alloc, mc_free_fn free_fn, void* ctx) {
  if (!m || !alloc || !free_fn || m->reserved) return MC_ERR_INVAL;
  m->alloc = alloc;
  m->dealloc = free_fn;
  m->actx = ctx;
  return MC_OK;
}

int mc_reserve(mc_model* m) {
  if (!m) return MC_ERR_INVAL;
  return reserve(m);
}

int mc_model_layout(const mc_model* m, mc_layout* out) {
  if (!m || !out) return MC_ERR_INVAL;
  std::memset(out, 0, sizeof(*out));
  out->key_bits = m->key_bits;
  out->key_words = m->key_words;
  out->used_bits = m->used_bits;
  out->P = m->P;
  out->n_bits = m->n_bits;
  out->ts_bits = m->ts_bits;
  out->wg_bits = m->wg_bits;
  out->ts_shift = m->ts_shift;
  out->wg_shift = m->wg_shift;
  out->max_level = m->max_level;
  for (uint32_t c = 0; c < m->P; ++c) out->n_shift[c] = (m->P - 1 - c) * m->n_bits;
  out->max_width = m->max_width;
  out->state_bound = m->state_bound;
  mc_model* mm = const_cast<mc_model*>(m);
  if (!m->reserved) size_buffers(mm);
  out->table_slots = m->table_slots;
  out->log_capacity = m->log_cap;
  out->device_bytes = m->device_bytes;
  out->probe_scheme = (uint32_t)resolve_scheme(m->opt.probe_scheme, m->key_words);
  out->engine = m->engine;
  out->log_tag_bits = m->engine == MC_ENGINE_CONFIG ? 0 : log_tag_bits(m);
  out->unit_width = m->unit_width;
  // threads that explore one configuration: 32 for warp units
  out->unit_threads = m->engine != MC_ENGINE_CONFIG ? 0 : m->cfg_warp ? 32u : (uint32_t)m->cfg_threads;
  return MC_OK;
}

int mc_check(mc_model* m, uint64_t T, mc_check_result* out, mc_trace** cex) {
  if (!m || !out) return MC_ERR_INVAL;
  if (cex) *cex = nullptr;
  DeviceGuard g(m->device);
  MC_TRY(reserve(m));
  MC_TRY(clear_ctrl(m, 1));
  MC_TRY(enqueue_pass(m, T, nullptr, 0, m->opt.prune, m->opt.early_exit, true, nullptr, 0));
  MC_TRY(fetch_ctrl(m));
  MC_TRY(sync(m));
  MC_TRY(pass_error(m, 0));
  fill_check(m, m->h_ctrl[0], out);
  if (!out->holds) MC_TRY(make_trace(m, m->h_ctrl[0], cex));
  return MC_OK;
}

int mc_count_states(mc_model* m, uint64_t* out) {
  if (!m || !out) return MC_ERR_INVAL;
  DeviceGuard g(m->device);
  MC_TRY(reserve(m));
  MC_TRY(clear_ctrl(m, 1));
  MC_TRY(enqueue_pass(m, UINT64_MAX, nullptr, 0, false, false, false, nullptr, 0));
  MC_TRY(fetch_ctrl(m));
  MC_TRY(sync(m));
  MC_TRY(pass_error(m, 0));
  *out = m->h_ctrl[0].states;
  return MC_OK;
}

int mc_simulate(mc_model* m, uint64_t seed, uint32_t walks, uint64_t* t_ini) {
  if (!m || !t_ini || walks == 0) return MC_ERR_INVAL;
  DeviceGuard g(m->device);
  MC_TRY(reserve(m));
  MC_TRY(run_simulation(m, seed, walks, m->d_tini));
  MC_CUDA(m, cudaMemcpyAsync(m->h_scalar, m->d_tini, 8, cudaMemcpyDeviceToHost, m->stream));
  m->stats.d2h_bytes += 8;
  MC_TRY(sync(m));
  *t_ini = m->h_scalar[0];
  return MC_OK;
}

int mc_min_time(mc_model* m, mc_min_result* out, mc_trace** trace) {
  if (!m || !out) return MC_ERR_INVAL;
  if (trace) *trace = nullptr;
  std::memset(out, 0, sizeof(*out));
  DeviceGuard g(m->device);
  MC_TRY(reserve(m));
  const bool prune = m->opt.prune, ee = m->opt.early_exit;
  // one memset for every slot and the scalars (T_min = 0), then T_ini
  MC_TRY(clear_ctrl(m, kSlots + 1));
  MC_TRY(run_simulation(m, m->opt.sim_seed, m->opt.sim_walks, m->d_tini));
  Ctrl c{};  // header of the check whose counterexample is the answer

  if (m->opt.search == MC_SEARCH_SINGLE) {
    // one pass with a device-side min-reduction over terminal times, then
    // the certificate checks at T_min - 1 (must hold) and T_min (fails);
    // thresholds stay on the device, so the host waits once
    MC_TRY(enqueue_pass(m, UINT64_MAX, prune ? m->d_tini : nullptr, 0, prune, false, false,
                        m->d_tmin, 0));
    int slot = 1;
    if (m->engine == MC_ENGINE_CONFIG) {
      // both checks in one launch: the certificate in slot 1 (with refine),
      // the counterexample in slot 2
      MC_TRY(enqueue_cfg_pair(m, prune, ee, m->opt.refine != 0));
      slot = 2;
    } else {
      if (m->opt.refine) MC_TRY(enqueue_pass(m, 0, m->d_tmin, -1, prune, ee, false, nullptr, slot++));
      MC_TRY(enqueue_pass(m, 0, m->d_tmin, 0, prune, ee, true, nullptr, slot));
    }
    const int final_slot = slot;
    MC_TRY(fetch_ctrl(m));
    MC_TRY(sync(m));
    out->t_ini = m->h_scalar[0];
    const int cert_slot = m->opt.refine ? 1 : -1;
    for (int s = 0; s <= final_slot; ++s) {
      if (s != 0 && s != cert_slot && s != final_slot) continue;  // no certificate check
      MC_TRY(pass_error(m, s));
      out->states += m->h_ctrl[s].states;
      out->checks += 1;
    }
    if (m->h_ctrl[0].best_pack == kNone) {
      m->last_err = "no terminal below T_ini";
      return MC_ERR_CUDA;
    }
    if ((m->opt.refine && m->h_ctrl[cert_slot].stop_level != 0) || m->h_ctrl[final_slot].stop_level == 0) {
      m->last_err = "certificate checks disagree with the minimum";
      return MC_ERR_CUDA;
    }
    c = m->h_ctrl[final_slot];
  } else if (m->opt.search == MC_SEARCH_LOWER) {
    // Step 3: check at T_ini, then one below each counterexample, until the
    // property holds.  The checks are chained on the device (each takes its
    // threshold from its predecessor's counterexample, and one after a check
    // that held does not run) in groups of three in slots 0..2; the host
    // waits once per group.  A group only follows one whose three checks all
    // failed: the last of them is copied into slot 3 and is the next group's
    // predecessor (and the answer if that group's first check holds).
    constexpr int kGroup = 3;
    static_assert(kGroup < kSlots, "slot kGroup keeps the predecessor");
    int last = -1;
    bool held = false;
    for (int group = 0; !held; ++group) {
      if (group > 0) {
        MC_CUDA(m, cudaMemcpyAsync(ctrl_at(m, kGroup), ctrl_at(m, kGroup - 1), sizeof(Ctrl),
                                   cudaMemcpyDeviceToDevice, m->stream));
        MC_TRY(clear_ctrl(m, kGroup));
        last = kGroup;
      }
      for (int k = 0; k < kGroup; ++k) {
        if (group == 0 && k == 0) MC_TRY(enqueue_pass(m, 0, m->d_tini, 0, prune, ee, true, nullptr, 0));
        else MC_TRY(enqueue_pass(m, 0, nullptr, 0, prune, ee, true, nullptr, k, k == 0 ? kGroup : k - 1));
      }
      // the trace buffer holds the last failing check's trace (a check that
      // holds or does not run leaves it alone); the fetch reads it too
      MC_TRY(fetch_ctrl(m));
      MC_TRY(sync(m));
      for (int k = 0; k < kGroup && !held; ++k) {
        if (m->h_ctrl[k].skipped) break;
        MC_TRY(pass_error(m, k));
        out->states += m->h_ctrl[k].states;
        out->checks += 1;
        if (m->h_ctrl[k].stop_level == 0) held = true;
        else last = k;
      }
    }
    out->t_ini = m->h_scalar[0];
    if (last < 0) {
      m->last_err = "search ended without a counterexample";
      return MC_ERR_CUDA;
    }
    c = m->h_ctrl[last];
  } else {
    MC_TRY(fetch_ctrl(m));
    MC_TRY(sync(m));
    out->t_ini = m->h_scalar[0];
    // run one check in slot 0 (the host keeps the last failing header)
    auto check = [&](uint64_t T) -> int {
      MC_TRY(clear_ctrl(m, 1));
      MC_TRY(enqueue_pass(m, T, nullptr, 0, prune, ee, true, nullptr, 0));
      MC_TRY(fetch_ctrl(m));
      MC_TRY(sync(m));
      MC_TRY(pass_error(m, 0));
      out->states += m->h_ctrl[0].states;
      out->checks += 1;
      return MC_OK;
    };
    bool have = false;  // c holds a failing check's header
    {
      // bisection (Fig. 1) between 0 (no terminal has time 0) and T_ini;
      // a counterexample at mid lowers hi to its own time
      uint64_t lo = 0, hi = out->t_ini;
      while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        MC_TRY(check(mid));
        if (m->h_ctrl[0].stop_level == 0) {
          lo = mid;
        } else {
          hi = mc::pack_time(m->h_ctrl[0].wpack);
          c = m->h_ctrl[0];
          have = true;
        }
      }
      if (!have || mc::pack_time(c.wpack) != hi) {
        MC_TRY(check(hi));
        c = m->h_ctrl[0];
        have = true;
      }
    }
    // the trace buffer (read by every fetch) holds the last failing check's trace
    if (!have || c.stop_level == 0) {
      m->last_err = "search ended without a counterexample";
      return MC_ERR_CUDA;
    }
  }
  out->t_min = mc::pack_time(c.wpack);
  out->wg_index = mc::pack_i(c.wpack);
  out->ts_index = mc::pack_j(c.wpack);
  out->wg = wg_value(m, out->wg_index);
  out->ts = ts_value(m, out->ts_index);
  out->level = c.stop_level;
  out->witness_key[0] = c.wkey_lo;
  out->witness_key[1] = m->key_words == 2 ? c.wkey_hi : 0;
  MC_TRY(make_trace(m, c, trace));
  return MC_OK;
}

int mc_swarm(mc_model* m, uint64_t seed, uint32_t walks_per_round, uint32_t max_rounds,
             mc_swarm_result* out, mc_trace** trace) {
  if (!m || !out || walks_per_round == 0 || walks_per_round > (1u << 24) || max_rounds == 0)
    return MC_ERR_INVAL;
  if (trace) *trace = nullptr;
  std::memset(out, 0, sizeof(*out));
  DeviceGuard g(m->device);
  MC_TRY(reserve(m));
  const auto t0 = std::chrono::steady_clock::now();
  auto ms_since = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  int sms = 0;
  MC_CUDA(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  unsigned long long* best = reinterpret_cast<unsigned long long*>(m->d_tmin);
  uint64_t bound = UINT64_MAX;
  for (uint32_t r = 0; r < max_rounds; ++r) {
    MC_CUDA(m, cudaMemsetAsync(best, 0xFF, 8, m->stream));
    MC_CUDA(m, mc::launch_swarm(m->params, seed, (uint64_t)r * walks_per_round, walks_per_round, bound,
                                best, sms * 8, m->stream));
    m->stats.other_launches += 1;
    MC_CUDA(m, cudaMemcpyAsync(m->h_scalar, best, 8, cudaMemcpyDeviceToHost, m->stream));
    m->stats.d2h_bytes += 8;
    MC_TRY(sync(m));
    out->rounds = r + 1;
    out->walks += walks_per_round;
    const uint64_t v = m->h_scalar[0];
    if (v == UINT64_MAX) break;  // nothing at or below the bound: stop
    out->best_time = v >> 24;
    out->best_walk = (uint64_t)r * walks_per_round + (v & 0xFFFFFFu);
    if (r == 0) {
      out->first_time = out->best_time;
      out->first_trail_ms = ms_since();
    }
    if (out->best_time == 0) break;
    bound = out->best_time - 1;
  }
  if (out->first_time == 0) {  // cannot happen: every run terminates
    m->last_err = "swarm found no terminal";
    return MC_ERR_CUDA;
  }
  // replay the best run: its states give the configuration and the trace
  uint32_t* d_len = reinterpret_cast<uint32_t*>(m->d_tini);
  MC_CUDA(m, mc::launch_replay_walk(m->params, seed, out->best_walk, (int)m->key_words, m->d_trace,
                                    d_len, m->stream));
  m->stats.other_launches += 1;
  const size_t L2 = m->max_level + 2;
  MC_CUDA(m, cudaMemcpyAsync(m->h_scalar, d_len, 4, cudaMemcpyDeviceToHost, m->stream));
  MC_CUDA(m, cudaMemcpyAsync(m->h_trace, m->d_trace, 16 * L2, cudaMemcpyDeviceToHost, m->stream));
  m->stats.d2h_bytes += 4 + 16 * L2;
  MC_TRY(sync(m));
  out->total_ms = ms_since();
  const uint32_t len = (uint32_t)(m->h_scalar[0] & 0xFFFFFFFFu);
  const uint64_t k2lo = m->h_trace[4], k2hi = m->h_trace[5];  // state 2: (i+1, j+1, 0)
  const unsigned __int128 k2 = ((unsigned __int128)k2hi << 64) | k2lo;
  out->wg_index = (uint32_t)((k2 >> m->wg_shift) & ((1u << m->wg_bits) - 1)) - 1;
  out->ts_index = (uint32_t)((k2 >> m->ts_shift) & ((1u << m->ts_bits) - 1)) - 1;
  out->wg = wg_value(m, out->wg_index);
  out->ts = ts_value(m, out->ts_index);
  out->key_words = m->key_words;
  if (trace) {
    mc::Ctrl c{};
    c.trace_len = len;
    MC_TRY(make_trace(m, c, trace));
  }
  return MC_OK;
}

int mc_last_widths(mc_model* m, uint64_t* out, uint32_t cap, uint32_t* n) {
  if (!m || !n || (!out && cap)) return MC_ERR_INVAL;
  *n = m->reserved ? m->last_levels : 0;
  if (!m->reserved || cap == 0) return MC_OK;
  DeviceGuard g(m->device);
  const uint32_t k = std::min(cap, *n);
  std::vector<uint64_t> rec(2ull * k);
  const uint64_t* src = m->engine == MC_ENGINE_CONFIG ? cfg_levels_at(m, m->last_slot) : m->d_levels;
  MC_CUDA(m, cudaMemcpyAsync(rec.data(), src, 16ull * k, cudaMemcpyDeviceToHost, m->stream));
  m->stats.d2h_bytes += 16ull * k;
  MC_TRY(sync(m));
  // the low 32 bits of a level's word are its width (the kernel's level
  // barrier counts arrivals in the high bits of the same word)
  for (uint32_t l = 0; l < k; ++l) out[l] = rec[2 * l] & 0xFFFFFFFFull;
  return MC_OK;
}

int mc_get_stats(const mc_model* m, mc_stats* out) {
  if (!m || !out) return MC_ERR_INVAL;
  // the times of timed launches are added here (a cache the call may fill)
  mc_model* w = const_cast<mc_model*>(m);
  if (w->ev_pending) {
    DeviceGuard g(w->device);
    const int rc = settle_timing(w);
    if (rc) return rc;
  }
  *out = m->stats;
  return MC_OK;
}

int mc_reset_stats(mc_model* m) {
  if (!m) return MC_ERR_INVAL;
  m->ev_pending = 0;  // launches before the reset do not count
  m->stats = mc_stats{};
  return MC_OK;
}

int mc_trace_length(const mc_trace* t) {
  return t ? (int)(t->keys.size() / t->words) : 0;
}

uint32_t mc_trace_key_words(const mc_trace* t) { return t ? t->words : 0; }

const uint64_t* mc_trace_states(const mc_trace* t) { return t && !t->keys.empty() ? t->keys.data() : nullptr; }

void mc_trace_free(mc_trace* t) { delete t; }

int mc_release_cached(void) {
  mc::release_cached();
  return MC_OK;
}

int mc_set_pool_retention(uint64_t bytes) { return mc::set_pool_retention(bytes); }

const char* mc_strerror(int code) {
  switch (code) {
    case MC_OK: return "ok";
    case MC_ERR_INVAL: return "invalid argument";
    case MC_ERR_NOMEM: return "out of memory";
    case MC_ERR_TABLE_FULL: return "visited set full (probe limit reached)";
    case MC_ERR_FRONTIER: return "frontier log capacity exceeded";
    case MC_ERR_TIMEOUT: return "device-side wait timed out";
    case MC_ERR_CUDA: return "CUDA error";
    case MC_ERR_OVERFLOW: return "overflow (key width, clock range or level width)";
  }
  return "unknown error";
}

const char* mc_last_error(const mc_model* m) { return m ? m->last_err.c_str() : ""; }

}  // extern "C"
