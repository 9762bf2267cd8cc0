// mc_check_noalloc: the property check of mc_check for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- inside a host framework that owns the whole device memory
// budget and hands out no allocator, in a latency-critical serving path
// where an allocation could block on the driver or fail under
// fragmentation, or in a plugin that may only launch work on a stream it is
// given.  Such a caller passes its inputs (the model description, in host
// memory) and its output (a result struct in host memory) and gets the same
// answer as mc_check, with every scratch buffer of the exploration -- the
// visited set, the frontier log, the control block and the device copy of
// the cost tables -- carved out of one fixed array that lives in the
// library's device image.
//
// The array is a file-scope static __device__ object of
// MC_NOALLOC_SCRATCH_BYTES bytes; every GPU that loads the library holds it
// until the process exits.  In host code its name is only a host-side
// stand-in, so its device address is looked up with cudaGetSymbolAddress,
// once per device, with that device current, the first time the entry point
// runs on that device; that first call should therefore come before any
// stream capture.  Models whose buffers do not fit are rejected with
// MC_ERR_NOMEM.  All calls share the array and it keeps the previous call's
// contents: the control block and barrier counters are cleared on every
// call, the kernel itself clears the visited set and initialises the level
// records, and every other byte is written before it is read.  Calls that
// overlap on the GPU (on different streams, or from different threads)
// race on the array.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mc.h"
#include "mc_internal.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[MC_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

uint32_t nbits(uint64_t x) {
  uint32_t b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

uint64_t choose_sat(uint64_t n, uint64_t k) {
  if (k > n) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (uint64_t i = 0; i < k; ++i) {
    r = r * (n - i) / (i + 1);
    if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
  }
  return (uint64_t)r;
}

uint64_t sat_add(uint64_t a, uint64_t b) { return a > UINT64_MAX - b ? UINT64_MAX : a + b; }
uint64_t sat_mul(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  return a > UINT64_MAX / b ? UINT64_MAX : a * b;
}

// Device address of the scratch array on the current device (set up once).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return MC_OK;
}

}  // namespace

extern "C" int mc_check_noalloc(const mc_model_desc* d, uint64_t T, uint32_t prune,
                                uint32_t early_exit, void* stream_handle, mc_check_result* out) {
  if (!d || !out) return MC_ERR_INVAL;
  if (d->n_wg == 0 || d->n_ts == 0 || d->P == 0 || d->P > mc::kMaxP) return MC_ERR_INVAL;
  if (!d->n_workgroups || !d->cost || d->rule > MC_GREEDY) return MC_ERR_INVAL;
  if (d->key_bits != 0 && d->key_bits != 64 && d->key_bits != 128) return MC_ERR_INVAL;
  if (d->n_wg > 4095 || d->n_ts > 4095) return MC_ERR_OVERFLOW;
  const uint32_t a = d->n_wg, b = d->n_ts, P = d->P;
  const uint64_t ab = (uint64_t)a * b;
  uint32_t ones[mc::kMaxP];
  for (uint32_t c = 0; c < P; ++c) ones[c] = 1;
  const uint32_t* speed = d->speed ? d->speed : ones;
  uint32_t n_max = 0, s_max = 0;
  for (uint64_t k = 0; k < ab; ++k) {
    if (d->n_workgroups[k] == 0 || d->cost[k] == 0) return MC_ERR_INVAL;
    if (d->n_workgroups[k] > n_max) n_max = d->n_workgroups[k];
  }
  for (uint32_t c = 0; c < P; ++c) {
    if (speed[c] == 0) return MC_ERR_INVAL;
    if (speed[c] > s_max) s_max = speed[c];
  }
  for (uint64_t k = 0; k < ab; ++k)
    if ((unsigned __int128)d->n_workgroups[k] * d->cost[k] * s_max >= ((unsigned __int128)1 << 40))
      return MC_ERR_OVERFLOW;

  // key layout (as mc_model_create)
  const uint32_t n_bits = nbits(n_max), ts_bits = nbits(b), wg_bits = nbits(a);
  const uint32_t used = wg_bits + ts_bits + P * n_bits;
  const uint32_t key_bits = d->key_bits ? d->key_bits : (used <= 64 ? 64 : 128);
  if (used > key_bits) return MC_ERR_OVERFLOW;
  const uint32_t key_words = key_bits / 64;
  const uint32_t max_level = n_max + 2;
  uint32_t tile = 1;
  while (tile < P) tile <<= 1;

  // Every configuration has at least one state per level 2 .. N_ij + 2
  // under either rule, so the frontier log holds at least 1 + a +
  // sum(N_ij + 1) states: a model whose log cannot fit is refused here, in
  // one pass over the table, before the bounds below (which cost time
  // proportional to max N) are computed.
  const uint64_t key_bytes = 8ull * key_words;
  const uint64_t params_bytes = align256(4 * (2 * ab + P));
  {
    uint64_t floor_states = 1 + (uint64_t)a;
    for (uint64_t k = 0; k < ab; ++k) floor_states += (uint64_t)d->n_workgroups[k] + 1;
    if (sat_add(params_bytes, sat_mul(floor_states, key_bytes + 4)) > MC_NOALLOC_SCRATCH_BYTES)
      return MC_ERR_NOMEM;
  }

  // closed-form bounds (as mc_model_create) and the scratch they need: the
  // configurations with N_ij >= k for every k from a suffix histogram (max N
  // is small here: the check above bounds it by the array's size)
  const uint64_t greedy_cap = choose_sat(P, P / 2);
  std::vector<uint64_t> at_least((size_t)n_max + 2, 0);
  for (uint64_t c = 0; c < ab; ++c) at_least[d->n_workgroups[c]] += 1;
  for (int64_t k = (int64_t)n_max - 1; k >= 0; --k) at_least[k] += at_least[k + 1];
  uint64_t total = sat_add(1 + (uint64_t)a, ab), widest = 0;
  uint64_t per_free = 1;  // C(k+P-1, P-1), updated incrementally (saturating)
  for (uint32_t k = 1; k <= n_max; ++k) {
    if (per_free != UINT64_MAX) {
      const unsigned __int128 nx = (unsigned __int128)per_free * (k + P - 1) / k;
      per_free = nx > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)nx;
    }
    uint64_t per = per_free;
    if (d->rule == MC_GREEDY && greedy_cap < per) per = greedy_cap;
    const uint64_t w = sat_mul(per, at_least[k]);
    if (w > widest) widest = w;
    total = sat_add(total, w);
    if (sat_mul(total, key_bytes + 4) > MC_NOALLOC_SCRATCH_BYTES) return MC_ERR_NOMEM;
  }
  const uint64_t per_bucket = key_words == 1 ? 4 : 2;
  const uint64_t want = sat_mul(widest ? widest : 1, 4) + 1;  // load factor 25%
  uint64_t slots = 64;
  while (slots < want && slots < (1ull << 40)) slots <<= 1;
  const uint64_t L2 = max_level + 2;
  const uint64_t ctrl_bytes = align256(256 + mc::kBarBytes + 16 * L2 + 8 * L2 + 16 * L2 + 64);
  const uint64_t table_bytes = align256(sat_mul(slots, key_bytes));
  const uint64_t keys_bytes = align256(sat_mul(total, key_bytes));
  const uint64_t par_bytes = align256(sat_mul(total, 4));
  uint64_t need = sat_add(params_bytes, ctrl_bytes);
  need = sat_add(need, table_bytes);
  need = sat_add(need, keys_bytes);
  need = sat_add(need, par_bytes);
  if (total == UINT64_MAX || need > MC_NOALLOC_SCRATCH_BYTES) return MC_ERR_NOMEM;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  int sms = 0, coop = 0, bps = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      mc::explore_kernel_occupancy(key_words, tile, d->rule, key_words == 1 ? MC_PROBE_SPLIT : MC_PROBE_CAS_FIRST,
                                   mc::kThreads, &bps) || bps < 1) {
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  cudaStream_t stream = (cudaStream_t)stream_handle;

  // carve the scratch array
  uint32_t* d_params = reinterpret_cast<uint32_t*>(base);
  unsigned char* q = base + params_bytes;
  mc::Ctrl* d_ctrl = reinterpret_cast<mc::Ctrl*>(q);
  uint32_t* d_bar = reinterpret_cast<uint32_t*>(q + 256);
  uint64_t* d_levels = reinterpret_cast<uint64_t*>(q + 256 + mc::kBarBytes);
  uint64_t* d_off = d_levels + 2 * L2;
  uint64_t* d_trace = d_off + L2;
  q += ctrl_bytes;
  void* d_table = q;
  q += table_bytes;
  void* d_keys = q;
  q += keys_bytes;
  uint32_t* d_par = reinterpret_cast<uint32_t*>(q);

  // inputs: the model tables; the control block and barrier start at zero
  if (cudaMemcpyAsync(d_params, d->n_workgroups, 4 * ab, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(d_params + ab, d->cost, 4 * ab, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(d_params + 2 * ab, speed, 4ull * P, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemsetAsync(d_ctrl, 0, 256 + mc::kBarBytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_CUDA;
  }

  mc::ExploreArgs A;
  std::memset(&A, 0, sizeof(A));
  mc::Params& p = A.p;
  p.a = a;
  p.b = b;
  p.P = P;
  p.rule = d->rule;
  p.n_bits = n_bits;
  p.ts_shift = P * n_bits;
  p.wg_shift = P * n_bits + ts_bits;
  p.ts_mask = (1u << ts_bits) - 1;
  p.wg_mask = (1u << wg_bits) - 1;
  p.max_level = max_level;
  p.n_mask = (1ull << n_bits) - 1;
  const uint32_t nf = P * n_bits;
  p.swar_ok = nf <= 64;
  p.swar_mask = nf >= 64 ? ~0ull : ((1ull << nf) - 1);
  for (uint32_t t = 0; t < P && t * n_bits < 64; ++t) p.swar_mul |= 1ull << (t * n_bits);
  p.N = d_params;
  p.cost = d_params + ab;
  p.speed = d_params + 2 * ab;
  A.table = d_table;
  A.bucket_mask = slots / per_bucket - 1;
  A.table_u64 = slots * key_words;
  A.max_probes = (uint32_t)(slots / per_bucket < 0xFFFFFFFFull ? slots / per_bucket : 0xFFFFFFFFull);
  A.prune = prune ? 1 : 0;
  A.early_exit = early_exit ? 1 : 0;
  A.want_witness = 1;
  A.log_keys = d_keys;
  A.log_par = d_par;
  A.log_cap = total;
  A.ctrl = d_ctrl;
  A.levels = d_levels;
  A.off = d_off;
  A.trace = d_trace;
  A.T = T;
  A.bar_lines = d_bar;
  A.stage_chunk = mc::kWarpCap;
  A.timeout_ns = 60ull * 1000000000ull;

  mc::Ctrl h;
  if (mc::launch_explore(key_words, tile, d->rule, key_words == 1 ? MC_PROBE_SPLIT : MC_PROBE_CAS_FIRST, sms * bps,
                         mc::kThreads, A, stream) !=
      cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  // from here the kernel may be running on the shared array: every return
  // waits for the stream first, so the next call cannot clear the array
  // under it
  if (cudaMemcpyAsync(&h, d_ctrl, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(stream);
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  if (h.err) return (int)h.err;

  std::memset(out, 0, sizeof(*out));
  out->holds = h.stop_level == 0;
  out->levels = h.levels;
  out->states = h.states;
  out->key_words = key_words;
  if (!out->holds) {
    out->cex_time = mc::pack_time(h.wpack);
    out->cex_wg_index = mc::pack_i(h.wpack);
    out->cex_ts_index = mc::pack_j(h.wpack);
    out->cex_wg = d->wg_values ? d->wg_values[out->cex_wg_index] : out->cex_wg_index;
    out->cex_ts = d->ts_values ? d->ts_values[out->cex_ts_index] : out->cex_ts_index;
    out->cex_level = h.stop_level;
    out->cex_key[0] = h.wkey_lo;
    out->cex_key[1] = key_words == 2 ? h.wkey_hi : 0;
  }
  return MC_OK;
}
