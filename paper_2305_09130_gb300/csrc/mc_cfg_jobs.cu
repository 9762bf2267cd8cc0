// Runs of many models on the configuration engine (mc_cfg.cu): the batches
// of mc_batch_run and the jobs of the request loop (mc_server_*).
//
// A run answers one query per model (mc_check, or mc_min_time in SINGLE
// mode) in four launches on one stream, whatever the number of models:
//   clear    every model's pass headers, level widths and {T_ini, T_min};
//   sim      the T_ini simulation of every min-time model (Section 4,
//            Step 3);
//   pass A   every model's first pass: the min pass of a min-time query
//            (pruned at T_ini, the least terminal time reduced on the
//            device), or the check itself -- one unit per (model,
//            configuration), deepest configurations first;
//   pass B   the certificate check at T_min - 1 and the counterexample
//            check at T_min of every min-time model, both reading T_min
//            from the device.
// The host uploads the run's descriptors (passes, units, clears, sims) with
// one copy before and reads every header back with one copy after, so a
// run costs the same API calls for one model as for a thousand.  Every
// model uses 128-bit keys (as the lockstep batch engine), so its results
// equal mc_check / mc_min_time on the model with key_bits = 128.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mc.h"
#include "mc_cfg_jobs.h"
#include "mc_host.h"
#include "mc_internal.h"

namespace mc {
namespace {

uint64_t al256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

int cfg_prepare(const mc_model_desc& d_in, const mc_options& o, CfgModelPrep& M) {
  mc_model_desc d = d_in;
  d.key_bits = 128;
  mc_options co = o;
  co.engine = MC_ENGINE_CONFIG;
  mc_model* m = nullptr;
  int rc = mc_model_create(&d, &co, &m);
  if (rc) return rc;
  CfgModelInfo info;
  rc = cfg_model_info(m, &info);
  if (rc == MC_OK && !info.eligible) rc = MC_ERR_INVAL;
  if (rc) {
    mc_model_destroy(m);
    return rc;
  }
  M.p = info.p;
  M.group = info.group;
  M.ab = d.n_wg * d.n_ts;
  M.L2 = info.p.max_level + 2;
  M.unit_width = info.unit_width;
  M.unit_log = info.unit_log;
  M.seg.assign(info.seg, info.seg + M.ab + 1);
  mc_model_destroy(m);
  M.params.assign(d.n_workgroups, d.n_workgroups + M.ab);
  M.params.insert(M.params.end(), d.cost, d.cost + M.ab);
  for (uint32_t c = 0; c < d.P; ++c) M.params.push_back(d.speed ? d.speed[c] : 1);
  M.wg.clear();
  M.ts.clear();
  if (d.wg_values) M.wg.assign(d.wg_values, d.wg_values + d.n_wg);
  if (d.ts_values) M.ts.assign(d.ts_values, d.ts_values + d.n_ts);
  // configurations deepest first (by work-groups)
  M.order.resize(M.ab);
  for (uint32_t k = 0; k < M.ab; ++k) M.order[k] = k;
  const uint32_t* N = M.params.data();
  std::stable_sort(M.order.begin(), M.order.end(), [N](uint32_t x, uint32_t y) { return N[x] > N[y]; });
  // threads a block needs for this model's widest level in one round
  uint32_t t = 64;
  while ((uint64_t)t < M.unit_width * M.group && t < kCfgMaxThreads) t <<= 1;
  M.threads = t;
  uint32_t w = 32;
  while (w < M.unit_width) w <<= 1;
  M.wcap = w;
  // region: [params][seg][rec x 3][levels x 3][trace][log keys][log parents]
  M.region = al256(4ull * M.params.size()) + al256(8ull * (M.ab + 1)) + al256(3ull * sizeof(CfgRec) * M.ab) +
             al256(48ull * M.L2) + al256(16ull * M.L2) + al256(16 * M.unit_log) + al256(4 * M.unit_log);
  return MC_OK;
}

void cfg_place(CfgModelPrep& M, uint8_t* q) {
  const uint64_t ab = M.ab;
  M.base = q;
  M.p.N = (const uint32_t*)q;
  M.p.cost = (const uint32_t*)q + ab;
  M.p.speed = (const uint32_t*)q + 2 * ab;
  q += al256(4ull * M.params.size());
  M.d_seg = (uint64_t*)q;
  q += al256(8ull * (ab + 1));
  M.d_rec = (CfgRec*)q;
  q += al256(3ull * sizeof(CfgRec) * ab);
  M.d_levels = (uint64_t*)q;
  q += al256(48ull * M.L2);
  M.d_trace = (uint64_t*)q;
  q += al256(16ull * M.L2);
  M.d_keys = q;
  q += al256(16 * M.unit_log);
  M.d_par = (uint32_t*)q;
}

uint64_t cfg_tables_bytes(const CfgModelPrep& M) {
  return al256(4ull * M.params.size()) + al256(8ull * (M.ab + 1));
}

void cfg_place_state(CfgModelPrep& M, uint8_t* q) {
  const uint64_t ab = M.ab;
  M.base = q;
  M.d_rec = (CfgRec*)q;
  q += al256(3ull * sizeof(CfgRec) * ab);
  M.d_levels = (uint64_t*)q;
  q += al256(48ull * M.L2);
  M.d_trace = (uint64_t*)q;
  q += al256(16ull * M.L2);
  M.d_keys = q;
  q += al256(16 * M.unit_log);
  M.d_par = (uint32_t*)q;
}

// ---------------------------------------------------------------- a run
uint64_t CfgRun::block_bytes(uint32_t n, uint64_t units, uint64_t tables_bytes) {
  return al256(sizeof(CfgPass) * 3ull * n) + al256(sizeof(CfgClear) * (uint64_t)n) +
         al256(sizeof(CfgSim) * (uint64_t)n) + al256(8 * 3 * units) + 256 + al256(tables_bytes) +  // upload
         al256(sizeof(Ctrl) * 3ull * n) + al256(16ull * n);                                        // result
}

bool CfgRun::place_tables(CfgModelPrep& M) {
  const uint64_t need = cfg_tables_bytes(M);
  if (tables_used + need > tables_cap) return false;
  uint8_t* h = h_tables + tables_used;
  uint8_t* d = d_tables + tables_used;
  std::memcpy(h, M.params.data(), 4 * M.params.size());
  const uint64_t o_seg = al256(4ull * M.params.size());
  std::memcpy(h + o_seg, M.seg.data(), 8 * M.seg.size());
  M.p.N = (const uint32_t*)d;
  M.p.cost = (const uint32_t*)d + M.ab;
  M.p.speed = (const uint32_t*)d + 2ull * M.ab;
  M.d_seg = (uint64_t*)(d + o_seg);
  tables_used += need;
  return true;
}

void CfgRun::layout(uint32_t n_max, uint64_t units_max, uint8_t* dev, uint8_t* host, uint64_t tables_bytes) {
  cap_n = n_max;
  cap_units = units_max;
  uint64_t o = 0;
  auto take = [&](uint64_t bytes) {
    const uint64_t at = o;
    o += al256(bytes);
    return at;
  };
  const uint64_t o_pass = take(sizeof(CfgPass) * 3ull * n_max);
  const uint64_t o_clear = take(sizeof(CfgClear) * (uint64_t)n_max);
  const uint64_t o_sim = take(sizeof(CfgSim) * (uint64_t)n_max);
  const uint64_t o_units = take(8 * 3 * units_max);  // pass A: units_max, pass B: 2 x units_max
  const uint64_t o_cnt = take(256);
  const uint64_t o_tab = take(tables_bytes);
  tables_cap = al256(tables_bytes);
  tables_used = 0;
  upload_bytes = o;
  const uint64_t o_ctrl = take(sizeof(Ctrl) * 3ull * n_max);
  const uint64_t o_scal = take(16ull * n_max);
  result_off = o_ctrl;
  result_bytes = o - o_ctrl;
  d_block = dev;
  h_block = host;
  d_pass = (CfgPass*)(dev + o_pass);
  d_clear = (CfgClear*)(dev + o_clear);
  d_sim = (CfgSim*)(dev + o_sim);
  d_units = (uint64_t*)(dev + o_units);
  d_cnt = (uint32_t*)(dev + o_cnt);
  d_ctrl = (Ctrl*)(dev + o_ctrl);
  d_scal = (uint64_t*)(dev + o_scal);
  h_pass = (CfgPass*)(host + o_pass);
  h_clear = (CfgClear*)(host + o_clear);
  h_sim = (CfgSim*)(host + o_sim);
  h_units = (uint64_t*)(host + o_units);
  h_cnt = (uint32_t*)(host + o_cnt);
  h_ctrl = (Ctrl*)(host + o_ctrl);
  h_scal = (uint64_t*)(host + o_scal);
  d_tables = dev + o_tab;
  h_tables = host + o_tab;
}

void CfgRun::prepare(const std::vector<CfgModelPrep*>& models, const mc_query* queries, const mc_options& opt) {
  const uint32_t n = (uint32_t)models.size();
  n_models = n;
  refine = opt.refine != 0;
  std::memset(h_cnt, 0, 256);
  uint32_t n_sim = 0;
  std::vector<std::pair<uint32_t, uint64_t>> ua, ub, wa, wb;  // (work-groups, unit) for sorting
  wcap = 32;
  threads = 64;
  any_min = false;
  for (uint32_t k = 0; k < n; ++k) {
    CfgModelPrep& M = *models[k];
    const mc_query& q = queries[k];
    const bool mt = q.kind == MC_QUERY_MIN_TIME;
    const bool warp = cfg_warp_model(M, opt);
    any_min |= mt;
    if (!warp) {  // blocks are sized for the models they explore
      wcap = std::max(wcap, M.wcap);
      threads = std::max(threads, M.threads);
    }
    uint64_t* scal = d_scal + 2ull * k;
    for (uint32_t s = 0; s < 3; ++s) {
      CfgPass& Q = h_pass[3 * k + s];
      std::memset(&Q, 0, sizeof(Q));
      Q.p = M.p;
      Q.prune = opt.prune;
      Q.group = M.group;
      Q.log_keys = M.d_keys;
      Q.log_par = M.d_par;
      Q.seg = M.d_seg;
      Q.levels = M.d_levels + 2ull * M.L2 * s;
      Q.rec = M.d_rec + (uint64_t)M.ab * s;
      Q.ctrl = d_ctrl + 3ull * k + s;
      Q.trace = M.d_trace;
      Q.order = nullptr;
    }
    CfgPass& A = h_pass[3 * k];
    if (mt) {
      // the min pass: pruned at T_ini (or unpruned), the least violating
      // terminal time to T_min; then the certificate check at T_min - 1 and
      // the counterexample check at T_min
      A.T = UINT64_MAX;
      A.T_src = opt.prune ? scal : nullptr;
      A.early_exit = 0;
      A.want_witness = 0;
      A.tmin_out = scal + 1;
      CfgPass& R = h_pass[3 * k + 1];
      R.T_src = scal + 1;
      R.T_delta = -1;
      R.early_exit = opt.early_exit;
      CfgPass& F = h_pass[3 * k + 2];
      F.T_src = scal + 1;
      F.early_exit = opt.early_exit;
      F.want_witness = 1;
      CfgSim& S = h_sim[n_sim++];
      S.p = M.p;
      S.tini = scal;
      S.seed = opt.sim_seed;
      S.walks = opt.sim_walks;
    } else {
      A.T = q.T;
      A.early_exit = opt.early_exit;
      A.want_witness = 1;
    }
    CfgClear& C = h_clear[k];
    C.levels = M.d_levels;
    C.level_words = 6ull * M.L2;
    C.ctrl = d_ctrl + 3ull * k;
    C.n_ctrl = 3;
    C.scal = scal;
    const uint32_t* N = M.params.data();
    auto& la = warp ? wa : ua;
    auto& lb = warp ? wb : ub;
    for (uint32_t c : M.order) {
      la.push_back({N[c], ((uint64_t)(3 * k) << 32) | c});
      if (mt) {
        if (refine) lb.push_back({N[c], ((uint64_t)(3 * k + 1) << 32) | c});
        lb.push_back({N[c], ((uint64_t)(3 * k + 2) << 32) | c});
      }
    }
  }
  // deepest configurations first within each launch
  auto deeper = [](const std::pair<uint32_t, uint64_t>& x, const std::pair<uint32_t, uint64_t>& y) {
    return x.first > y.first;
  };
  std::stable_sort(ua.begin(), ua.end(), deeper);
  std::stable_sort(ub.begin(), ub.end(), deeper);
  std::stable_sort(wa.begin(), wa.end(), deeper);
  std::stable_sort(wb.begin(), wb.end(), deeper);
  n_units_a = ua.size();
  n_units_b = ub.size();
  n_wunits_a = wa.size();
  n_wunits_b = wb.size();
  // pass A's region [0, cap), pass B's [cap, 3 cap): block units from the
  // start, warp units from the end backwards (a model's configurations are
  // in one list or the other, so the two never meet)
  for (uint64_t x = 0; x < ua.size(); ++x) h_units[x] = ua[x].second;
  for (uint64_t x = 0; x < ub.size(); ++x) h_units[cap_units + x] = ub[x].second;
  for (uint64_t x = 0; x < wa.size(); ++x) h_units[cap_units - 1 - x] = wa[x].second;
  for (uint64_t x = 0; x < wb.size(); ++x) h_units[3 * cap_units - 1 - x] = wb[x].second;
  // counters: [0] next unit of pass A, [1] of pass B, [2] units of A,
  // [3] units of B, [4] models to clear, [5] min-time models to simulate,
  // [6] warp units of A, [7] of B, [8] next warp unit of A, [9] of B
  h_cnt[2] = (uint32_t)n_units_a;
  h_cnt[3] = (uint32_t)n_units_b;
  h_cnt[4] = n;
  h_cnt[5] = n_sim;
  h_cnt[6] = (uint32_t)n_wunits_a;
  h_cnt[7] = (uint32_t)n_wunits_b;
  walks_max = std::max<uint32_t>(opt.sim_walks, 1);
  tsize = 2 * wcap;
  if (opt.unit_threads) threads = opt.unit_threads;
  // blocks of warp units: from pass A's count, which depends on the models
  // only (a replayed graph keeps them while the queries change), and twice
  // that for pass B (every warp model a min-time query with both checks)
  const uint64_t wpb = threads / 32;
  auto blocks = [wpb](uint64_t units) {
    return (uint32_t)std::min<uint64_t>((units + wpb - 1) / wpb, kCfgMaxWarpBlocks);
  };
  wblocks_a = blocks(n_wunits_a);
  wblocks_b = blocks(2 * n_wunits_a);
}

cudaError_t CfgRun::enqueue(cudaStream_t st, int grid_a, int grid_b, size_t smem, cudaEvent_t ev0,
                            cudaEvent_t ev1, bool capturing) {
  cudaError_t e;
  const uint64_t up = tables_cap ? (uint64_t)(h_tables - h_block) + tables_used : upload_bytes;
  if ((e = cudaMemcpyAsync(d_block, h_block, up, cudaMemcpyHostToDevice, st))) return e;
  if ((e = launch_cfg_clear(d_clear, d_cnt + 4, cap_n, st))) return e;
  if ((e = launch_cfg_sim(d_sim, d_cnt + 5, cap_n, walks_max, st))) return e;
  if (ev0 && (e = capturing ? cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal) : cudaEventRecord(ev0, st)))
    return e;
  CfgLaunch L{};
  L.passes = d_pass;
  L.units = d_units;
  L.n_units_dev = d_cnt + 2;
  L.next = d_cnt + 0;
  L.wcap = wcap;
  L.tsize = tsize;
  L.wunits = d_units + cap_units - 1;
  L.wunits_rev = 1;
  L.n_wunits_dev = d_cnt + 6;
  L.wnext = d_cnt + 8;
  L.warp_blocks = wblocks_a;
  if ((e = launch_cfg(2, grid_a + (int)wblocks_a, threads, smem, L, st))) return e;
  L.units = d_units + cap_units;
  L.n_units_dev = d_cnt + 3;
  L.next = d_cnt + 1;
  L.wunits = d_units + 3 * cap_units - 1;
  L.n_wunits_dev = d_cnt + 7;
  L.wnext = d_cnt + 9;
  L.warp_blocks = wblocks_b;
  if ((e = launch_cfg(2, grid_b + (int)wblocks_b, threads, smem, L, st))) return e;
  if (ev1 && (e = capturing ? cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal) : cudaEventRecord(ev1, st)))
    return e;
  return cudaMemcpyAsync(h_block + result_off, d_block + result_off, result_bytes, cudaMemcpyDeviceToHost, st);
}

void CfgRun::result(const CfgModelPrep& M, uint32_t k, const mc_query& q, mc_batch_result& r, uint32_t* trace_len,
                    uint64_t* states_explored) const {
  std::memset(&r, 0, sizeof(r));
  r.kind = q.kind;
  const Ctrl* c = h_ctrl + 3ull * k;
  const Ctrl* last;
  uint64_t states = 0;
  int status = 0;
  if (q.kind == MC_QUERY_MIN_TIME) {
    const int passes[3] = {0, 1, 2};
    for (int s : passes) {
      if (s == 1 && !refine) continue;
      if (!status && c[s].err) status = (int)c[s].err;
      states += c[s].states;
      r.checks += 1;
    }
    last = c + 2;
    r.t_ini = h_scal[2ull * k];
    if (!status && (c[0].best_pack == kNone || (refine && c[1].stop_level != 0) || c[2].stop_level == 0))
      status = MC_ERR_CUDA;  // cannot happen: the certificate checks follow from the minimum
  } else {
    last = c;
    status = (int)c[0].err;
    states = c[0].states;
    r.checks = 1;
  }
  r.status = status;
  r.states = states;
  r.levels = last->levels;
  r.holds = last->stop_level == 0;
  if (states_explored) *states_explored = states;
  if (trace_len) *trace_len = status ? 0 : last->trace_len;
  if (!status && last->stop_level) {
    r.time = pack_time(last->wpack);
    r.wg_index = pack_i(last->wpack);
    r.ts_index = pack_j(last->wpack);
    r.wg = M.wg.empty() ? r.wg_index : M.wg[r.wg_index];
    r.ts = M.ts.empty() ? r.ts_index : M.ts[r.ts_index];
    r.level = last->stop_level;
    r.key[0] = last->wkey_lo;
    r.key[1] = last->wkey_hi;
  }
}

}  // namespace mc
