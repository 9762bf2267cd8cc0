// Runs of many models on the configuration engine (mc_cfg_jobs.cu): the
// batches of mc_batch_run and the jobs of the request loop.  Internal.
#pragma once

#include <cstdint>
#include <vector>

#include "mc.h"
#include "mc_internal.h"

namespace mc {

// One model prepared for the configuration engine (128-bit keys), with its
// device region once placed: [params][segment starts][records of 3 passes]
// [level widths of 3 passes][trace][log keys][log parents].
struct CfgModelPrep {
  Params p;                    // table pointers into the region once placed
  uint32_t group = 1, ab = 0, L2 = 0, threads = 64, wcap = 32;
  uint64_t unit_width = 0, unit_log = 0, region = 0;
  std::vector<uint32_t> params;  // N, cost, speed
  std::vector<uint64_t> seg;     // [ab + 1]
  std::vector<uint32_t> order;   // configurations, deepest first
  std::vector<uint32_t> wg, ts;  // values echoed in results
  uint8_t* base = nullptr;
  uint64_t* d_seg = nullptr;
  CfgRec* d_rec = nullptr;
  uint64_t* d_levels = nullptr;
  uint64_t* d_trace = nullptr;
  void* d_keys = nullptr;
  uint32_t* d_par = nullptr;
};

// Validate the description and lay the model out (host only).  Errors: as
// mc_model_create, INVAL when the configuration engine cannot take it.
int cfg_prepare(const mc_model_desc& d, const mc_options& o, CfgModelPrep& M);
// One warp per configuration: the widest level's lanes fit a warp and the
// options leave the block's threads to the library.
inline bool cfg_warp_model(const CfgModelPrep& M, const mc_options& o) {
  return !o.unit_threads && M.unit_width * M.group <= kCfgWarpLanes;
}
// Point the model at its region (M.region bytes, 256-byte aligned); the
// caller uploads M.params and M.seg to M.base and M.d_seg.
void cfg_place(CfgModelPrep& M, uint8_t* base);
// The same without the tables: the region holds M.region - cfg_tables_bytes(M)
// bytes, and the tables travel in a run's upload (CfgRun::place_tables).
uint64_t cfg_tables_bytes(const CfgModelPrep& M);
void cfg_place_state(CfgModelPrep& M, uint8_t* base);

// One run's descriptors and results: a device block and its pinned mirror,
// [passes][clears][sims][units][counters] uploaded, [headers][T_ini, T_min]
// read back.
struct CfgRun {
  uint32_t cap_n = 0;
  uint64_t cap_units = 0;
  uint64_t upload_bytes = 0, result_off = 0, result_bytes = 0;
  uint8_t *d_block = nullptr, *h_block = nullptr;
  CfgPass *d_pass = nullptr, *h_pass = nullptr;
  CfgClear *d_clear = nullptr, *h_clear = nullptr;
  CfgSim *d_sim = nullptr, *h_sim = nullptr;
  uint64_t *d_units = nullptr, *h_units = nullptr;
  uint32_t *d_cnt = nullptr, *h_cnt = nullptr;
  Ctrl *d_ctrl = nullptr, *h_ctrl = nullptr;
  uint64_t *d_scal = nullptr, *h_scal = nullptr;
  // set by prepare
  uint32_t n_models = 0, wcap = 32, tsize = 64, threads = 64, walks_max = 1;
  uint64_t n_units_a = 0, n_units_b = 0;
  // warp units (models whose widest configuration level fits a warp): in
  // the same unit regions, from their ends backwards; blocks serving them
  uint64_t n_wunits_a = 0, n_wunits_b = 0;
  uint32_t wblocks_a = 0, wblocks_b = 0;
  bool refine = true, any_min = false;

  uint64_t tables_cap = 0, tables_used = 0;     // model tables carried by the upload
  uint8_t *d_tables = nullptr, *h_tables = nullptr;

  static uint64_t block_bytes(uint32_t n_max, uint64_t units_max, uint64_t tables_bytes = 0);
  void layout(uint32_t n_max, uint64_t units_max, uint8_t* dev, uint8_t* host, uint64_t tables_bytes = 0);
  // Copy M's tables and segment starts into the upload and point M at them
  // (false when they do not fit); reset with tables_used = 0 per run.
  bool place_tables(CfgModelPrep& M);
  // Fill the pinned descriptors for queries[k] on *models[k].
  void prepare(const std::vector<CfgModelPrep*>& models, const mc_query* queries, const mc_options& opt);
  // Upload, clear, simulate, both pass launches, read back (events around
  // the pass launches if given).
  cudaError_t enqueue(cudaStream_t st, int grid_a, int grid_b, size_t smem, cudaEvent_t ev0, cudaEvent_t ev1,
                      bool capturing);
  // Model k's result from the read-back headers.
  void result(const CfgModelPrep& M, uint32_t k, const mc_query& q, mc_batch_result& r, uint32_t* trace_len,
              uint64_t* states_explored) const;
};

}  // namespace mc
