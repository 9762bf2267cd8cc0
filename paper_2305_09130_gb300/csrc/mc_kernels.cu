// Device side of the explorer besides the exploration pass (mc_explore.cuh):
// the simulation kernel that gives T_ini, the swarm kernels, and the launch
// helpers with their dispatch over key width, tile, rule and probe scheme.
#include <cstdint>

#include "mc_explore.cuh"

namespace mc {
namespace {

using namespace mc::dev;

// ------------------------------------------------------------------ simulation (T_ini)
// One random run per thread (Section 4, Step 3: a simulation gives T_ini).
__global__ void simulate_kernel(const Params p, uint64_t seed, uint32_t walks, uint64_t* t_out) {
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w = gtid; w < walks; w += nthreads)
    atomicMin(reinterpret_cast<unsigned long long*>(t_out),
              (unsigned long long)simulate_walk(p, seed, w));
}

// ------------------------------------------------------------------ swarm (Section 5)
// Walks w0 .. w0 + walks - 1, each cut as soon as a clock passes `bound`;
// the least (time, walk) over the runs that end at or below the bound goes to
// *best as (time << 24) | (w - w0).
__global__ void swarm_kernel(const Params p, uint64_t seed, uint64_t w0, uint32_t walks,
                             uint64_t bound, unsigned long long* best) {
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long mine = kNone;
  for (uint64_t k = gtid; k < walks; k += nthreads) {
    const uint64_t t = walk_time(p, seed, w0 + k, bound);
    if (t != kNone) {
      const unsigned long long v = ((unsigned long long)t << 24) | k;
      mine = v < mine ? v : mine;
    }
  }
  mine = warp_min(mine);
  if ((threadIdx.x & 31u) == 0 && mine != kNone) atomicMin(best, mine);
}

// Replays walk w and writes its states (keys {lo, hi}) into trace[0..];
// *len receives the number of states.
template <class K>
__device__ void replay_walk(const Params& p, uint64_t seed, uint64_t w, uint64_t* trace, uint32_t* len) {
  uint64_t ctr = w << 32;
  const uint32_t i = (uint32_t)(splitmix64_at(seed, ctr++) % p.a);
  const uint32_t j = (uint32_t)(splitmix64_at(seed, ctr++) % p.b);
  const uint32_t cfg = i * p.b + j;
  const uint32_t N = p.N[cfg];
  const uint64_t cost = p.cost[cfg];
  K key = 0;
  uint32_t l = 0;
  auto put = [&](K k) {
    trace[2 * l] = (uint64_t)k;
    trace[2 * l + 1] = sizeof(K) == 16 ? (uint64_t)((u128)k >> 64) : 0;
    ++l;
  };
  put(key);
  key = (K)(i + 1) << p.wg_shift;
  put(key);
  key |= (K)(j + 1) << p.ts_shift;
  put(key);
  uint64_t clk[kMaxP], t[kMaxP];
  for (uint32_t c = 0; c < p.P; ++c) {
    t[c] = cost * p.speed[c];
    clk[c] = 0;
  }
  for (uint32_t k = 0; k < N; ++k) {
    uint32_t c = 0;
    if (p.rule == MC_FREE) {
      c = (uint32_t)(splitmix64_at(seed, ctr++) % p.P);
    } else {
      uint64_t mn = kNone;
      for (uint32_t u = 0; u < p.P; ++u) mn = clk[u] < mn ? clk[u] : mn;
      uint32_t cnt = 0;
      for (uint32_t u = 0; u < p.P; ++u) cnt += clk[u] == mn;
      uint32_t pick = (uint32_t)(splitmix64_at(seed, ctr++) % cnt);
      for (uint32_t u = 0; u < p.P; ++u) {
        if (clk[u] == mn) {
          if (pick == 0) { c = u; break; }
          --pick;
        }
      }
    }
    clk[c] += t[c];
    key += (K)1 << ((p.P - 1 - c) * p.n_bits);
    put(key);
  }
  *len = l;
}

__global__ void replay_walk_kernel(const Params p, uint64_t seed, uint64_t w, int key_words,
                                   uint64_t* trace, uint32_t* len) {
  if (blockIdx.x || threadIdx.x) return;
  if (key_words == 1) replay_walk<uint64_t>(p, seed, w, trace, len);
  else replay_walk<u128>(p, seed, w, trace, len);
}

template <class K>
const void* pick_scheme(int tile, int rule, int scheme) {
  switch (scheme) {
    case MC_PROBE_SPLIT: return pick_rule<K, MC_PROBE_SPLIT>(tile, rule);
    case MC_PROBE_ONE_CALL: return pick_rule<K, MC_PROBE_ONE_CALL>(tile, rule);
  }
  return nullptr;
}

const void* pick_kernel(int key_words, int tile, int rule, int scheme) {
  if (scheme == MC_PROBE_CAS_FIRST || scheme == MC_PROBE_CAS_CLEAR)
    return pick_explore_cas(key_words, tile, rule, scheme);  // mc_explore_cas.cu
  if (key_words == 1) return pick_scheme<uint64_t>(tile, rule, scheme);
  if (key_words == 2) return pick_scheme<u128>(tile, rule, scheme);
  return nullptr;
}

}  // namespace

int explore_kernel_occupancy(int key_words, int tile, int rule, int scheme, int threads, int* blocks_per_sm) {
  const void* f = pick_kernel(key_words, tile, rule, scheme);
  if (!f) return -1;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, 0) == cudaSuccess
             ? 0
             : -1;
}

cudaError_t launch_explore(int key_words, int tile, int rule, int scheme, int grid, int threads,
                           const ExploreArgs& args, cudaStream_t stream) {
  const void* f = pick_kernel(key_words, tile, rule, scheme);
  if (!f) return cudaErrorInvalidValue;
  void* params[] = {const_cast<ExploreArgs*>(&args)};
  return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(threads), params, 0, stream);
}

cudaError_t launch_swarm(const Params& p, uint64_t seed, uint64_t w0, uint32_t walks, uint64_t bound,
                         unsigned long long* best, int grid, cudaStream_t stream) {
  swarm_kernel<<<grid, 256, 0, stream>>>(p, seed, w0, walks, bound, best);
  return cudaGetLastError();
}

cudaError_t launch_replay_walk(const Params& p, uint64_t seed, uint64_t w, int key_words,
                               uint64_t* trace, uint32_t* len, cudaStream_t stream) {
  replay_walk_kernel<<<1, 32, 0, stream>>>(p, seed, w, key_words, trace, len);
  return cudaGetLastError();
}

cudaError_t launch_simulate(const Params& p, uint64_t seed, uint32_t walks, uint64_t* t_out,
                            cudaStream_t stream) {
  const int threads = 128;
  int grid = (int)((walks + threads - 1) / threads);
  if (grid > 1024) grid = 1024;
  simulate_kernel<<<grid, threads, 0, stream>>>(p, seed, walks, t_out);
  return cudaGetLastError();
}

}  // namespace mc
