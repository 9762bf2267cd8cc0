// Random-access roofline of the device: the rate at which independent random
// 32-byte sector reads (read + atomicCAS, or atomicCAS alone) can be served
// from a buffer far larger than L2.  The visited set of a large exploration
// is accessed this way -- one random 32-byte bucket read per generated
// successor and one CAS per new state (split and one-call inserts), or one
// CAS per generated successor (CAS-first inserts) -- so this, not the
// streaming copy bandwidth, is the ceiling of the HBM-bound regime.  A measurement utility: it allocates its buffer with
// cudaMalloc and frees it before returning.
#include <cstdint>

#include "mc.h"
#include "mc_internal.h"

namespace {

__device__ __forceinline__ uint64_t rr_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Each thread performs `per_thread` accesses (four in flight at a time) to pseudo-random 32-byte sectors
// (a splitmix64 sequence per thread); op 0 reads the sector, op 1 reads it and
// CASes its first word, op 2 only CASes its first word from 0 (the first
// probe of the CAS-first inserts).  The xor of what was read goes to `sink`
// so nothing is optimised away.
__global__ void random_sector_kernel(uint64_t* buf, uint64_t sectors, uint32_t per_thread, int op,
                                     unsigned long long* sink) {
  constexpr int kUnroll = 4;  // independent accesses in flight per thread
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t x = 0, state = t * 0x9E3779B97F4A7C15ull + 12345;
  for (uint32_t k = 0; k < per_thread; k += kUnroll) {
    uint64_t sec[kUnroll];
    ulonglong2 a[kUnroll], b[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      state += 0x9E3779B97F4A7C15ull;
      sec[u] = rr_mix(state) % sectors;
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(buf + sec[u] * 4);
      if (op == 2) {
        a[u] = make_ulonglong2(
            atomicCAS(reinterpret_cast<unsigned long long*>(buf + sec[u] * 4), 0ull, (unsigned long long)state | 1ull),
            0ull);
        b[u] = make_ulonglong2(0ull, 0ull);
      } else {
        a[u] = __ldcg(p);
        b[u] = __ldcg(p + 1);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      x ^= a[u].x ^ a[u].y ^ b[u].x ^ b[u].y;
      if (op == 1)
        x ^= atomicCAS(reinterpret_cast<unsigned long long*>(buf + sec[u] * 4),
                       (unsigned long long)a[u].x, (unsigned long long)(a[u].x + 1));
    }
  }
  if (x == 0x5A5A5A5A5A5A5A5Aull) atomicAdd(sink, 1ull);
}

}  // namespace

extern "C" int mc_measure_random_access(uint64_t buffer_bytes, uint64_t accesses, int op,
                                        double* sectors_per_s, double* ms_out) {
  if (!sectors_per_s || buffer_bytes < (1u << 20) || accesses == 0 || op < 0 || op > 2)
    return MC_ERR_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  uint64_t* buf = nullptr;
  unsigned long long* sink = nullptr;
  if (cudaMalloc(&buf, buffer_bytes) != cudaSuccess || cudaMalloc(&sink, 8) != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    return MC_ERR_NOMEM;
  }
  const uint64_t sectors = buffer_bytes / 32;
  const int threads = 256;
  const int grid = sms * 8;
  const uint64_t total_threads = (uint64_t)grid * threads;
  uint32_t per_thread = (uint32_t)((accesses + total_threads - 1) / total_threads);
  per_thread = (per_thread + 3) & ~3u;  // whole unrolled groups
  if (per_thread == 0) per_thread = 4;
  cudaEvent_t e0, e1;
  int rc = MC_OK;
  if (cudaMemset(buf, 0, buffer_bytes) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = MC_ERR_CUDA;
  } else {
    random_sector_kernel<<<grid, threads>>>(buf, sectors, per_thread, op, sink);  // warm-up
    cudaEventRecord(e0);
    random_sector_kernel<<<grid, threads>>>(buf, sectors, per_thread, op, sink);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      rc = MC_ERR_CUDA;
    } else {
      *sectors_per_s = (double)total_threads * per_thread / (ms / 1e3);
      if (ms_out) *ms_out = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaFree(buf);
  cudaFree(sink);
  return rc;
}
