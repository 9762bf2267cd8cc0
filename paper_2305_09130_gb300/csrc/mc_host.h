// Host-side resources shared by the model kinds (defined in mc_api.cu).
// Internal; thread-safe.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

namespace mc {

// Pinned host blocks reused across models.
void* pinned_alloc(size_t bytes);
void pinned_free(void* p, size_t bytes);

// The library's stream-ordered device pool of a device.
cudaMemPool_t device_pool(int device);

// Trim every device pool and free the cached pinned blocks.
void release_cached();
int set_pool_retention(uint64_t bytes);

}  // namespace mc
