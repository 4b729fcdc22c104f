// Host-side internals shared by the C-ABI translation unit and the kernel
// translation units of the GPU library.
#pragma once

#include <cuda_runtime.h>

#include "vsr_device.cuh"

namespace vsr {

struct LaunchArgs {
    DevScene sc;
    IsectParams ip;
    const float4* rays;
    unsigned long long n;
    float4* hits;
    uint2* counters;  // COUNT intersector: (boxes, tris) per ray, may be null
    uint4* stats;     // measurement variant: (boxes, tris, cands, 0), may be null
    int query;
    uint32_t block;
    uint32_t persistent;
    uint32_t refill;
    uint32_t blocks_per_sm;
    unsigned long long* work;  // persistent: ray counter, zeroed before launch
    const DevScene* dyn_user;  // dynamic dispatch: scene copy in device memory
    cudaStream_t stream;
};

// Static injection: one instantiation per (query, intersector, stats).
cudaError_t launch_static(const LaunchArgs& a, int kind, bool stats);
// Dynamic injection: run-time checked function-pointer table.
cudaError_t launch_dynamic(const LaunchArgs& a, int kind);
// Resident blocks per SM for the given kernel configuration (0 on error).
int persistent_grid(const LaunchArgs& a, const void* kernel, size_t smem);

}  // namespace vsr
