// Trace kernels with the intersector injected at compile time (Section 3.2:
// "the traversal function, at compile time, is passed the custom
// intersector"), one instantiation per query and intersector.
//
// Two launch shapes:
//   k_trace            one ray per thread, grid over the rays;
//   k_trace_persistent persistent warps that claim rays from a global counter
//                      with one atomic per warp and refill idle lanes when the
//                      number of active lanes drops below a threshold
//                      (ballot + popc), after Aila and Laine's persistent
//                      threads, which the paper's traversal scheme cites.
#include "vsr_internal.h"

namespace vsr {

template <int Q, class H, bool STATS>
__global__ void __launch_bounds__(256) k_trace(DevScene sc, IsectParams ip,
                                               const float4* __restrict__ rays,
                                               RayMap map, float4* __restrict__ hits,
                                               uint2* __restrict__ counters,
                                               uint4* __restrict__ stats) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= map.threads) return;
    const unsigned long long i = ray_of_thread(g, map);
    if (i >= map.n) return;
    const Ray r = make_ray(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1));
    H h;
    Best best;
    Stats st;
    traverse<Q, H, STATS>(sc, ip, r, h, best, st, s_stack + threadIdx.x, blockDim.x);
    hits[i] = hit_record(best);
    if (H::kCounts && counters) counters[i] = h.counters();
    if (STATS) stats[i] = make_uint4(st.boxes, st.tris, st.cands, st.texs);
}

// Persistent variant.  Per-lane traversal state lives in registers and the
// shared-memory stack column; a lane that finishes its ray idles until the
// warp refills.  The counter hands out thread slots of the ray map; a slot
// past the image edge takes no ray.  Every wait is a plain loop over claimed
// work: no lane ever waits on another warp or block.  Each outer iteration
// either advances some lane's traversal (bounded per ray by the node count)
// or claims at least one ray, so the kernel terminates.
template <int Q, class H, bool STATS>
__global__ void __launch_bounds__(256) k_trace_persistent(
    DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint2* __restrict__ counters, uint4* __restrict__ stats,
    unsigned long long* __restrict__ work, uint32_t refill) {
    extern __shared__ uint32_t s_stack[];
    uint32_t* stack = s_stack + threadIdx.x;
    const uint32_t stride = blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;

    bool has = false;        // lane holds a ray in flight
    bool exhausted = false;  // warp-uniform: the counter passed n
    unsigned long long ri = 0;
    Ray r;
    Best best;
    Stats st;
    H h;
    uint32_t ref = 0, sp = 0, steps = 0;

    auto finish = [&]() {
        finish_miss(best);
        hits[ri] = hit_record(best);
        if (H::kCounts && counters) counters[ri] = h.counters();
        if (STATS) stats[ri] = make_uint4(st.boxes, st.tris, st.cands, st.texs);
        has = false;
    };

    for (;;) {
        const uint32_t busy = __ballot_sync(0xFFFFFFFFu, has);
        if (!exhausted && (uint32_t)__popc(busy) < refill) {
            const uint32_t idle = ~busy;
            const uint32_t nidle = (uint32_t)__popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)nidle);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + nidle >= map.threads) exhausted = true;
            if (!has) {
                const unsigned long long slot = base + (unsigned long long)__popc(idle & lt_mask);
                ri = slot < map.threads ? ray_of_thread(slot, map) : map.n;
                if (ri < map.n) {
                    r = make_ray(VSR_LDG(rays + 2 * ri), VSR_LDG(rays + 2 * ri + 1));
                    h = H();
                    st = Stats();
                    has = true;
                    if (!traverse_start<Q, H, STATS>(sc, ip, r, h, best, st, ref, sp, steps))
                        finish();
                }
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, has) == 0u) {
            if (exhausted) break;
            continue;
        }
        if (!has) continue;
        if (traverse_step<Q, H, STATS>(sc, ip, r, h, best, st, ref, sp, steps, stack, stride))
            finish();
    }
}

int persistent_grid(const LaunchArgs& a, const void* kernel, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (a.blocks_per_sm) {
        per_sm = (int)a.blocks_per_sm;
    } else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)a.block, smem) !=
               cudaSuccess) {
        return 0;
    }
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

namespace {

template <class K>
cudaError_t ensure_smem(K kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int Q, class H, bool STATS>
cudaError_t launch_one(const LaunchArgs& a) {
    const size_t smem = (size_t)a.sc.stack_depth * a.block * sizeof(uint32_t);
    if (!a.persistent) {
        auto k = k_trace<Q, H, STATS>;
        cudaError_t e = ensure_smem(k, smem);
        if (e != cudaSuccess) return e;
        const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
        k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits,
                                                         a.counters, a.stats);
        return cudaGetLastError();
    }
    auto k = k_trace_persistent<Q, H, STATS>;
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid(a, reinterpret_cast<const void*>(k), smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), a.stream);
    if (e != cudaSuccess) return e;
    k<<<grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits, a.counters, a.stats,
                                         a.work, a.refill);
    return cudaGetLastError();
}

template <int Q, bool STATS>
cudaError_t launch_kind(const LaunchArgs& a, int kind) {
    switch (kind) {
        case 0: return launch_one<Q, IsectNone, STATS>(a);
        case 1: return launch_one<Q, IsectDefault, STATS>(a);
        case 2: return launch_one<Q, IsectAlphaTex, STATS>(a);
        case 3: return launch_one<Q, IsectProcAlpha, STATS>(a);
        case 4: return launch_one<Q, IsectCount, STATS>(a);
        case 5: return launch_one<Q, IsectClip, STATS>(a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_static(const LaunchArgs& a, int kind, bool stats) {
    if (a.query == kClosest)
        return stats ? launch_kind<kClosest, true>(a, kind) : launch_kind<kClosest, false>(a, kind);
    return stats ? launch_kind<kAny, true>(a, kind) : launch_kind<kAny, false>(a, kind);
}

}  // namespace vsr
