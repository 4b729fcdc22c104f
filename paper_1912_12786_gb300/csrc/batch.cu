// Batched persistent trace: many independent scenes, each with its own ray
// batch, in one launch.
//
// The rays of all scenes form one index space [0, total) with per-scene
// prefix offsets.  Warps claim rays from a global counter with one atomic
// per warp and refill idle lanes when fewer than `refill` lanes are still
// busy (the persistent scheme of k_trace_persistent).  A lane locates the
// scene of its ray by binary search over the offsets and copies that scene's
// descriptor, so lanes of one warp may trace different scenes.  Per-ray
// results are identical to a per-scene vsr_trace: the traversal code is the
// same (traverse_start / traverse_step).
#include "vsr_internal.h"

namespace vsr {

__device__ __forceinline__ uint32_t scene_of(const unsigned long long* __restrict__ offsets,
                                             uint32_t nbatch, unsigned long long g) {
    // largest s with offsets[s] <= g; offsets[0] = 0, offsets[nbatch] = total
    uint32_t lo = 0, hi = nbatch;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (VSR_LDG(offsets + mid) <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <int Q, class H>
__global__ void __launch_bounds__(256) k_trace_batch(const BatchItem* __restrict__ items,
                                                     const unsigned long long* __restrict__ offsets,
                                                     uint32_t nbatch, IsectParams ip,
                                                     unsigned long long total,
                                                     unsigned long long* __restrict__ work,
                                                     uint32_t refill) {
    extern __shared__ uint32_t s_stack[];
    uint32_t* stack = s_stack + threadIdx.x;
    const uint32_t stride = blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;

    bool has = false;
    bool exhausted = false;
    unsigned long long ri = 0;
    float4* hp = nullptr;
    DevScene sc;
    Ray r;
    Best best;
    Stats st;
    H h;
    uint32_t ref = 0, sp = 0, steps = 0;

    for (;;) {
        const uint32_t busy = __ballot_sync(0xFFFFFFFFu, has);
        if (!exhausted && (uint32_t)__popc(busy) < refill) {
            const uint32_t idle = ~busy;
            const uint32_t nidle = (uint32_t)__popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)nidle);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + nidle >= total) exhausted = true;
            if (!has) {
                const unsigned long long g = base + (unsigned long long)__popc(idle & lt_mask);
                if (g < total) {
                    const uint32_t s = scene_of(offsets, nbatch, g);
                    ri = g - VSR_LDG(offsets + s);
                    sc = items[s].sc;
                    const float4* rays = items[s].rays;
                    hp = items[s].hits;
                    r = make_ray(VSR_LDG(rays + 2 * ri), VSR_LDG(rays + 2 * ri + 1));
                    h = H();
                    has = true;
                    if (!traverse_start<Q, H, false>(sc, ip, r, h, best, st, ref, sp, steps)) {
                        finish_miss(best);
                        hp[ri] = hit_record(best);
                        has = false;
                    }
                }
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, has) == 0u) {
            if (exhausted) break;
            continue;
        }
        if (!has) continue;
        if (traverse_step<Q, H, false>(sc, ip, r, h, best, st, ref, sp, steps, stack, stride)) {
            finish_miss(best);
            hp[ri] = hit_record(best);
            has = false;
        }
    }
}

namespace {

template <int Q, class H>
cudaError_t batch_one(const BatchLaunch& b, cudaStream_t stream, uint32_t* grid_out) {
    auto k = k_trace_batch<Q, H>;
    const size_t smem = (size_t)b.stack_max * b.block * sizeof(uint32_t);
    uint32_t grid = b.grid;
    if (grid == 0) {
        if (smem > 48 * 1024) {
            cudaError_t e =
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int dev = 0, sms = 0, per_sm = (int)b.blocks_per_sm;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess && per_sm == 0)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)b.block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        grid = (uint32_t)(sms * per_sm);
    }
    if (grid_out) {
        *grid_out = grid;
        return cudaSuccess;
    }
    cudaError_t e = cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    k<<<grid, b.block, smem, stream>>>(b.items, b.offsets, b.nbatch, b.ip, b.total, b.work,
                                       b.refill);
    return cudaGetLastError();
}

template <int Q>
cudaError_t batch_kind(const BatchLaunch& b, int kind, cudaStream_t stream, uint32_t* grid) {
    switch (kind) {
        case 0: return batch_one<Q, IsectNone>(b, stream, grid);
        case 1: return batch_one<Q, IsectDefault>(b, stream, grid);
        case 2: return batch_one<Q, IsectAlphaTex>(b, stream, grid);
        case 3: return batch_one<Q, IsectProcAlpha>(b, stream, grid);
        case 4: return batch_one<Q, IsectCount>(b, stream, grid);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_batch(const BatchLaunch& b, int kind, int query, cudaStream_t stream) {
    return query == kClosest ? batch_kind<kClosest>(b, kind, stream, nullptr)
                             : batch_kind<kAny>(b, kind, stream, nullptr);
}

cudaError_t batch_grid(const BatchLaunch& b, int kind, int query, uint32_t* grid) {
    return query == kClosest ? batch_kind<kClosest>(b, kind, nullptr, grid)
                             : batch_kind<kAny>(b, kind, nullptr, grid);
}

}  // namespace vsr
