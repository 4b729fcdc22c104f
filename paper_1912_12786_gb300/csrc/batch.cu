// Batched persistent trace: many independent scenes, each with its own ray
// batch, in one launch.
//
// The rays of all scenes form one index space [0, total) with per-scene
// prefix offsets.  Warps claim rays from a global counter with one atomic
// per warp and refill idle lanes when fewer than `refill` lanes are still
// busy (the persistent scheme of k_trace_persistent).  A claim is a run of
// consecutive indices, so it usually lies in one scene: the warp finds the
// scene of the run's first index by a 32-way search over the offsets, and each
// claiming lane walks forward from there to its own scene (past scenes with
// no rays) and keeps a pointer to that scene's descriptor in the item table
// (fields are read from L1 as the traversal needs them, instead of a
// 128-byte copy held in registers).  Lanes of one warp may still trace
// different scenes.  In coherence order (sort.cu) the claims walk the sorted
// order instead: slot k names the ray perm[k], and scene s still owns slots
// [offsets[s], offsets[s+1]) because the sort key is scene-major.  Per-ray
// results are identical to a per-scene vsr_trace: the traversal code is the
// same (traverse_start / traverse_step).
#include "vsr_internal.h"

namespace vsr {

// Largest s with offsets[s] <= g (offsets[0] = 0, offsets[nbatch] = total),
// found by the whole warp: each round the 32 lanes probe 32 evenly spaced
// offsets of the remaining range at once and a ballot keeps the segment
// that holds g, so 256 scenes take two rounds of loads (a binary search by
// one lane takes eight dependent ones).  Called by all 32 lanes with the
// same g; returns the same s on every lane.
__device__ __forceinline__ uint32_t scene_of_warp(const unsigned long long* __restrict__ offsets,
                                                  uint32_t nbatch, unsigned long long g,
                                                  uint32_t lane) {
    uint32_t lo = 0, hi = nbatch;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t idx = lo + lane * step;
        const bool le = idx < hi && VSR_LDG(offsets + idx) <= g;
        const uint32_t m = __ballot_sync(kFullMask, le);  // a prefix of the lanes (lane 0 set)
        const uint32_t k = 31u - (uint32_t)__clz(m);
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Control flow as k_trace_persistent (trace_static.cuh): converged votes at
// the top of every iteration, one divergent traversal step closed by
// __syncwarp, uniform exits, and the watchdog.
template <int Q, class H, int K, bool LS>
__global__ void __launch_bounds__(256, 4) k_trace_batch(const BatchItem* __restrict__ items,
                                                     const unsigned long long* __restrict__ offsets,
                                                     uint32_t nbatch, IsectParams ip,
                                                     unsigned long long total,
                                                     unsigned long long* __restrict__ work,
                                                     uint32_t refill, Watchdog wd,
                                                     const uint32_t* __restrict__ perm,
                                                     uint32_t stack_max) {
    extern __shared__ uint32_t s_stack[];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    ShortStack<K> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    // closest-hit speculation's entry distances (lock step), after the stack
    float* tcol =
        reinterpret_cast<float*>(s_stack + stack_words(stack_max, K) * blockDim.x) + threadIdx.x;

    bool has = false;
    bool exhausted = false;
    unsigned long long ri = 0;
    float4* hp = nullptr;
    const DevScene* scp = &items[0].sc;
    Ray r;
    Best best;
    Stats st;
    H h;
    uint32_t ref = 0, steps = 0, leaf = 0;
    bool more = false, pend = false;
    uint32_t* err0 = items[0].sc.err;  // the watchdog also reports to scene 0's word
    const unsigned long long t0 = wd.max_ns ? global_ns() : 0ull;
    unsigned long long iters = 0;

    for (;;) {
        const uint32_t busy = __ballot_sync(kFullMask, has);
        if (!exhausted && (uint32_t)__popc(busy) < refill) {
            const uint32_t idle = ~busy;
            const uint32_t nidle = (uint32_t)__popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)nidle);
            base = __shfl_sync(kFullMask, base, 0);
            if (base + nidle >= total) exhausted = true;
            const uint32_t s0 = base < total ? scene_of_warp(offsets, nbatch, base, lane) : 0u;
            if (!has) {
                const unsigned long long slot = base + (unsigned long long)__popc(idle & lt_mask);
                if (slot < total) {
                    // slots of scene s are [offsets[s], offsets[s+1]) in either order
                    uint32_t s = s0;
                    while (s + 1 < nbatch && VSR_LDG(offsets + s + 1) <= slot) ++s;
                    const unsigned long long g = perm ? (unsigned long long)VSR_LDG(perm + slot)
                                                      : slot;
                    const unsigned long long lo_s = VSR_LDG(offsets + s);
                    ri = g - lo_s;
                    scp = &items[s].sc;
                    if (perm && (g < lo_s || g >= VSR_LDG(offsets + s + 1))) {
                        // a sorted slot naming a ray of another scene cannot
                        // happen with a scene-major sort; never index with it
                        atomicOr(scp->err, kErrHit);
                    } else {
                        const float4* rays = items[s].rays;
                        hp = items[s].hits;
                        r = make_ray(VSR_LDG(rays + 2 * ri), VSR_LDG(rays + 2 * ri + 1));
                        h = H();
                        has = true;
                        more = true;
                        pend = false;
                        if (!traverse_start<Q, H, false>(*scp, ip, r, h, best, st, ref, steps,
                                                         stk)) {
                            finish_miss(best);
                            hp[ri] = hit_record(best);
                            has = false;
                        }
                    }
                }
            }
        }
        const uint32_t live = __ballot_sync(kFullMask, has);
        if (live == 0u && exhausted) break;
        if (watchdog_expired(wd, ++iters, t0)) {
            if (lane == 0) atomicOr(err0, kErrTimeout);
            if (has) {
                atomicOr(scp->err, kErrTimeout);
                best.fail();
                finish_miss(best);
                hp[ri] = hit_record(best);
                has = false;
            }
            break;
        }
        if constexpr (LS) {
            if (warp_step<Q, H, false>(*scp, ip, r, h, best, st, has, ref, more, leaf, pend,
                                       steps, stk, tcol)) {
                finish_miss(best);
                hp[ri] = hit_record(best);
                has = false;
            }
        } else {
            if (has) {
                if (traverse_step<Q, H, false>(*scp, ip, r, h, best, st, ref, steps, stk)) {
                    finish_miss(best);
                    hp[ri] = hit_record(best);
                    has = false;
                }
            }
            __syncwarp();
        }
    }
}

namespace {

template <int Q, class H, int K, bool LS>
cudaError_t batch_one(const BatchLaunch& b, cudaStream_t stream, uint32_t* grid_out) {
    auto k = k_trace_batch<Q, H, K, LS>;
    const uint32_t words =
        stack_words(b.stack_max, K) + (LS ? spec_words<Q, H, false, K>(b.stack_max) : 0u);
    const size_t smem = (size_t)words * b.block * sizeof(uint32_t);
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
    uint32_t* perm = nullptr;
    if (b.sort_scratch) {
        cudaError_t e = launch_coherence_sort(b.items, b.offsets, b.sort_tiles, b.tile_scene,
                                              b.sort_ntiles, (uint32_t)b.total, b.sort_scratch,
                                              &perm, stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(b.work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    k<<<grid, b.block, smem, stream>>>(b.items, b.offsets, b.nbatch, b.ip, b.total, b.work,
                                       b.refill, b.wd, perm, b.stack_max);
    return cudaGetLastError();
}

template <int Q, class H, bool LS>
cudaError_t batch_depth(const BatchLaunch& b, cudaStream_t stream, uint32_t* grid) {
    switch (b.stack_regs) {
        case 0: return batch_one<Q, H, 0, LS>(b, stream, grid);
        case 2: return batch_one<Q, H, 2, LS>(b, stream, grid);
        case 4: return batch_one<Q, H, 4, LS>(b, stream, grid);
        default: return cudaErrorInvalidValue;
    }
}

template <int Q, class H>
cudaError_t batch_regs(const BatchLaunch& b, cudaStream_t stream, uint32_t* grid) {
    return b.lockstep ? batch_depth<Q, H, true>(b, stream, grid)
                      : batch_depth<Q, H, false>(b, stream, grid);
}

template <int Q>
cudaError_t batch_kind(const BatchLaunch& b, int kind, cudaStream_t stream, uint32_t* grid) {
    switch (kind) {
        case 0: return batch_regs<Q, IsectNone>(b, stream, grid);
        case 1: return batch_regs<Q, IsectDefault>(b, stream, grid);
        case 2: return batch_regs<Q, IsectAlphaTex>(b, stream, grid);
        case 3: return batch_regs<Q, IsectProcAlpha>(b, stream, grid);
        case 4: return batch_regs<Q, IsectCount>(b, stream, grid);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool batch_stack_regs_supported(uint32_t k) { return k == 0 || k == 2 || k == 4; }

cudaError_t launch_batch(const BatchLaunch& b, int kind, int query, cudaStream_t stream) {
    return query == kClosest ? batch_kind<kClosest>(b, kind, stream, nullptr)
                             : batch_kind<kAny>(b, kind, stream, nullptr);
}

cudaError_t batch_grid(const BatchLaunch& b, int kind, int query, uint32_t* grid) {
    return query == kClosest ? batch_kind<kClosest>(b, kind, nullptr, grid)
                             : batch_kind<kAny>(b, kind, nullptr, grid);
}

}  // namespace vsr
