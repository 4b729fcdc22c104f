// Trace kernels with the intersector injected at compile time (Section 3.2:
// the traversal receives the custom intersector as a template argument, so
// its hooks are inlined where the box and primitive tests are), one
// instantiation per query, intersector and register-stack depth K.
//
// Two launch shapes:
//   k_trace            one ray per thread, grid over the rays;
//   k_trace_persistent persistent warps that claim rays from a global counter
//                      with one atomic per warp and refill idle lanes when the
//                      number of active lanes drops below a threshold
//                      (ballot + popc), after Aila and Laine's persistent
//                      threads, which the paper's traversal scheme cites.
// and two ways for a warp's lanes to run the traversal: each lane its own
// while-while loop (traverse / traverse_step), or the warp in lock step
// (k_trace_ls, and k_trace_persistent with LS: warp_step, whose loops run
// while any lane needs them and end every pass in a warp vote; speculative
// descent for the any-hit query).  Both visit the same nodes and leaves in
// the same order per ray, so every result is the same.
//
// Each translation unit trace_k<K>.cu includes this file and instantiates
// the kernels for one K, so the instantiations compile in parallel.
#pragma once

#include "vsr_internal.h"

namespace vsr {

template <int Q, class H, bool STATS, int K>
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
    ShortStack<K> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    traverse<Q, H, STATS>(sc, ip, r, h, best, st, stk);
    hits[i] = hit_record(best);
    if (H::kCounts && counters) counters[i] = h.counters();
    if (STATS) stats[i] = make_uint4(st.boxes, st.tris, st.cands, st.texs);
}

// One ray per thread, the warp in lock step (warp_step).  Every lane stays
// in the loop to the end (lanes past the rays with busy = false), since each
// pass ends in a full-warp vote; launches are whole warps (block a multiple
// of 32).  Each pass finishes a ray or tests one leaf of every busy lane, so
// the loop ends.
template <int Q, class H, bool STATS, int K>
__device__ __forceinline__ void trace_ls(DevScene sc, IsectParams ip,
                                         const float4* __restrict__ rays, RayMap map,
                                         float4* __restrict__ hits, uint2* __restrict__ counters,
                                         uint4* __restrict__ stats,
                                         const DevScene* __restrict__ user) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long i = g < map.threads ? ray_of_thread(g, map) : map.n;
    bool busy = i < map.n;
    Ray r;
    H h;
    isect_setup(h, ip, user);
    Best best;
    Stats st;
    ShortStack<K> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    // closest-hit speculation's entry distances, after the stack columns
    float* tcol = reinterpret_cast<float*>(s_stack + stack_words(sc.stack_depth, K) * blockDim.x) +
                  threadIdx.x;
    uint32_t ref = 0, steps = 0, leaf = 0;
    bool more = false, pend = false;
    auto finish = [&]() {
        finish_miss(best);
        hits[i] = hit_record(best);
        if (H::kCounts && counters) counters[i] = h.counters();
        if (STATS) stats[i] = make_uint4(st.boxes, st.tris, st.cands, st.texs);
        busy = false;
    };
    if (busy) {
        r = make_ray(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1));
        more = traverse_start<Q, H, STATS>(sc, ip, r, h, best, st, ref, steps, stk);
        if (!more) finish();
    }
    while (__any_sync(kFullMask, busy)) {
        if (warp_step<Q, H, STATS>(sc, ip, r, h, best, st, busy, ref, more, leaf, pend, steps,
                                   stk, tcol))
            finish();
    }
}

// The kernels: the compiler's own register choice (the static intersectors),
// or a budget of MINB resident 256-thread blocks per SM (min_blocks: the
// dynamic intersector).
template <int Q, class H, bool STATS, int K>
__global__ void __launch_bounds__(256)
    k_trace_ls(DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
               float4* __restrict__ hits, uint2* __restrict__ counters,
               uint4* __restrict__ stats, const DevScene* __restrict__ user) {
    trace_ls<Q, H, STATS, K>(sc, ip, rays, map, hits, counters, stats, user);
}
template <int Q, class H, bool STATS, int K, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_trace_ls_budget(DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
                      float4* __restrict__ hits, uint2* __restrict__ counters,
                      uint4* __restrict__ stats, const DevScene* __restrict__ user) {
    trace_ls<Q, H, STATS, K>(sc, ip, rays, map, hits, counters, stats, user);
}

// k_trace under a register budget: __launch_bounds__(256, MINB) asks the
// compiler to fit MINB blocks of 256 threads per SM (at most 65536 /
// (256 MINB) registers per thread).  Used to compare static injection with
// the callback kernel at equal register budgets (trace_caps.cu); stack in
// shared memory.
template <int Q, class H, int MINB>
__global__ void __launch_bounds__(256, MINB) k_trace_cap(DevScene sc, IsectParams ip,
                                                         const float4* __restrict__ rays,
                                                         RayMap map, float4* __restrict__ hits,
                                                         uint2* __restrict__ counters) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= map.threads) return;
    const unsigned long long i = ray_of_thread(g, map);
    if (i >= map.n) return;
    const Ray r = make_ray(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1));
    H h;
    Best best;
    Stats st;
    ShortStack<0> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    traverse<Q, H, false>(sc, ip, r, h, best, st, stk);
    hits[i] = hit_record(best);
    if (H::kCounts && counters) counters[i] = h.counters();
}

// Persistent variant (persistent_rays: warps claim rays from a global
// counter and refill idle lanes).  Per-lane traversal state lives in
// registers and the shared-memory stack column; a lane that finishes its ray
// idles until the warp refills.  A counter slot past the image edge takes no
// ray.  Per-lane loops: the traversal step (traverse_step) is the only
// divergent region besides the claim, and the warp reconverges after it.
// With LS the step is warp_step, called by all 32 lanes (converged
// throughout).
template <int Q, class H, bool STATS, int K, bool LS>
__device__ __forceinline__ void trace_persistent(
    DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint2* __restrict__ counters, uint4* __restrict__ stats,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd,
    const DevScene* __restrict__ user) {
    extern __shared__ uint32_t s_stack[];
    ShortStack<K> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    // closest-hit speculation's entry distances (lock step), after the stack
    float* tcol = reinterpret_cast<float*>(s_stack + stack_words(sc.stack_depth, K) * blockDim.x) +
                  threadIdx.x;
    Ray r;
    Best best;
    Stats st;
    H h;
    uint32_t ref = 0, steps = 0, leaf = 0;
    bool more = false, pend = false;
    persistent_rays<LS>(
        map, work, refill, wd, sc.err,
        [&](unsigned long long ri) {
            r = make_ray(VSR_LDG(rays + 2 * ri), VSR_LDG(rays + 2 * ri + 1));
            h = H();
            isect_setup(h, ip, user);
            st = Stats();
            more = true;
            pend = false;
            return traverse_start<Q, H, STATS>(sc, ip, r, h, best, st, ref, steps, stk);
        },
        [&](bool busy) {
            if constexpr (LS)
                return warp_step<Q, H, STATS>(sc, ip, r, h, best, st, busy, ref, more, leaf, pend,
                                              steps, stk, tcol);
            else
                return traverse_step<Q, H, STATS>(sc, ip, r, h, best, st, ref, steps, stk);
        },
        [&](unsigned long long ri) {
            finish_miss(best);
            hits[ri] = hit_record(best);
            if (H::kCounts && counters) counters[ri] = h.counters();
            if (STATS) stats[ri] = make_uint4(st.boxes, st.tris, st.cands, st.texs);
        },
        [&]() { best.fail(); });
}

template <int Q, class H, bool STATS, int K, bool LS>
__global__ void __launch_bounds__(256) k_trace_persistent(
    DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint2* __restrict__ counters, uint4* __restrict__ stats,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd,
    const DevScene* __restrict__ user) {
    trace_persistent<Q, H, STATS, K, LS>(sc, ip, rays, map, hits, counters, stats, work, refill,
                                         wd, user);
}
template <int Q, class H, bool STATS, int K, bool LS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_trace_persistent_budget(
    DevScene sc, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint2* __restrict__ counters, uint4* __restrict__ stats,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd,
    const DevScene* __restrict__ user) {
    trace_persistent<Q, H, STATS, K, LS>(sc, ip, rays, map, hits, counters, stats, work, refill,
                                         wd, user);
}

namespace detail {

// The kernel of each shape under a budget of MINB resident 256-thread
// blocks per SM (MINB <= 1: the compiler's own register choice).
template <int Q, class H, bool STATS, int K, bool LS, int MINB>
inline auto persistent_kernel() {
    if constexpr (MINB > 1)
        return k_trace_persistent_budget<Q, H, STATS, K, LS, MINB>;
    else
        return k_trace_persistent<Q, H, STATS, K, LS>;
}
template <int Q, class H, bool STATS, int K, int MINB>
inline auto lockstep_kernel() {
    if constexpr (MINB > 1)
        return k_trace_ls_budget<Q, H, STATS, K, MINB>;
    else
        return k_trace_ls<Q, H, STATS, K>;
}

template <class Kern>
cudaError_t ensure_smem(Kern kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// The persistent launch (also the dynamic dispatcher's, with H =
// IsectDynamic and a.dyn_user the scene copy its callbacks see; the static
// intersectors ignore it), under H's register budget unless MINB says
// otherwise.
template <int Q, class H, bool STATS, int K, bool LS, int MINB = min_blocks<Q, H>()>
cudaError_t launch_persistent(const LaunchArgs& a) {
    const uint32_t words = stack_words(a.sc.stack_depth, K) +
                           (LS ? spec_words<Q, H, STATS, K>(a.sc.stack_depth) : 0u);
    const size_t smem = (size_t)words * a.block * sizeof(uint32_t);
    auto k = persistent_kernel<Q, H, STATS, K, LS, MINB>();
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid(a, reinterpret_cast<const void*>(k), smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    return with_ray_counter(a.work, a.stream, [&](unsigned long long* work) {
        k<<<grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits, a.counters,
                                             a.stats, work, a.refill, a.wd, a.dyn_user);
        return cudaGetLastError();
    });
}

// One ray per thread in lock step (budget as launch_persistent).
template <int Q, class H, bool STATS, int K, int MINB = min_blocks<Q, H>()>
cudaError_t launch_lockstep(const LaunchArgs& a) {
    const uint32_t words =
        stack_words(a.sc.stack_depth, K) + spec_words<Q, H, STATS, K>(a.sc.stack_depth);
    const size_t smem = (size_t)words * a.block * sizeof(uint32_t);
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    auto k = lockstep_kernel<Q, H, STATS, K, MINB>();
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits, a.counters,
                                                     a.stats, a.dyn_user);
    return cudaGetLastError();
}

template <int Q, class H, bool STATS, int K, bool LS>
cudaError_t launch_shape(const LaunchArgs& a) {
    if (a.persistent) return launch_persistent<Q, H, STATS, K, LS>(a);
    if constexpr (LS) {
        return launch_lockstep<Q, H, STATS, K>(a);
    } else {
        const size_t smem = (size_t)stack_words(a.sc.stack_depth, K) * a.block * sizeof(uint32_t);
        const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
        auto k = k_trace<Q, H, STATS, K>;
        cudaError_t e = ensure_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits,
                                                         a.counters, a.stats);
        return cudaGetLastError();
    }
}

template <int Q, class H, bool STATS, int K>
cudaError_t launch_one(const LaunchArgs& a) {
    return a.lockstep ? launch_shape<Q, H, STATS, K, true>(a)
                      : launch_shape<Q, H, STATS, K, false>(a);
}

template <int Q, bool STATS, int K>
cudaError_t launch_kind(const LaunchArgs& a, int kind) {
    switch (kind) {
        case 0: return launch_one<Q, IsectNone, STATS, K>(a);
        case 1: return launch_one<Q, IsectDefault, STATS, K>(a);
        case 2: return launch_one<Q, IsectAlphaTex, STATS, K>(a);
        case 3: return launch_one<Q, IsectProcAlpha, STATS, K>(a);
        case 4: return launch_one<Q, IsectCount, STATS, K>(a);
        case 5: return launch_one<Q, IsectClip, STATS, K>(a);
        default: return cudaErrorInvalidValue;
    }
}

// Launchers of one K; the measurement (stats) variant is instantiated with
// the shared-memory-only stack alone (K == 0).
template <int K>
cudaError_t launch_static_k(const LaunchArgs& a, int kind, bool stats) {
    if (stats) {
        if constexpr (K == 0) {
            return a.query == kClosest ? launch_kind<kClosest, true, 0>(a, kind)
                                       : launch_kind<kAny, true, 0>(a, kind);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    return a.query == kClosest ? launch_kind<kClosest, false, K>(a, kind)
                               : launch_kind<kAny, false, K>(a, kind);
}

}  // namespace detail

}  // namespace vsr
