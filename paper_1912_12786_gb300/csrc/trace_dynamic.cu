// Trace kernels with the intersector reached at run time through device
// function pointers (dynamic.cuh), the callback approach of the libraries
// that the paper contrasts with static injection (Sections 1 and 5).  The
// traversal itself is the same template as the static kernels, so the two
// variants differ only in how the intersector is reached.  Persistent and
// lock-step launches take the static launch shapes (trace_static.cuh) with
// the dynamic intersector as their template argument.
#include "dynamic.cuh"
#include "trace_static.cuh"

namespace vsr {

// Register budget: __launch_bounds__(256, MINB) fits MINB blocks of 256
// threads per SM.  The indirect calls make the callback kernel register-
// hungry (about 100 uncapped, MINB == 1), and it runs faster at higher
// occupancy despite a few spills: 3 blocks (80 registers) for closest-hit and
// 4 (64) for any-hit were the fastest of the budgets measured, and are the
// defaults.  The other budgets exist to compare with the static kernel at
// equal budgets.
template <int Q, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_trace_dyn(DevScene sc, IsectParams ip, const DevScene* __restrict__ user,
                const float4* __restrict__ rays, RayMap map, float4* __restrict__ hits,
                uint2* __restrict__ counters) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= map.threads) return;
    const unsigned long long i = ray_of_thread(g, map);
    if (i >= map.n) return;
    const Ray r = make_ray(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1));
    IsectDynamic h;
    bind_callbacks(h, ip);
    set_callback_scene(h, user);
    Best best;
    Stats st;
    ShortStack<0> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    traverse<Q, IsectDynamic, false>(sc, ip, r, h, best, st, stk);
    hits[i] = hit_record(best);
    if (counters) counters[i] = h.counters();
}

// Persistent warps (per-lane loops or lock step) and one ray per thread in
// lock step, the callbacks bound per ray by isect_setup; register budget
// MINB resident 256-thread blocks per SM (1: none).
template <int Q, int MINB>
cudaError_t launch_dynamic_budget(const LaunchArgs& a) {
    if (a.persistent)
        return a.lockstep ? detail::launch_persistent<Q, IsectDynamic, false, 0, true, MINB>(a)
                          : detail::launch_persistent<Q, IsectDynamic, false, 0, false, MINB>(a);
    return detail::launch_lockstep<Q, IsectDynamic, false, 0, MINB>(a);
}

// a.reg_cap 0: the intersector's budget (3 blocks closest hit, 4 any hit);
// 1: none; 3 or 4 blocks.
template <int Q>
cudaError_t launch_dynamic_shape(const LaunchArgs& a) {
    switch (a.reg_cap) {
        case 0: return launch_dynamic_budget<Q, min_blocks<Q, IsectDynamic>()>(a);
        case 1: return launch_dynamic_budget<Q, 1>(a);
        case 3: return launch_dynamic_budget<Q, 3>(a);
        case 4: return launch_dynamic_budget<Q, 4>(a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dynamic(const LaunchArgs& a, int kind) {
    (void)kind;
    cudaError_t e0 = ensure_callbacks_registered();
    if (e0 != cudaSuccess) return e0;
    if (a.persistent || a.lockstep)
        return a.query == kClosest ? launch_dynamic_shape<kClosest>(a)
                                   : launch_dynamic_shape<kAny>(a);
    const size_t smem = (size_t)a.sc.stack_depth * a.block * sizeof(uint32_t);
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    const uint32_t cap = a.reg_cap ? a.reg_cap : (a.query == kClosest ? 3u : 4u);
    void (*k)(DevScene, IsectParams, const DevScene*, const float4*, RayMap, float4*, uint2*);
    if (cap == 1)
        k = a.query == kClosest ? k_trace_dyn<kClosest, 1> : k_trace_dyn<kAny, 1>;
    else if (cap == 3)
        k = a.query == kClosest ? k_trace_dyn<kClosest, 3> : k_trace_dyn<kAny, 3>;
    else if (cap == 4)
        k = a.query == kClosest ? k_trace_dyn<kClosest, 4> : k_trace_dyn<kAny, 4>;
    else
        return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.dyn_user, a.rays, a.map, a.hits,
                                                     a.counters);
    return cudaGetLastError();
}

}  // namespace vsr
