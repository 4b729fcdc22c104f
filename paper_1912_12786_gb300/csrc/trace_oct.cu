// One ray per thread (per-lane while-while loops, stack in shared memory)
// with the node box test specialised to the direction octant of the warp's
// rays.  The slab test (Section 3.2, intersect(ray, aabb)) takes, per axis,
// the minimum and the maximum of the two plane distances; when the sign of
// the ray's direction along the axis is known, the entry plane and the exit
// plane are known too, and box_hit_o<OCT> reads each from its plane with
// five ALU instructions instead of eleven.  The sign pattern is a per-ray
// value, so it becomes a compile-time constant only where all rays of a warp
// share it: the warp votes once, and a warp with one octant runs the
// traversal instantiated for it; any other warp runs the generic one.  Both
// test the same boxes with the same outcome, so the nodes, leaves, hits and
// counts are those of k_trace (K = 0) bit for bit.
#include "trace_static.cuh"

namespace vsr {

namespace {

template <int Q, class H>
__global__ void __launch_bounds__(256) k_trace_oct(DevScene sc, IsectParams ip,
                                                   const float4* __restrict__ rays, RayMap map,
                                                   float4* __restrict__ hits,
                                                   uint2* __restrict__ counters) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long i = g < map.threads ? ray_of_thread(g, map) : map.n;
    const bool live = i < map.n;
    Ray r{};
    if (live) r = make_ray(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1));
    // Whether all of the warp's rays share one direction octant: each lane's
    // code against lane 0's, and one vote (launches are whole warps, since
    // the block is a multiple of 32, so every lane takes part).  The switch
    // below then takes the same case in every lane of the warp.  A form that
    // computed the set of octants with __reduce_or_sync, whose result the
    // compiler knows to be warp-uniform, gave wrong closest hits on a few
    // rays whose warps diverged (nvcc 13.0, sm_103a); this form gives the
    // generic kernel's records bit for bit.
    const uint32_t code = live ? r.negmask : 8u;
    const uint32_t first = __shfl_sync(kFullMask, code, 0);
    const bool one = __all_sync(kFullMask, !live || code == first);
    if (!live) return;
    H h;
    Best best;
    Stats st;
    ShortStack<0> stk;
    stk.init(s_stack + threadIdx.x, blockDim.x);
    const int oct = (sc.boxes_ordered && one) ? (int)code : -1;
    switch (oct) {
        case 0: traverse<Q, H, false, 0>(sc, ip, r, h, best, st, stk); break;
        case 1: traverse<Q, H, false, 1>(sc, ip, r, h, best, st, stk); break;
        case 2: traverse<Q, H, false, 2>(sc, ip, r, h, best, st, stk); break;
        case 3: traverse<Q, H, false, 3>(sc, ip, r, h, best, st, stk); break;
        case 4: traverse<Q, H, false, 4>(sc, ip, r, h, best, st, stk); break;
        case 5: traverse<Q, H, false, 5>(sc, ip, r, h, best, st, stk); break;
        case 6: traverse<Q, H, false, 6>(sc, ip, r, h, best, st, stk); break;
        case 7: traverse<Q, H, false, 7>(sc, ip, r, h, best, st, stk); break;
        default: traverse<Q, H, false, -1>(sc, ip, r, h, best, st, stk); break;
    }
    hits[i] = hit_record(best);
    if (H::kCounts && counters) counters[i] = h.counters();
}

template <int Q, class H>
cudaError_t launch_oct_one(const LaunchArgs& a) {
    const size_t smem = (size_t)stack_words(a.sc.stack_depth, 0) * a.block * sizeof(uint32_t);
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    auto k = k_trace_oct<Q, H>;
    cudaError_t e = detail::ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits, a.counters);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_oct_kind(const LaunchArgs& a, int kind) {
    switch (kind) {
        case 0: return launch_oct_one<Q, IsectNone>(a);
        case 1: return launch_oct_one<Q, IsectDefault>(a);
        case 2: return launch_oct_one<Q, IsectAlphaTex>(a);
        case 3: return launch_oct_one<Q, IsectProcAlpha>(a);
        case 4: return launch_oct_one<Q, IsectCount>(a);
        case 5: return launch_oct_one<Q, IsectClip>(a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_static_octant(const LaunchArgs& a, int kind) {
    return a.query == kClosest ? launch_oct_kind<kClosest>(a, kind)
                               : launch_oct_kind<kAny>(a, kind);
}

}  // namespace vsr
