// Multi-hit query with the intersector injected at compile time: the first
// n accepted hits of each ray in ascending (t, prim) order.  This is the third
// visibility query of the library the paper extends (Section 3.1, next to
// closest-hit and any-hit), and the custom intersector reaches it the same
// way (Section 3.2).  The traversal is the closest-hit traversal with the n-th
// entry of a sorted buffer as its bound (MultiBest, in shared memory after
// the traversal stack), so the intersector is consulted for exactly the
// candidates that would enter the buffer; with n == 1 it is the closest-hit
// query.  The intersector is compiled in (static dispatch) or reached
// through this module's callback tables (dynamic dispatch, dynamic.cuh).
// Launch shapes: one ray per thread, or persistent warps with per-lane loops
// or in lock step.
//
// The first launch of the unchecked build raised a misaligned-address fault
// that reading the code did not explain (every access here uses a cudaMalloc
// or caller base and an index that keeps the access width's alignment), so,
// as for the render kernels, every load goes through the alignment-checked
// path and the hit and counter stores check their address: a misaligned
// access is skipped and its source line reported (device error bit 2).
#define VSR_CHECKED_LOADS 1
#include "dynamic.cuh"

namespace vsr {

namespace {

// Hit record of a kept entry: the triangle test again on the original
// vertices, with the edges formed as the device triangle layout forms them
// (k_build_tris), which reproduces t, u and v bit for bit.  A kept entry
// passed this test during the traversal, so it passes it again.
__device__ __forceinline__ float4 multi_record(const Ray& r, const float* __restrict__ verts,
                                               const uint32_t* __restrict__ idx, uint32_t p) {
    if (p == kMiss) return make_float4(__int_as_float(0x7f800000), 0.0f, 0.0f, __uint_as_float(p));
    const float* a = verts + 3ull * VSR_LDG(idx + 3ull * p);
    const float* b = verts + 3ull * VSR_LDG(idx + 3ull * p + 1);
    const float* c = verts + 3ull * VSR_LDG(idx + 3ull * p + 2);
    const float4 v0 = make_float4(VSR_LDG(a), VSR_LDG(a + 1), VSR_LDG(a + 2), 0.0f);
    const float4 e1 = make_float4(__fsub_rn(VSR_LDG(b), v0.x), __fsub_rn(VSR_LDG(b + 1), v0.y),
                                  __fsub_rn(VSR_LDG(b + 2), v0.z), 0.0f);
    const float4 e2 = make_float4(__fsub_rn(VSR_LDG(c), v0.x), __fsub_rn(VSR_LDG(c + 1), v0.y),
                                  __fsub_rn(VSR_LDG(c + 2), v0.z), 0.0f);
    float t = 0.0f, u = 0.0f, v = 0.0f;
    tri_test(r, v0, e1, e2, t, u, v);
    return make_float4(t, u, v, __uint_as_float(p));
}

// Write ray i's nh records (and its counters) with the address checks.
template <class H>
__device__ __forceinline__ void write_multi(const Ray& r, const float* __restrict__ verts,
                                            const uint32_t* __restrict__ idx,
                                            const MultiBest& mb, const H& h, unsigned long long i,
                                            uint32_t nh, float4* __restrict__ hits,
                                            uint2* __restrict__ counters) {
    float4* out = hits + i * nh;
    for (uint32_t k = 0; k < nh; ++k) {
        const float4 rec = multi_record(r, verts, idx, mb.pk[k * mb.stride]);
        if (reinterpret_cast<unsigned long long>(out + k) % 16)
            atomicCAS(&g_vsr_align_line, 0u, (unsigned)__LINE__);
        else
            out[k] = rec;
    }
    if (H::kCounts && counters) {
        if (reinterpret_cast<unsigned long long>(counters + i) % 8)
            atomicCAS(&g_vsr_align_line, 0u, (unsigned)__LINE__);
        else
            counters[i] = h.counters();
    }
}

template <class H>
__global__ void __launch_bounds__(256) k_trace_multi(DevScene sc, IsectParams ip,
                                                     const float* __restrict__ verts,
                                                     const uint32_t* __restrict__ idx,
                                                     const float4* __restrict__ rays, RayMap map,
                                                     uint32_t nh, float4* __restrict__ hits,
                                                     uint2* __restrict__ counters,
                                                     const DevScene* __restrict__ user) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= map.threads) return;
    const unsigned long long i = ray_of_thread(g, map);
    if (i >= map.n) return;
    const Ray r = make_ray(VSR_LDG(rays + 2 * i), VSR_LDG(rays + 2 * i + 1));
    H h;
    bind_callbacks(h, ip);
    set_callback_scene(h, user);
    // shared memory: stack (depth x block words), then the buffer's t and
    // prim columns (nh x block words each)
    const uint32_t stride = blockDim.x;
    uint32_t* buf = s_stack + sc.stack_depth * stride;
    MultiBest mb;
    mb.tk = reinterpret_cast<float*>(buf) + threadIdx.x;
    mb.pk = buf + nh * stride + threadIdx.x;
    mb.stride = stride;
    mb.n = nh;
    Stats st;
    ShortStack<0> stk;
    stk.init(s_stack + threadIdx.x, stride);
    traverse_body<kClosest, H, false>(sc, ip, r, h, mb, st, stk);
    write_multi(r, verts, idx, mb, h, i, nh, hits, counters);
}

// Persistent multi-hit (persistent_rays: warps claim rays from a counter and
// refill idle lanes): each lane's traversal resumable (traverse_start /
// traverse_step), or the warp in lock step (warp_step, whose closest-hit
// speculation works with the buffer's last entry as the far limit).  Shared
// memory per thread: stack, the buffer's t and prim columns, and with LS the
// speculation's entry distances.
template <class H, bool LS>
__device__ __forceinline__ void trace_multi_persistent(
    DevScene sc, IsectParams ip, const float* __restrict__ verts,
    const uint32_t* __restrict__ idx, const float4* __restrict__ rays, RayMap map, uint32_t nh,
    float4* __restrict__ hits, uint2* __restrict__ counters, unsigned long long* __restrict__ work,
    uint32_t refill, Watchdog wd, const DevScene* __restrict__ user) {
    extern __shared__ uint32_t s_stack[];
    const uint32_t stride = blockDim.x;
    uint32_t* buf = s_stack + sc.stack_depth * stride;
    MultiBest mb;
    mb.tk = reinterpret_cast<float*>(buf) + threadIdx.x;
    mb.pk = buf + nh * stride + threadIdx.x;
    mb.stride = stride;
    mb.n = nh;
    float* tcol = reinterpret_cast<float*>(buf + 2u * nh * stride) + threadIdx.x;
    ShortStack<0> stk;
    stk.init(s_stack + threadIdx.x, stride);
    Ray r;
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
            more = true;
            pend = false;
            return traverse_start<kClosest, H, false>(sc, ip, r, h, mb, st, ref, steps, stk);
        },
        [&](bool busy) {
            if constexpr (LS)
                return warp_step<kClosest, H, false>(sc, ip, r, h, mb, st, busy, ref, more, leaf,
                                                     pend, steps, stk, tcol);
            else
                return traverse_step<kClosest, H, false>(sc, ip, r, h, mb, st, ref, steps, stk);
        },
        [&](unsigned long long ri) { write_multi(r, verts, idx, mb, h, ri, nh, hits, counters); },
        [&]() { mb.fail(); });
}

// Kernel with the compiler's register choice (static intersectors) or the
// intersector's budget of MINB resident blocks per SM (min_blocks).
template <class H, bool LS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_trace_multi_persistent_budget(
    DevScene sc, IsectParams ip, const float* __restrict__ verts,
    const uint32_t* __restrict__ idx, const float4* __restrict__ rays, RayMap map, uint32_t nh,
    float4* __restrict__ hits, uint2* __restrict__ counters, unsigned long long* __restrict__ work,
    uint32_t refill, Watchdog wd, const DevScene* __restrict__ user) {
    trace_multi_persistent<H, LS>(sc, ip, verts, idx, rays, map, nh, hits, counters, work, refill,
                                  wd, user);
}
template <class H, bool LS>
__global__ void __launch_bounds__(256) k_trace_multi_persistent(
    DevScene sc, IsectParams ip, const float* __restrict__ verts,
    const uint32_t* __restrict__ idx, const float4* __restrict__ rays, RayMap map, uint32_t nh,
    float4* __restrict__ hits, uint2* __restrict__ counters, unsigned long long* __restrict__ work,
    uint32_t refill, Watchdog wd, const DevScene* __restrict__ user) {
    trace_multi_persistent<H, LS>(sc, ip, verts, idx, rays, map, nh, hits, counters, work, refill,
                                  wd, user);
}
template <class H, bool LS>
inline auto multi_persistent_kernel() {
    if constexpr (min_blocks<kClosest, H>() > 1)
        return k_trace_multi_persistent_budget<H, LS, min_blocks<kClosest, H>()>;
    else
        return k_trace_multi_persistent<H, LS>;
}

template <class H, bool LS>
cudaError_t multi_persistent(const LaunchArgs& a, const float* verts, const uint32_t* idx,
                             uint32_t nh) {
    const uint32_t words = a.sc.stack_depth + 2u * nh +
                           (LS ? spec_words<kClosest, H, false, 0>(a.sc.stack_depth) : 0u);
    const size_t smem = (size_t)words * a.block * sizeof(uint32_t);
    auto k = multi_persistent_kernel<H, LS>();
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = persistent_grid(a, reinterpret_cast<const void*>(k), smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    return with_ray_counter(a.work, a.stream, [&](unsigned long long* work) {
        k<<<grid, a.block, smem, a.stream>>>(a.sc, a.ip, verts, idx, a.rays, a.map, nh, a.hits,
                                             a.counters, work, a.refill, a.wd, a.dyn_user);
        return cudaGetLastError();
    });
}

template <class H>
cudaError_t multi_one(const LaunchArgs& a, const float* verts, const uint32_t* idx, uint32_t nh) {
    if (a.persistent)
        return a.lockstep ? multi_persistent<H, true>(a, verts, idx, nh)
                          : multi_persistent<H, false>(a, verts, idx, nh);
    const size_t smem = ((size_t)a.sc.stack_depth + 2u * nh) * a.block * sizeof(uint32_t);
    auto k = k_trace_multi<H>;
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, verts, idx, a.rays, a.map, nh,
                                                     a.hits, a.counters, a.dyn_user);
    return cudaGetLastError();
}

}  // namespace

cudaError_t multi_align_error(unsigned* line) {
    cudaError_t e = cudaMemcpyFromSymbol(line, g_vsr_align_line, sizeof(unsigned));
    if (e != cudaSuccess || *line == 0) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_vsr_align_line, &zero, sizeof(unsigned));
}

cudaError_t launch_multi(const LaunchArgs& a, int kind, const float* verts, const uint32_t* idx,
                         uint32_t nh, bool dynamic) {
    if (nh < 1 || nh > 16) return cudaErrorInvalidValue;
    if (dynamic) {
        cudaError_t e = ensure_callbacks_registered();
        return e != cudaSuccess ? e : multi_one<IsectDynamic>(a, verts, idx, nh);
    }
    switch (kind) {
        case 0: return multi_one<IsectNone>(a, verts, idx, nh);
        case 1: return multi_one<IsectDefault>(a, verts, idx, nh);
        case 2: return multi_one<IsectAlphaTex>(a, verts, idx, nh);
        case 3: return multi_one<IsectProcAlpha>(a, verts, idx, nh);
        case 4: return multi_one<IsectCount>(a, verts, idx, nh);
        case 5: return multi_one<IsectClip>(a, verts, idx, nh);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vsr
