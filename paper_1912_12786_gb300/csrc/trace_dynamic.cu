// Trace kernels with the intersector reached at run time through device
// function pointers, the "usual function pointer approach" of callback
// libraries that the paper contrasts with static injection (Sections 1 and
// 5): the library checks whether a callback is registered and, if so, calls
// it indirectly for every box test, triangle test and candidate.  The
// traversal itself is the same template as the static kernels, so the two
// variants differ only in how the intersector is reached.
#include <mutex>

#include "vsr_internal.h"

namespace vsr {

// The callbacks receive the intersector parameters they read by value, 16
// bytes (the clip box of the static intersectors is not among them).
struct DynParams {
    uint32_t cutoff_u8;
    float cutoff_f;
    float freq;
    uint32_t kind;
};
typedef bool (*AcceptFn)(const DevScene*, DynParams, uint32_t, float, float);
// Counting callbacks take the running count by value and return it
// incremented, so no callback ever receives a pointer into the caller's
// local memory.
typedef uint32_t (*CountFn)(uint32_t);

__device__ __forceinline__ IsectParams from_dyn(DynParams d) {
    IsectParams ip{};
    ip.cutoff_u8 = d.cutoff_u8;
    ip.cutoff_f = d.cutoff_f;
    ip.freq = d.freq;
    ip.kind = d.kind;
    return ip;
}
__device__ __noinline__ bool dyn_accept_default(const DevScene*, DynParams, uint32_t, float,
                                                float) {
    return true;
}
__device__ __noinline__ bool dyn_accept_alpha(const DevScene* sc, DynParams dp, uint32_t prim,
                                              float u, float v) {
    return alpha_tex_accept(*sc, from_dyn(dp), prim, u, v);
}
__device__ __noinline__ bool dyn_accept_proc(const DevScene* sc, DynParams dp, uint32_t prim,
                                             float u, float v) {
    return proc_alpha_accept(*sc, from_dyn(dp), prim, u, v);
}
__device__ __noinline__ uint32_t dyn_count_box(uint32_t n) { return n + 1u; }
__device__ __noinline__ uint32_t dyn_count_tri(uint32_t n) { return n + 1u; }

// Registration tables indexed by vsr_isect_kind; a null entry means "no
// callback registered" and is skipped after the run-time check.  They are
// filled on the device by k_dyn_register before the first dynamic trace.
__device__ AcceptFn g_accept[5];
__device__ CountFn g_on_box[5];
__device__ CountFn g_on_tri[5];

__global__ void k_dyn_register() {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int k = 0; k < 5; ++k) {
        g_accept[k] = nullptr;
        g_on_box[k] = nullptr;
        g_on_tri[k] = nullptr;
    }
    g_accept[1] = dyn_accept_default;
    g_accept[2] = dyn_accept_alpha;
    g_accept[3] = dyn_accept_proc;
    g_on_box[4] = dyn_count_box;
    g_on_tri[4] = dyn_count_tri;
}

struct IsectDynamic {
    static constexpr bool kCounts = true;
    static constexpr bool kTexcoords = false;
    AcceptFn acc = nullptr;
    CountFn on_box = nullptr, on_tri = nullptr;
    const DevScene* user = nullptr;
    uint32_t boxes = 0, tris = 0;
    __device__ __forceinline__ void begin(const Ray&, const IsectParams&) {}
    __device__ __forceinline__ float far(float tfar) const { return tfar; }
    __device__ __forceinline__ void box() {
        if (on_box) boxes = on_box(boxes);
    }
    __device__ __forceinline__ void tri() {
        if (on_tri) tris = on_tri(tris);
    }
    __device__ __forceinline__ bool keep(const IsectParams&, float4, float4) const { return true; }
    __device__ __forceinline__ bool accept(const DevScene&, const IsectParams& ip, uint32_t prim,
                                           float u, float v, float) {
        return acc ? acc(user, DynParams{ip.cutoff_u8, ip.cutoff_f, ip.freq, ip.kind}, prim, u, v)
                   : true;
    }
    __device__ __forceinline__ uint2 counters() const { return make_uint2(boxes, tris); }
};

// Register cap per query: the indirect calls make the callback kernel
// register-hungry (about 100 uncapped), and it runs faster at higher
// occupancy despite a few spills -- 80 registers for closest-hit and 64 for
// any-hit were the fastest of the caps measured (none, 80, 64).
template <int Q>
__global__ void __launch_bounds__(256, Q == kClosest ? 3 : 4)
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
    const uint32_t kind = ip.kind < 5u ? ip.kind : 0u;
    h.acc = g_accept[kind];
    h.on_box = g_on_box[kind];
    h.on_tri = g_on_tri[kind];
    h.user = user;
    Best best;
    Stats st;
    traverse<Q, IsectDynamic, false>(sc, ip, r, h, best, st, s_stack + threadIdx.x, blockDim.x);
    hits[i] = hit_record(best);
    if (counters) counters[i] = h.counters();
}

namespace {
std::mutex g_reg_mutex;
bool g_registered[64] = {};
}  // namespace

cudaError_t launch_dynamic(const LaunchArgs& a, int kind) {
    (void)kind;
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_reg_mutex);
        if (!g_registered[dev]) {
            k_dyn_register<<<1, 1>>>();
            e0 = cudaGetLastError();
            if (e0 == cudaSuccess) e0 = cudaDeviceSynchronize();
            if (e0 != cudaSuccess) return e0;
            g_registered[dev] = true;
        }
    }
    const size_t smem = (size_t)a.sc.stack_depth * a.block * sizeof(uint32_t);
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    auto k = (a.query == kClosest) ? k_trace_dyn<kClosest> : k_trace_dyn<kAny>;
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
