// The intersector reached at run time through device function pointers: the
// callback approach that the paper contrasts with static injection (Sections
// 1 and 5).  The library checks whether a callback is registered and, if so,
// calls it indirectly for every box test, triangle test and candidate.
//
// Each translation unit that includes this header gets its own registration
// tables and registration kernel (internal linkage): device function
// pointers and __device__ tables belong to one module, so every module that
// calls through them fills its own, once per device, before its first
// dynamic launch (ensure_callbacks_registered).
#pragma once

#include <mutex>

#include "vsr_internal.h"

namespace vsr {
namespace {

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
// callback registered" and is skipped after the run-time check.  Filled on
// the device by k_dyn_register.
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
    // lock-step descent may speculate past a held leaf when the bound kind
    // has no box callback (box_hooks_silent below decides for each ray)
    static constexpr bool kMaySpeculate = true;
    // the indirect calls take 128-160 registers uncapped: the persistent and
    // lock-step kernels are compiled for 3 (closest hit) or 4 (any hit)
    // resident 256-thread blocks per SM, as the one-ray-per-thread kernel
    static constexpr int kMinBlocksClosest = 3;
    static constexpr int kMinBlocksAny = 4;
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

// Look the callbacks of intersector kind ip.kind up in the tables (the run-
// time registration check happens at each call: a null entry is skipped).
__device__ __forceinline__ void bind_callbacks(IsectDynamic& h, const IsectParams& ip) {
    const uint32_t kind = ip.kind < 5u ? ip.kind : 0u;
    h.acc = g_accept[kind];
    h.on_box = g_on_box[kind];
    h.on_tri = g_on_tri[kind];
}
template <class H>
__device__ __forceinline__ void bind_callbacks(H&, const IsectParams&) {}

// The scene a callback sees (its device copy), for the dynamic intersector.
__device__ __forceinline__ void set_callback_scene(IsectDynamic& h, const DevScene* sc) {
    h.user = sc;
}
template <class H>
__device__ __forceinline__ void set_callback_scene(H&, const DevScene*) {}

// The box hooks observe nothing when the bound kind registered no box
// callback (every kind but count).
__device__ __forceinline__ bool box_hooks_silent(const IsectDynamic& h) {
    return h.on_box == nullptr;
}

// Per-ray setup in the persistent loop: bind the callbacks and their scene.
__device__ __forceinline__ void isect_setup(IsectDynamic& h, const IsectParams& ip,
                                            const DevScene* user) {
    bind_callbacks(h, ip);
    set_callback_scene(h, user);
}

std::mutex g_dyn_reg_mutex;
bool g_dyn_registered[64] = {};

// Fill this module's tables on the current device (once per device).
cudaError_t ensure_callbacks_registered() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_dyn_reg_mutex);
    if (g_dyn_registered[dev]) return cudaSuccess;
    k_dyn_register<<<1, 1>>>();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) g_dyn_registered[dev] = true;
    return e;
}

}  // namespace
}  // namespace vsr
