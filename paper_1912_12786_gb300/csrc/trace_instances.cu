// Instancing: BVHs acting as compound primitives (Section 3.2).  The
// visibility query runs over a top-level BVH whose leaves hold instances; an
// instance is a mesh (a scene with its own BVH) seen through a world-to-object
// affine map, and the custom intersector is passed on to the mesh's own
// traversal, where it replaces both calls to intersect exactly as for a
// single mesh.  Closest-hit ties between instances go to the lower instance
// id, then the lower primitive id.
//
// One ray per thread (k_trace_inst), or persistent warps with per-lane
// loops (k_trace_inst_persistent).  The top-level while-while loop uses the
// bottom of the thread's shared-memory stack; a mesh traversal runs on the stack above the
// top-level entries, continuing the running result.  The intersector is
// compiled in (static dispatch) or reached through this module's callback
// tables (dynamic dispatch, dynamic.cuh), the callbacks seeing the mesh of
// the instance being traversed.
//
// Two new kernels (the render and multi-hit kernels) raised an unexplained
// misaligned-address fault on the first launch of their unchecked builds and
// ran clean with checked accesses, so this translation unit starts checked:
// every load goes through the alignment-checked path and the stores check
// their address (a skipped access is reported with its line, device error
// bit 2).
#define VSR_CHECKED_LOADS 1
#include "dynamic.cuh"

namespace vsr {

namespace {

// Running result across instances, in the interface the mesh traversal
// expects (see Best): init() leaves the result alone because it spans
// instances (reset() starts a ray), before() orders by (t, instance, prim) and
// take() records the current instance.
struct InstBest {
    float t, u, v;
    uint32_t prim, inst, cur;
    bool failed;
    __device__ __forceinline__ void reset(float tmax) {
        t = tmax;
        u = 0.0f;
        v = 0.0f;
        prim = kMiss;
        inst = kMiss;
        failed = false;
    }
    __device__ __forceinline__ void init(float) {}
    __device__ __forceinline__ bool before(float tc, uint32_t pc) const {
        return tc < t || (tc == t && (cur < inst || (cur == inst && pc < prim)));
    }
    __device__ __forceinline__ void take(float tc, float uc, float vc, uint32_t pc) {
        t = tc;
        u = uc;
        v = vc;
        prim = pc;
        inst = cur;
    }
    __device__ __forceinline__ void fail() {
        prim = kMiss;
        failed = true;
    }
};

// Ray in the instance's object space: o' = W (o, 1), d' = W (d, 0) with the
// rounding order fixed (rows of W in w0..w2, translation in .w); the interval
// is unchanged, so t is the same parameter in both spaces.
__device__ __forceinline__ Ray to_object(const float4 ra, const float4 rb, const float4 w0,
                                         const float4 w1, const float4 w2) {
    const float4 o = make_float4(
        __fmaf_rn(w0.x, ra.x, __fmaf_rn(w0.y, ra.y, __fmaf_rn(w0.z, ra.z, w0.w))),
        __fmaf_rn(w1.x, ra.x, __fmaf_rn(w1.y, ra.y, __fmaf_rn(w1.z, ra.z, w1.w))),
        __fmaf_rn(w2.x, ra.x, __fmaf_rn(w2.y, ra.y, __fmaf_rn(w2.z, ra.z, w2.w))), ra.w);
    const float4 d = make_float4(
        __fmaf_rn(w0.x, rb.x, __fmaf_rn(w0.y, rb.y, __fmul_rn(w0.z, rb.z))),
        __fmaf_rn(w1.x, rb.x, __fmaf_rn(w1.y, rb.y, __fmul_rn(w1.z, rb.z))),
        __fmaf_rn(w2.x, rb.x, __fmaf_rn(w2.y, rb.y, __fmul_rn(w2.z, rb.z))), rb.w);
    return make_ray(o, d);
}

// Write ray i's record, instance id and counters with the address checks
// (a miss as t = +inf, u = v = 0, prim and instance kMiss).
template <class H>
__device__ __forceinline__ void write_inst(InstBest best, const H& h, unsigned long long i,
                                           float4* __restrict__ hits,
                                           uint32_t* __restrict__ inst_ids,
                                           uint2* __restrict__ counters) {
    if (best.prim == kMiss) {
        best.t = __int_as_float(0x7f800000);
        best.u = 0.0f;
        best.v = 0.0f;
        best.inst = kMiss;
    }
    if (reinterpret_cast<unsigned long long>(hits + i) % 16)
        atomicCAS(&g_vsr_align_line, 0u, (unsigned)__LINE__);
    else
        hits[i] = make_float4(best.t, best.u, best.v, __uint_as_float(best.prim));
    if (inst_ids) {
        if (reinterpret_cast<unsigned long long>(inst_ids + i) % 4)
            atomicCAS(&g_vsr_align_line, 0u, (unsigned)__LINE__);
        else
            inst_ids[i] = best.inst;
    }
    if (H::kCounts && counters) {
        if (reinterpret_cast<unsigned long long>(counters + i) % 8)
            atomicCAS(&g_vsr_align_line, 0u, (unsigned)__LINE__);
        else
            counters[i] = h.counters();
    }
}

template <int Q, class H>
__global__ void __launch_bounds__(256) k_trace_inst(InstDev is, IsectParams ip,
                                                    const float4* __restrict__ rays, RayMap map,
                                                    float4* __restrict__ hits,
                                                    uint32_t* __restrict__ inst_ids,
                                                    uint2* __restrict__ counters) {
    extern __shared__ uint32_t s_stack[];
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= map.threads) return;
    const unsigned long long i = ray_of_thread(g, map);
    if (i >= map.n) return;
    const float4 ra = VSR_LDG(rays + 2 * i), rb = VSR_LDG(rays + 2 * i + 1);
    const Ray r = make_ray(ra, rb);
    uint32_t* stack = s_stack + threadIdx.x;
    const uint32_t stride = blockDim.x;
    H h;
    bind_callbacks(h, ip);
    InstBest best;
    best.reset(r.tmax);
    Stats st;
    if (is.ninst > 0) {
        h.box();
        if (box_hit(r, is.root_a, is.root_b, Q == kClosest ? best.t : r.tmax)) {
            uint32_t ref = is.root_ref, sp = 0, leaves = 0;
            for (;;) {
                // descent ends by construction (children follow their parent)
                while (!(ref & kLeafBit)) {
                    const float4* p = is.nodes + 4ull * (ref >> 2);
                    const float4 la = VSR_LDG(p), lb = VSR_LDG(p + 1), qa = VSR_LDG(p + 2),
                                 qb = VSR_LDG(p + 3);
                    const float tfar = (Q == kClosest) ? best.t : r.tmax;
                    h.box();
                    h.box();
                    const bool hl = box_hit(r, la, lb, tfar);
                    const bool hr = box_hit(r, qa, qb, tfar);
                    const uint32_t rl = __float_as_uint(la.w), rr = __float_as_uint(qa.w);
                    if (hl && hr) {
                        const bool neg = (r.negmask >> (ref & 3u)) & 1u;
                        if (sp >= is.top_depth) {  // unreachable for a validated blob
                            atomicOr(is.err, kErrStack);
                            best.fail();
                            goto done;
                        }
                        stack[sp * stride] = neg ? rl : rr;
                        ++sp;
                        ref = neg ? rr : rl;
                    } else if (hl) {
                        ref = rl;
                    } else if (hr) {
                        ref = rr;
                    } else {
                        if (sp == 0) goto done;
                        --sp;
                        ref = stack[sp * stride];
                    }
                }
                if (++leaves > is.max_leaves) {  // unreachable for a validated blob
                    atomicOr(is.err, kErrSteps);
                    best.fail();
                    goto done;
                }
                {
                    const uint32_t first = (ref >> 3) & 0x0FFFFFFFu, cnt = (ref & 7u) + 1u;
                    for (uint32_t k = 0; k < cnt; ++k) {
                        const uint32_t id = VSR_LDG(is.order + first + k);
                        const float4* w = is.inst + 4ull * id;
                        const Ray ro =
                            to_object(ra, rb, VSR_LDG(w), VSR_LDG(w + 1), VSR_LDG(w + 2));
                        const DevScene& msc = is.meshes[__float_as_uint(VSR_LDG(w + 3).x)];
                        best.cur = id;
                        set_callback_scene(h, &msc);
                        ShortStack<0> stk;
                        stk.init(stack + sp * stride, stride);
                        traverse_body<Q, H, false>(msc, ip, ro, h, best, st, stk);
                        if (best.failed || (Q == kAny && best.prim != kMiss)) goto done;
                    }
                }
                if (sp == 0) break;
                --sp;
                ref = stack[sp * stride];
            }
        }
    }
done:
    write_inst(best, h, i, hits, inst_ids, counters);
}

// The instanced traversal of k_trace_inst split into resumable steps for
// the persistent kernel.  Per lane: the top-level loop's position (`tref`
// the node to descend from when `tfresh`, `tsp` entries on the stack's
// bottom, the current top-level leaf's instances first..first+cnt with the
// next at k) and, while `in_mesh`, the current instance's mesh traversal
// (traverse_start / traverse_step on the stack above the top-level entries,
// continuing the running result).  Composed, the steps visit top-level
// nodes, instances and mesh nodes in the order of k_trace_inst, so every
// result and count is the same.
template <int Q, class H>
struct InstWalk {
    float4 ra, rb;  // the world ray as loaded
    Ray r, ro;      // world ray; the ray in the current instance's object space
    InstBest best;
    Stats st;
    H h;
    const DevScene* msc;
    ShortStack<0> mstk;
    uint32_t tref, tsp, tleaves, first, cnt, k, mref, msteps;
    bool tfresh, in_mesh;

    // Begin a ray; false when it needs no steps (no instances, root missed).
    __device__ __forceinline__ bool start(const InstDev& is, const IsectParams& ip, float4 a,
                                          float4 b) {
        ra = a;
        rb = b;
        r = make_ray(a, b);
        h = H();
        bind_callbacks(h, ip);
        best.reset(r.tmax);
        in_mesh = false;
        tfresh = true;
        tsp = 0;
        tleaves = 0;
        cnt = 0;
        k = 0;
        if (is.ninst == 0) return false;
        h.box();
        if (!box_hit(r, is.root_a, is.root_b, Q == kClosest ? best.t : r.tmax)) return false;
        tref = is.root_ref;
        return true;
    }

    // The next top-level leaf: descend from tref (or from the next stack
    // entry after a leaf).  False when the top level is exhausted or failed.
    __device__ __forceinline__ bool top_next(const InstDev& is, uint32_t* stack,
                                             uint32_t stride) {
        if (!tfresh) {
            if (tsp == 0) return false;
            --tsp;
            tref = stack[tsp * stride];
        }
        tfresh = false;
        // descent ends by construction (children follow their parent)
        while (!(tref & kLeafBit)) {
            const float4* p = is.nodes + 4ull * (tref >> 2);
            const float4 la = VSR_LDG(p), lb = VSR_LDG(p + 1), qa = VSR_LDG(p + 2),
                         qb = VSR_LDG(p + 3);
            const float tfar = (Q == kClosest) ? best.t : r.tmax;
            h.box();
            h.box();
            const bool hl = box_hit(r, la, lb, tfar);
            const bool hr = box_hit(r, qa, qb, tfar);
            const uint32_t rl = __float_as_uint(la.w), rr = __float_as_uint(qa.w);
            if (hl && hr) {
                const bool neg = (r.negmask >> (tref & 3u)) & 1u;
                if (tsp >= is.top_depth) {  // unreachable for a validated blob
                    atomicOr(is.err, kErrStack);
                    best.fail();
                    return false;
                }
                stack[tsp * stride] = neg ? rl : rr;
                ++tsp;
                tref = neg ? rr : rl;
            } else if (hl) {
                tref = rl;
            } else if (hr) {
                tref = rr;
            } else {
                if (tsp == 0) return false;
                --tsp;
                tref = stack[tsp * stride];
            }
        }
        if (++tleaves > is.max_leaves) {  // unreachable for a validated blob
            atomicOr(is.err, kErrSteps);
            best.fail();
            return false;
        }
        first = (tref >> 3) & 0x0FFFFFFFu;
        cnt = (tref & 7u) + 1u;
        k = 0;
        return true;
    }

    // One step: a step of the current mesh traversal, or the top level's
    // advance to the next instance whose mesh root the ray hits.  True when
    // the ray has finished.
    __device__ __forceinline__ bool step(const InstDev& is, const IsectParams& ip,
                                         uint32_t* stack, uint32_t stride) {
        if (in_mesh) {
            if (!traverse_step<Q, H, false>(*msc, ip, ro, h, best, st, mref, msteps, mstk))
                return false;
            in_mesh = false;
            if (best.failed || (Q == kAny && best.prim != kMiss)) return true;
        }
        for (;;) {
            while (k < cnt) {
                const uint32_t id = VSR_LDG(is.order + first + k);
                ++k;
                const float4* w = is.inst + 4ull * id;
                ro = to_object(ra, rb, VSR_LDG(w), VSR_LDG(w + 1), VSR_LDG(w + 2));
                msc = is.meshes + __float_as_uint(VSR_LDG(w + 3).x);
                best.cur = id;
                set_callback_scene(h, msc);
                mstk.init(stack + tsp * stride, stride);
                if (traverse_start<Q, H, false>(*msc, ip, ro, h, best, st, mref, msteps, mstk)) {
                    in_mesh = true;
                    return false;
                }
            }
            if (!top_next(is, stack, stride)) return true;
        }
    }
};

// Persistent instanced trace (persistent_rays: warps claim rays from a
// counter and refill idle lanes), per-lane loops over InstWalk steps.
template <int Q, class H>
__device__ __forceinline__ void trace_inst_persistent(
    InstDev is, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint32_t* __restrict__ inst_ids, uint2* __restrict__ counters,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd) {
    extern __shared__ uint32_t s_stack[];
    uint32_t* stack = s_stack + threadIdx.x;
    const uint32_t stride = blockDim.x;
    InstWalk<Q, H> w;
    persistent_rays<false>(
        map, work, refill, wd, is.err,
        [&](unsigned long long ri) {
            return w.start(is, ip, VSR_LDG(rays + 2 * ri), VSR_LDG(rays + 2 * ri + 1));
        },
        [&](bool) { return w.step(is, ip, stack, stride); },
        [&](unsigned long long ri) { write_inst(w.best, w.h, ri, hits, inst_ids, counters); },
        [&]() { w.best.fail(); });
}

// Kernel with the compiler's register choice (static intersectors) or the
// intersector's budget of MINB resident blocks per SM (min_blocks).
template <int Q, class H>
__global__ void __launch_bounds__(256) k_trace_inst_persistent(
    InstDev is, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint32_t* __restrict__ inst_ids, uint2* __restrict__ counters,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd) {
    trace_inst_persistent<Q, H>(is, ip, rays, map, hits, inst_ids, counters, work, refill, wd);
}
template <int Q, class H, int MINB>
__global__ void __launch_bounds__(256, MINB) k_trace_inst_persistent_budget(
    InstDev is, IsectParams ip, const float4* __restrict__ rays, RayMap map,
    float4* __restrict__ hits, uint32_t* __restrict__ inst_ids, uint2* __restrict__ counters,
    unsigned long long* __restrict__ work, uint32_t refill, Watchdog wd) {
    trace_inst_persistent<Q, H>(is, ip, rays, map, hits, inst_ids, counters, work, refill, wd);
}
template <int Q, class H>
inline auto inst_persistent_kernel() {
    if constexpr (min_blocks<Q, H>() > 1)
        return k_trace_inst_persistent_budget<Q, H, min_blocks<Q, H>()>;
    else
        return k_trace_inst_persistent<Q, H>;
}

template <int Q, class H>
cudaError_t inst_persistent(const InstLaunch& L) {
    const size_t smem = (size_t)L.stack_words * L.block * sizeof(uint32_t);
    auto k = inst_persistent_kernel<Q, H>();
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid =
        persistent_grid(L.block, L.blocks_per_sm, reinterpret_cast<const void*>(k), smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    return with_ray_counter(nullptr, L.stream, [&](unsigned long long* work) {
        k<<<grid, L.block, smem, L.stream>>>(L.is, L.ip, L.rays, L.map, L.hits, L.inst_ids,
                                             L.counters, work, L.refill, L.wd);
        return cudaGetLastError();
    });
}

template <int Q, class H>
cudaError_t inst_one(const InstLaunch& L) {
    if (L.persistent) return inst_persistent<Q, H>(L);
    const size_t smem = (size_t)L.stack_words * L.block * sizeof(uint32_t);
    auto k = k_trace_inst<Q, H>;
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned long long grid = (L.map.threads + L.block - 1) / L.block;
    k<<<(unsigned)grid, L.block, smem, L.stream>>>(L.is, L.ip, L.rays, L.map, L.hits, L.inst_ids,
                                                   L.counters);
    return cudaGetLastError();
}

template <int Q>
cudaError_t inst_kind(const InstLaunch& L, int kind) {
    switch (kind) {
        case 0: return inst_one<Q, IsectNone>(L);
        case 1: return inst_one<Q, IsectDefault>(L);
        case 2: return inst_one<Q, IsectAlphaTex>(L);
        case 3: return inst_one<Q, IsectProcAlpha>(L);
        case 4: return inst_one<Q, IsectCount>(L);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t instances_align_error(unsigned* line) {
    cudaError_t e = cudaMemcpyFromSymbol(line, g_vsr_align_line, sizeof(unsigned));
    if (e != cudaSuccess || *line == 0) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_vsr_align_line, &zero, sizeof(unsigned));
}

cudaError_t launch_instances(const InstLaunch& L, int kind, int query, bool dynamic) {
    if (dynamic) {
        cudaError_t e = ensure_callbacks_registered();
        if (e != cudaSuccess) return e;
        return query == kClosest ? inst_one<kClosest, IsectDynamic>(L)
                                 : inst_one<kAny, IsectDynamic>(L);
    }
    return query == kClosest ? inst_kind<kClosest>(L, kind) : inst_kind<kAny>(L, kind);
}

}  // namespace vsr
