// C ABI of the GPU library: scene upload, BVH load, trace dispatch, secondary
// ray generation and error reporting.  Every entry point validates its
// arguments on the host before anything is launched, so an invalid call
// returns an error instead of reaching a kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "vsr.h"
#include "vsr_internal.h"

using namespace vsr;

struct vsr_scene {
    int device = 0;
    uint32_t ntri = 0, nverts = 0, ntex = 0;
    float* d_verts = nullptr;
    uint32_t* d_idx = nullptr;
    float2* d_uvs = nullptr;
    uint32_t* d_geom = nullptr;
    TexDesc* d_tex = nullptr;
    uint8_t* d_texels = nullptr;
    float4* d_nodes = nullptr;
    float4* d_tris = nullptr;
    uint32_t num_nodes = 0, max_depth = 0;
    bool has_bvh = false;
    DevScene dev{};
    DevScene* d_user = nullptr;
    uint32_t* d_err = nullptr;  // [0] device error word; [1] refit box state
    // kept for updates: leaf order, node ids by tree level (deepest first),
    // host copies of the texture descriptors
    uint32_t* d_order = nullptr;
    uint32_t* d_levels = nullptr;
    std::vector<uint32_t> level_offsets;
    std::vector<TexDesc> h_tex;
    // launch configurations chosen by vsr_trace_tune, per (intersector kind,
    // dispatch, query); read by vsr_trace with params == NULL
    struct Tuned {
        int32_t kind, dispatch, query;
        vsr_trace_params p;
    };
    std::mutex tune_mutex;
    std::vector<Tuned> tuned;
};

namespace {

thread_local std::string g_err;

vsr_status fail(vsr_status s, const std::string& m) {
    g_err = m;
    return s;
}

vsr_status cuda_fail(cudaError_t e, const std::string& what) {
    g_err = what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? VSR_ERR_OOM : VSR_ERR_CUDA;
}

#define VSR_CUDA(call, what)                        \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            ok = false;
            return;
        }
        if (prev != d) ok = cudaSetDevice(d) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

typedef int (*AddressRangeFn)(unsigned long long*, size_t*, unsigned long long);

AddressRangeFn address_range_fn() {
    static AddressRangeFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (AddressRangeFn) nullptr;
        }
        return reinterpret_cast<AddressRangeFn>(f);
    }();
    return fn;
}

// The driver's cuPointerGetAttributes: several attributes of a pointer in
// one call (a pointer the driver does not know gets zeroed attributes).
typedef int (*PointerAttrsFn)(unsigned, int*, void**, unsigned long long);

PointerAttrsFn pointer_attrs_fn() {
    static PointerAttrsFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttributes", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PointerAttrsFn) nullptr;
        }
        return reinterpret_cast<PointerAttrsFn>(f);
    }();
    return fn;
}

// Attribute codes and the device memory type of the driver API (cuda.h).
constexpr int kAttrMemoryType = 2, kAttrIsManaged = 8, kAttrDeviceOrdinal = 9,
              kAttrRangeStart = 11, kAttrRangeSize = 12;
constexpr unsigned kMemoryTypeDevice = 2;

// A device pointer on `device`, aligned, with `bytes` inside its allocation.
// One driver query gives the memory type, managed flag, device and
// allocation range; without it the runtime's attributes and the address
// range are queried separately.
vsr_status check_dev(const void* p, int device, const char* name, size_t align, size_t bytes) {
    if (!p) return fail(VSR_ERR_ARG, std::string(name) + " is null");
    if (reinterpret_cast<uintptr_t>(p) % align)
        return fail(VSR_ERR_ARG, std::string(name) + " is not " + std::to_string(align) +
                                     "-byte aligned");
    if (PointerAttrsFn fn = pointer_attrs_fn()) {
        unsigned mem_type = 0, managed = 0;
        int ordinal = -1;
        unsigned long long start = 0;
        size_t size = 0;
        int attrs[5] = {kAttrMemoryType, kAttrIsManaged, kAttrDeviceOrdinal, kAttrRangeStart,
                        kAttrRangeSize};
        void* data[5] = {&mem_type, &managed, &ordinal, &start, &size};
        const unsigned long long addr = reinterpret_cast<uintptr_t>(p);
        if (fn(5, attrs, data, addr) == 0) {
            if (managed) return VSR_OK;
            if (mem_type != kMemoryTypeDevice)
                return fail(VSR_ERR_ARG, std::string(name) + " is not device memory");
            if (ordinal != device)
                return fail(VSR_ERR_ARG, std::string(name) + " lives on another device");
            if (size && (addr + bytes > start + size || addr + bytes < addr))
                return fail(VSR_ERR_ARG, std::string(name) + " is smaller than " +
                                             std::to_string(bytes) + " bytes");
            return VSR_OK;
        }
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(VSR_ERR_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(VSR_ERR_ARG, std::string(name) + " is not device memory");
    if (at.type == cudaMemoryTypeDevice && at.device != device)
        return fail(VSR_ERR_ARG, std::string(name) + " lives on another device");
    if (at.type == cudaMemoryTypeDevice) {
        if (AddressRangeFn fn = address_range_fn()) {
            unsigned long long base = 0;
            size_t size = 0;
            if (fn(&base, &size, (unsigned long long)reinterpret_cast<uintptr_t>(p)) == 0) {
                const unsigned long long end = base + size;
                const unsigned long long addr = reinterpret_cast<uintptr_t>(p);
                if (addr + bytes > end || addr + bytes < addr)
                    return fail(VSR_ERR_ARG, std::string(name) + " is smaller than " +
                                                 std::to_string(bytes) + " bytes");
            }
        }
    }
    return VSR_OK;
}

uint32_t texel_size(int32_t fmt) {
    return fmt == VSR_TEX_U8 ? 1u : (fmt == VSR_TEX_RGBA8 ? 4u : 16u);
}

// Convert one blob node to the packed device reference.
uint32_t node_ref(const vsr_bvh_node& n) {
    const uint32_t count = n.count_axis >> 2;
    if (count == 0) return ((n.left_or_first >> 1) << 2) | (n.count_axis & 3u);
    return kLeafBit | (n.left_or_first << 3) | (count - 1u);
}

__global__ void k_build_tris(const float* __restrict__ verts, const uint32_t* __restrict__ idx,
                             const uint32_t* __restrict__ order, uint32_t n,
                             float4* __restrict__ tris) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t p = order[s];
    const float* a = verts + 3ull * idx[3ull * p];
    const float* b = verts + 3ull * idx[3ull * p + 1];
    const float* c = verts + 3ull * idx[3ull * p + 2];
    tris[3ull * s] = make_float4(a[0], a[1], a[2], __uint_as_float(p));
    tris[3ull * s + 1] =
        make_float4(__fsub_rn(b[0], a[0]), __fsub_rn(b[1], a[1]), __fsub_rn(b[2], a[2]), 0.0f);
    tris[3ull * s + 2] =
        make_float4(__fsub_rn(c[0], a[0]), __fsub_rn(c[1], a[1]), __fsub_rn(c[2], a[2]), 0.0f);
}

__global__ void k_shadow_rays(const float4* __restrict__ rays, const float4* __restrict__ hits,
                              unsigned long long n, float lx, float ly, float lz, float eps,
                              float4* __restrict__ out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = hits[i];
    if (__float_as_uint(h.w) == kMiss) {
        out[2 * i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        out[2 * i + 1] = make_float4(lx, ly, lz, -1.0f);
        return;
    }
    const float4 a = rays[2 * i], b = rays[2 * i + 1];
    out[2 * i] = make_float4(__fmaf_rn(h.x, b.x, a.x), __fmaf_rn(h.x, b.y, a.y),
                             __fmaf_rn(h.x, b.z, a.z), eps);
    out[2 * i + 1] = make_float4(lx, ly, lz, __int_as_float(0x7f800000));
}

// Ambient-occlusion rays: spp per primary hit, cosine-distributed about the
// face normal turned against the primary direction, tangent frame of Duff et
// al. (2017), FP32.  Output ray i*spp + k.
__global__ void k_ao_rays(const float* __restrict__ verts, const uint32_t* __restrict__ idx,
                          const float4* __restrict__ rays, const float4* __restrict__ hits,
                          unsigned long long n, uint32_t spp, const float2* __restrict__ xi,
                          float tmax, float eps, uint32_t nprims, uint32_t* __restrict__ err,
                          float4* __restrict__ out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = hits[i];
    const bool bad = __float_as_uint(h.w) != kMiss && __float_as_uint(h.w) >= nprims;
    if (bad) atomicOr(err, kErrHit);
    if (__float_as_uint(h.w) == kMiss || bad) {
        for (uint32_t k = 0; k < spp; ++k) {
            out[2 * (i * spp + k)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            out[2 * (i * spp + k) + 1] = make_float4(0.0f, 0.0f, 1.0f, -1.0f);
        }
        return;
    }
    const float4 a = rays[2 * i], b = rays[2 * i + 1];
    const AoFrame f = ao_frame(verts, idx, __float_as_uint(h.w), b.x, b.y, b.z);
    const float ox = __fmaf_rn(h.x, b.x, a.x), oy = __fmaf_rn(h.x, b.y, a.y),
                oz = __fmaf_rn(h.x, b.z, a.z);
    for (uint32_t k = 0; k < spp; ++k) {
        out[2 * (i * spp + k)] = make_float4(ox, oy, oz, eps);
        out[2 * (i * spp + k) + 1] = ao_direction(f, xi[i * spp + k], tmax);
    }
}

// Occluded rays per pixel from the ambient-occlusion rays' any-hit records
// (pixel i's rays at i * spp .. i * spp + spp - 1), as integers, so the
// counts do not depend on the traversal order.
__global__ void k_ao_count(const float4* __restrict__ hits, unsigned long long n, uint32_t spp,
                           uint32_t* __restrict__ cnt) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = 0;
    for (uint32_t k = 0; k < spp; ++k) c += __float_as_uint(hits[i * spp + k].w) != kMiss;
    cnt[i] = c;
}

void free_bvh(vsr_scene* s) {
    dfree(s->d_nodes);
    dfree(s->d_tris);
    dfree(s->d_order);
    dfree(s->d_levels);
    s->level_offsets.clear();
    s->has_bvh = false;
}

// Node ids grouped by depth, deepest level first (for the bottom-up refit).
void node_levels(const vsr_bvh_node* nodes, uint32_t num_nodes, uint32_t max_depth,
                 std::vector<uint32_t>& ids, std::vector<uint32_t>& offsets) {
    std::vector<std::vector<uint32_t>> by_depth(max_depth + 1);
    std::vector<std::pair<uint32_t, uint32_t>> st{{0u, 0u}};
    while (!st.empty()) {
        auto [id, depth] = st.back();
        st.pop_back();
        by_depth[depth].push_back(id);
        const uint32_t count = nodes[id].count_axis >> 2;
        if (count == 0 && id < num_nodes) {
            st.push_back({nodes[id].left_or_first, depth + 1});
            st.push_back({nodes[id].left_or_first + 1, depth + 1});
        }
    }
    ids.clear();
    offsets.assign(1, 0u);
    for (int dpt = (int)max_depth; dpt >= 0; --dpt) {
        ids.insert(ids.end(), by_depth[dpt].begin(), by_depth[dpt].end());
        offsets.push_back((uint32_t)ids.size());
    }
}

vsr_status validate_isect(const vsr_intersector* is, int32_t query) {
    if (!is) return fail(VSR_ERR_ARG, "intersector is null");
    if (is->kind < VSR_ISECT_NONE || is->kind > VSR_ISECT_CLIP)
        return fail(VSR_ERR_ARG, "unknown intersector kind");
    if (is->dispatch != VSR_DISPATCH_STATIC && is->dispatch != VSR_DISPATCH_DYNAMIC)
        return fail(VSR_ERR_ARG, "unknown dispatch mode");
    if (is->alpha_cutoff_u8 > 256) return fail(VSR_ERR_ARG, "alpha_cutoff_u8 above 256");
    if (std::isnan(is->alpha_cutoff_f) || !std::isfinite(is->proc_freq))
        return fail(VSR_ERR_ARG, "non-finite intersector parameter");
    if (is->kind == VSR_ISECT_CLIP) {
        if (is->dispatch != VSR_DISPATCH_STATIC)
            return fail(VSR_ERR_ARG, "the clip-box intersector uses static dispatch only");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(is->clip_lo[a]) || !std::isfinite(is->clip_hi[a]) ||
                is->clip_lo[a] > is->clip_hi[a])
                return fail(VSR_ERR_ARG, "clip box must be finite with clip_lo <= clip_hi");
    }
    if (query != VSR_CLOSEST && query != VSR_ANY) return fail(VSR_ERR_ARG, "unknown query");
    return VSR_OK;
}

IsectParams isect_params(const vsr_intersector* is) {
    IsectParams ip{};
    ip.cutoff_u8 = is->alpha_cutoff_u8;
    ip.cutoff_f = is->alpha_cutoff_f;
    ip.freq = is->proc_freq;
    ip.kind = (uint32_t)is->kind;
    for (int a = 0; a < 3; ++a) {
        ip.clip_lo[a] = is->clip_lo[a];
        ip.clip_hi[a] = is->clip_hi[a];
    }
    return ip;
}

// Thread -> ray map for n rays laid out as a row-major image `width` pixels
// wide (0: buffer order).  The padded thread count is at most 8n; layouts
// whose count would not fit one launch are refused.
vsr_status make_map(uint64_t n, uint32_t width, RayMap& m) {
    constexpr uint64_t kMaxThreads = (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull;
    m = RayMap{n, n, 0u, 0u, nullptr};
    if (width == 0 || n == 0) return VSR_OK;
    if (width > n) width = (uint32_t)n;  // one partial row: the same rays
    const uint64_t rows = (n + width - 1) / width;
    const uint64_t tiles_x = (width + 3ull) / 4ull, tiles_y = (rows + 7ull) / 8ull;
    if (tiles_y > kMaxThreads / 32ull / tiles_x)
        return fail(VSR_ERR_ARG, "image_width gives too many threads for one launch");
    m.threads = tiles_x * tiles_y * 32ull;
    m.width = width;
    m.tiles_x = (uint32_t)tiles_x;
    return VSR_OK;
}

constexpr vsr_trace_params kDefaultParams{128u, 0u, 16u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
constexpr uint32_t kDefaultWatchdogMs = 60000u;

// Watchdog of a persistent loop from the launch parameters (0 ms: the
// default budget; 0xFFFFFFFF ms: none).
Watchdog make_watchdog(const vsr_trace_params& p) {
    Watchdog w{};
    w.max_iters = p.watchdog_iterations;
    const uint32_t ms = p.watchdog_ms == 0 ? kDefaultWatchdogMs : p.watchdog_ms;
    w.max_ns = ms == 0xFFFFFFFFu ? 0ull : (unsigned long long)ms * 1000000ull;
    return w;
}

// The fields of a launch that the parameters decide (validated already).
vsr_status apply_params(LaunchArgs& a, uint64_t n, const vsr_trace_params& prm) {
    vsr_status st = make_map(n, prm.image_width, a.map);
    if (st != VSR_OK) return st;
    a.block = prm.block_size;
    a.persistent = prm.persistent;
    a.refill = prm.refill_threshold;
    a.blocks_per_sm = prm.blocks_per_sm;
    a.stack_regs = prm.stack_regs;
    a.wd = make_watchdog(prm);
    a.reg_cap = prm.reg_cap_blocks;
    a.lockstep = prm.lockstep;
    a.octant = prm.octant;
    return VSR_OK;
}

vsr_status prepare_launch(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                          const vsr_intersector* is, int32_t query, vsr_hit* hits,
                          const vsr_trace_params* p, LaunchArgs& a) {
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    if (!s->has_bvh) return fail(VSR_ERR_STATE, "no BVH loaded into the scene");
    vsr_status st = validate_isect(is, query);
    if (st != VSR_OK) return st;
    vsr_trace_params prm = kDefaultParams;
    if (p) prm = *p;
    if (prm.block_size < 32 || prm.block_size > 256 || prm.block_size % 32)
        return fail(VSR_ERR_ARG, "block_size must be a multiple of 32 in 32..256");
    if (prm.persistent > 1) return fail(VSR_ERR_ARG, "persistent must be 0 or 1");
    if (prm.refill_threshold < 1 || prm.refill_threshold > 32)
        return fail(VSR_ERR_ARG, "refill_threshold must be in 1..32");
    if (prm.blocks_per_sm > 32) return fail(VSR_ERR_ARG, "blocks_per_sm above 32");
    if (!stack_regs_supported(prm.stack_regs))
        return fail(VSR_ERR_ARG, "stack_regs must be 0, 1, 2, 4 or 8");
    if (prm.ray_order != 0)
        return fail(VSR_ERR_ARG, "ray_order 1 (coherence order) is for vsr_trace and batched launches");
    if (prm.reg_cap_blocks == 2 || prm.reg_cap_blocks > 6)
        return fail(VSR_ERR_ARG, "reg_cap_blocks must be 0, 1, 3, 4, 5 or 6");
    if (prm.lockstep > 1) return fail(VSR_ERR_ARG, "lockstep must be 0 or 1");
    if (prm.lockstep && prm.reg_cap_blocks && is->dispatch == VSR_DISPATCH_STATIC)
        return fail(VSR_ERR_ARG, "lockstep 1 with static dispatch takes reg_cap_blocks 0");
    if (prm.octant > 1) return fail(VSR_ERR_ARG, "octant must be 0 or 1");
    if (prm.octant && (prm.persistent || prm.lockstep || prm.stack_regs ||
                       prm.reg_cap_blocks >= 3 || is->dispatch != VSR_DISPATCH_STATIC))
        return fail(VSR_ERR_ARG,
                    "octant 1 takes static dispatch, persistent 0, lockstep 0, stack_regs 0 "
                    "and reg_cap_blocks 0 or 1");
    if (prm.reg_cap_blocks >= 5 && is->dispatch == VSR_DISPATCH_DYNAMIC)
        return fail(VSR_ERR_ARG, "reg_cap_blocks 5 and 6 are for static dispatch");
    if (prm.reg_cap_blocks >= 3 && is->dispatch == VSR_DISPATCH_STATIC &&
        (prm.persistent || prm.stack_regs || is->kind < VSR_ISECT_DEFAULT ||
         is->kind > VSR_ISECT_COUNT))
        return fail(VSR_ERR_ARG,
                    "reg_cap_blocks 3 to 6 with static dispatch: one ray per thread, stack_regs "
                    "0, intersector default, alpha texture, procedural alpha or count");
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull)
        return fail(VSR_ERR_ARG, "too many rays for one launch");
    if (n > 0) {
        st = check_dev(rays, s->device, "rays", 16, n * sizeof(vsr_ray));
        if (st != VSR_OK) return st;
        st = check_dev(hits, s->device, "hits", 16, n * sizeof(vsr_hit));
        if (st != VSR_OK) return st;
    }
    a = LaunchArgs{};
    st = apply_params(a, n, prm);
    if (st != VSR_OK) return st;
    a.sc = s->dev;
    a.ip = isect_params(is);
    a.rays = reinterpret_cast<const float4*>(rays);
    a.n = n;
    a.hits = reinterpret_cast<float4*>(hits);
    a.query = query;
    a.work = nullptr;  // persistent launches take their own counter
    a.dyn_user = s->d_user;
    return VSR_OK;
}

// Launch `a` in the rays' coherence order (vsr_trace with ray_order 1):
// scratch from the stream-ordered allocator, the sort of the rays by origin
// and direction, the trace through the resulting permutation, the scratch
// freed on the stream.
cudaError_t launch_ordered(LaunchArgs a, int kind, bool dynamic) {
    if (a.n > coherence_sort_max_rays()) return cudaErrorInvalidValue;
    uint32_t* scratch = nullptr;
    const uint32_t ntiles = (uint32_t)((a.n + kSortTileRays - 1) / kSortTileRays);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch),
                                    coherence_sort_words((uint32_t)a.n, ntiles) * sizeof(uint32_t),
                                    a.stream);
    if (e != cudaSuccess) return e;
    uint32_t* perm = nullptr;
    e = launch_coherence_sort_scene(a.sc, a.rays, (uint32_t)a.n, scratch, &perm, a.stream);
    if (e == cudaSuccess) {
        a.map = RayMap{a.n, a.n, 0u, 0u, perm};
        e = dynamic ? launch_dynamic(a, kind) : launch_static(a, kind, false);
    }
    const cudaError_t f = cudaFreeAsync(scratch, a.stream);
    return e != cudaSuccess ? e : f;
}

// Time `c` on the launch `base` describes (the caller's rays and hit
// buffer): one warm-up launch, then the mean of two launches between CUDA
// events on base.stream.
cudaError_t time_params(const LaunchArgs& base, const vsr_trace_params& c, int kind,
                        bool dynamic, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    LaunchArgs a = base;
    if (apply_params(a, a.n, c) != VSR_OK) return cudaErrorInvalidValue;
    auto launch = [&]() {
        if (c.ray_order) return launch_ordered(a, kind, dynamic);
        return dynamic ? launch_dynamic(a, kind) : launch_static(a, kind, false);
    };
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, a.stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, a.stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    *ms *= 0.5f;
    return e;
}

// Choose a launch configuration for (scene, intersector, query) by timing
// candidates on the caller's rays, and remember it in the scene.  First pass:
// one ray per thread, per-lane loops and lock step x block 64/128/256 x
// register-stack depth 0/1/2/4/8 (static dispatch; dynamic: depth 0),
// starting from the default (128, 0, per-lane loops), and with static
// dispatch the octant-specialised box test at block 64/128/256; then the
// best of these in coherence order (its sort timed with it); last, the
// persistent launch at
// the best configuration with per-lane loops and in lock step, refill
// thresholds 1/8/16/24.  Every candidate but the coherence-order one keeps
// the caller's image_width.
vsr_status tune_trace(vsr_scene* s, const LaunchArgs& base, const vsr_intersector* is,
                      int32_t query, uint32_t image_width, vsr_trace_params* out) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    VSR_CUDA(cudaStreamIsCapturing(base.stream, &cap), "capture status");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(VSR_ERR_STATE, "cannot tune while the stream is being captured");
    const bool dynamic = is->dispatch == VSR_DISPATCH_DYNAMIC;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    VSR_CUDA(cudaEventCreate(&e0), "tune events");
    cudaError_t e = cudaEventCreate(&e1);
    vsr_trace_params best = kDefaultParams;
    best.image_width = image_width;
    float best_ms = 0.0f;
    bool have = false;
    // A candidate replaces the best only if it is at least 2% faster, and the
    // default comes first, so timing noise between near-equal candidates
    // does not change the choice from one run to the next.
    auto consider = [&](const vsr_trace_params& c) {
        float ms = 0.0f;
        if (e == cudaSuccess) e = time_params(base, c, is->kind, dynamic, e0, e1, &ms);
        if (e == cudaSuccess && (!have || ms < 0.98f * best_ms)) {
            best = c;
            best_ms = ms;
            have = true;
        }
    };
    consider(vsr_trace_params{128u, 0u, 16u, 0u, image_width, 0u, 0u, 0u, 0u, 0u, 0u});
    for (uint32_t ls : {0u, 1u})
        for (uint32_t b : {64u, 128u, 256u})
            for (uint32_t k : {0u, 1u, 2u, 4u, 8u})
                if ((!dynamic || k == 0) && !(b == 128u && k == 0u && ls == 0u))
                    consider(vsr_trace_params{b, 0u, 16u, 0u, image_width, k, 0u, 0u, 0u, 0u, ls});
    if (!dynamic)  // box tests specialised to a warp's direction octant
        for (uint32_t b : {64u, 128u, 256u}) {
            vsr_trace_params c{b, 0u, 16u, 0u, image_width, 0u, 0u, 0u, 0u, 0u, 0u};
            c.octant = 1u;
            consider(c);
        }
    if (base.n <= coherence_sort_max_rays()) {
        // the fastest one-ray-per-thread configuration in coherence order
        // (the sort is part of every timed launch)
        vsr_trace_params c = best;
        c.image_width = 0;
        c.ray_order = 1;
        consider(c);
    }
    {
        const vsr_trace_params one = best;
        for (uint32_t ls : {0u, 1u})
            for (uint32_t r : {1u, 8u, 16u, 24u}) {
                vsr_trace_params c = one;
                c.persistent = 1u;
                c.refill_threshold = r;
                c.lockstep = ls;
                c.octant = 0u;
                consider(c);
            }
    }
    if (e1) cudaEventDestroy(e1);
    cudaEventDestroy(e0);
    if (e != cudaSuccess) return cuda_fail(e, "trace tuning");
    {
        std::lock_guard<std::mutex> lock(s->tune_mutex);
        bool found = false;
        for (auto& t : s->tuned)
            if (t.kind == is->kind && t.dispatch == is->dispatch && t.query == query) {
                t.p = best;
                found = true;
            }
        if (!found) s->tuned.push_back({is->kind, is->dispatch, query, best});
    }
    *out = best;
    return VSR_OK;
}

bool tuned_params(vsr_scene* s, const vsr_intersector* is, int32_t query, vsr_trace_params* out) {
    std::lock_guard<std::mutex> lock(s->tune_mutex);
    for (const auto& t : s->tuned)
        if (t.kind == is->kind && t.dispatch == is->dispatch && t.query == query) {
            *out = t.p;
            return true;
        }
    return false;
}

}  // namespace

extern "C" {

int32_t vsr_version(void) { return 100; }

const char* vsr_last_error(void) { return g_err.c_str(); }

vsr_status vsr_scene_create_indexed(const float* verts, uint32_t nverts, const uint32_t* idx,
                                    const float* uvs, const uint32_t* geom_id, uint32_t ntri,
                                    const vsr_texture_desc* tex, uint32_t ntex,
                                    vsr_scene** out) {
    g_err.clear();
    if (!out) return fail(VSR_ERR_ARG, "out is null");
    *out = nullptr;
    if (ntri > (1u << 28)) return fail(VSR_ERR_ARG, "more than 2^28 triangles");
    if (ntri > 0 && (!verts || !idx || !uvs || !geom_id))
        return fail(VSR_ERR_ARG, "null geometry pointer");
    if (ntex > 0 && !tex) return fail(VSR_ERR_ARG, "null texture array");
    for (uint64_t k = 0; k < 3ull * ntri; ++k)
        if (idx[k] >= nverts) return fail(VSR_ERR_ARG, "vertex index out of range");
    for (uint32_t p = 0; p < ntri; ++p)
        if (geom_id[p] != VSR_NO_TEXTURE && geom_id[p] >= ntex)
            return fail(VSR_ERR_ARG, "geom_id references a missing texture");
    std::vector<TexDesc> td(ntex);
    unsigned long long texel_bytes = 0;
    for (uint32_t k = 0; k < ntex; ++k) {
        const vsr_texture_desc& t = tex[k];
        if (t.fmt < VSR_TEX_U8 || t.fmt > VSR_TEX_RGBA32F)
            return fail(VSR_ERR_ARG, "unknown texture format");
        if (t.w < 1 || t.h < 1 || t.w > 16384 || t.h > 16384)
            return fail(VSR_ERR_ARG, "texture size outside 1..16384");
        if (!t.texels) return fail(VSR_ERR_ARG, "null texels");
        td[k] = TexDesc{(uint32_t)t.fmt, t.w, t.h, 0u, texel_bytes, 0ull};
        texel_bytes += ((unsigned long long)t.w * t.h * texel_size(t.fmt) + 15ull) & ~15ull;
    }
    vsr_scene* s = new (std::nothrow) vsr_scene();
    if (!s) return fail(VSR_ERR_OOM, "host allocation failed");
    cudaGetDevice(&s->device);
    s->ntri = ntri;
    s->nverts = nverts;
    s->ntex = ntex;
    auto bail = [&](vsr_status st) {
        vsr_scene_destroy(s);
        return st;
    };
    cudaError_t e = cudaSuccess;
    if ((e = dmalloc(&s->d_verts, 3ull * nverts)) != cudaSuccess ||
        (e = dmalloc(&s->d_idx, 3ull * ntri)) != cudaSuccess ||
        (e = dmalloc(&s->d_uvs, 3ull * ntri)) != cudaSuccess ||
        (e = dmalloc(&s->d_geom, (size_t)ntri)) != cudaSuccess ||
        (e = dmalloc(&s->d_tex, (size_t)ntex)) != cudaSuccess ||
        (e = dmalloc(&s->d_texels, (size_t)texel_bytes)) != cudaSuccess ||
        (e = dmalloc(&s->d_user, 1)) != cudaSuccess || (e = dmalloc(&s->d_err, 2)) != cudaSuccess)
        return bail(cuda_fail(e, "scene allocation"));
    if ((nverts && (e = cudaMemcpy(s->d_verts, verts, 12ull * nverts, cudaMemcpyHostToDevice))) ||
        (ntri && (e = cudaMemcpy(s->d_idx, idx, 12ull * ntri, cudaMemcpyHostToDevice))) ||
        (ntri && (e = cudaMemcpy(s->d_uvs, uvs, 24ull * ntri, cudaMemcpyHostToDevice))) ||
        (ntri && (e = cudaMemcpy(s->d_geom, geom_id, 4ull * ntri, cudaMemcpyHostToDevice))) ||
        (ntex && (e = cudaMemcpy(s->d_tex, td.data(), sizeof(TexDesc) * ntex,
                                 cudaMemcpyHostToDevice))) ||
        (e = cudaMemset(s->d_err, 0, 2 * sizeof(uint32_t))))
        return bail(cuda_fail(e, "scene upload"));
    for (uint32_t k = 0; k < ntex; ++k) {
        const size_t b = (size_t)tex[k].w * tex[k].h * texel_size(tex[k].fmt);
        if ((e = cudaMemcpy(s->d_texels + td[k].offset, tex[k].texels, b,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(cuda_fail(e, "texture upload"));
    }
    s->h_tex = td;
    *out = s;
    return VSR_OK;
}

vsr_status vsr_scene_create(const float* verts_xyz, const float* uvs, const uint32_t* geom_id,
                            uint32_t ntri, const vsr_texture_desc* tex, uint32_t ntex,
                            vsr_scene** out) {
    g_err.clear();
    if (ntri > (1u << 28)) return fail(VSR_ERR_ARG, "more than 2^28 triangles");
    std::vector<uint32_t> idx(3ull * ntri);
    for (uint64_t k = 0; k < idx.size(); ++k) idx[k] = (uint32_t)k;
    return vsr_scene_create_indexed(verts_xyz, 3u * ntri, idx.data(), uvs, geom_id, ntri, tex,
                                    ntex, out);
}

vsr_status vsr_scene_destroy(vsr_scene* s) {
    if (!s) return VSR_OK;
    DeviceGuard g(s->device);
    cudaDeviceSynchronize();
    free_bvh(s);
    dfree(s->d_verts);
    dfree(s->d_idx);
    dfree(s->d_uvs);
    dfree(s->d_geom);
    dfree(s->d_tex);
    dfree(s->d_texels);
    dfree(s->d_user);
    dfree(s->d_err);
    delete s;
    return VSR_OK;
}

vsr_status vsr_bvh_load(vsr_scene* s, const void* blob, size_t bytes) {
    g_err.clear();
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    if (vsr_bvh_validate(blob, bytes) != 0)
        return fail(VSR_ERR_BLOB, std::string("invalid BVH blob: ") + vsr_bvh_last_error());
    DeviceGuard g(s->device);
    if (!g.ok) return fail(VSR_ERR_CUDA, "cannot select the scene's device");
    uint32_t hdr[8];
    std::memcpy(hdr, static_cast<const uint8_t*>(blob) + 8, sizeof(hdr));
    const uint32_t num_nodes = hdr[2], num_prims = hdr[3], max_depth = hdr[4];
    if (num_prims != s->ntri)
        return fail(VSR_ERR_BLOB, "BVH was built over a different number of triangles");
    const vsr_bvh_node* nodes =
        reinterpret_cast<const vsr_bvh_node*>(static_cast<const uint8_t*>(blob) + 64);
    const uint32_t* order = reinterpret_cast<const uint32_t*>(
        static_cast<const uint8_t*>(blob) + 64 + 32ull * num_nodes);
    free_bvh(s);
    std::vector<float4> hn(2ull * num_nodes);
    for (uint32_t i = 0; i < num_nodes; ++i) {
        const vsr_bvh_node& nd = nodes[i];
        const uint32_t ref = (i == 1) ? 0u : node_ref(nd);
        float ref_bits;
        std::memcpy(&ref_bits, &ref, sizeof(ref_bits));
        hn[2ull * i] = make_float4(nd.lo[0], nd.lo[1], nd.lo[2], ref_bits);
        hn[2ull * i + 1] = make_float4(nd.hi[0], nd.hi[1], nd.hi[2], 0.0f);
    }
    cudaError_t e;
    if ((e = dmalloc(&s->d_nodes, hn.size())) != cudaSuccess)
        return cuda_fail(e, "node allocation");
    if ((e = cudaMemcpy(s->d_nodes, hn.data(), sizeof(float4) * hn.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_bvh(s);
        return cuda_fail(e, "node upload");
    }
    if ((e = dmalloc(&s->d_tris, 3ull * num_prims)) != cudaSuccess) {
        free_bvh(s);
        return cuda_fail(e, "triangle allocation");
    }
    if (num_prims) {
        if ((e = dmalloc(&s->d_order, (size_t)num_prims)) != cudaSuccess) {
            free_bvh(s);
            return cuda_fail(e, "order allocation");
        }
        e = cudaMemcpy(s->d_order, order, 4ull * num_prims, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            k_build_tris<<<(num_prims + 255) / 256, 256>>>(s->d_verts, s->d_idx, s->d_order,
                                                            num_prims, s->d_tris);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess) {
            free_bvh(s);
            return cuda_fail(e, "triangle layout");
        }
        std::vector<uint32_t> ids;
        node_levels(nodes, num_nodes, max_depth, ids, s->level_offsets);
        if ((e = dmalloc(&s->d_levels, ids.size())) != cudaSuccess ||
            (e = cudaMemcpy(s->d_levels, ids.data(), 4ull * ids.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_bvh(s);
            return cuda_fail(e, "level list upload");
        }
    }
    s->num_nodes = num_nodes;
    s->max_depth = max_depth;
    DevScene& d = s->dev;
    d.nodes = s->d_nodes;
    d.tris = s->d_tris;
    d.uvs = s->d_uvs;
    d.geom = s->d_geom;
    d.tex = s->d_tex;
    d.texels = s->d_texels;
    d.err = s->d_err;
    d.nprims = num_prims;
    d.ntex = s->ntex;
    d.root_ref = node_ref(nodes[0]);
    d.stack_depth = max_depth > 0 ? max_depth : 1u;
    d.max_steps = num_nodes + 2u;
    d.boxes_ordered = 1u;  // the validator checked every box: finite, lo <= hi
    d.root_a = make_float4(nodes[0].lo[0], nodes[0].lo[1], nodes[0].lo[2], 0.0f);
    d.root_b = make_float4(nodes[0].hi[0], nodes[0].hi[1], nodes[0].hi[2], 0.0f);
    if ((e = cudaMemcpy(s->d_user, &d, sizeof(DevScene), cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_bvh(s);
        return cuda_fail(e, "scene descriptor upload");
    }
    s->has_bvh = true;
    return VSR_OK;
}

vsr_status vsr_trace(vsr_scene* s, const vsr_ray* rays, uint64_t n, const vsr_intersector* is,
                     int32_t query, vsr_hit* hits, uint32_t* counters,
                     const vsr_trace_params* p, vsr_stream stream) {
    g_err.clear();
    // coherence order: checked here, then the launch is prepared without it
    vsr_trace_params given;
    bool ordered = false;
    if (p && p->ray_order) {
        if (p->ray_order > 1) return fail(VSR_ERR_ARG, "ray_order must be 0 or 1");
        if (p->image_width)
            return fail(VSR_ERR_ARG, "ray_order 1 replaces the pixel-tile map: image_width 0");
        if (n > coherence_sort_max_rays())
            return fail(VSR_ERR_ARG, "too many rays for the coherence order (2^28)");
        given = *p;
        given.ray_order = 0;
        p = &given;
        ordered = true;
    }
    LaunchArgs a;
    vsr_status st = prepare_launch(s, rays, n, is, query, hits, p, a);
    if (st != VSR_OK) return st;
    vsr_trace_params tp;
    if (!p && n > 0) {
        // the configuration tuned for this scene, intersector and query; the
        // first such call tunes on its own rays unless the stream is being
        // captured, in which case the defaults apply
        bool have = tuned_params(s, is, query, &tp);
        if (!have) {
            a.stream = reinterpret_cast<cudaStream_t>(stream);
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(a.stream, &cap) != cudaSuccess) {
                cudaGetLastError();
                cap = cudaStreamCaptureStatusActive;
            }
            if (cap == cudaStreamCaptureStatusNone) {
                DeviceGuard g(s->device);
                st = tune_trace(s, a, is, query, 0u, &tp);
                if (st != VSR_OK) return st;
                have = true;
            }
        }
        if (have) {
            st = apply_params(a, n, tp);
            if (st != VSR_OK) return st;
            ordered = tp.ray_order != 0 && n <= coherence_sort_max_rays();
        }
    }
    if (counters) {
        if (is->kind != VSR_ISECT_COUNT)
            return fail(VSR_ERR_ARG, "counters are written by the COUNT intersector only");
        if (n) {
            st = check_dev(counters, s->device, "counters", 8, n * 8);
            if (st != VSR_OK) return st;
        }
        a.counters = reinterpret_cast<uint2*>(counters);
    }
    if (n == 0) return VSR_OK;
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    const bool dynamic = is->dispatch == VSR_DISPATCH_DYNAMIC;
    cudaError_t e = ordered    ? launch_ordered(a, is->kind, dynamic)
                    : dynamic ? launch_dynamic(a, is->kind)
                              : launch_static(a, is->kind, false);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    return VSR_OK;
}

vsr_status vsr_trace_tune(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                          const vsr_intersector* is, int32_t query, uint32_t image_width,
                          vsr_hit* hits, vsr_trace_params* out, vsr_stream stream) {
    g_err.clear();
    if (!out) return fail(VSR_ERR_ARG, "out is null");
    if (n == 0) return fail(VSR_ERR_ARG, "tuning needs at least one ray");
    vsr_trace_params base = kDefaultParams;
    base.image_width = image_width;
    LaunchArgs a;
    vsr_status st = prepare_launch(s, rays, n, is, query, hits, &base, a);
    if (st != VSR_OK) return st;
    if (is->kind == VSR_ISECT_COUNT) a.counters = nullptr;  // counters are not written
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    return tune_trace(s, a, is, query, image_width, out);
}

vsr_status vsr_trace_tuned_params(vsr_scene* s, const vsr_intersector* is, int32_t query,
                                  vsr_trace_params* out) {
    g_err.clear();
    if (!s || !out) return fail(VSR_ERR_ARG, "null argument");
    vsr_status st = validate_isect(is, query);
    if (st != VSR_OK) return st;
    if (!tuned_params(s, is, query, out))
        return fail(VSR_ERR_STATE, "no tuned configuration for this intersector and query");
    return VSR_OK;
}

vsr_status vsr_trace_multi(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                           const vsr_intersector* is, uint32_t max_hits, vsr_hit* hits,
                           uint32_t* counters, const vsr_trace_params* p, vsr_stream stream) {
    g_err.clear();
    if (max_hits < 1 || max_hits > 16) return fail(VSR_ERR_ARG, "max_hits must be in 1..16");
    if (p && p->lockstep && !p->persistent)
        return fail(VSR_ERR_ARG, "the multi-hit query runs lockstep 1 with persistent 1");
    if (p && p->octant)
        return fail(VSR_ERR_ARG, "octant 1 is for vsr_trace, vsr_render and vsr_path_trace");
    LaunchArgs a;
    vsr_status st = prepare_launch(s, rays, n, is, VSR_CLOSEST, hits, p, a);
    if (st != VSR_OK) return st;
    if (n) {
        st = check_dev(hits, s->device, "hits", 16, n * max_hits * sizeof(vsr_hit));
        if (st != VSR_OK) return st;
    }
    if (counters) {
        if (is->kind != VSR_ISECT_COUNT)
            return fail(VSR_ERR_ARG, "counters are written by the COUNT intersector only");
        if (n) {
            st = check_dev(counters, s->device, "counters", 8, n * 8);
            if (st != VSR_OK) return st;
        }
        a.counters = reinterpret_cast<uint2*>(counters);
    }
    if (n == 0) return VSR_OK;
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    cudaError_t e = launch_multi(a, is->kind, s->d_verts, s->d_idx, max_hits,
                                 is->dispatch == VSR_DISPATCH_DYNAMIC);
    if (e != cudaSuccess) return cuda_fail(e, "multi-hit launch");
    return VSR_OK;
}

vsr_status vsr_trace_stats(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                           const vsr_intersector* is, int32_t query, vsr_hit* hits,
                           uint32_t* stats, vsr_stream stream) {
    g_err.clear();
    LaunchArgs a;
    vsr_status st = prepare_launch(s, rays, n, is, query, hits, nullptr, a);
    if (st != VSR_OK) return st;
    if (n == 0) return VSR_OK;
    st = check_dev(stats, s->device, "stats", 16, n * 16);
    if (st != VSR_OK) return st;
    a.stats = reinterpret_cast<uint4*>(stats);
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    cudaError_t e = launch_static(a, is->kind, true);
    if (e != cudaSuccess) return cuda_fail(e, "trace_stats launch");
    return VSR_OK;
}

vsr_status vsr_make_shadow_rays(const vsr_ray* prim_rays, const vsr_hit* prim_hits, uint64_t n,
                                const float light[3], float eps, vsr_ray* out,
                                vsr_stream stream) {
    g_err.clear();
    if (!light) return fail(VSR_ERR_ARG, "light is null");
    if (!std::isfinite(eps) || !std::isfinite(light[0]) || !std::isfinite(light[1]) ||
        !std::isfinite(light[2]))
        return fail(VSR_ERR_ARG, "non-finite light or eps");
    if (n == 0) return VSR_OK;
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 256ull)
        return fail(VSR_ERR_ARG, "too many rays");
    int dev = 0;
    cudaGetDevice(&dev);
    vsr_status st = check_dev(prim_rays, dev, "prim_rays", 16, n * 32);
    if (st == VSR_OK) st = check_dev(prim_hits, dev, "prim_hits", 16, n * 16);
    if (st == VSR_OK) st = check_dev(out, dev, "out", 16, n * 32);
    if (st != VSR_OK) return st;
    k_shadow_rays<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4*>(prim_rays), reinterpret_cast<const float4*>(prim_hits), n,
        light[0], light[1], light[2], eps, reinterpret_cast<float4*>(out));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "shadow ray launch");
    return VSR_OK;
}

vsr_status vsr_make_ao_rays(vsr_scene* s, const vsr_ray* prim_rays, const vsr_hit* prim_hits,
                            uint64_t n, uint32_t spp, const float* xi, float tmax, float eps,
                            vsr_ray* out, vsr_stream stream) {
    g_err.clear();
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    if (spp < 1 || spp > 64) return fail(VSR_ERR_ARG, "spp must be in 1..64");
    if (!std::isfinite(eps) || std::isnan(tmax)) return fail(VSR_ERR_ARG, "bad eps or tmax");
    if (n == 0) return VSR_OK;
    if (n * spp > (uint64_t)(std::numeric_limits<int>::max() - 1) * 256ull)
        return fail(VSR_ERR_ARG, "too many rays");
    vsr_status st = check_dev(prim_rays, s->device, "prim_rays", 16, n * 32);
    if (st == VSR_OK) st = check_dev(prim_hits, s->device, "prim_hits", 16, n * 16);
    if (st == VSR_OK) st = check_dev(xi, s->device, "xi", 8, n * spp * 8);
    if (st == VSR_OK) st = check_dev(out, s->device, "out", 16, n * spp * 32);
    if (st != VSR_OK) return st;
    DeviceGuard g(s->device);
    k_ao_rays<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        s->d_verts, s->d_idx, reinterpret_cast<const float4*>(prim_rays),
        reinterpret_cast<const float4*>(prim_hits), n, spp, reinterpret_cast<const float2*>(xi),
        tmax, eps, s->dev.nprims, s->dev.err, reinterpret_cast<float4*>(out));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ao ray launch");
    return VSR_OK;
}

vsr_status vsr_read_probe(const void* buf, uint64_t bytes, uint32_t reps, vsr_stream stream) {
    g_err.clear();
    if (bytes == 0 || bytes % 16)
        return fail(VSR_ERR_ARG, "bytes must be a nonzero multiple of 16");
    if (reps == 0) return fail(VSR_ERR_ARG, "reps must be >= 1");
    int dev = 0;
    VSR_CUDA(cudaGetDevice(&dev), "current device");
    vsr_status st = check_dev(buf, dev, "buf", 16, bytes);
    if (st != VSR_OK) return st;
    VSR_CUDA(launch_read_probe(buf, bytes, reps, reinterpret_cast<cudaStream_t>(stream)),
             "read probe launch");
    return VSR_OK;
}

vsr_status vsr_read_probe_l1(const void* buf, uint64_t bytes, uint32_t reps,
                             uint64_t* bytes_read, vsr_stream stream) {
    g_err.clear();
    if (bytes == 0 || bytes % 16 || bytes > 65536)
        return fail(VSR_ERR_ARG, "bytes must be a nonzero multiple of 16 up to 65536");
    if (reps == 0) return fail(VSR_ERR_ARG, "reps must be >= 1");
    if (!bytes_read) return fail(VSR_ERR_ARG, "bytes_read is null");
    int dev = 0;
    VSR_CUDA(cudaGetDevice(&dev), "current device");
    vsr_status st = check_dev(buf, dev, "buf", 16, bytes);
    if (st != VSR_OK) return st;
    unsigned long long total = 0;
    VSR_CUDA(launch_read_probe_l1(buf, bytes, reps, &total, reinterpret_cast<cudaStream_t>(stream)),
             "L1 read probe launch");
    *bytes_read = total;
    return VSR_OK;
}

vsr_status vsr_get_device_error(vsr_scene* s, uint32_t* word) {
    g_err.clear();
    if (!s || !word) return fail(VSR_ERR_ARG, "null argument");
    DeviceGuard g(s->device);
    VSR_CUDA(cudaDeviceSynchronize(), "synchronise");
    VSR_CUDA(cudaMemcpy(word, s->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost),
             "read error word");
    VSR_CUDA(cudaMemset(s->d_err, 0, sizeof(uint32_t)), "clear error word");
    unsigned line = 0;
    VSR_CUDA(render_align_error(&line), "read alignment check");
    if (line) {
        *word |= kErrAlign;
        g_err = "render kernel skipped a misaligned load at render.cu/vsr_device.cuh line " +
                std::to_string(line);
    }
    line = 0;
    VSR_CUDA(path_align_error(&line), "read alignment check");
    if (line) {
        *word |= kErrAlign;
        g_err += (g_err.empty() ? "" : "; ") +
                 std::string("path kernel skipped a misaligned load at "
                             "path.cu/vsr_device.cuh line ") +
                 std::to_string(line);
    }
    line = 0;
    VSR_CUDA(multi_align_error(&line), "read alignment check");
    if (line) {
        *word |= kErrAlign;
        g_err += (g_err.empty() ? "" : "; ") +
                 std::string("multi-hit kernel skipped a misaligned access at "
                             "trace_multi.cu/vsr_device.cuh line ") +
                 std::to_string(line);
    }
    return VSR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Differentiable shading (render.cu kernels)

namespace {

vsr_status prepare_shade(const vsr_scene* s, const vsr_shade_params* sh, ShadeDev& out) {
    if (!sh) return fail(VSR_ERR_ARG, "shade params are null");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(sh->light[k]) || !std::isfinite(sh->background[k]))
            return fail(VSR_ERR_ARG, "non-finite light or background");
    if (sh->grad_tex != VSR_NO_TEXTURE && sh->grad_tex >= s->ntex)
        return fail(VSR_ERR_ARG, "grad_tex references a missing texture");
    out = ShadeDev{{sh->light[0], sh->light[1], sh->light[2]},
                   {sh->background[0], sh->background[1], sh->background[2]},
                   sh->grad_tex,
                   0u};
    return VSR_OK;
}

vsr_status prepare_render(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                          const vsr_intersector* is, const vsr_shade_params* sh,
                          const vsr_trace_params* p, LaunchArgs& a, ShadeDev& shd) {
    if (is && is->dispatch != VSR_DISPATCH_STATIC)
        return fail(VSR_ERR_ARG, "rendering uses static dispatch only");
    if (is && is->kind == VSR_ISECT_CLIP)
        return fail(VSR_ERR_ARG, "the clip-box intersector is for vsr_trace and vsr_trace_multi");
    // hits are checked by the callers; a placeholder keeps prepare_launch's
    // hit check out of the way when n == 0
    vsr_status st = prepare_launch(s, rays, 0, is, VSR_CLOSEST, nullptr, p, a);
    if (st != VSR_OK) return st;
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull)
        return fail(VSR_ERR_ARG, "too many rays for one launch");
    if (n) {
        st = check_dev(rays, s->device, "rays", 16, n * sizeof(vsr_ray));
        if (st != VSR_OK) return st;
    }
    a.n = n;
    st = make_map(n, p ? p->image_width : 0u, a.map);
    if (st != VSR_OK) return st;
    a.rays = reinterpret_cast<const float4*>(rays);
    return prepare_shade(s, sh, shd);
}

}  // namespace

extern "C" vsr_status vsr_render(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                                 const vsr_intersector* is, const vsr_shade_params* sh,
                                 float* image, vsr_hit* hits, const vsr_trace_params* p,
                                 vsr_stream stream) {
    g_err.clear();
    LaunchArgs a;
    ShadeDev shd;
    vsr_status st = prepare_render(s, rays, n, is, sh, p, a, shd);
    if (st != VSR_OK) return st;
    if (n == 0) return VSR_OK;
    st = check_dev(image, s->device, "image", 4, n * 12);
    if (st == VSR_OK && hits) st = check_dev(hits, s->device, "hits", 16, n * 16);
    if (st != VSR_OK) return st;
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    // the closest-hit trace into `hits` (or stream-ordered scratch), then the
    // shading pass from the records
    float4* h = reinterpret_cast<float4*>(hits);
    cudaError_t e = cudaSuccess;
    if (!h) e = cudaMallocAsync(reinterpret_cast<void**>(&h), n * sizeof(float4), a.stream);
    if (e != cudaSuccess) return cuda_fail(e, "render scratch");
    a.hits = h;
    e = launch_static(a, is->kind, false);
    if (e == cudaSuccess)
        e = launch_shade_hits(s->dev, shd, s->d_verts, s->d_idx, a.rays, h, n, image, a.stream);
    if (!hits) {
        const cudaError_t f = cudaFreeAsync(h, a.stream);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_trace_backward(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                                         const vsr_intersector* is,
                                         const vsr_shade_params* sh, const float* dL_dimage,
                                         float* grad_verts, float* grad_texels,
                                         const vsr_trace_params* p, vsr_stream stream) {
    g_err.clear();
    LaunchArgs a;
    ShadeDev shd;
    vsr_status st = prepare_render(s, rays, n, is, sh, p, a, shd);
    if (st != VSR_OK) return st;
    if (grad_texels) {
        if (shd.grad_tex == VSR_NO_TEXTURE || s->h_tex[shd.grad_tex].fmt != VSR_TEX_RGBA32F)
            return fail(VSR_ERR_ARG, "texel gradients need an RGBA32F grad_tex");
    }
    if (n == 0) return VSR_OK;
    st = check_dev(dL_dimage, s->device, "dL_dimage", 4, n * 12);
    if (st == VSR_OK) st = check_dev(grad_verts, s->device, "grad_verts", 4, 12ull * s->nverts);
    if (st == VSR_OK && grad_texels) {
        const TexDesc& t = s->h_tex[shd.grad_tex];
        st = check_dev(grad_texels, s->device, "grad_texels", 4, 16ull * t.w * t.h);
    }
    if (st != VSR_OK) return st;
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    // the closest hits traced again into stream-ordered scratch, then the
    // adjoint from them
    float4* h = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&h), n * sizeof(float4), a.stream);
    if (e != cudaSuccess) return cuda_fail(e, "backward scratch");
    a.hits = h;
    e = launch_static(a, is->kind, false);
    if (e == cudaSuccess)
        e = launch_render_backward_hits(s->dev, shd, s->d_verts, s->d_idx, a.rays, h, n,
                                        dL_dimage, grad_verts, grad_texels, a.stream);
    const cudaError_t f = cudaFreeAsync(h, a.stream);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_render_backward_hits(vsr_scene* s, const vsr_ray* rays,
                                               const vsr_hit* hits, uint64_t n,
                                               const vsr_shade_params* sh,
                                               const float* dL_dimage, float* grad_verts,
                                               float* grad_texels, vsr_stream stream) {
    g_err.clear();
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    if (!s->has_bvh) return fail(VSR_ERR_STATE, "no BVH loaded into the scene");
    ShadeDev shd;
    vsr_status st = prepare_shade(s, sh, shd);
    if (st != VSR_OK) return st;
    if (grad_texels) {
        if (shd.grad_tex == VSR_NO_TEXTURE || s->h_tex[shd.grad_tex].fmt != VSR_TEX_RGBA32F)
            return fail(VSR_ERR_ARG, "texel gradients need an RGBA32F grad_tex");
    }
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 256ull)
        return fail(VSR_ERR_ARG, "too many pixels for one launch");
    if (n == 0) return VSR_OK;
    st = check_dev(rays, s->device, "rays", 16, n * sizeof(vsr_ray));
    if (st == VSR_OK) st = check_dev(hits, s->device, "hits", 16, n * sizeof(vsr_hit));
    if (st == VSR_OK) st = check_dev(dL_dimage, s->device, "dL_dimage", 4, n * 12);
    if (st == VSR_OK) st = check_dev(grad_verts, s->device, "grad_verts", 4, 12ull * s->nverts);
    if (st == VSR_OK && grad_texels) {
        const TexDesc& t = s->h_tex[shd.grad_tex];
        st = check_dev(grad_texels, s->device, "grad_texels", 4, 16ull * t.w * t.h);
    }
    if (st != VSR_OK) return st;
    DeviceGuard g(s->device);
    cudaError_t e = launch_render_backward_hits(
        s->dev, shd, s->d_verts, s->d_idx, reinterpret_cast<const float4*>(rays),
        reinterpret_cast<const float4*>(hits), n, dL_dimage, grad_verts, grad_texels,
        reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    return VSR_OK;
}

namespace {

vsr_status prepare_ao(vsr_scene* s, uint64_t n, uint32_t spp, const float* xi, float tmax,
                      float eps) {
    if (spp < 1 || spp > 64) return fail(VSR_ERR_ARG, "spp must be in 1..64");
    if (!std::isfinite(eps) || std::isnan(tmax)) return fail(VSR_ERR_ARG, "bad eps or tmax");
    // one thread per occlusion ray, blocks of at least 32 threads
    if (n * spp > (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull)
        return fail(VSR_ERR_ARG, "too many occlusion rays for one launch");
    if (n) return check_dev(xi, s->device, "xi", 8, n * spp * 8);
    return VSR_OK;
}

}  // namespace

extern "C" vsr_status vsr_render_ao(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                                    const vsr_intersector* is, uint32_t spp, const float* xi,
                                    float ao_tmax, float eps, const vsr_shade_params* sh,
                                    float* image, vsr_hit* hits, float* occlusion,
                                    vsr_stream stream) {
    g_err.clear();
    LaunchArgs a;
    ShadeDev shd;
    vsr_status st = prepare_render(s, rays, n, is, sh, nullptr, a, shd);
    if (st == VSR_OK) st = prepare_ao(s, n, spp, xi, ao_tmax, eps);
    if (st != VSR_OK) return st;
    if (n == 0) return VSR_OK;
    st = check_dev(image, s->device, "image", 4, n * 12);
    if (st == VSR_OK) st = check_dev(hits, s->device, "hits", 16, n * sizeof(vsr_hit));
    if (st == VSR_OK) st = check_dev(occlusion, s->device, "occlusion", 4, n * 4);
    if (st != VSR_OK) return st;
    AoArgs ao{shd, s->d_verts, s->d_idx, spp, reinterpret_cast<const float2*>(xi), ao_tmax, eps,
              reinterpret_cast<float4*>(hits), occlusion, image, nullptr, nullptr};
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    a.hits = ao.hits;
    DeviceGuard g(s->device);
    // the primary trace at the configuration tuned for the closest-hit query
    // (its pixel tiles included), else the default
    vsr_trace_params pp;
    if (tuned_params(s, is, VSR_CLOSEST, &pp) && pp.ray_order == 0 &&
        apply_params(a, n, pp) != VSR_OK) {
        st = apply_params(a, n, kDefaultParams);
        if (st != VSR_OK) return st;
    }
    cudaError_t e = launch_static(a, is->kind, false);
    if (e != cudaSuccess) return cuda_fail(e, "ao primary trace launch");
    // occlusion: the AO rays (as vsr_make_ao_rays makes them) and their
    // any-hit records in stream-ordered scratch, traced by the trace kernels
    // at the configuration tuned for this scene, intersector and the any-hit
    // query (else the default), then counted per pixel
    const uint64_t m = n * spp;
    float4* ao_rays = nullptr;
    float4* ao_hits = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&ao_rays), m * 32, a.stream);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&ao_hits), m * 16, a.stream);
    if (e == cudaSuccess) {
        k_ao_rays<<<(unsigned)((n + 255) / 256), 256, 0, a.stream>>>(
            s->d_verts, s->d_idx, a.rays, ao.hits, n, spp, ao.xi, ao_tmax, eps, s->dev.nprims,
            s->dev.err, ao_rays);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchArgs b = a;
        b.query = VSR_ANY;
        b.rays = ao_rays;
        b.n = m;
        b.hits = ao_hits;
        b.counters = nullptr;
        vsr_trace_params tp;
        if (!tuned_params(s, is, VSR_ANY, &tp) || tp.image_width) tp = kDefaultParams;
        if (apply_params(b, m, tp) != VSR_OK) e = cudaErrorInvalidValue;
        if (e == cudaSuccess)
            e = tp.ray_order ? launch_ordered(b, is->kind, false) : launch_static(b, is->kind, false);
    }
    if (e == cudaSuccess) {
        k_ao_count<<<(unsigned)((n + 255) / 256), 256, 0, a.stream>>>(
            ao_hits, n, spp, reinterpret_cast<uint32_t*>(occlusion));
        e = cudaGetLastError();
    }
    if (ao_hits) cudaFreeAsync(ao_hits, a.stream);
    if (ao_rays) cudaFreeAsync(ao_rays, a.stream);
    if (e != cudaSuccess) return cuda_fail(e, "ao occlusion");
    e = launch_ao_shade(a.sc, ao, n, a.stream);
    if (e != cudaSuccess) return cuda_fail(e, "ao shade launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_render_ao_backward(vsr_scene* s, const vsr_hit* hits,
                                             const float* occlusion, uint64_t n,
                                             const vsr_shade_params* sh, const float* dL_dimage,
                                             float* grad_texels, vsr_stream stream) {
    g_err.clear();
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    ShadeDev shd;
    vsr_status st = prepare_shade(s, sh, shd);
    if (st != VSR_OK) return st;
    if (shd.grad_tex == VSR_NO_TEXTURE || s->h_tex[shd.grad_tex].fmt != VSR_TEX_RGBA32F)
        return fail(VSR_ERR_ARG, "texel gradients need an RGBA32F grad_tex");
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 256ull)
        return fail(VSR_ERR_ARG, "too many pixels for one launch");
    if (n == 0) return VSR_OK;
    const TexDesc& t = s->h_tex[shd.grad_tex];
    st = check_dev(hits, s->device, "hits", 16, n * sizeof(vsr_hit));
    if (st == VSR_OK) st = check_dev(occlusion, s->device, "occlusion", 4, n * 4);
    if (st == VSR_OK) st = check_dev(dL_dimage, s->device, "dL_dimage", 4, n * 12);
    if (st == VSR_OK) st = check_dev(grad_texels, s->device, "grad_texels", 4, 16ull * t.w * t.h);
    if (st != VSR_OK) return st;
    AoArgs ao{shd, nullptr, nullptr, 0, nullptr, 0.0f, 0.0f,
              reinterpret_cast<float4*>(const_cast<vsr_hit*>(hits)),
              const_cast<float*>(occlusion), nullptr, dL_dimage, grad_texels};
    DeviceGuard g(s->device);
    cudaError_t e = launch_ao_backward(s->dev, ao, n, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ao backward launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_scene_update(vsr_scene* s, const float* verts, uint32_t tex_index,
                                       const void* texels, vsr_stream stream) {
    g_err.clear();
    if (!s) return fail(VSR_ERR_ARG, "scene is null");
    vsr_status st = VSR_OK;
    if (verts && s->nverts) st = check_dev(verts, s->device, "verts", 4, 12ull * s->nverts);
    if (st != VSR_OK) return st;
    size_t tex_bytes = 0;
    if (texels) {
        if (tex_index >= s->ntex)
            return fail(VSR_ERR_ARG, "tex_index references a missing texture");
        const TexDesc& t = s->h_tex[tex_index];
        tex_bytes = (size_t)t.w * t.h * texel_size((int32_t)t.fmt);
        st = check_dev(texels, s->device, "texels", 4, tex_bytes);
        if (st != VSR_OK) return st;
    }
    DeviceGuard g(s->device);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (texels)
        VSR_CUDA(cudaMemcpyAsync(s->d_texels + s->h_tex[tex_index].offset, texels, tex_bytes,
                                 cudaMemcpyDeviceToDevice, cs),
                 "texel update");
    if (verts && s->nverts) {
        VSR_CUDA(cudaMemcpyAsync(s->d_verts, verts, 12ull * s->nverts, cudaMemcpyDeviceToDevice,
                                 cs),
                 "vertex update");
        if (s->has_bvh && s->dev.nprims) {
            // word 1 of the error allocation: set by the refit if a box comes
            // out non-finite or inverted
            VSR_CUDA(cudaMemsetAsync(s->d_err + 1, 0, sizeof(uint32_t), cs), "box state");
            k_build_tris<<<(s->dev.nprims + 255) / 256, 256, 0, cs>>>(s->d_verts, s->d_idx,
                                                                    s->d_order, s->dev.nprims,
                                                                    s->d_tris);
            VSR_CUDA(cudaGetLastError(), "triangle layout");
            VSR_CUDA(launch_refit(s->d_nodes, s->d_levels, s->level_offsets.data(),
                                  (uint32_t)s->level_offsets.size() - 1u, s->d_verts, s->d_idx,
                                  s->d_order, s->d_err + 1, cs),
                     "refit");
        }
    }
    VSR_CUDA(cudaStreamSynchronize(cs), "update");
    if (verts && s->has_bvh && s->dev.nprims) {
        float4 root[2];
        VSR_CUDA(cudaMemcpy(root, s->d_nodes, sizeof(root), cudaMemcpyDeviceToHost), "root box");
        s->dev.root_a = make_float4(root[0].x, root[0].y, root[0].z, 0.0f);
        s->dev.root_b = make_float4(root[1].x, root[1].y, root[1].z, 0.0f);
        uint32_t unordered = 0;
        VSR_CUDA(cudaMemcpy(&unordered, s->d_err + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost),
                 "box state");
        s->dev.boxes_ordered = unordered ? 0u : 1u;
        VSR_CUDA(cudaMemcpy(s->d_user, &s->dev, sizeof(DevScene), cudaMemcpyHostToDevice),
                 "scene descriptor upload");
    }
    return VSR_OK;
}

// ---------------------------------------------------------------------------
// Persistent trace whose scratch comes from a static device array.
//
// The persistent kernel needs one piece of scratch memory: the 64-bit counter
// from which warps claim rays.  vsr_trace keeps it in a word the scene
// allocated with cudaMalloc; this variant keeps it in the array below, which
// is part of the library image: every GPU that loads the library holds these
// 256 bytes until the process exits, and the entry point itself allocates
// nothing.  All calls share the array, so calls that overlap on the GPU race
// on the counter.  The counter is cleared on the caller's stream before each
// launch.

namespace {

constexpr unsigned kNoallocWords = 32;  // 256 bytes
constexpr unsigned kNoallocWordsPerCall = 1;
// the limit of any single launch here: (2^31 - 2) * 32 rays
constexpr uint64_t kNoallocMaxRays = (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull;
static_assert(kNoallocWordsPerCall <= kNoallocWords, "scratch array too small");

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocWords];

typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

// Unique id of the calling thread's current CUDA context (ids are never
// reused within a process), read through the driver's entry points.
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
struct NoallocSlot {
    unsigned long long ctx_id;
    unsigned long long* ptr;
};
NoallocSlot g_noalloc[kNoallocMaxDevices] = {};

// Device address of the scratch array on `device` (current).  Set up once
// per device: the address is looked up with cudaGetSymbolAddress on the first
// call and kept with the id of the context it belongs to.  If that context
// was destroyed and another created (cudaDeviceReset, for example), the ids
// differ and the address is looked up again, so a stale address is never
// used.  The host-side name of the array is only a stand-in.
vsr_status noalloc_scratch(int device, unsigned long long** out) {
    if (device < 0 || device >= kNoallocMaxDevices)
        return fail(VSR_ERR_ARG, "device index above the supported maximum of 64");
    unsigned long long id = 0;
    if (!current_context_id(&id))
        return fail(VSR_ERR_CUDA, "cannot identify the current CUDA context");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocSlot& slot = g_noalloc[device];
    if (!slot.ptr || slot.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        slot.ptr = static_cast<unsigned long long*>(p);
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return VSR_OK;
}

}  // namespace

extern "C" vsr_status vsr_trace_persistent_noalloc(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                                                   const vsr_intersector* is, int32_t query,
                                                   vsr_hit* hits, uint32_t* counters,
                                                   const vsr_trace_params* p,
                                                   vsr_stream stream) {
    g_err.clear();
    if (n > kNoallocMaxRays)
        return fail(VSR_ERR_ARG, "vsr_trace_persistent_noalloc: n = " + std::to_string(n) +
                                     " exceeds the maximum of (2^31 - 2) * 32 rays");
    if (is && is->dispatch != VSR_DISPATCH_STATIC)
        return fail(VSR_ERR_ARG, "vsr_trace_persistent_noalloc: static dispatch only");
    vsr_trace_params prm = kDefaultParams;
    if (p) prm = *p;
    prm.persistent = 1u;
    LaunchArgs a;
    vsr_status st = prepare_launch(s, rays, n, is, query, hits, &prm, a);
    if (st != VSR_OK) return st;
    if (counters) {
        if (is->kind != VSR_ISECT_COUNT)
            return fail(VSR_ERR_ARG, "counters are written by the COUNT intersector only");
        if (n) {
            st = check_dev(counters, s->device, "counters", 8, n * 8);
            if (st != VSR_OK) return st;
        }
        a.counters = reinterpret_cast<uint2*>(counters);
    }
    if (n == 0) return VSR_OK;
    DeviceGuard g(s->device);
    if (!g.ok) return fail(VSR_ERR_CUDA, "cannot select the scene's device");
    unsigned long long* scratch = nullptr;
    st = noalloc_scratch(s->device, &scratch);
    if (st != VSR_OK) return st;
    a.work = scratch;  // zeroed on the stream by the launcher before the kernel
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_static(a, is->kind, false);
    if (e != cudaSuccess) return cuda_fail(e, "persistent trace launch");
    return VSR_OK;
}

// ---------------------------------------------------------------------------
// Batched persistent launch: device tables built once, launch configuration
// autotuned, the launch captured in a CUDA graph and replayed.

struct vsr_batch {
    int device = 0;
    uint32_t nbatch = 0;
    unsigned long long total = 0;
    int kind = 0, query = 0;
    IsectParams ip{};
    uint32_t stack_max = 1;
    BatchItem* d_items = nullptr;
    unsigned long long* d_offsets = nullptr;
    unsigned long long* d_work = nullptr;
    vsr_trace_params params{128u, 1u, 16u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    bool tuned = false;
    uint32_t* d_sort = nullptr;  // coherence-order scratch (allocated when used)
    SortTile* d_sort_tiles = nullptr;      // the sort's scene-aligned tiles
    uint32_t* d_tile_scene = nullptr;
    std::vector<SortTile> sort_tiles;      // host copy, made at creation
    std::vector<uint32_t> tile_scene;
    uint64_t shape = 0;  // workload signature for the tuning cache
    cudaStream_t side = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

uint64_t fnv_mix(uint64_t h, uint64_t v) {
    for (int k = 0; k < 8; ++k) {
        h ^= (v >> (8 * k)) & 0xFFu;
        h *= 1099511628211ull;
    }
    return h;
}

std::mutex g_tune_mutex;
std::vector<std::pair<uint64_t, vsr_trace_params>> g_tune_cache;
bool g_tune_file_loaded = false;

const char* tune_file() {
    const char* f = std::getenv("VSR_TUNE_CACHE");
    return (f && *f) ? f : nullptr;
}

bool tune_lookup(uint64_t shape, vsr_trace_params* out) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (!g_tune_file_loaded) {
        g_tune_file_loaded = true;
        if (const char* f = tune_file()) {
            if (FILE* fp = std::fopen(f, "r")) {
                // one line per entry: "v4 <shape hex> <block> <refill> <blocks
                // per SM> <stack regs> <ray order> <lockstep>"; lines in any
                // other form are skipped
                char line[256];
                while (std::fgets(line, sizeof line, fp)) {
                    unsigned long long sh;
                    unsigned b, r, bps, k, o, ls;
                    if (std::sscanf(line, "v4 %llx %u %u %u %u %u %u", &sh, &b, &r, &bps, &k, &o,
                                    &ls) == 7 && ls <= 1u && o <= 1u)
                        g_tune_cache.push_back(
                            {sh, vsr_trace_params{b, 1u, r, bps, 0u, k, 0u, 0u, 0u, o, ls}});
                }
                std::fclose(fp);
            }
        }
    }
    for (const auto& e : g_tune_cache)
        if (e.first == shape) {
            *out = e.second;
            return true;
        }
    return false;
}

void tune_store(uint64_t shape, const vsr_trace_params& p) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.push_back({shape, p});
    if (const char* f = tune_file()) {
        if (FILE* fp = std::fopen(f, "a")) {
            std::fprintf(fp, "v4 %llx %u %u %u %u %u %u\n", (unsigned long long)shape,
                         p.block_size, p.refill_threshold, p.blocks_per_sm, p.stack_regs,
                         p.ray_order, p.lockstep);
            std::fclose(fp);
        }
    }
}

vsr_status validate_params(const vsr_trace_params& p) {
    if (p.block_size < 32 || p.block_size > 256 || p.block_size % 32)
        return fail(VSR_ERR_ARG, "block_size must be a multiple of 32 in 32..256");
    if (p.refill_threshold < 1 || p.refill_threshold > 32)
        return fail(VSR_ERR_ARG, "refill_threshold must be in 1..32");
    if (p.blocks_per_sm > 32) return fail(VSR_ERR_ARG, "blocks_per_sm above 32");
    if (!batch_stack_regs_supported(p.stack_regs))
        return fail(VSR_ERR_ARG, "batched launches take stack_regs 0, 2 or 4");
    if (p.ray_order > 1) return fail(VSR_ERR_ARG, "ray_order must be 0 or 1");
    if (p.reg_cap_blocks != 0) return fail(VSR_ERR_ARG, "batched launches take reg_cap_blocks 0");
    if (p.lockstep > 1) return fail(VSR_ERR_ARG, "lockstep must be 0 or 1");
    if (p.octant) return fail(VSR_ERR_ARG, "batched launches take octant 0");
    if (p.image_width != 0)
        return fail(VSR_ERR_ARG, "batched launches take rays in buffer order (image_width 0)");
    return VSR_OK;
}

BatchLaunch batch_launch_args(const vsr_batch* b, const vsr_trace_params& p) {
    BatchLaunch L;
    L.items = b->d_items;
    L.offsets = b->d_offsets;
    L.nbatch = b->nbatch;
    L.ip = b->ip;
    L.total = b->total;
    L.work = b->d_work;
    L.block = p.block_size;
    L.refill = p.refill_threshold;
    L.blocks_per_sm = p.blocks_per_sm;
    L.stack_max = b->stack_max;
    L.stack_regs = p.stack_regs;
    L.wd = make_watchdog(p);
    L.sort_scratch = p.ray_order ? b->d_sort : nullptr;
    L.sort_tiles = b->d_sort_tiles;
    L.tile_scene = b->d_tile_scene;
    L.sort_ntiles = (uint32_t)b->sort_tiles.size();
    L.lockstep = p.lockstep;
    return L;
}

// Coherence-order scratch of the batch (allocated once, when first needed).
cudaError_t ensure_sort_scratch(vsr_batch* b) {
    if (b->d_sort) return cudaSuccess;
    const size_t nt = b->sort_tiles.size();
    cudaError_t e = dmalloc(&b->d_sort, coherence_sort_words((uint32_t)b->total, (uint32_t)nt));
    if (e == cudaSuccess && !b->d_sort_tiles && nt) {
        e = dmalloc(&b->d_sort_tiles, nt);
        if (e == cudaSuccess) e = dmalloc(&b->d_tile_scene, nt);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_sort_tiles, b->sort_tiles.data(), sizeof(SortTile) * nt,
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_tile_scene, b->tile_scene.data(), sizeof(uint32_t) * nt,
                           cudaMemcpyHostToDevice);
    }
    return e;
}

// Whether the batch fits the coherence sort (ray and tile counts).
bool sort_fits(const vsr_batch* b) {
    return b->total > 0 && b->total <= coherence_sort_max_rays() &&
           b->sort_tiles.size() <= coherence_sort_max_tiles();
}

// Time candidate configurations on the batch itself (one warm-up run, then
// the mean of two timed runs) and keep the fastest.  First pass: block
// 64/128/256 x refill threshold 1/8/16/24/32 x blocks per SM (occupancy or
// 4), lock step, stack in shared memory; then the winner with 2 and 4 stack
// entries in registers, with per-lane loops, and in coherence order.  The
// caller's watchdog budget applies to every run.
vsr_status batch_tune(vsr_batch* b) {
    static const uint32_t blocks[] = {64u, 128u, 256u};
    static const uint32_t refills[] = {1u, 8u, 16u, 24u, 32u};
    static const uint32_t per_sm[] = {0u, 4u};
    cudaEvent_t e0, e1;
    VSR_CUDA(cudaEventCreate(&e0), "tune events");
    VSR_CUDA(cudaEventCreate(&e1), "tune events");
    float best_ms = 0.0f;
    vsr_trace_params best = b->params;
    bool have = false;
    cudaError_t e = cudaSuccess;
    auto consider = [&](const vsr_trace_params& cand) {
        if (e != cudaSuccess) return;
        const BatchLaunch L = batch_launch_args(b, cand);
        float ms[2] = {0.0f, 0.0f};
        e = launch_batch(L, b->kind, b->query, b->side);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventRecord(e0, b->side);
            if (e == cudaSuccess) e = launch_batch(L, b->kind, b->query, b->side);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->side);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k], e0, e1);
        }
        if (e != cudaSuccess) return;
        const float m = 0.5f * (ms[0] + ms[1]);
        if (!have || m < best_ms) {
            best_ms = m;
            best = cand;
            have = true;
        }
    };
    for (uint32_t bl : blocks) {
        if ((size_t)b->stack_max * bl * 4 > 200 * 1024) continue;
        for (uint32_t rf : refills)
            for (uint32_t ps : per_sm) {
                vsr_trace_params cand = b->params;
                cand.block_size = bl;
                cand.persistent = 1u;
                cand.refill_threshold = rf;
                cand.blocks_per_sm = ps;
                cand.stack_regs = 0u;
                cand.lockstep = 1u;
                consider(cand);
            }
    }
    const vsr_trace_params first = best;
    for (uint32_t k : {2u, 4u}) {
        vsr_trace_params cand = first;
        cand.stack_regs = k;
        consider(cand);
    }
    {
        vsr_trace_params cand = best;
        cand.lockstep = 0u;
        consider(cand);
    }
    // third pass: the winner in coherence order (the sort runs in every
    // timed launch), if the batch is small enough for it
    if (e == cudaSuccess && sort_fits(b)) {
        const bool had = b->d_sort != nullptr;
        e = ensure_sort_scratch(b);
        if (e == cudaSuccess) {
            vsr_trace_params cand = best;
            cand.ray_order = 1u;
            consider(cand);
            if (e == cudaSuccess && best.ray_order == 0 && !had) dfree(b->d_sort);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    b->params = best;
    b->tuned = true;
    tune_store(b->shape, best);
    return VSR_OK;
}

void batch_free(vsr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->side) cudaStreamDestroy(b->side);
    dfree(b->d_items);
    dfree(b->d_offsets);
    dfree(b->d_work);
    dfree(b->d_sort);
    dfree(b->d_sort_tiles);
    dfree(b->d_tile_scene);
    delete b;
}

}  // namespace

extern "C" vsr_status vsr_batch_create(vsr_scene* const* scenes, const vsr_ray* const* rays,
                                       const uint64_t* n, vsr_hit* const* hits, uint32_t nbatch,
                                       const vsr_intersector* is, int32_t query,
                                       const vsr_trace_params* params, vsr_batch** out) {
    g_err.clear();
    if (!out) return fail(VSR_ERR_ARG, "out is null");
    *out = nullptr;
    if (nbatch < 1 || nbatch > 65536) return fail(VSR_ERR_ARG, "nbatch must be in 1..65536");
    if (!scenes || !rays || !n || !hits) return fail(VSR_ERR_ARG, "null batch array");
    vsr_status st = validate_isect(is, query);
    if (st != VSR_OK) return st;
    if (is->dispatch != VSR_DISPATCH_STATIC)
        return fail(VSR_ERR_ARG, "batched launches use static dispatch only");
    if (is->kind == VSR_ISECT_CLIP)
        return fail(VSR_ERR_ARG, "the clip-box intersector is for vsr_trace and vsr_trace_multi");
    vsr_trace_params prm = kDefaultParams;
    prm.persistent = 1u;
    if (params) {
        prm = *params;
        prm.persistent = 1u;
        st = validate_params(prm);
        if (st != VSR_OK) return st;
    }
    if (!scenes[0]) return fail(VSR_ERR_ARG, "scene 0 is null");
    const int device = scenes[0]->device;
    std::vector<BatchItem> items(nbatch);
    std::vector<unsigned long long> offsets(nbatch + 1, 0ull);
    uint32_t stack_max = 1;
    uint64_t shape = fnv_mix(fnv_mix(fnv_mix(1469598103934665603ull, (uint64_t)is->kind),
                                     (uint64_t)query),
                             nbatch);
    for (uint32_t k = 0; k < nbatch; ++k) {
        vsr_scene* s = scenes[k];
        if (!s) return fail(VSR_ERR_ARG, "scene " + std::to_string(k) + " is null");
        if (!s->has_bvh) return fail(VSR_ERR_STATE, "scene " + std::to_string(k) + " has no BVH");
        if (s->device != device) return fail(VSR_ERR_ARG, "scenes live on different devices");
        if (n[k] > (1ull << 36)) return fail(VSR_ERR_ARG, "ray batch too large");
        if (n[k]) {
            st = check_dev(rays[k], device, "rays", 16, n[k] * sizeof(vsr_ray));
            if (st == VSR_OK) st = check_dev(hits[k], device, "hits", 16, n[k] * sizeof(vsr_hit));
            if (st != VSR_OK) return fail(st, vsr_last_error() + std::string(" (batch entry ") +
                                                  std::to_string(k) + ")");
        }
        items[k].sc = s->dev;
        items[k].rays = reinterpret_cast<const float4*>(rays[k]);
        items[k].hits = reinterpret_cast<float4*>(hits[k]);
        offsets[k + 1] = offsets[k] + n[k];
        stack_max = std::max(stack_max, s->dev.stack_depth);
        shape = fnv_mix(fnv_mix(shape, s->ntri), n[k]);
    }
    if (offsets[nbatch] > (1ull << 40)) return fail(VSR_ERR_ARG, "more than 2^40 rays in a batch");
    DeviceGuard g(device);
    if (!g.ok) return fail(VSR_ERR_CUDA, "cannot select the scenes' device");
    vsr_batch* b = new (std::nothrow) vsr_batch();
    if (!b) return fail(VSR_ERR_OOM, "host allocation failed");
    b->device = device;
    b->nbatch = nbatch;
    b->total = offsets[nbatch];
    b->kind = is->kind;
    b->query = query;
    b->ip = isect_params(is);
    b->stack_max = stack_max;
    b->shape = shape;
    b->params = prm;
    b->tuned = params != nullptr || tune_lookup(shape, &b->params);
    coherence_sort_tiles(offsets.data(), nbatch, &b->sort_tiles, &b->tile_scene);
    cudaError_t e;
    if ((e = dmalloc(&b->d_items, (size_t)nbatch)) != cudaSuccess ||
        (e = dmalloc(&b->d_offsets, (size_t)nbatch + 1)) != cudaSuccess ||
        (e = dmalloc(&b->d_work, 1)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * nbatch,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_offsets, offsets.data(), 8ull * (nbatch + 1),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch set-up");
    }
    *out = b;
    return VSR_OK;
}

extern "C" vsr_status vsr_batch_launch(vsr_batch* b, vsr_stream stream) {
    g_err.clear();
    if (!b) return fail(VSR_ERR_ARG, "batch is null");
    DeviceGuard g(b->device);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (!b->exec) {
        // first launch: inputs produced on the caller's stream must be ready
        // before tuning runs on the side stream
        VSR_CUDA(cudaStreamSynchronize(cs), "synchronise before the first batch launch");
        if (!b->tuned) {
            vsr_status st = batch_tune(b);
            if (st != VSR_OK) return st;
        }
        if (b->params.ray_order) {
            if (!sort_fits(b))
                return fail(VSR_ERR_ARG, "too many rays in the batch for the coherence order");
            VSR_CUDA(ensure_sort_scratch(b), "coherence-order scratch");
        }
        BatchLaunch L = batch_launch_args(b, b->params);
        // one plain launch resolves the grid and shared-memory attribute
        VSR_CUDA(launch_batch(L, b->kind, b->query, b->side), "batch launch");
        VSR_CUDA(cudaStreamSynchronize(b->side), "batch launch");
        VSR_CUDA(batch_grid(L, b->kind, b->query, &L.grid), "batch grid");
        VSR_CUDA(cudaStreamBeginCapture(b->side, cudaStreamCaptureModeThreadLocal), "capture");
        cudaError_t e = launch_batch(L, b->kind, b->query, b->side);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->side, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e != cudaSuccess ? e : e2, "batch graph capture");
        }
        b->graph = graph;
        VSR_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "batch graph instantiate");
    }
    VSR_CUDA(cudaGraphLaunch(b->exec, cs), "batch graph launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_batch_params(const vsr_batch* b, vsr_trace_params* out) {
    g_err.clear();
    if (!b || !out) return fail(VSR_ERR_ARG, "null argument");
    *out = b->params;
    return VSR_OK;
}

extern "C" vsr_status vsr_batch_destroy(vsr_batch* b) {
    if (!b) return VSR_OK;
    DeviceGuard g(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    return VSR_OK;
}

namespace {
struct BatchCacheEntry {
    uint64_t key;
    vsr_batch* batch;
};
std::mutex g_batch_cache_mutex;
std::vector<BatchCacheEntry> g_batch_cache;
constexpr size_t kBatchCacheSize = 8;
}  // namespace

extern "C" vsr_status vsr_trace_batch(vsr_scene* const* scenes, const vsr_ray* const* rays,
                                      const uint64_t* n, vsr_hit* const* hits, uint32_t nbatch,
                                      const vsr_intersector* is, int32_t query,
                                      const vsr_trace_params* params, vsr_stream stream) {
    g_err.clear();
    if (!scenes || !rays || !n || !hits || !is || nbatch < 1 || nbatch > 65536)
        return fail(VSR_ERR_ARG, "invalid batch arguments");
    uint64_t key = 1469598103934665603ull;
    for (uint32_t k = 0; k < nbatch; ++k) {
        key = fnv_mix(key, reinterpret_cast<uintptr_t>(scenes[k]));
        key = fnv_mix(key, reinterpret_cast<uintptr_t>(rays[k]));
        key = fnv_mix(key, reinterpret_cast<uintptr_t>(hits[k]));
        key = fnv_mix(key, n[k]);
    }
    key = fnv_mix(fnv_mix(fnv_mix(key, nbatch), (uint64_t)query),
                  ((uint64_t)(uint32_t)is->kind << 32) | (uint32_t)is->dispatch);
    uint32_t fbits;
    std::memcpy(&fbits, &is->alpha_cutoff_f, 4);
    key = fnv_mix(fnv_mix(key, is->alpha_cutoff_u8), fbits);
    std::memcpy(&fbits, &is->proc_freq, 4);
    key = fnv_mix(key, fbits);
    if (params) {
        key = fnv_mix(fnv_mix(key, params->block_size),
                      ((uint64_t)params->refill_threshold << 32) | params->blocks_per_sm);
        key = fnv_mix(fnv_mix(key, ((uint64_t)params->stack_regs << 32) | params->ray_order),
                      ((uint64_t)params->watchdog_iterations << 32) | params->watchdog_ms);
        key = fnv_mix(key, params->lockstep);
    }
    vsr_batch* b = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_batch_cache_mutex);
        for (auto& e : g_batch_cache)
            if (e.key == key) b = e.batch;
        if (!b) {
            vsr_status st = vsr_batch_create(scenes, rays, n, hits, nbatch, is, query, params, &b);
            if (st != VSR_OK) return st;
            if (g_batch_cache.size() >= kBatchCacheSize) {
                vsr_batch_destroy(g_batch_cache.front().batch);
                g_batch_cache.erase(g_batch_cache.begin());
            }
            g_batch_cache.push_back({key, b});
        }
    }
    return vsr_batch_launch(b, stream);
}

// ---------------------------------------------------------------------------
// Instancing: BVHs as compound primitives of a top-level BVH (Section 3.2).
// The instance set snapshots the meshes' device descriptors; the meshes must
// outlive it and keep their geometry and BVH while it exists.

struct vsr_instances {
    int device = 0;
    uint32_t nmeshes = 0, ninst = 0;
    DevScene* d_meshes = nullptr;
    float4* d_inst = nullptr;
    float4* d_nodes = nullptr;
    uint32_t* d_order = nullptr;
    uint32_t* d_err = nullptr;
    InstDev dev{};
    uint32_t stack_words = 1;
};

namespace {

void free_instances(vsr_instances* x) {
    dfree(x->d_meshes);
    dfree(x->d_inst);
    dfree(x->d_nodes);
    dfree(x->d_order);
    dfree(x->d_err);
    delete x;
}

}  // namespace

extern "C" vsr_status vsr_instances_create(vsr_scene* const* meshes, uint32_t nmeshes,
                                           const uint32_t* inst_mesh,
                                           const float* world_to_object, uint32_t ninst,
                                           const void* top_blob, size_t top_bytes,
                                           vsr_instances** out) {
    g_err.clear();
    if (!out) return fail(VSR_ERR_ARG, "out is null");
    *out = nullptr;
    if (!meshes || nmeshes < 1 || nmeshes > 65536)
        return fail(VSR_ERR_ARG, "nmeshes must be in 1..65536 with a mesh array");
    if (ninst > (1u << 28)) return fail(VSR_ERR_ARG, "more than 2^28 instances");
    if (ninst && (!inst_mesh || !world_to_object))
        return fail(VSR_ERR_ARG, "null instance arrays");
    uint32_t mesh_depth = 1;
    for (uint32_t m = 0; m < nmeshes; ++m) {
        if (!meshes[m]) return fail(VSR_ERR_ARG, "mesh " + std::to_string(m) + " is null");
        if (!meshes[m]->has_bvh)
            return fail(VSR_ERR_STATE, "mesh " + std::to_string(m) + " has no BVH loaded");
        if (meshes[m]->device != meshes[0]->device)
            return fail(VSR_ERR_ARG, "meshes live on different devices");
        mesh_depth = std::max(mesh_depth, meshes[m]->dev.stack_depth);
    }
    for (uint32_t i = 0; i < ninst; ++i) {
        if (inst_mesh[i] >= nmeshes)
            return fail(VSR_ERR_ARG, "instance " + std::to_string(i) + " names a missing mesh");
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(world_to_object[12ull * i + k]))
                return fail(VSR_ERR_ARG, "instance " + std::to_string(i) +
                                             " has a non-finite transform");
    }
    if (vsr_bvh_validate(top_blob, top_bytes) != 0)
        return fail(VSR_ERR_BLOB, std::string("invalid top-level blob: ") + vsr_bvh_last_error());
    uint32_t hdr[8];
    std::memcpy(hdr, static_cast<const uint8_t*>(top_blob) + 8, sizeof(hdr));
    const uint32_t num_nodes = hdr[2], num_prims = hdr[3], max_depth = hdr[4];
    if (num_prims != ninst)
        return fail(VSR_ERR_BLOB, "top-level BVH was built over a different number of instances");
    const vsr_bvh_node* nodes =
        reinterpret_cast<const vsr_bvh_node*>(static_cast<const uint8_t*>(top_blob) + 64);
    const uint32_t* order = reinterpret_cast<const uint32_t*>(
        static_cast<const uint8_t*>(top_blob) + 64 + 32ull * num_nodes);
    DeviceGuard g(meshes[0]->device);
    if (!g.ok) return fail(VSR_ERR_CUDA, "cannot select the meshes' device");
    vsr_instances* x = new (std::nothrow) vsr_instances;
    if (!x) return fail(VSR_ERR_OOM, "out of host memory");
    x->device = meshes[0]->device;
    x->nmeshes = nmeshes;
    x->ninst = ninst;
    std::vector<DevScene> descs(nmeshes);
    for (uint32_t m = 0; m < nmeshes; ++m) descs[m] = meshes[m]->dev;
    std::vector<float4> inst(4ull * std::max(ninst, 1u));
    for (uint32_t i = 0; i < ninst; ++i) {
        const float* w = world_to_object + 12ull * i;
        for (int r = 0; r < 3; ++r)
            inst[4ull * i + r] = make_float4(w[4 * r], w[4 * r + 1], w[4 * r + 2], w[4 * r + 3]);
        float mesh_bits;
        std::memcpy(&mesh_bits, &inst_mesh[i], sizeof(mesh_bits));
        inst[4ull * i + 3] = make_float4(mesh_bits, 0.0f, 0.0f, 0.0f);
    }
    std::vector<float4> hn(2ull * num_nodes);
    for (uint32_t i = 0; i < num_nodes; ++i) {
        const vsr_bvh_node& nd = nodes[i];
        const uint32_t ref = (i == 1) ? 0u : node_ref(nd);
        float ref_bits;
        std::memcpy(&ref_bits, &ref, sizeof(ref_bits));
        hn[2ull * i] = make_float4(nd.lo[0], nd.lo[1], nd.lo[2], ref_bits);
        hn[2ull * i + 1] = make_float4(nd.hi[0], nd.hi[1], nd.hi[2], 0.0f);
    }
    cudaError_t e;
    if ((e = dmalloc(&x->d_meshes, (size_t)nmeshes)) != cudaSuccess ||
        (e = dmalloc(&x->d_inst, inst.size())) != cudaSuccess ||
        (e = dmalloc(&x->d_nodes, hn.size())) != cudaSuccess ||
        (e = dmalloc(&x->d_order, (size_t)std::max(ninst, 1u))) != cudaSuccess ||
        (e = dmalloc(&x->d_err, 1)) != cudaSuccess) {
        free_instances(x);
        return e == cudaErrorMemoryAllocation ? fail(VSR_ERR_OOM, "instance set allocation")
                                              : cuda_fail(e, "instance set allocation");
    }
    if ((e = cudaMemcpy(x->d_meshes, descs.data(), sizeof(DevScene) * nmeshes,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(x->d_inst, inst.data(), sizeof(float4) * inst.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(x->d_nodes, hn.data(), sizeof(float4) * hn.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (ninst && (e = cudaMemcpy(x->d_order, order, 4ull * ninst, cudaMemcpyHostToDevice)) !=
                      cudaSuccess) ||
        (e = cudaMemset(x->d_err, 0, sizeof(uint32_t))) != cudaSuccess) {
        free_instances(x);
        return cuda_fail(e, "instance set upload");
    }
    InstDev& d = x->dev;
    d.nodes = x->d_nodes;
    d.order = x->d_order;
    d.inst = x->d_inst;
    d.meshes = x->d_meshes;
    d.err = x->d_err;
    d.ninst = ninst;
    d.root_ref = node_ref(nodes[0]);
    d.top_depth = max_depth > 0 ? max_depth : 1u;
    d.max_leaves = num_nodes + 2u;
    d.root_a = make_float4(nodes[0].lo[0], nodes[0].lo[1], nodes[0].lo[2], 0.0f);
    d.root_b = make_float4(nodes[0].hi[0], nodes[0].hi[1], nodes[0].hi[2], 0.0f);
    x->stack_words = d.top_depth + mesh_depth;
    *out = x;
    return VSR_OK;
}

extern "C" vsr_status vsr_instances_destroy(vsr_instances* x) {
    g_err.clear();
    if (!x) return VSR_OK;
    DeviceGuard g(x->device);
    free_instances(x);
    return VSR_OK;
}

extern "C" vsr_status vsr_trace_instances(vsr_instances* x, const vsr_ray* rays, uint64_t n,
                                          const vsr_intersector* is, int32_t query,
                                          vsr_hit* hits, uint32_t* inst_ids, uint32_t* counters,
                                          const vsr_trace_params* p, vsr_stream stream) {
    g_err.clear();
    if (!x) return fail(VSR_ERR_ARG, "instance set is null");
    vsr_status st = validate_isect(is, query);
    if (st != VSR_OK) return st;
    if (is->kind == VSR_ISECT_CLIP)
        return fail(VSR_ERR_ARG, "the clip-box intersector is for vsr_trace and vsr_trace_multi");
    vsr_trace_params prm = kDefaultParams;
    if (p) prm = *p;
    if (prm.block_size < 32 || prm.block_size > 256 || prm.block_size % 32)
        return fail(VSR_ERR_ARG, "block_size must be a multiple of 32 in 32..256");
    if (prm.persistent > 1) return fail(VSR_ERR_ARG, "persistent must be 0 or 1");
    if (prm.refill_threshold < 1 || prm.refill_threshold > 32)
        return fail(VSR_ERR_ARG, "refill_threshold must be in 1..32");
    if (prm.blocks_per_sm > 32) return fail(VSR_ERR_ARG, "blocks_per_sm above 32");
    if (prm.lockstep) return fail(VSR_ERR_ARG, "instanced traces take lockstep 0");
    if (prm.octant) return fail(VSR_ERR_ARG, "instanced traces take octant 0");
    if (prm.ray_order) return fail(VSR_ERR_ARG, "instanced traces take ray_order 0");
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull)
        return fail(VSR_ERR_ARG, "too many rays for one launch");
    InstLaunch L{};
    st = make_map(n, prm.image_width, L.map);
    if (st != VSR_OK) return st;
    if (n == 0) return VSR_OK;
    if ((st = check_dev(rays, x->device, "rays", 16, n * sizeof(vsr_ray))) != VSR_OK ||
        (st = check_dev(hits, x->device, "hits", 16, n * sizeof(vsr_hit))) != VSR_OK)
        return st;
    if (inst_ids && (st = check_dev(inst_ids, x->device, "inst_ids", 4, n * 4)) != VSR_OK)
        return st;
    if (counters) {
        if (is->kind != VSR_ISECT_COUNT)
            return fail(VSR_ERR_ARG, "counters are written by the COUNT intersector only");
        if ((st = check_dev(counters, x->device, "counters", 8, n * 8)) != VSR_OK) return st;
    }
    L.is = x->dev;
    L.ip = isect_params(is);
    L.rays = reinterpret_cast<const float4*>(rays);
    L.hits = reinterpret_cast<float4*>(hits);
    L.inst_ids = inst_ids;
    L.counters = reinterpret_cast<uint2*>(counters);
    L.block = prm.block_size;
    L.stack_words = x->stack_words;
    L.stream = reinterpret_cast<cudaStream_t>(stream);
    L.persistent = prm.persistent;
    L.refill = prm.refill_threshold;
    L.blocks_per_sm = prm.blocks_per_sm;
    L.wd = make_watchdog(prm);
    DeviceGuard g(x->device);
    cudaError_t e = launch_instances(L, is->kind, query, is->dispatch == VSR_DISPATCH_DYNAMIC);
    if (e != cudaSuccess) return cuda_fail(e, "instanced trace launch");
    return VSR_OK;
}

extern "C" vsr_status vsr_instances_device_error(vsr_instances* x, uint32_t* word) {
    g_err.clear();
    if (!x || !word) return fail(VSR_ERR_ARG, "null argument");
    DeviceGuard g(x->device);
    VSR_CUDA(cudaDeviceSynchronize(), "synchronise");
    VSR_CUDA(cudaMemcpy(word, x->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost),
             "read error word");
    VSR_CUDA(cudaMemset(x->d_err, 0, sizeof(uint32_t)), "clear error word");
    unsigned line = 0;
    VSR_CUDA(instances_align_error(&line), "read alignment check");
    if (line) {
        *word |= kErrAlign;
        g_err = "instanced kernel skipped a misaligned access at "
                "trace_instances.cu/vsr_device.cuh line " + std::to_string(line);
    }
    return VSR_OK;
}

// ---------------------------------------------------------------------------
// Diffuse path tracing on the closest-hit query (path.cu): one trace launch
// per segment depth over every path, then the shading launch.

extern "C" vsr_status vsr_path_trace(vsr_scene* s, const vsr_ray* rays, uint64_t n,
                                     const vsr_intersector* is, const vsr_path_params* pp,
                                     const float* dirs, float* radiance, uint32_t* segments,
                                     const vsr_trace_params* p, vsr_stream stream) {
    g_err.clear();
    if (!pp) return fail(VSR_ERR_ARG, "path parameters are null");
    if (pp->bounces > 64) return fail(VSR_ERR_ARG, "bounces must be in 0..64");
    if (!std::isfinite(pp->eps) || pp->eps < 0.0f)
        return fail(VSR_ERR_ARG, "eps must be finite and >= 0");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(pp->sky[c]) || !std::isfinite(pp->untextured[c]))
            return fail(VSR_ERR_ARG, "non-finite sky or albedo");
    LaunchArgs a;
    // n == 0 keeps prepare_launch's ray and hit checks out of the way
    vsr_status st = prepare_launch(s, rays, 0, is, VSR_CLOSEST, nullptr, p, a);
    if (st != VSR_OK) return st;
    if (n > (uint64_t)(std::numeric_limits<int>::max() - 1) * 32ull)
        return fail(VSR_ERR_ARG, "too many rays for one launch");
    if (n == 0) return VSR_OK;
    if ((st = check_dev(rays, s->device, "rays", 16, n * sizeof(vsr_ray))) != VSR_OK ||
        (st = check_dev(radiance, s->device, "radiance", 4, n * 12)) != VSR_OK)
        return st;
    if (pp->bounces &&
        (st = check_dev(dirs, s->device, "dirs", 4, n * pp->bounces * 12ull)) != VSR_OK)
        return st;
    if (segments && (st = check_dev(segments, s->device, "segments", 4, n * 4)) != VSR_OK)
        return st;
    st = make_map(n, p ? p->image_width : 0u, a.map);
    if (st != VSR_OK) return st;
    a.n = n;
    PathDev pd{};
    pd.bounces = pp->bounces;
    pd.eps = pp->eps;
    for (int c = 0; c < 3; ++c) {
        pd.sky[c] = pp->sky[c];
        pd.untex[c] = pp->untextured[c];
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    DeviceGuard g(s->device);
    if (!g.ok) return fail(VSR_ERR_CUDA, "cannot select the scene's device");
    float4* work = nullptr;
    float4* hits = nullptr;
    float* f = nullptr;
    // after each bounce the live paths are compacted to the front of a
    // permutation the next segment's trace follows (ray indices are 32-bit)
    const bool compact = pp->bounces > 0 && n <= 0xFFFFFFFFull;
    uint32_t* perm = nullptr;
    uint32_t* counts = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&work), n * 32, cs);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&hits), n * 16, cs);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&f), n * 12, cs);
    if (e == cudaSuccess && compact)
        e = cudaMallocAsync(reinterpret_cast<void**>(&perm), n * 4, cs);
    if (e == cudaSuccess && compact)
        e = cudaMallocAsync(reinterpret_cast<void**>(&counts),
                            (path_compact_blocks(n) + 1ull) * 4, cs);
    if (e == cudaSuccess)
        e = launch_path_init(reinterpret_cast<const float4*>(rays), n, work, f, radiance, segments,
                             cs);
    a.rays = work;
    a.hits = hits;
    a.stream = cs;
    for (uint32_t k = 0; e == cudaSuccess && k <= pp->bounces; ++k) {
        if (k == 1 && compact) a.map = RayMap{n, n, 0u, 0u, perm};
        e = is->dispatch == VSR_DISPATCH_STATIC ? launch_static(a, is->kind, false)
                                                : launch_dynamic(a, is->kind);
        if (e == cudaSuccess)
            e = launch_path_bounce(s->dev, pd, s->d_verts, s->d_idx, work, hits, f, dirs, k, n,
                                   radiance, segments, cs);
        if (e == cudaSuccess && compact && k < pp->bounces)
            e = launch_path_compact(f, n, counts, perm, cs);
    }
    if (counts) cudaFreeAsync(counts, cs);
    if (perm) cudaFreeAsync(perm, cs);
    if (f) cudaFreeAsync(f, cs);
    if (hits) cudaFreeAsync(hits, cs);
    if (work) cudaFreeAsync(work, cs);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(VSR_ERR_OOM, "path scratch allocation")
                                              : cuda_fail(e, "path tracing launch");
    return VSR_OK;
}
