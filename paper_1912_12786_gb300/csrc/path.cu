// Diffuse path tracing on the closest-hit query with the custom intersector
// (a workload of many incoherent segments; the paper has no shading).  The
// host runs it wavefront-style: for each bounce, one closest-hit launch over
// every path (the trace kernels; finished paths carry an inactive ray that
// leaves at the root box test), then k_path_bounce, which shades the hits and
// writes the next segment in place.  FP32 with the operation order fixed, so
// every bounce reproduces the oracle's bit for bit:
//   miss      radiance = throughput * sky, the path ends;
//   hit       throughput *= albedo (the nearest texel's colour, RGBA8 / 255 or
//             RGBA32F; `untex` for untextured triangles and u8 textures);
//             after `bounces` bounces the path ends with radiance 0;
//   bounce    origin fmaf(t, d, o); face normal m = e1 x e2 (the triangle
//             test's cross), n = m / sqrt(m . m) (IEEE; (0, 0, 1) for m = 0),
//             turned against d; Duff et al. (2017) frame s = copysign(1, n.z),
//             a = -1 / (s + n.z), b = (n.x n.y) a, t1 = (1 + ((s n.x) n.x) a,
//             s b, -(s n.x)), t2 = (b, s + (n.y n.y) a, -n.y); direction
//             fmaf(l.x, t1, fmaf(l.y, t2, l.z n)) for the given local unit
//             vector l; interval (eps, +inf).
//
// The bounce kernel reads vertices through the index buffer, the access
// pattern of the two kernels whose unchecked builds raised unexplained
// misaligned-address faults, so this translation unit uses the checked
// loads (a skipped access is reported with its line, device error bit 2).
#define VSR_CHECKED_LOADS 1
#include "vsr_internal.h"

namespace vsr {

namespace {

__device__ __forceinline__ void path_albedo(const DevScene& sc, uint32_t prim, float u, float v,
                                            const PathDev& pd, float alb[3]) {
    alb[0] = pd.untex[0];
    alb[1] = pd.untex[1];
    alb[2] = pd.untex[2];
    const uint32_t g = VSR_LDG(sc.geom + prim);
    if (g == kMiss) return;
    const uint4 d = VSR_LDG(reinterpret_cast<const uint4*>(sc.tex + g));
    if (d.x == kTexU8) return;
    const unsigned long long off = VSR_LDG(&sc.tex[g].offset);
    const float2 uv = lerp_uv(sc.uvs, prim, u, v);
    const unsigned long long k =
        (unsigned long long)texel_coord(uv.y, d.z) * d.y + texel_coord(uv.x, d.y);
    for (int c = 0; c < 3; ++c)
        alb[c] = d.x == kTexRGBA8
                     ? __fdiv_rn((float)VSR_LDG(sc.texels + off + 4 * k + c), 255.0f)
                     : VSR_LDG(reinterpret_cast<const float*>(sc.texels + off) + 4 * k + c);
}

__global__ void k_path_init(const float4* __restrict__ rays, unsigned long long n,
                            float4* __restrict__ work, float* __restrict__ f,
                            float* __restrict__ radiance, uint32_t* __restrict__ segments) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    work[2 * i] = VSR_LDG(rays + 2 * i);
    work[2 * i + 1] = VSR_LDG(rays + 2 * i + 1);
    f[3 * i] = 1.0f;
    f[3 * i + 1] = 1.0f;
    f[3 * i + 2] = 1.0f;
    radiance[3 * i] = 0.0f;
    radiance[3 * i + 1] = 0.0f;
    radiance[3 * i + 2] = 0.0f;
    if (segments) segments[i] = 0;
}

// Shading of segment k of every live path (f[3i] < 0 marks a finished path).
__global__ void k_path_bounce(DevScene sc, PathDev pd, const float* __restrict__ verts,
                              const uint32_t* __restrict__ idx, float4* __restrict__ work,
                              const float4* __restrict__ hits, float* __restrict__ f,
                              const float* __restrict__ dirs, uint32_t k,
                              unsigned long long n, float* __restrict__ radiance,
                              uint32_t* __restrict__ segments) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float fr = f[3 * i], fg = f[3 * i + 1], fb = f[3 * i + 2];
    if (fr < 0.0f) return;
    if (segments) segments[i] = k + 1;
    const float4 h = VSR_LDG(hits + i);
    const uint32_t prim = __float_as_uint(h.w);
    bool done = false;
    if (prim == kMiss) {
        radiance[3 * i] = __fmul_rn(fr, pd.sky[0]);
        radiance[3 * i + 1] = __fmul_rn(fg, pd.sky[1]);
        radiance[3 * i + 2] = __fmul_rn(fb, pd.sky[2]);
        done = true;
    } else {
        float alb[3];
        path_albedo(sc, prim, h.y, h.z, pd, alb);
        fr = __fmul_rn(fr, alb[0]);
        fg = __fmul_rn(fg, alb[1]);
        fb = __fmul_rn(fb, alb[2]);
        done = k == pd.bounces;
    }
    if (done) {
        f[3 * i] = -1.0f;
        work[2 * i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        work[2 * i + 1] = make_float4(0.0f, 0.0f, 1.0f, -1.0f);
        return;
    }
    f[3 * i] = fr;
    f[3 * i + 1] = fg;
    f[3 * i + 2] = fb;
    // the next segment
    const float4 ra = work[2 * i], rb = work[2 * i + 1];
    const float* a = verts + 3ull * VSR_LDG(idx + 3ull * prim);
    const float* b = verts + 3ull * VSR_LDG(idx + 3ull * prim + 1);
    const float* c = verts + 3ull * VSR_LDG(idx + 3ull * prim + 2);
    const float ax = VSR_LDG(a), ay = VSR_LDG(a + 1), az = VSR_LDG(a + 2);
    const float e1x = __fsub_rn(VSR_LDG(b), ax), e1y = __fsub_rn(VSR_LDG(b + 1), ay),
                e1z = __fsub_rn(VSR_LDG(b + 2), az);
    const float e2x = __fsub_rn(VSR_LDG(c), ax), e2y = __fsub_rn(VSR_LDG(c + 1), ay),
                e2z = __fsub_rn(VSR_LDG(c + 2), az);
    const float mx = __fmaf_rn(e1y, e2z, -__fmul_rn(e1z, e2y));
    const float my = __fmaf_rn(e1z, e2x, -__fmul_rn(e1x, e2z));
    const float mz = __fmaf_rn(e1x, e2y, -__fmul_rn(e1y, e2x));
    const float len = __fsqrt_rn(dot3(mx, my, mz, mx, my, mz));
    float nx = 0.0f, ny = 0.0f, nz = 1.0f;
    if (len > 0.0f) {
        nx = __fdiv_rn(mx, len);
        ny = __fdiv_rn(my, len);
        nz = __fdiv_rn(mz, len);
    }
    if (dot3(nx, ny, nz, rb.x, rb.y, rb.z) > 0.0f) {
        nx = -nx;
        ny = -ny;
        nz = -nz;
    }
    const float sg = copysignf(1.0f, nz);
    const float aa = __fdiv_rn(-1.0f, __fadd_rn(sg, nz));
    const float bb = __fmul_rn(__fmul_rn(nx, ny), aa);
    const float sx = __fmul_rn(sg, nx);
    const float t1x = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(sx, nx), aa)), t1y = __fmul_rn(sg, bb),
                t1z = -sx;
    const float t2x = bb, t2y = __fadd_rn(sg, __fmul_rn(__fmul_rn(ny, ny), aa)), t2z = -ny;
    const float* l = dirs + 3ull * ((unsigned long long)i * pd.bounces + k);
    const float lx = VSR_LDG(l), ly = VSR_LDG(l + 1), lz = VSR_LDG(l + 2);
    const float t = h.x;
    work[2 * i] = make_float4(__fmaf_rn(t, rb.x, ra.x), __fmaf_rn(t, rb.y, ra.y),
                              __fmaf_rn(t, rb.z, ra.z), pd.eps);
    work[2 * i + 1] =
        make_float4(__fmaf_rn(lx, t1x, __fmaf_rn(ly, t2x, __fmul_rn(lz, nx))),
                    __fmaf_rn(lx, t1y, __fmaf_rn(ly, t2y, __fmul_rn(lz, ny))),
                    __fmaf_rn(lx, t1z, __fmaf_rn(ly, t2z, __fmul_rn(lz, nz))),
                    __int_as_float(0x7f800000));
}

// Live-path compaction between bounces: a stable partition of the path
// indices with the live paths (f[3i] >= 0) first, in index order, and the
// finished ones after them.  The next segment's trace then takes ray perm[g]
// in thread g, so live rays fill whole warps instead of sharing them with
// finished paths, whose inactive rays end at the root box test.  Each ray is
// traced exactly as before, so every result is unchanged.
constexpr uint32_t kCompactThreads = 256;

__device__ __forceinline__ bool path_live(const float* __restrict__ f, unsigned long long i,
                                          unsigned long long n) {
    return i < n && f[3 * i] >= 0.0f;
}

// Number of live paths of this block before the thread's path, and the
// block's live count in *total.  Every thread of the block calls it.
__device__ __forceinline__ uint32_t block_live_rank(bool live, uint32_t* s_warp,
                                                    uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(kFullMask, live);
    if (lane == 0) s_warp[warp] = __popc(b);
    __syncthreads();
    uint32_t before = 0, sum = 0;
    for (uint32_t w = 0; w < kCompactThreads / 32u; ++w) {
        const uint32_t c = s_warp[w];
        if (w < warp) before += c;
        sum += c;
    }
    *total = sum;
    return before + __popc(b & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kCompactThreads)
    k_live_count(const float* __restrict__ f, unsigned long long n, uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_warp[kCompactThreads / 32];
    const unsigned long long i = (unsigned long long)blockIdx.x * kCompactThreads + threadIdx.x;
    uint32_t total = 0;
    block_live_rank(path_live(f, i, n), s_warp, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Exclusive scan of the nb block counts in place, 1,024 at a time with a
// running carry; counts[nb] receives the number of live paths.
__global__ void __launch_bounds__(1024) k_live_scan(uint32_t* __restrict__ counts, uint32_t nb) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024u) {
        const uint32_t j = base + threadIdx.x;
        const uint32_t v = j < nb ? counts[j] : 0u;
        uint32_t x = v;  // inclusive scan within the warp
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane];
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullMask, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const uint32_t excl = s_carry + (warp ? s_warp[warp - 1] : 0u) + x - v;
        if (j < nb) counts[j] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[nb] = s_carry;
}

__global__ void __launch_bounds__(kCompactThreads)
    k_live_scatter(const float* __restrict__ f, unsigned long long n,
                   const uint32_t* __restrict__ offsets, uint32_t nb, uint32_t* __restrict__ perm) {
    __shared__ uint32_t s_warp[kCompactThreads / 32];
    const unsigned long long i = (unsigned long long)blockIdx.x * kCompactThreads + threadIdx.x;
    const bool live = path_live(f, i, n);
    uint32_t total = 0;
    const uint32_t rank = block_live_rank(live, s_warp, &total);
    if (i >= n) return;
    const uint32_t live_before = offsets[blockIdx.x];
    if (live) {
        perm[live_before + rank] = (uint32_t)i;
    } else {
        // finished paths before this one: in earlier blocks, then in this one
        const uint32_t dead_before = blockIdx.x * kCompactThreads - live_before;
        perm[offsets[nb] + dead_before + (threadIdx.x - rank)] = (uint32_t)i;
    }
}

}  // namespace

uint32_t path_compact_blocks(unsigned long long n) {
    return (uint32_t)((n + kCompactThreads - 1) / kCompactThreads);
}

cudaError_t launch_path_compact(const float* f, unsigned long long n, uint32_t* counts,
                                uint32_t* perm, cudaStream_t stream) {
    const uint32_t nb = path_compact_blocks(n);
    k_live_count<<<nb, kCompactThreads, 0, stream>>>(f, n, counts);
    k_live_scan<<<1, 1024, 0, stream>>>(counts, nb);
    k_live_scatter<<<nb, kCompactThreads, 0, stream>>>(f, n, counts, nb, perm);
    return cudaGetLastError();
}

cudaError_t launch_path_init(const float4* rays, unsigned long long n, float4* work, float* f,
                             float* radiance, uint32_t* segments, cudaStream_t stream) {
    k_path_init<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(rays, n, work, f, radiance,
                                                                 segments);
    return cudaGetLastError();
}

cudaError_t launch_path_bounce(const DevScene& sc, const PathDev& pd, const float* verts,
                               const uint32_t* idx, float4* work, const float4* hits, float* f,
                               const float* dirs, uint32_t k, unsigned long long n,
                               float* radiance, uint32_t* segments, cudaStream_t stream) {
    k_path_bounce<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
        sc, pd, verts, idx, work, hits, f, dirs, k, n, radiance, segments);
    return cudaGetLastError();
}

cudaError_t path_align_error(unsigned* line) {
    cudaError_t e = cudaMemcpyFromSymbol(line, g_vsr_align_line, sizeof(unsigned));
    if (e != cudaSuccess || *line == 0) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_vsr_align_line, &zero, sizeof(unsigned));
}

}  // namespace vsr
