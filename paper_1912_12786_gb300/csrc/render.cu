// Differentiable shading on top of the closest-hit query with a custom
// intersector, and its adjoint at fixed visibility.
//
//   forward   c = albedo_rgb(uv) * max(0, n_f . L) for a hit, background for
//             a miss; n = normalize(e1 x e2) flipped to face the ray, uv the
//             interpolated texture coordinate, albedo the bilinear lookup
//             (texel centres at ((i + 0.5)/W, (j + 0.5)/H), clamp-to-edge
//             texel indices).
//             The render is the closest-hit trace (the trace kernels), then
//             a shading pass over its hit records.
//   backward  from closest-hit records -- the forward's, or those a trace
//             writes again -- the shading is recomputed and its adjoint is
//             scattered with atomics into the vertex gradients (through u, v
//             of the Moller-Trumbore solve and through the face normal) and
//             the texel gradients (through the bilinear weights).
//
// Also: the BVH refit used after a vertex update.
// The shading, adjoint and occlusion kernels use alignment-checked loads
// (see VSR_LDG).
#define VSR_CHECKED_LOADS 1
#include "vsr_internal.h"

namespace vsr {

namespace {

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 load_v3(const float* p) { return v3(p[0], p[1], p[2]); }

// Bilinear footprint of one lookup.
struct Bilinear {
    float rgb[3];
    float t[4][3];   // texel colours: (j0,i0), (j0,i1), (j1,i0), (j1,i1)
    uint32_t k[4];   // texel indices j*W + i
    float fx, fy;
    uint32_t W, H;
    bool varying;    // albedo depends on uv (a colour texture)
    bool rgba32f;
};

__device__ __forceinline__ float texel_channel(const DevScene& sc, const TexDesc& d,
                                               uint32_t k, int ch) {
    if (d.fmt == kTexRGBA32F)
        return VSR_LDG(reinterpret_cast<const float*>(sc.texels + d.offset) + 4ull * k + ch);
    return (float)VSR_LDG(sc.texels + d.offset + 4ull * k + ch) * (1.0f / 255.0f);
}

// Albedo of texture g at uv.  Untextured triangles and alpha-only (u8)
// textures have albedo 1.
__device__ __forceinline__ void albedo(const DevScene& sc, uint32_t g, float2 uv, Bilinear& b) {
    b.varying = false;
    b.rgba32f = false;
    b.rgb[0] = b.rgb[1] = b.rgb[2] = 1.0f;
    if (g == kMiss) return;
    TexDesc d;
    const uint4 h = VSR_LDG(reinterpret_cast<const uint4*>(sc.tex + g));
    d.fmt = h.x;
    d.w = h.y;
    d.h = h.z;
    d.offset = VSR_LDG(&sc.tex[g].offset);
    if (d.fmt == kTexU8) return;
    b.varying = true;
    b.rgba32f = d.fmt == kTexRGBA32F;
    b.W = d.w;
    b.H = d.h;
    const float x = uv.x * (float)d.w - 0.5f, y = uv.y * (float)d.h - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    b.fx = x - x0;
    b.fy = y - y0;
    const int ix = (int)fmaxf(fminf(x0, 2147483520.0f), -2147483520.0f);
    const int iy = (int)fmaxf(fminf(y0, 2147483520.0f), -2147483520.0f);
    const int wm = (int)d.w - 1, hm = (int)d.h - 1;
    const uint32_t i0 = (uint32_t)min(max(ix, 0), wm), i1 = (uint32_t)min(max(ix + 1, 0), wm);
    const uint32_t j0 = (uint32_t)min(max(iy, 0), hm), j1 = (uint32_t)min(max(iy + 1, 0), hm);
    b.k[0] = j0 * d.w + i0;
    b.k[1] = j0 * d.w + i1;
    b.k[2] = j1 * d.w + i0;
    b.k[3] = j1 * d.w + i1;
    const float w[4] = {(1.0f - b.fx) * (1.0f - b.fy), b.fx * (1.0f - b.fy),
                        (1.0f - b.fx) * b.fy, b.fx * b.fy};
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
        for (int c = 0; c < 4; ++c) {
            b.t[c][ch] = texel_channel(sc, d, b.k[c], ch);
            acc += w[c] * b.t[c][ch];
        }
        b.rgb[ch] = acc;
    }
}

// Geometry of a hit needed by the shading and its adjoint.
struct Surface {
    V3 a, e1, e2, m, n;
    float len, flip, ndl, s;
    uint32_t vi[3];
};

__device__ __forceinline__ void surface(const float* __restrict__ verts,
                                        const uint32_t* __restrict__ idx, uint32_t prim, V3 d,
                                        V3 L, Surface& f) {
    for (int k = 0; k < 3; ++k) f.vi[k] = VSR_LDG(idx + 3ull * prim + k);
    f.a = load_v3(verts + 3ull * f.vi[0]);
    f.e1 = load_v3(verts + 3ull * f.vi[1]) - f.a;
    f.e2 = load_v3(verts + 3ull * f.vi[2]) - f.a;
    f.m = cross(f.e1, f.e2);
    f.len = sqrtf(dot(f.m, f.m));
    f.n = f.len > 0.0f ? (1.0f / f.len) * f.m : v3(0.0f, 0.0f, 0.0f);
    f.flip = dot(f.n, d) < 0.0f ? 1.0f : -1.0f;
    f.ndl = f.flip * dot(f.n, L);
    f.s = fmaxf(f.ndl, 0.0f);
}

}  // namespace

// The forward shading from the closest hits the trace kernels wrote (the
// render is that trace, then this pass): one thread per ray.  A hit record
// whose primitive is out of range gives the background and is flagged
// (kErrHit).
__global__ void __launch_bounds__(256) k_shade_hits(DevScene sc, ShadeDev sh,
                                                    const float* __restrict__ verts,
                                                    const uint32_t* __restrict__ idx,
                                                    const float4* __restrict__ rays,
                                                    const float4* __restrict__ hits,
                                                    unsigned long long n,
                                                    float* __restrict__ image) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = VSR_LDG(hits + i);
    const uint32_t prim = __float_as_uint(h.w);
    float c[3] = {sh.bg[0], sh.bg[1], sh.bg[2]};
    if (prim != kMiss && prim >= sc.nprims) {
        atomicOr(sc.err, kErrHit);
    } else if (prim != kMiss) {
        const float4 rb = VSR_LDG(rays + 2 * i + 1);
        Surface f;
        surface(verts, idx, prim, v3(rb.x, rb.y, rb.z), v3(sh.light[0], sh.light[1], sh.light[2]),
                f);
        Bilinear b;
        albedo(sc, VSR_LDG(sc.geom + prim), lerp_uv(sc.uvs, prim, h.y, h.z), b);
        for (int ch = 0; ch < 3; ++ch) c[ch] = b.rgb[ch] * f.s;
    }
    image[3 * i] = c[0];
    image[3 * i + 1] = c[1];
    image[3 * i + 2] = c[2];
}

// Add (a, b, c) to the RGB of texel k in a gradient array of 4 floats per
// texel: one 16-byte vector atomic when the array is 16-byte aligned (the
// fourth float gets +0), else three scalar atomics.  `vec` is the same for
// the whole launch.
__device__ __forceinline__ void add_texel_grad(float* grad, uint32_t k, float a, float b, float c,
                                               bool vec) {
    if (vec) {
        atomicAdd(reinterpret_cast<float4*>(grad) + k, make_float4(a, b, c, 0.0f));
    } else {
        atomicAdd(grad + 4ull * k, a);
        atomicAdd(grad + 4ull * k + 1, b);
        atomicAdd(grad + 4ull * k + 2, c);
    }
}

// Adjoint of the shading at fixed visibility.  g = dL/dc for the pixel.
//   texels: dc/dT(corner) = s * w(corner)                      (rgb channels)
//   uv:     dc/duv.x = s * W * [(1-fy)(T01-T00) + fy(T11-T10)]   (and y)
//   (u, v): duv/du = tc1 - tc0, duv/dv = tc2 - tc0
//   normal: dc/dn_f = albedo * L where n_f . L > 0, n_f = flip * m/|m|,
//           dL/dm = (dL/dn - n (n . dL/dn)) / |m|, m = e1 x e2
//   solve:  (t, u, v) = M^-1 (o - v0) with M = [-d, e1, e2] gives
//           dL/dv_k = -b_k y with y = M^-T (0, dL/du, dL/dv) and
//           b = (1 - u - v, u, v).
// shade_adjoint: that adjoint for pixel i, from its hit (prim, bu, bv: the
// closest hit's primitive and barycentrics) and ray direction d; scatters
// into grad_verts and (if not null) grad_texels.
__device__ __forceinline__ void shade_adjoint(const DevScene& sc, const ShadeDev& sh,
                                              const float* __restrict__ verts,
                                              const uint32_t* __restrict__ idx,
                                              unsigned long long i, V3 d, uint32_t prim,
                                              float bu, float bv,
                                              const float* __restrict__ dL_dimage,
                                              float* __restrict__ grad_verts,
                                              float* __restrict__ grad_texels,
                                              bool vec_texels) {
    const float g[3] = {VSR_LDG(dL_dimage + 3 * i), VSR_LDG(dL_dimage + 3 * i + 1),
                        VSR_LDG(dL_dimage + 3 * i + 2)};
    if (g[0] == 0.0f && g[1] == 0.0f && g[2] == 0.0f) return;
    const V3 L = v3(sh.light[0], sh.light[1], sh.light[2]);
    Surface f;
    surface(verts, idx, prim, d, L, f);
    const uint32_t geom = VSR_LDG(sc.geom + prim);
    const float2 c0 = VSR_LDG(sc.uvs + 3ull * prim), c1 = VSR_LDG(sc.uvs + 3ull * prim + 1),
                 c2 = VSR_LDG(sc.uvs + 3ull * prim + 2);
    Bilinear b;
    albedo(sc, geom, lerp_uv(sc.uvs, prim, bu, bv), b);

    // texel gradients
    if (grad_texels && b.rgba32f && geom == sh.grad_tex && f.s > 0.0f) {
        const float w[4] = {(1.0f - b.fx) * (1.0f - b.fy), b.fx * (1.0f - b.fy),
                            (1.0f - b.fx) * b.fy, b.fx * b.fy};
        for (int c = 0; c < 4; ++c)
            add_texel_grad(grad_texels, b.k[c], g[0] * f.s * w[c], g[1] * f.s * w[c],
                           g[2] * f.s * w[c], vec_texels);
    }
    // through the texture coordinate
    float dL_du = 0.0f, dL_dv = 0.0f;
    if (b.varying && f.s > 0.0f) {
        float gx = 0.0f, gy = 0.0f;
        for (int ch = 0; ch < 3; ++ch) {
            const float dx = (1.0f - b.fy) * (b.t[1][ch] - b.t[0][ch]) +
                             b.fy * (b.t[3][ch] - b.t[2][ch]);
            const float dy = (1.0f - b.fx) * (b.t[2][ch] - b.t[0][ch]) +
                             b.fx * (b.t[3][ch] - b.t[1][ch]);
            gx += g[ch] * f.s * dx;
            gy += g[ch] * f.s * dy;
        }
        gx *= (float)b.W;
        gy *= (float)b.H;
        dL_du = gx * (c1.x - c0.x) + gy * (c1.y - c0.y);
        dL_dv = gx * (c2.x - c0.x) + gy * (c2.y - c0.y);
    }
    // through the face normal
    V3 dL_de1 = v3(0.0f, 0.0f, 0.0f), dL_de2 = v3(0.0f, 0.0f, 0.0f);
    if (f.ndl > 0.0f && f.len > 0.0f) {
        const float dL_ds = g[0] * b.rgb[0] + g[1] * b.rgb[1] + g[2] * b.rgb[2];
        const V3 dL_dn = (f.flip * dL_ds) * L;
        const V3 dL_dm = (1.0f / f.len) * (dL_dn - dot(f.n, dL_dn) * f.n);
        dL_de1 = cross(f.e2, dL_dm);
        dL_de2 = cross(dL_dm, f.e1);
    }
    // through the solve for (t, u, v): rows of M^T are -d, e1, e2
    V3 y = v3(0.0f, 0.0f, 0.0f);
    const V3 nd = v3(-d.x, -d.y, -d.z);
    const float det = dot(nd, f.m);
    if (det != 0.0f && (dL_du != 0.0f || dL_dv != 0.0f))
        y = (1.0f / det) * (dL_du * cross(f.e2, nd) + dL_dv * cross(nd, f.e1));
    const float w0 = 1.0f - bu - bv;
    const V3 gv0 = (-w0) * y - dL_de1 - dL_de2;
    const V3 gv1 = (-bu) * y + dL_de1;
    const V3 gv2 = (-bv) * y + dL_de2;
    const V3 gk[3] = {gv0, gv1, gv2};
    for (int k = 0; k < 3; ++k) {
        float* p = grad_verts + 3ull * f.vi[k];
        atomicAdd(p, gk[k].x);
        atomicAdd(p + 1, gk[k].y);
        atomicAdd(p + 2, gk[k].z);
    }
}

// The adjoint from closest-hit records (the forward's saved hits, or those a
// trace writes again for vsr_trace_backward), one thread per pixel, no
// traversal.  A hit record whose primitive is out of range is skipped and
// flagged (kErrHit).
__global__ void __launch_bounds__(256) k_render_backward_hits(
    DevScene sc, ShadeDev sh, const float* __restrict__ verts, const uint32_t* __restrict__ idx,
    const float4* __restrict__ rays, const float4* __restrict__ hits, unsigned long long n,
    const float* __restrict__ dL_dimage, float* __restrict__ grad_verts,
    float* __restrict__ grad_texels, bool vec_texels) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = VSR_LDG(hits + i);
    const uint32_t prim = __float_as_uint(h.w);
    if (prim == kMiss) return;
    if (prim >= sc.nprims) {
        atomicOr(sc.err, kErrHit);
        return;
    }
    const float4 rb = VSR_LDG(rays + 2 * i + 1);
    shade_adjoint(sc, sh, verts, idx, i, v3(rb.x, rb.y, rb.z), prim, h.y, h.z, dL_dimage,
                  grad_verts, grad_texels, vec_texels);
}

// Ambient-occlusion render: c = albedo_rgb(uv) * (1 - occluded / spp) for a
// primary hit, background for a miss.  The closest-hit trace, the occlusion
// rays traced any-hit and counted (the trace kernels; api.cu), then the
// shading of the saved hits here.

// Shading of the saved hits; occ enters as the integer counts of
// k_ao_count and leaves as the occluded fraction (0 for a miss).
__global__ void __launch_bounds__(256) k_ao_shade(DevScene sc, ShadeDev sh,
                                                  const float4* __restrict__ hits,
                                                  unsigned long long n, uint32_t spp,
                                                  float* __restrict__ occ,
                                                  float* __restrict__ image) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = VSR_LDG(hits + i);
    const uint32_t prim = __float_as_uint(h.w);
    float c[3] = {sh.bg[0], sh.bg[1], sh.bg[2]};
    float o = 0.0f;
    if (prim != kMiss) {
        o = (float)reinterpret_cast<const uint32_t*>(occ)[i] / (float)spp;
        const float vis = 1.0f - o;
        Bilinear b;
        albedo(sc, VSR_LDG(sc.geom + prim), lerp_uv(sc.uvs, prim, h.y, h.z), b);
        for (int ch = 0; ch < 3; ++ch) c[ch] = b.rgb[ch] * vis;
    }
    image[3 * i] = c[0];
    image[3 * i + 1] = c[1];
    image[3 * i + 2] = c[2];
    occ[i] = o;
}

// Adjoint with respect to the colour texels of texture sh.grad_tex at fixed
// visibility, from the forward's saved hits and occluded fractions (no
// traversal): dc/dT(corner) = (1 - occ) * w(corner).  A hit record whose
// primitive is out of range is skipped and flagged (kErrHit).
__global__ void __launch_bounds__(256) k_ao_backward(DevScene sc, ShadeDev sh,
                                                     const float4* __restrict__ hits,
                                                     const float* __restrict__ occ,
                                                     unsigned long long n,
                                                     const float* __restrict__ dL_dimage,
                                                     float* __restrict__ grad_texels,
                                                     bool vec_texels) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g[3] = {VSR_LDG(dL_dimage + 3 * i), VSR_LDG(dL_dimage + 3 * i + 1),
                        VSR_LDG(dL_dimage + 3 * i + 2)};
    if (g[0] == 0.0f && g[1] == 0.0f && g[2] == 0.0f) return;
    const float4 h = VSR_LDG(hits + i);
    const uint32_t prim = __float_as_uint(h.w);
    if (prim == kMiss) return;
    if (prim >= sc.nprims) {
        atomicOr(sc.err, kErrHit);
        return;
    }
    const uint32_t geom = VSR_LDG(sc.geom + prim);
    if (geom != sh.grad_tex) return;
    Bilinear b;
    albedo(sc, geom, lerp_uv(sc.uvs, prim, h.y, h.z), b);
    if (!b.rgba32f) return;
    const float vis = 1.0f - VSR_LDG(occ + i);
    if (vis == 0.0f) return;
    const float w[4] = {(1.0f - b.fx) * (1.0f - b.fy), b.fx * (1.0f - b.fy),
                        (1.0f - b.fx) * b.fy, b.fx * b.fy};
    for (int c = 0; c < 4; ++c)
        add_texel_grad(grad_texels, b.k[c], g[0] * vis * w[c], g[1] * vis * w[c],
                       g[2] * vis * w[c], vec_texels);
}

// Bottom-up refit of the node boxes after a vertex update: one launch per
// tree level, deepest first.  Leaves take the bounds of their triangles'
// vertices (as the builder does); inner nodes the union of their children.
// Topology and the packed references are unchanged.
__global__ void k_refit(float4* __restrict__ nodes, const uint32_t* __restrict__ level_nodes,
                        uint32_t count, const float* __restrict__ verts,
                        const uint32_t* __restrict__ idx, const uint32_t* __restrict__ order,
                        uint32_t* __restrict__ unordered) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint32_t id = level_nodes[t];
    const float4 a = nodes[2ull * id];
    const uint32_t ref = __float_as_uint(a.w);
    float lo[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000),
                   __int_as_float(0x7f800000)};
    float hi[3] = {-lo[0], -lo[1], -lo[2]};
    if (ref & kLeafBit) {
        const uint32_t first = (ref >> 3) & 0x0FFFFFFFu, cnt = (ref & 7u) + 1u;
        for (uint32_t s = first; s < first + cnt; ++s) {
            const uint32_t p = order[s];
            for (int k = 0; k < 3; ++k) {
                const float* v = verts + 3ull * idx[3ull * p + k];
                for (int c = 0; c < 3; ++c) {
                    lo[c] = fminf(lo[c], v[c]);
                    hi[c] = fmaxf(hi[c], v[c]);
                }
            }
        }
    } else {
        const uint64_t l = 2ull * (ref >> 2);
        for (uint64_t c = l; c <= l + 1; ++c) {
            const float4 ca = nodes[2 * c], cb = nodes[2 * c + 1];
            lo[0] = fminf(lo[0], ca.x);
            lo[1] = fminf(lo[1], ca.y);
            lo[2] = fminf(lo[2], ca.z);
            hi[0] = fmaxf(hi[0], cb.x);
            hi[1] = fmaxf(hi[1], cb.y);
            hi[2] = fmaxf(hi[2], cb.z);
        }
    }
    nodes[2ull * id] = make_float4(lo[0], lo[1], lo[2], a.w);
    nodes[2ull * id + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    // the octant-specialised box test needs finite boxes with lo <= hi
    bool ordered = true;
    for (int c = 0; c < 3; ++c)
        ordered = ordered && isfinite(lo[c]) && isfinite(hi[c]) && lo[c] <= hi[c];
    if (!ordered) atomicOr(unordered, 1u);
}

cudaError_t launch_shade_hits(const DevScene& sc, const ShadeDev& sh, const float* verts,
                              const uint32_t* idx, const float4* rays, const float4* hits,
                              unsigned long long n, float* image, cudaStream_t stream) {
    k_shade_hits<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(sc, sh, verts, idx, rays, hits,
                                                                  n, image);
    return cudaGetLastError();
}

cudaError_t launch_render_backward_hits(const DevScene& sc, const ShadeDev& sh,
                                        const float* verts, const uint32_t* idx,
                                        const float4* rays, const float4* hits,
                                        unsigned long long n, const float* g, float* gv,
                                        float* gt, cudaStream_t stream) {
    const bool vec = (reinterpret_cast<uintptr_t>(gt) & 15u) == 0;
    k_render_backward_hits<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
        sc, sh, verts, idx, rays, hits, n, g, gv, gt, vec);
    return cudaGetLastError();
}

cudaError_t render_align_error(unsigned* line) {
    cudaError_t e = cudaMemcpyFromSymbol(line, g_vsr_align_line, sizeof(unsigned));
    if (e != cudaSuccess || *line == 0) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(g_vsr_align_line, &zero, sizeof(unsigned));
}

cudaError_t launch_refit(float4* nodes, const uint32_t* level_nodes,
                         const uint32_t* level_offsets, uint32_t levels, const float* verts,
                         const uint32_t* idx, const uint32_t* order, uint32_t* unordered,
                         cudaStream_t stream) {
    for (uint32_t l = 0; l < levels; ++l) {
        const uint32_t begin = level_offsets[l], count = level_offsets[l + 1] - begin;
        if (count == 0) continue;
        k_refit<<<(count + 255) / 256, 256, 0, stream>>>(nodes, level_nodes + begin, count, verts,
                                                         idx, order, unordered);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ao_shade(const DevScene& sc, const AoArgs& ao, unsigned long long n,
                            cudaStream_t stream) {
    k_ao_shade<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(sc, ao.sh, ao.hits, n, ao.spp,
                                                                ao.occ, ao.image);
    return cudaGetLastError();
}

cudaError_t launch_ao_backward(const DevScene& sc, const AoArgs& ao, unsigned long long n,
                               cudaStream_t stream) {
    const bool vec = (reinterpret_cast<uintptr_t>(ao.grad_texels) & 15u) == 0;
    k_ao_backward<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(sc, ao.sh, ao.hits, ao.occ, n,
                                                                   ao.g, ao.grad_texels, vec);
    return cudaGetLastError();
}

}  // namespace vsr
