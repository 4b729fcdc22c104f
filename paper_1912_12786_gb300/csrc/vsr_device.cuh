// Device-side layout, FP32 tests and the while-while traversal with an
// injected intersector (Zellmann, Section 3.2).
//
// Device layout (built by vsr_bvh_load):
//   nodes  2 x float4 per node: {lo.xyz, ref}, {hi.xyz, 0}.  Siblings are
//          adjacent and start at an even index, so the two children of an
//          inner node are one 64-byte aligned pair (4 x 128-bit loads).
//   ref    packed node reference: inner = (left/2) << 2 | split axis,
//          leaf = 1 << 31 | first << 3 | (count - 1).
//   tris   3 x float4 per leaf slot: {v0.xyz, prim id}, {e1.xyz, 0},
//          {e2.xyz, 0} with e1 = v1 - v0, e2 = v2 - v0, in leaf order.
//   uvs    3 x float2 per original triangle id; geom: texture id per id.
//
// Rounding: the file is compiled with -fmad=false and every product, sum and
// fused multiply-add below is an explicit __fmul_rn / __fadd_rn / __fmaf_rn,
// divisions are IEEE (__fdiv_rn) and denormals are kept, so hit distances,
// barycentrics, box decisions and counts are reproducible bit for bit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Loads through the read-only path.  A translation unit that defines
// VSR_CHECKED_LOADS before including this header gets loads that first check
// the address against the access width, record the source line of a
// misaligned one in g_vsr_align_line (see render.cu) and skip it, so that such
// an access becomes an error code instead of a fault.
#ifdef VSR_CHECKED_LOADS
__device__ unsigned int g_vsr_align_line;
template <class T>
__device__ __forceinline__ T vsr_checked_ldg(const T* p, unsigned line) {
    if (reinterpret_cast<unsigned long long>(p) % sizeof(T)) {
        atomicCAS(&g_vsr_align_line, 0u, line);
        return T{};
    }
    return __ldg(p);
}
#define VSR_LDG(p) ::vsr_checked_ldg((p), __LINE__)
#else
#define VSR_LDG(p) __ldg(p)
#endif

namespace vsr {

constexpr uint32_t kMiss = 0xFFFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kFullMask = 0xFFFFFFFFu;  // all 32 lanes of a warp
constexpr int kClosest = 0;
constexpr int kAny = 1;

enum : uint32_t { kTexU8 = 0, kTexRGBA8 = 1, kTexRGBA32F = 2 };
// Device error word bits: stack overflow and more node visits than nodes
// (neither can happen for a validated blob), a misaligned load skipped, a
// caller-supplied hit record out of range, and a persistent loop that ran
// out of its iteration or time budget (the watchdog).  The checks turn a
// corrupted structure or input into an error instead of a fault or an
// endless loop.
enum : uint32_t {
    kErrStack = 1u,
    kErrSteps = 2u,
    kErrAlign = 4u,
    kErrHit = 8u,
    kErrTimeout = 16u
};

struct TexDesc {
    uint32_t fmt, w, h, pad;
    unsigned long long offset;  // byte offset into texels
    unsigned long long pad2;
};

// Everything a kernel needs to know about a scene (passed by value).
struct DevScene {
    const float4* nodes;
    const float4* tris;
    const float2* uvs;
    const uint32_t* geom;
    const TexDesc* tex;
    const uint8_t* texels;
    uint32_t* err;
    uint32_t nprims, ntex, root_ref, stack_depth;
    uint32_t max_steps;     // node visits per ray never exceed the node count
    uint32_t boxes_ordered; // 1: every node box is finite with lo <= hi (a
                            // validated blob; rechecked by each refit)
    uint32_t pad[2];
    float4 root_a, root_b;  // root box (lo, hi) in .xyz
};

// Which ray each thread traces.  width == 0: thread g takes ray g.  width >
// 0: the rays form a row-major image `width` pixels wide and each warp takes
// a 4 x 8 pixel tile (tiles in row-major order, lanes row-major inside the
// tile), so a warp's rays are neighbours in both image directions.  The
// grid then covers `threads` = tiles_x * tiles_y * 32 threads; threads past
// the image's right or bottom edge take no ray.  perm != null (coherence
// order, width 0): thread g takes ray perm[g], a permutation of the rays
// sorted by origin and direction.  Rays and hits keep the caller's layout in
// every case.
struct RayMap {
    unsigned long long n;        // rays
    unsigned long long threads;  // threads the grid covers
    uint32_t width, tiles_x;
    const uint32_t* perm;        // coherence order, or null
};

// Ray of thread g (< map.threads), or map.n when the thread takes none.
__device__ __forceinline__ unsigned long long ray_of_thread(unsigned long long g,
                                                            const RayMap& m) {
    if (m.perm) return __ldg(m.perm + g);
    if (m.width == 0) return g;
    const uint32_t tile = (uint32_t)(g >> 5), lane = (uint32_t)g & 31u;
    const uint32_t ty = tile / m.tiles_x, tx = tile - ty * m.tiles_x;
    const uint32_t px = tx * 4u + (lane & 3u);
    if (px >= m.width) return m.n;
    const unsigned long long i =
        ((unsigned long long)ty * 8u + (lane >> 2)) * m.width + px;
    return i < m.n ? i : m.n;
}

struct IsectParams {
    uint32_t cutoff_u8;
    float cutoff_f;
    float freq;
    uint32_t kind;
    float clip_lo[3], clip_hi[3];  // clip-box intersector
};

// --------------------------------------------------------------------------
// exact FP32 helpers

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by,
                                      float bz) {
    return __fmaf_rn(ax, bx, __fmaf_rn(ay, by, __fmul_rn(az, bz)));
}

struct Ray {
    float ox, oy, oz, tmin, dx, dy, dz, tmax;
    float ix, iy, iz;     // guarded inverse direction
    float nox, noy, noz;  // -(o * inv)
    uint32_t negmask;     // bit a set iff the sign bit of d[a] is set
};

// Three-input minimum / maximum (one ALU instruction on sm_100-family GPUs).
// Like fminf/fmaxf they ignore a NaN operand; min and max are exact, so any
// grouping of the operands gives the same value.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The two children of an inner node: a 64-byte aligned pair of 32-byte
// records, read as two 256-bit loads (the address is 32-byte aligned by
// construction: the node array comes from cudaMalloc and pair k sits at byte
// 64 k).  Checked builds read them as four checked 128-bit loads.
__device__ __forceinline__ void load_pair(const float4* p, float4& la, float4& lb, float4& ra,
                                          float4& rb) {
#ifdef VSR_CHECKED_LOADS
    la = VSR_LDG(p);
    lb = VSR_LDG(p + 1);
    ra = VSR_LDG(p + 2);
    rb = VSR_LDG(p + 3);
#else
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(la.x), "=f"(la.y), "=f"(la.z), "=f"(la.w), "=f"(lb.x), "=f"(lb.y), "=f"(lb.z),
          "=f"(lb.w)
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(ra.x), "=f"(ra.y), "=f"(ra.z), "=f"(ra.w), "=f"(rb.x), "=f"(rb.y), "=f"(rb.z),
          "=f"(rb.w)
        : "l"(p + 2));
#endif
}

__device__ __forceinline__ float guard_dir(float d) {
    return fabsf(d) < 0x1p-80f ? copysignf(0x1p-80f, d) : d;
}

__device__ __forceinline__ Ray make_ray(float4 a, float4 b) {
    Ray r;
    r.ox = a.x; r.oy = a.y; r.oz = a.z; r.tmin = a.w;
    r.dx = b.x; r.dy = b.y; r.dz = b.z; r.tmax = b.w;
    r.ix = __fdiv_rn(1.0f, guard_dir(b.x));
    r.iy = __fdiv_rn(1.0f, guard_dir(b.y));
    r.iz = __fdiv_rn(1.0f, guard_dir(b.z));
    r.nox = -__fmul_rn(a.x, r.ix);
    r.noy = -__fmul_rn(a.y, r.iy);
    r.noz = -__fmul_rn(a.z, r.iz);
    r.negmask = (signbit(b.x) ? 1u : 0u) | (signbit(b.y) ? 2u : 0u) | (signbit(b.z) ? 4u : 0u);
    return r;
}

// intersect(ray, aabb, inv_dir): slab test over [tmin, tfar].
__device__ __forceinline__ bool box_hit(const Ray& r, float4 lo, float4 hi, float tfar) {
    const float t0x = __fmaf_rn(lo.x, r.ix, r.nox), t1x = __fmaf_rn(hi.x, r.ix, r.nox);
    const float t0y = __fmaf_rn(lo.y, r.iy, r.noy), t1y = __fmaf_rn(hi.y, r.iy, r.noy);
    const float t0z = __fmaf_rn(lo.z, r.iz, r.noz), t1z = __fmaf_rn(hi.z, r.iz, r.noz);
    const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), r.tmin));
    const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tfar));
    return tn <= tf;
}

// box_hit for rays whose direction signs are known at compile time: OCT bit
// a is set iff d[a] has its sign bit set (Ray::negmask).  The guarded inverse
// direction has the sign of d, so along axis a the entry plane is lo[a] for a
// clear bit and hi[a] for a set one, and each axis needs no min/max: five
// ALU-pipe instructions (two three-input max/min, the two limits, one
// compare) instead of eleven.  For a box with finite lo <= hi this is box_hit
// bit for bit: FMA rounding is monotone in the plane coordinate, so the
// plane picked is the one min/max would pick (equal values, at most of
// opposite zero sign, which the comparison does not see); a NaN or infinite
// slab value comes out of both planes alike.  Inverted or non-finite boxes do
// not occur in a validated blob; after a refit the kernels that use this test
// check the scene's box-state word first.  OCT < 0 is box_hit.
template <int OCT>
__device__ __forceinline__ bool box_hit_o(const Ray& r, float4 lo, float4 hi, float tfar) {
    if constexpr (OCT < 0) {
        return box_hit(r, lo, hi, tfar);
    } else {
        const float nx = __fmaf_rn((OCT & 1) ? hi.x : lo.x, r.ix, r.nox);
        const float fx = __fmaf_rn((OCT & 1) ? lo.x : hi.x, r.ix, r.nox);
        const float ny = __fmaf_rn((OCT & 2) ? hi.y : lo.y, r.iy, r.noy);
        const float fy = __fmaf_rn((OCT & 2) ? lo.y : hi.y, r.iy, r.noy);
        const float nz = __fmaf_rn((OCT & 4) ? hi.z : lo.z, r.iz, r.noz);
        const float fz = __fmaf_rn((OCT & 4) ? lo.z : hi.z, r.iz, r.noz);
        return fmax3(nx, ny, fmaxf(nz, r.tmin)) <= fmin3(fx, fy, fminf(fz, tfar));
    }
}

// box_hit that also gives the entry distance tn: the box is hit with a
// smaller far limit t' iff it was hit and tn <= t' (the exit side of the
// comparison does not depend on the far limit).
__device__ __forceinline__ bool box_hit_tn(const Ray& r, float4 lo, float4 hi, float tfar,
                                           float& tn) {
    const float t0x = __fmaf_rn(lo.x, r.ix, r.nox), t1x = __fmaf_rn(hi.x, r.ix, r.nox);
    const float t0y = __fmaf_rn(lo.y, r.iy, r.noy), t1y = __fmaf_rn(hi.y, r.iy, r.noy);
    const float t0z = __fmaf_rn(lo.z, r.iz, r.noz), t1z = __fmaf_rn(hi.z, r.iz, r.noz);
    tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), r.tmin));
    const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tfar));
    return tn <= tf;
}

// intersect(ray, basic_triangle<3,float>): Moller-Trumbore with the fixed
// rounding order.  Returns false when det == 0 (no t, u, v) and, as a shortcut
// that changes no decision, when u alone already rules out a geometric hit
// (u < 0, u > 1 or NaN: with v >= 0 the rounded u + v is at least u).
__device__ __forceinline__ bool tri_test(const Ray& r, float4 a, float4 e1, float4 e2,
                                         float& t, float& u, float& v) {
    const float px = __fmaf_rn(r.dy, e2.z, -__fmul_rn(r.dz, e2.y));
    const float py = __fmaf_rn(r.dz, e2.x, -__fmul_rn(r.dx, e2.z));
    const float pz = __fmaf_rn(r.dx, e2.y, -__fmul_rn(r.dy, e2.x));
    const float det = dot3(e1.x, e1.y, e1.z, px, py, pz);
    if (det == 0.0f) return false;
    const float inv = __fdiv_rn(1.0f, det);
    const float sx = __fsub_rn(r.ox, a.x), sy = __fsub_rn(r.oy, a.y), sz = __fsub_rn(r.oz, a.z);
    u = __fmul_rn(dot3(sx, sy, sz, px, py, pz), inv);
    if (!(u >= 0.0f && u <= 1.0f)) return false;
    const float qx = __fmaf_rn(sy, e1.z, -__fmul_rn(sz, e1.y));
    const float qy = __fmaf_rn(sz, e1.x, -__fmul_rn(sx, e1.z));
    const float qz = __fmaf_rn(sx, e1.y, -__fmul_rn(sy, e1.x));
    v = __fmul_rn(dot3(r.dx, r.dy, r.dz, qx, qy, qz), inv);
    t = __fmul_rn(dot3(e2.x, e2.y, e2.z, qx, qy, qz), inv);
    return true;
}

// --------------------------------------------------------------------------
// intersector arithmetic (Section 4 use cases)

// Interpolated texture coordinate: w0 = (1-u)-v, uv = v*tc2 + (u*tc1 + w0*tc0).
__device__ __forceinline__ float2 lerp_uv(const float2* __restrict__ uvs, uint32_t prim, float u,
                                          float v) {
    const float2 c0 = VSR_LDG(uvs + 3ull * prim), c1 = VSR_LDG(uvs + 3ull * prim + 1),
                 c2 = VSR_LDG(uvs + 3ull * prim + 2);
    const float w0 = __fsub_rn(__fsub_rn(1.0f, u), v);
    float2 r;
    r.x = __fmaf_rn(v, c2.x, __fmaf_rn(u, c1.x, __fmul_rn(w0, c0.x)));
    r.y = __fmaf_rn(v, c2.y, __fmaf_rn(u, c1.y, __fmul_rn(w0, c0.y)));
    return r;
}

__device__ __forceinline__ uint32_t texel_coord(float c, uint32_t n) {
    const float cl = fminf(fmaxf(c, 0.0f), 1.0f);
    const int i = (int)floorf(__fmul_rn(cl, (float)n));
    return (uint32_t)min(i, (int)n - 1);
}

// Alpha-mask decision: nearest texel, clamp to edge.
__device__ __forceinline__ bool alpha_tex_accept(const DevScene& sc, const IsectParams& ip,
                                                 uint32_t prim, float u, float v) {
    const uint32_t g = VSR_LDG(sc.geom + prim);
    if (g == kMiss) return true;
    const float2 uv = lerp_uv(sc.uvs, prim, u, v);
    const uint4 d = VSR_LDG(reinterpret_cast<const uint4*>(sc.tex + g));
    const unsigned long long off = VSR_LDG(&sc.tex[g].offset);
    const uint32_t i = texel_coord(uv.x, d.y), j = texel_coord(uv.y, d.z);
    const unsigned long long k = (unsigned long long)j * d.y + i;
    if (d.x == kTexU8) return VSR_LDG(sc.texels + off + k) >= ip.cutoff_u8;
    if (d.x == kTexRGBA8) return VSR_LDG(sc.texels + off + 4 * k + 3) >= ip.cutoff_u8;
    const float a = VSR_LDG(reinterpret_cast<const float*>(sc.texels + off) + 4 * k + 3);
    return a >= ip.cutoff_f;
}

// Sign of sin(x) (-1, 0 or +1) without evaluating the sine.  With
// k = rint(x / pi) and r = x - k pi, sin(x) = (-1)^k sin(r) and |r| < pi, so
// the sign is (-1)^k sign(r).  r is reduced with pi split in three float32
// parts (Cody and Waite's additive reduction): kPiA has 8 significant bits,
// so x - k kPiA is exact for |x| < 2^22, and each fused multiply-add then
// rounds once.  Near a multiple of pi the error of r is below 2e-11 there,
// while every float32 with |x| < 2^22 lies at least 8.4e-9 from a multiple
// of pi (the closest is next to 161 pi), so the sign is that of the true
// sine for every such x.  For larger |x| the result is deterministic but may
// differ from a correctly rounded sine where |sin x| is tiny.  The parts are
// pi rounded to 8 significant bits, then the remainder rounded to float32
// twice over (kPiA + kPiB + kPiC = pi - 1.7e-19).
constexpr float kInvPi = 0x1.45f306p-2f;  // float32(1 / pi)
constexpr float kPiA = 0x1.92p+1f;        // 3.140625
constexpr float kPiB = 0x1.fb5444p-11f;
constexpr float kPiC = 0x1.68c234p-38f;

__device__ __forceinline__ int sin_sign(float x) {
    const float k = rintf(__fmul_rn(x, kInvPi));
    float r = __fmaf_rn(-k, kPiA, x);
    r = __fmaf_rn(-k, kPiB, r);
    r = __fmaf_rn(-k, kPiC, r);
    const int s = (r > 0.0f) - (r < 0.0f);
    return (__float2int_rz(k) & 1) ? -s : s;
}

// Procedural alpha: accept iff sin(f u) sin(f v) > 0 at the texture
// coordinate, decided from the signs of the two sines (their float32 product
// differs only where it underflows, i.e. both sines below 1e-22).
__device__ __forceinline__ bool proc_alpha_accept(const DevScene& sc, const IsectParams& ip,
                                                  uint32_t prim, float u, float v) {
    const uint32_t g = VSR_LDG(sc.geom + prim);
    if (g == kMiss) return true;
    const float2 uv = lerp_uv(sc.uvs, prim, u, v);
    return sin_sign(__fmul_rn(ip.freq, uv.x)) * sin_sign(__fmul_rn(ip.freq, uv.y)) > 0;
}

// --------------------------------------------------------------------------
// statically injected intersectors: hooks on every box test and triangle
// test, and a verdict on each geometric candidate ("hr.hit &= ...").

// Hooks: begin() sees the ray once; box() and tri() run on every box and
// triangle test (bvh_costs); far() may lower the far limit of node box tests
// and keep() may turn a box the ray hits into a miss (both part of the
// intersector's intersect(ray, aabb) overload, Section 3.2); accept() gives
// the verdict on a candidate hit at distance t.
struct IsectNone {
    static constexpr bool kCounts = false;
    static constexpr bool kTexcoords = false;  // reads geom id and texcoords
    // box hooks that may observe nothing, so that a lane may test boxes
    // ahead of the plain order (warp_step); whether they do for a ray is
    // box_hooks_silent's answer
    static constexpr bool kMaySpeculate = true;
    // resident 256-thread blocks per SM the persistent and lock-step kernels
    // are compiled for, per query (1: no register budget)
    static constexpr int kMinBlocksClosest = 1;
    static constexpr int kMinBlocksAny = 1;
    __device__ __forceinline__ void begin(const Ray&, const IsectParams&) {}
    __device__ __forceinline__ void box() {}
    __device__ __forceinline__ void tri() {}
    __device__ __forceinline__ float far(float tfar) const { return tfar; }
    __device__ __forceinline__ bool keep(const IsectParams&, float4, float4) const { return true; }
    __device__ __forceinline__ bool accept(const DevScene&, const IsectParams&, uint32_t, float,
                                           float, float) {
        return true;
    }
    __device__ __forceinline__ uint2 counters() const { return make_uint2(0, 0); }
};

// basic_intersector: forwards intersect() unchanged.
struct IsectDefault : IsectNone {};

struct IsectAlphaTex : IsectNone {
    static constexpr bool kTexcoords = true;
    __device__ __forceinline__ bool accept(const DevScene& sc, const IsectParams& ip,
                                           uint32_t prim, float u, float v, float) {
        return alpha_tex_accept(sc, ip, prim, u, v);
    }
};

struct IsectProcAlpha : IsectNone {
    static constexpr bool kTexcoords = true;
    __device__ __forceinline__ bool accept(const DevScene& sc, const IsectParams& ip,
                                           uint32_t prim, float u, float v, float) {
        return proc_alpha_accept(sc, ip, prim, u, v);
    }
};

// bvh_costs: ++num_boxes per box test, ++num_tris per triangle test.
struct IsectCount : IsectNone {
    static constexpr bool kCounts = true;
    static constexpr bool kMaySpeculate = false;  // every box test is counted
    uint32_t num_boxes = 0, num_tris = 0;
    __device__ __forceinline__ void box() { ++num_boxes; }
    __device__ __forceinline__ void tri() { ++num_tris; }
    __device__ __forceinline__ uint2 counters() const { return make_uint2(num_boxes, num_tris); }
};

// Clip box: a node box that does not overlap [clip_lo, clip_hi] counts as
// missed (its subtree is skipped), node box tests stop where the ray leaves
// the clip box, and a candidate is accepted iff its hit point fmaf(t, d, o)
// lies in the closed box.
struct IsectClip : IsectNone {
    float ox, oy, oz, dx, dy, dz, t_exit;
    __device__ __forceinline__ void begin(const Ray& r, const IsectParams& ip) {
        ox = r.ox;
        oy = r.oy;
        oz = r.oz;
        dx = r.dx;
        dy = r.dy;
        dz = r.dz;
        const float t0x = __fmaf_rn(ip.clip_lo[0], r.ix, r.nox);
        const float t1x = __fmaf_rn(ip.clip_hi[0], r.ix, r.nox);
        const float t0y = __fmaf_rn(ip.clip_lo[1], r.iy, r.noy);
        const float t1y = __fmaf_rn(ip.clip_hi[1], r.iy, r.noy);
        const float t0z = __fmaf_rn(ip.clip_lo[2], r.iz, r.noz);
        const float t1z = __fmaf_rn(ip.clip_hi[2], r.iz, r.noz);
        const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fminf(t0z, t1z));
        const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fmaxf(t0z, t1z));
        t_exit = tn <= tf ? tf : __int_as_float(0xff800000);
    }
    __device__ __forceinline__ float far(float tfar) const { return fminf(tfar, t_exit); }
    __device__ __forceinline__ bool keep(const IsectParams& ip, float4 lo, float4 hi) const {
        return lo.x <= ip.clip_hi[0] && hi.x >= ip.clip_lo[0] && lo.y <= ip.clip_hi[1] &&
               hi.y >= ip.clip_lo[1] && lo.z <= ip.clip_hi[2] && hi.z >= ip.clip_lo[2];
    }
    __device__ __forceinline__ bool accept(const DevScene&, const IsectParams& ip, uint32_t,
                                           float, float, float t) {
        const float px = __fmaf_rn(t, dx, ox), py = __fmaf_rn(t, dy, oy),
                    pz = __fmaf_rn(t, dz, oz);
        return px >= ip.clip_lo[0] && px <= ip.clip_hi[0] && py >= ip.clip_lo[1] &&
               py <= ip.clip_hi[1] && pz >= ip.clip_lo[2] && pz <= ip.clip_hi[2];
    }
};

// Measurement counters: box tests, triangle tests, intersector
// consultations, and consultations that fetched texture coordinates.
struct Stats {
    uint32_t boxes = 0, tris = 0, cands = 0, texs = 0;
};

// (t, prim) comes before (t2, prim2) in the closest-hit / multi-hit order.
__device__ __forceinline__ bool hit_before(float t, uint32_t p, float t2, uint32_t p2) {
    return t < t2 || (t == t2 && p < p2);
}

// The running result of the closest-hit and any-hit queries.  The traversal
// bounds its search by t, asks before() whether a candidate would improve the
// result and hands every accepted candidate to take().
struct Best {
    float t, u, v;
    uint32_t prim;
    __device__ __forceinline__ void init(float tmax) {
        t = tmax;
        u = 0.0f;
        v = 0.0f;
        prim = kMiss;
    }
    __device__ __forceinline__ void take(float tc, float uc, float vc, uint32_t pc) {
        t = tc;
        u = uc;
        v = vc;
        prim = pc;
    }
    __device__ __forceinline__ bool before(float tc, uint32_t pc) const {
        return hit_before(tc, pc, t, prim);
    }
    __device__ __forceinline__ void fail() { prim = kMiss; }
};

// The running result of the multi-hit query: the first n accepted hits in
// ascending (t, prim) order, kept as (t, prim) in this thread's columns of
// shared memory (stride words apart, like the traversal stack; the
// barycentrics are recomputed for the final entries).  (t, prim) mirror entry
// n - 1, so the traversal's closest-hit bound is the multi-hit bound; with
// n == 1 the query is the closest-hit query.  An insertion shifts only the
// entries the new hit passes, and hits tend to arrive front to back.
struct MultiBest {
    float* tk;
    uint32_t* pk;
    uint32_t stride, n;
    float t;
    uint32_t prim;
    __device__ __forceinline__ void init(float tmax) {
        for (uint32_t k = 0; k < n; ++k) {
            tk[k * stride] = tmax;
            pk[k * stride] = kMiss;
        }
        t = tmax;
        prim = kMiss;
    }
    // Insert a candidate that comes before entry n - 1 (the caller checked).
    __device__ __forceinline__ void take(float tc, float, float, uint32_t pc) {
        uint32_t k = n - 1;
        while (k > 0) {
            const float tp = tk[(k - 1) * stride];
            const uint32_t pp = pk[(k - 1) * stride];
            if (!hit_before(tc, pc, tp, pp)) break;
            tk[k * stride] = tp;
            pk[k * stride] = pp;
            --k;
        }
        tk[k * stride] = tc;
        pk[k * stride] = pc;
        t = tk[(n - 1) * stride];
        prim = pk[(n - 1) * stride];
    }
    __device__ __forceinline__ bool before(float tc, uint32_t pc) const {
        return hit_before(tc, pc, t, prim);
    }
    __device__ __forceinline__ void fail() {
        for (uint32_t k = 0; k < n; ++k) pk[k * stride] = kMiss;
        prim = kMiss;
    }
};

// --------------------------------------------------------------------------
// The traversal stack of node references: the top K entries in registers,
// the rest in this thread's column of a shared-memory stack (`col`, `stride`
// words between levels).  A push with K entries held moves the deepest one
// to shared memory; a pop refills it from there, so a pop never waits on
// shared memory for the node it returns.  K == 0 keeps every entry in
// shared memory.  The order of entries is the LIFO order either way, so the
// traversal visits nodes in the same order for every K.
template <int K>
struct ShortStack {
    static constexpr int kRegs = K;
    uint32_t top[K > 0 ? K : 1];
    uint32_t* col;
    uint32_t stride;
    uint32_t n;  // entries held (registers and shared memory)
    __device__ __forceinline__ void init(uint32_t* column, uint32_t words_apart) {
        col = column;
        stride = words_apart;
        n = 0;
    }
    // The caller checked n against the tree depth.
    __device__ __forceinline__ void push(uint32_t x) {
        if (K == 0) {
            col[n * stride] = x;
        } else {
            if (n >= (uint32_t)K) col[(n - K) * stride] = top[K - 1];
#pragma unroll
            for (int j = K - 1; j > 0; --j) top[j] = top[j - 1];
            top[0] = x;
        }
        ++n;
    }
    // The caller checked n > 0.
    __device__ __forceinline__ uint32_t pop() {
        --n;
        if (K == 0) return col[n * stride];
        const uint32_t x = top[0];
#pragma unroll
        for (int j = 0; j < K - 1; ++j) top[j] = top[j + 1];
        if (n >= (uint32_t)K) top[K - 1] = col[(n - K) * stride];
        return x;
    }
};

// Shared-memory words per thread for a tree of `depth` levels with K
// entries in registers.
__host__ __device__ __forceinline__ uint32_t stack_words(uint32_t depth, uint32_t k) {
    return depth > k ? depth - k : 1u;
}

// The while-while traversal (Section 3.2) with the intersector's hooks.
// OCT >= 0: every node box test is box_hit_o<OCT> (the caller checked that
// the ray's direction octant is OCT and that the scene's boxes are finite
// and ordered), so the visits and results are those of OCT = -1.
template <int Q, class H, bool STATS, int OCT = -1, class B = Best, class S>
__device__ __forceinline__ void traverse_body(const DevScene& sc, const IsectParams& ip,
                                              const Ray& r, H& h, B& best, Stats& st, S& stk) {
    best.init(r.tmax);
    stk.n = 0;
    if (sc.nprims == 0) return;
    h.begin(r, ip);
    h.box();
    if (STATS) st.boxes++;
    if (!box_hit_o<OCT>(r, sc.root_a, sc.root_b, h.far(best.t)) ||
        !h.keep(ip, sc.root_a, sc.root_b))
        return;
    uint32_t ref = sc.root_ref;
    uint32_t steps = 0;
    for (;;) {  // while ray not terminated
        // While the node is inner.  Descent ends by construction: a loaded
        // blob is a tree whose children sit at higher node indices than
        // their parent, so no counter is needed here (leaf visits are
        // counted below).
        while (!(ref & kLeafBit)) {
            const float4* p = sc.nodes + 4ull * (ref >> 2);
            float4 la, lb, ra, rb;
            load_pair(p, la, lb, ra, rb);
            const float tfar = h.far((Q == kClosest) ? best.t : r.tmax);
            h.box();
            h.box();
            if (STATS) st.boxes += 2;
            const bool hl = box_hit_o<OCT>(r, la, lb, tfar) && h.keep(ip, la, lb);
            const bool hr = box_hit_o<OCT>(r, ra, rb, tfar) && h.keep(ip, ra, rb);
            const uint32_t rl = __float_as_uint(la.w), rr = __float_as_uint(ra.w);
            if (hl && hr) {
                const bool neg = OCT >= 0 ? (((unsigned)OCT >> (ref & 3u)) & 1u)
                                          : ((r.negmask >> (ref & 3u)) & 1u);
                if (stk.n >= sc.stack_depth) {  // unreachable for a validated blob
                    atomicOr(sc.err, kErrStack);
                    best.fail();
                    return;
                }
                stk.push(neg ? rl : rr);
                ref = neg ? rr : rl;
            } else if (hl) {
                ref = rl;
            } else if (hr) {
                ref = rr;
            } else {
                if (stk.n == 0) return;
                ref = stk.pop();
            }
        }
        {  // found a leaf: test its primitives
            if (++steps > sc.max_steps) {
                atomicOr(sc.err, kErrSteps);
                best.fail();
                return;
            }
            const uint32_t first = (ref >> 3) & 0x0FFFFFFFu;
            const uint32_t cnt = (ref & 7u) + 1u;
            const float4* tp = sc.tris + 3ull * first;
            for (uint32_t k = 0; k < cnt; ++k) {
                const float4 a = VSR_LDG(tp + 3 * k), e1 = VSR_LDG(tp + 3 * k + 1),
                             e2 = VSR_LDG(tp + 3 * k + 2);
                h.tri();
                if (STATS) st.tris++;
                float t, u, v;
                if (!tri_test(r, a, e1, e2, t, u, v)) continue;
                const bool geo = u >= 0.0f && v >= 0.0f && __fadd_rn(u, v) <= 1.0f;
                if (!geo || !(t > r.tmin) || !(t < r.tmax)) continue;
                const uint32_t prim = __float_as_uint(a.w);
                if (Q == kClosest) {
                    if (!best.before(t, prim)) continue;
                }
                if (STATS) {
                    st.cands++;
                    if (H::kTexcoords && VSR_LDG(sc.geom + prim) != kMiss) st.texs++;
                }
                if (!h.accept(sc, ip, prim, u, v, t)) continue;
                best.take(t, u, v, prim);
                if (Q == kAny) return;
            }
        }
        if (stk.n == 0) return;
        ref = stk.pop();
    }
}

// Full query: traversal, then every miss (root missed, empty or inactive
// interval, nothing accepted) is reported as t = +inf, u = v = 0.
template <int Q, class H, bool STATS, int OCT = -1, class S>
__device__ __forceinline__ void traverse(const DevScene& sc, const IsectParams& ip, const Ray& r,
                                         H& h, Best& best, Stats& st, S& stk) {
    traverse_body<Q, H, STATS, OCT>(sc, ip, r, h, best, st, stk);
    if (best.prim == kMiss) {
        best.t = __int_as_float(0x7f800000);
        best.u = 0.0f;
        best.v = 0.0f;
    }
}

// The same traversal split into resumable pieces for persistent kernels,
// whose lanes interleave rays: traverse_start tests the root box and
// returns whether the ray is still live; each traverse_step runs one outer
// iteration of the while-while loop (descend to a leaf, test it, pop the
// next node) and returns true when the ray has finished.  Composed, they
// visit nodes and primitives in exactly the order of traverse_body.  The
// running result B is Best or one with its interface (MultiBest, the
// instancing result).
template <int Q, class H, bool STATS, class B, class S>
__device__ __forceinline__ bool traverse_start(const DevScene& sc, const IsectParams& ip,
                                               const Ray& r, H& h, B& best, Stats& st,
                                               uint32_t& ref, uint32_t& steps, S& stk) {
    best.init(r.tmax);
    stk.n = 0;
    steps = 0;
    if (sc.nprims == 0) return false;
    h.begin(r, ip);
    h.box();
    if (STATS) st.boxes++;
    if (!box_hit(r, sc.root_a, sc.root_b, h.far(best.t)) || !h.keep(ip, sc.root_a, sc.root_b))
        return false;
    ref = sc.root_ref;
    return true;
}

template <int Q, class H, bool STATS, class B, class S>
__device__ __forceinline__ bool traverse_step(const DevScene& sc, const IsectParams& ip,
                                              const Ray& r, H& h, B& best, Stats& st,
                                              uint32_t& ref, uint32_t& steps, S& stk) {
    // Descent ends by construction as in traverse_body; the persistent and
    // batched kernels that run these steps keep the per-node visit bound as
    // well, so their outer loops stay bounded whatever the node data.
    while (!(ref & kLeafBit)) {
        if (++steps > sc.max_steps) {
            atomicOr(sc.err, kErrSteps);
            best.fail();
            return true;
        }
        const float4* p = sc.nodes + 4ull * (ref >> 2);
        float4 la, lb, ra, rb;
        load_pair(p, la, lb, ra, rb);
        const float tfar = h.far((Q == kClosest) ? best.t : r.tmax);
        h.box();
        h.box();
        if (STATS) st.boxes += 2;
        const bool hl = box_hit(r, la, lb, tfar) && h.keep(ip, la, lb);
        const bool hr = box_hit(r, ra, rb, tfar) && h.keep(ip, ra, rb);
        const uint32_t rl = __float_as_uint(la.w), rr = __float_as_uint(ra.w);
        if (hl && hr) {
            const bool neg = (r.negmask >> (ref & 3u)) & 1u;
            if (stk.n >= sc.stack_depth) {
                atomicOr(sc.err, kErrStack);
                best.fail();
                return true;
            }
            stk.push(neg ? rl : rr);
            ref = neg ? rr : rl;
        } else if (hl) {
            ref = rl;
        } else if (hr) {
            ref = rr;
        } else {
            if (stk.n == 0) return true;
            ref = stk.pop();
        }
    }
    if (++steps > sc.max_steps) {
        atomicOr(sc.err, kErrSteps);
        best.fail();
        return true;
    }
    const uint32_t first = (ref >> 3) & 0x0FFFFFFFu;
    const uint32_t cnt = (ref & 7u) + 1u;
    const float4* tp = sc.tris + 3ull * first;
    for (uint32_t k = 0; k < cnt; ++k) {
        const float4 a = VSR_LDG(tp + 3 * k), e1 = VSR_LDG(tp + 3 * k + 1),
                     e2 = VSR_LDG(tp + 3 * k + 2);
        h.tri();
        if (STATS) st.tris++;
        float t, u, v;
        if (!tri_test(r, a, e1, e2, t, u, v)) continue;
        const bool geo = u >= 0.0f && v >= 0.0f && __fadd_rn(u, v) <= 1.0f;
        if (!geo || !(t > r.tmin) || !(t < r.tmax)) continue;
        const uint32_t prim = __float_as_uint(a.w);
        if (Q == kClosest) {
            if (!best.before(t, prim)) continue;
        }
        if (STATS) {
            st.cands++;
            if (H::kTexcoords && VSR_LDG(sc.geom + prim) != kMiss) st.texs++;
        }
        if (!h.accept(sc, ip, prim, u, v, t)) continue;
        best.take(t, u, v, prim);
        if (Q == kAny) return true;
    }
    if (stk.n == 0) return true;
    ref = stk.pop();
    return false;
}

// The primitive loop body of the traversal for one triangle of a leaf (tp:
// its three float4).  Returns true when the query has its answer (an
// accepted any hit).
template <int Q, class H, bool STATS, class B>
__device__ __forceinline__ bool test_prim(const DevScene& sc, const IsectParams& ip,
                                          const Ray& r, H& h, B& best, Stats& st,
                                          const float4* tp) {
    const float4 a = VSR_LDG(tp), e1 = VSR_LDG(tp + 1), e2 = VSR_LDG(tp + 2);
    h.tri();
    if (STATS) st.tris++;
    float t, u, v;
    if (!tri_test(r, a, e1, e2, t, u, v)) return false;
    const bool geo = u >= 0.0f && v >= 0.0f && __fadd_rn(u, v) <= 1.0f;
    if (!geo || !(t > r.tmin) || !(t < r.tmax)) return false;
    const uint32_t prim = __float_as_uint(a.w);
    if (Q == kClosest) {
        if (!best.before(t, prim)) return false;
    }
    if (STATS) {
        st.cands++;
        if (H::kTexcoords && VSR_LDG(sc.geom + prim) != kMiss) st.texs++;
    }
    if (!h.accept(sc, ip, prim, u, v, t)) return false;
    best.take(t, u, v, prim);
    return Q == kAny;
}

// Where a lane that holds a leaf may keep descending (warp_step): an
// intersector whose box hooks may observe nothing, and no measurement
// counters (box_hooks_silent then decides for the ray, at compile time for
// the static intersectors).  Any hit: the far limit is the ray's tmax, which
// never changes, so speculation needs no bookkeeping.  Closest hit: the far
// limit shrinks when the held leaf improves the result, so speculation
// records entry distances (in a shared-memory column beside the stack's,
// for the shared-memory stack, K == 0) and undoes what the new limit culls.
template <int Q, class H, bool STATS, int K>
struct Speculate {
    static constexpr bool any = Q == kAny && H::kMaySpeculate && !STATS;
    static constexpr bool closest = Q == kClosest && H::kMaySpeculate && !STATS && K == 0;
    static constexpr bool value = any || closest;
};

// Whether h's box hooks observe nothing (a static intersector: unless it
// counts).  The dynamic intersector overloads this with a run-time answer.
template <class H>
__device__ __forceinline__ bool box_hooks_silent(const H&) {
    return !H::kCounts;
}

// Register budget of the persistent and lock-step kernels with intersector
// H for query Q, as resident 256-thread blocks per SM (__launch_bounds__).
template <int Q, class H>
__host__ __device__ constexpr int min_blocks() {
    return Q == kClosest ? H::kMinBlocksClosest : H::kMinBlocksAny;
}

// Per-ray setup of the intersector of a ray a persistent loop claims: none
// for the static intersectors; the dynamic intersector overloads this to
// bind its callbacks.
template <class H>
__device__ __forceinline__ void isect_setup(H&, const IsectParams&, const DevScene*) {}

// A reached leaf is held for testing and the next node taken from the stack.
template <class S>
__device__ __forceinline__ void hold_leaf(uint32_t& ref, bool& more, uint32_t& leaf, bool& pend,
                                          S& stk) {
    if (more && !pend && (ref & kLeafBit)) {
        leaf = ref;
        pend = true;
        if (stk.n)
            ref = stk.pop();
        else
            more = false;
    }
}

// One outer iteration of the while-while traversal (Section 3.2) run by the
// whole warp in lock step: all 32 lanes call it, lanes without a ray with
// busy = false.  The node loop and the primitive loop repeat while any lane
// needs them and every pass ends in a full-warp vote, so lanes that diverge
// inside a pass meet again at the next one.  (With independent thread
// scheduling a divergent loop lets the lanes of a warp drift onto different
// iterations, each group then issuing on its own.)
//
// Per lane: `ref` is the next node to visit when `more`; `leaf` is a leaf
// reached and not yet tested when `pend`.  The descent runs until every busy
// lane holds a leaf or has run out of nodes.  Where Speculate holds, a lane
// that already holds a leaf keeps descending toward its next one while other
// lanes are still looking (the speculative traversal of Aila and Laine,
// 2009).  Then each lane holding a leaf tests its primitives, one per pass.
//
// Speculation leaves every result and the sequence of tested leaves as in
// traverse_body:
//   - any hit: the far limit is the ray's tmax, so a speculating lane visits
//     the nodes the plain order visits after the held leaf, in that order;
//   - closest hit: a speculating lane tests boxes against the far limit of
//     before the held leaf (tf0), which the leaf may lower (to tf).  Each
//     entry pushed while speculating keeps, in `tcol`, the largest entry
//     distance on the way to it (`path`: the node it was pushed from and its
//     ancestors up to the last entry popped, itself included).  The plain
//     order would have reached that node iff this distance is <= tf: box
//     tests along the way passed with tf0 >= tf, and a box hit with far
//     limit tf0 is hit with tf iff its entry distance is <= tf.  So after
//     the leaf test, entries above `sbase` (pushed while speculating) whose
//     distance exceeds tf are dropped, order kept, and so is `ref` when its
//     own path distance exceeds tf; what is left is what the plain order
//     holds at the same point, and the leaves come in its order.
// Returns true on busy lanes whose ray has finished (result in best).
template <int Q, class H, bool STATS, class B, class S>
__device__ __forceinline__ bool warp_step(const DevScene& sc, const IsectParams& ip,
                                          const Ray& r, H& h, B& best, Stats& st, bool busy,
                                          uint32_t& ref, bool& more, uint32_t& leaf, bool& pend,
                                          uint32_t& steps, S& stk, float* tcol) {
    using Spec = Speculate<Q, H, STATS, S::kRegs>;
    const bool spec = Spec::value && box_hooks_silent(h);
    const bool track = Spec::closest && spec;
    const float kNegInf = -__int_as_float(0x7f800000);
    bool done = false;
    uint32_t sbase = 0;           // track: entries at or above were pushed speculating
    float path = kNegInf;         // track: largest entry distance on the way to ref
    float tf0 = 0.0f;             // track: the far limit speculation used
    if (busy) hold_leaf(ref, more, leaf, pend, stk);
    if (track && busy && pend) {
        sbase = stk.n;
        tf0 = h.far(best.t);
    }
    for (;;) {  // while some lane is still looking for a leaf
        const bool seek = busy && !done && more && !pend;  // then ref is an inner node
        if (!__any_sync(kFullMask, seek)) break;
        if (busy && !done && more && !(ref & kLeafBit) && (spec || !pend)) {
            if (++steps > sc.max_steps) {
                atomicOr(sc.err, kErrSteps);
                best.fail();
                done = true;
            } else {
                const float4* p = sc.nodes + 4ull * (ref >> 2);
                float4 la, lb, ra, rb;
                load_pair(p, la, lb, ra, rb);
                const float tfar = h.far((Q == kClosest) ? best.t : r.tmax);
                h.box();
                h.box();
                if (STATS) st.boxes += 2;
                float tnl = 0.0f, tnr = 0.0f;
                const bool hl = box_hit_tn(r, la, lb, tfar, tnl) && h.keep(ip, la, lb);
                const bool hr = box_hit_tn(r, ra, rb, tfar, tnr) && h.keep(ip, ra, rb);
                const uint32_t rl = __float_as_uint(la.w), rr = __float_as_uint(ra.w);
                if (hl && hr) {
                    const bool neg = (r.negmask >> (ref & 3u)) & 1u;
                    if (stk.n >= sc.stack_depth) {
                        atomicOr(sc.err, kErrStack);
                        best.fail();
                        done = true;
                    } else {
                        if (track) tcol[stk.n * stk.stride] = fmaxf(path, neg ? tnl : tnr);
                        stk.push(neg ? rl : rr);
                        ref = neg ? rr : rl;
                        if (track) path = fmaxf(path, neg ? tnr : tnl);
                    }
                } else if (hl) {
                    ref = rl;
                    if (track) path = fmaxf(path, tnl);
                } else if (hr) {
                    ref = rr;
                    if (track) path = fmaxf(path, tnr);
                } else if (stk.n) {
                    ref = stk.pop();
                    if (track) {
                        if (stk.n >= sbase) {
                            path = tcol[stk.n * stk.stride];
                        } else {  // an entry of the plain order
                            sbase = stk.n;
                            path = kNegInf;
                        }
                    }
                } else {
                    more = false;
                }
                if (!done) {
                    const bool held = pend;
                    hold_leaf(ref, more, leaf, pend, stk);
                    if (track && pend && !held) {  // speculation starts here
                        sbase = stk.n;
                        path = kNegInf;
                        tf0 = h.far(best.t);
                    }
                }
            }
        }
    }
    // test the held leaves, one primitive of every lane per pass
    uint32_t cnt = 0;
    const float4* tp = nullptr;
    if (busy && !done && pend) {
        if (++steps > sc.max_steps) {
            atomicOr(sc.err, kErrSteps);
            best.fail();
            done = true;
        } else {
            cnt = (leaf & 7u) + 1u;
            tp = sc.tris + 3ull * ((leaf >> 3) & 0x0FFFFFFFu);
        }
    }
    for (uint32_t k = 0; __any_sync(kFullMask, k < cnt); ++k) {
        if (k < cnt && test_prim<Q, H, STATS>(sc, ip, r, h, best, st, tp + 3 * k)) {
            done = true;
            cnt = 0;
        }
    }
    if (busy && !done) {
        if (track && pend) {
            const float tf = h.far(best.t);
            if (tf < tf0) {  // the leaf lowered the far limit: drop what it culls
                uint32_t j = sbase;
                for (uint32_t i = sbase; i < stk.n; ++i) {
                    const float tn = tcol[i * stk.stride];
                    if (tn <= tf) {
                        stk.col[j * stk.stride] = stk.col[i * stk.stride];
                        tcol[j * stk.stride] = tn;
                        ++j;
                    }
                }
                stk.n = j;
                if (more && path > tf) {
                    if (stk.n)
                        ref = stk.pop();
                    else
                        more = false;
                }
            }
        }
        pend = false;
        hold_leaf(ref, more, leaf, pend, stk);
        if (!pend && !more) done = true;
    }
    return busy && done;
}

// Shared-memory words per thread of the entry-distance column that
// closest-hit speculation keeps beside the stack (0 where it does not run).
template <int Q, class H, bool STATS, int K>
__host__ __device__ constexpr uint32_t spec_words(uint32_t depth) {
    return Speculate<Q, H, STATS, K>::closest ? depth : 0u;
}

// Budget of a persistent loop: outer iterations per warp (0: no limit) and
// nanoseconds of the global timer per warp (0: no limit).  When either runs
// out the warp records kErrTimeout, marks its rays in flight as failed and
// leaves the loop.
struct Watchdog {
    unsigned long long max_iters;
    unsigned long long max_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Whether a persistent warp has used up its budget.  Called by all 32 lanes
// with the same `iters`; the result is the same on every lane.
__device__ __forceinline__ bool watchdog_expired(const Watchdog& wd, unsigned long long iters,
                                                 unsigned long long t0) {
    if (wd.max_iters && iters > wd.max_iters) return true;
    if (wd.max_ns && (iters & 255ull) == 0ull)
        return __any_sync(kFullMask, global_ns() - t0 > wd.max_ns) != 0;
    return false;
}

// The claim loop of the persistent kernels: warps that take rays from a
// global counter (`work`, thread slots of `map`) with one atomic per warp and
// refill idle lanes when fewer than `refill` of 32 hold a ray (ballot +
// popc), after Aila and Laine's persistent threads.  Per ray:
//   start(i)  begins ray i on this lane, returns whether it needs steps;
//   step(b)   one step of the lane's ray; returns true when it has finished.
//             With LS all 32 lanes call it (b: the lane holds a ray) and it
//             must be a converged, warp-synchronous step; otherwise only
//             lanes holding a ray call it (b true) and the warp reconverges
//             after it;
//   finish(i) writes ray i's results;
//   fail()    marks the lane's result as failed (the watchdog ran out).
//
// Control flow: every iteration starts with all 32 lanes converged at the
// first vote.  The claim block runs on a warp-uniform condition; inside it
// only the lanes without a ray take new ones, and the second vote closes
// that divergent part.  The loop's exits (all lanes idle and the counter
// passed the end, or the watchdog) are uniform decisions.  No lane waits on
// another warp or block.  Each iteration claims at least one ray or advances
// some lane's ray (bounded per ray by the traversal's own visit bound), so
// the loop ends; the watchdog bounds it whatever happens.
template <bool LS, class Start, class Step, class Finish, class Fail>
__device__ __forceinline__ void persistent_rays(const RayMap& map, unsigned long long* work,
                                                uint32_t refill, const Watchdog& wd,
                                                uint32_t* err, Start&& start, Step&& step,
                                                Finish&& finish, Fail&& fail) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    bool has = false;        // lane holds a ray in flight
    bool exhausted = false;  // warp-uniform: the counter passed the last slot
    unsigned long long ri = 0;
    const unsigned long long t0 = wd.max_ns ? global_ns() : 0ull;
    unsigned long long iters = 0;
    for (;;) {
        const uint32_t busy = __ballot_sync(kFullMask, has);
        if (!exhausted && (uint32_t)__popc(busy) < refill) {
            const uint32_t idle = ~busy;
            const uint32_t nidle = (uint32_t)__popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)nidle);
            base = __shfl_sync(kFullMask, base, 0);
            if (base + nidle >= map.threads) exhausted = true;
            if (!has) {
                const unsigned long long slot = base + (unsigned long long)__popc(idle & lt_mask);
                ri = slot < map.threads ? ray_of_thread(slot, map) : map.n;
                if (ri < map.n) {
                    has = start(ri);
                    if (!has) finish(ri);
                }
            }
        }
        const uint32_t live = __ballot_sync(kFullMask, has);
        if (live == 0u && exhausted) break;
        if (watchdog_expired(wd, ++iters, t0)) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            if (has) {
                fail();
                finish(ri);
                has = false;
            }
            break;
        }
        if constexpr (LS) {
            if (step(has)) {
                finish(ri);
                has = false;
            }
        } else {
            if (has && step(true)) {
                finish(ri);
                has = false;
            }
            __syncwarp();
        }
    }
}

// Ambient-occlusion sampling frame at a hit: face normal of the triangle
// (v1 - v0) x (v2 - v0) turned against the ray direction d, tangent frame of
// Duff et al. (2017, "Building an orthonormal basis, revisited").  FP32.
struct AoFrame {
    float nx, ny, nz, t1x, t1y, t1z, t2x, t2y, t2z;
};

__device__ __forceinline__ AoFrame ao_frame(const float* __restrict__ verts,
                                            const uint32_t* __restrict__ idx, uint32_t prim,
                                            float dx, float dy, float dz) {
    const float* v0 = verts + 3ull * idx[3ull * prim];
    const float* v1 = verts + 3ull * idx[3ull * prim + 1];
    const float* v2 = verts + 3ull * idx[3ull * prim + 2];
    const float e1x = v1[0] - v0[0], e1y = v1[1] - v0[1], e1z = v1[2] - v0[2];
    const float e2x = v2[0] - v0[0], e2y = v2[1] - v0[1], e2z = v2[2] - v0[2];
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    if (len > 0.0f) {
        nx /= len;
        ny /= len;
        nz /= len;
    } else {
        nx = 0.0f;
        ny = 0.0f;
        nz = 1.0f;
    }
    if (nx * dx + ny * dy + nz * dz > 0.0f) {
        nx = -nx;
        ny = -ny;
        nz = -nz;
    }
    const float sg = copysignf(1.0f, nz);
    const float ca = -1.0f / (sg + nz);
    const float cb = nx * ny * ca;
    return AoFrame{nx, ny, nz, 1.0f + sg * nx * nx * ca, sg * cb, -sg * nx,
                   cb, sg + ny * ny * ca, -ny};
}

// Cosine-distributed direction for the uniforms (x1, x2).
__device__ __forceinline__ float4 ao_direction(const AoFrame& f, float2 x, float tmax) {
    const float rr = sqrtf(x.x), z = sqrtf(1.0f - x.x);
    float sp, cp;
    sincospif(2.0f * x.y, &sp, &cp);
    return make_float4(rr * cp * f.t1x + rr * sp * f.t2x + z * f.nx,
                       rr * cp * f.t1y + rr * sp * f.t2y + z * f.ny,
                       rr * cp * f.t1z + rr * sp * f.t2z + z * f.nz, tmax);
}

// Miss record normalisation shared by all kernels.
__device__ __forceinline__ void finish_miss(Best& best) {
    if (best.prim == kMiss) {
        best.t = __int_as_float(0x7f800000);
        best.u = 0.0f;
        best.v = 0.0f;
    }
}

__device__ __forceinline__ float4 hit_record(const Best& b) {
    return make_float4(b.t, b.u, b.v, __uint_as_float(b.prim));
}

}  // namespace vsr
