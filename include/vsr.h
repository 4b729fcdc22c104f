/*
 * vsr.h -- C ABI of the GB300 custom-intersector ray traversal library.
 *
 * Method (Zellmann, "Adding Custom Intersectors to the C++ Ray Tracing
 * Template Library Visionaray"):
 *   - Section 3.1: a custom intersector wraps intersect(ray, primitive); it
 *     calls the built-in test, may inspect the hit record (barycentrics,
 *     primitive id) and clears hr.hit to reject a candidate, which makes the
 *     traversal continue.  The default intersector forwards the built-in
 *     result unchanged.  Queries: closest hit and any hit over a BVH.
 *   - Section 3.2: the BVH traversal (while-while, after Aila and Laine 2009)
 *     calls intersect for node boxes and for primitives; both calls are
 *     replaced by the intersector, statically at compile time.
 *   - Section 1: callback libraries instead check at run time whether a
 *     callback is registered and call it through a function pointer.
 *   - Section 4: intersectors for an alpha-mask texture, a procedural alpha
 *     function of the texture coordinate, and bvh_costs, which counts box and
 *     triangle tests for a heat map.
 *
 * Here the intersectors are compiled in as template instantiations
 * (VSR_DISPATCH_STATIC) and, for comparison, reached through a device
 * function-pointer table checked at run time (VSR_DISPATCH_DYNAMIC).
 *
 * Conventions for every entry point:
 *   - returns vsr_status; no C++ exception crosses the ABI;
 *   - invalid arguments are rejected before any launch (VSR_ERR_ARG) and
 *     vsr_last_error() gives a message for the calling thread;
 *   - "device" pointers must be CUDA device (or managed) memory on the
 *     scene's device; they are checked with cudaPointerGetAttributes and a
 *     host pointer is rejected, never dereferenced by a kernel; a buffer
 *     that ends past its CUDA allocation is rejected (the check sees whole
 *     allocations: a buffer carved from a larger allocation, as caching
 *     allocators do, is only checked against the enclosing allocation);
 *   - work is enqueued on the given stream and is asynchronous unless stated;
 *   - CUDA failures map to VSR_ERR_CUDA, allocation failures to VSR_ERR_OOM.
 *
 * Floating point: the triangle and box tests use FP32 with a fixed rounding
 * order (explicit fused multiply-adds, IEEE division, no flush to zero) so
 * that results are reproducible bit for bit by an independent CPU program.
 */
#ifndef VSR_H
#define VSR_H

#include <stddef.h>
#include <stdint.h>

#include "vsr_bvh.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vsr_stream; /* == cudaStream_t; NULL = legacy default */

typedef enum vsr_status {
    VSR_OK = 0,
    VSR_ERR_ARG = 1,     /* invalid argument, nothing launched */
    VSR_ERR_CUDA = 2,    /* a CUDA runtime call or launch failed */
    VSR_ERR_OOM = 3,     /* device or host allocation failed */
    VSR_ERR_BLOB = 4,    /* BVH blob failed validation */
    VSR_ERR_STACK = 5,   /* a traversal stack overflowed (device error word) */
    VSR_ERR_TIMEOUT = 6, /* a bounded device wait gave up */
    VSR_ERR_STATE = 7    /* call order violated (e.g. trace before bvh_load) */
} vsr_status;

/* ---------------------------------------------------------------- data */

#define VSR_NO_TEXTURE 0xFFFFFFFFu /* geom_id of an untextured, opaque triangle */
#define VSR_MISS 0xFFFFFFFFu       /* prim_id of a miss */

typedef enum vsr_tex_format {
    VSR_TEX_U8 = 0,     /* 1 byte per texel: alpha */
    VSR_TEX_RGBA8 = 1,  /* 4 bytes per texel, alpha in byte 3 */
    VSR_TEX_RGBA32F = 2 /* 16 bytes per texel, alpha in component 3 */
} vsr_tex_format;

/* A 2-D texture, row-major: texel (i, j) at index j*w + i; row j covers
 * v in [j/h, (j+1)/h), column i covers u in [i/w, (i+1)/w). */
typedef struct vsr_texture_desc {
    int32_t fmt;         /* vsr_tex_format */
    uint32_t w, h;       /* 1 .. 16384 */
    uint32_t reserved;   /* 0 */
    const void* texels;  /* host pointer, w*h texels, copied by the library */
} vsr_texture_desc;

/* A ray: origin, direction and the open parametric interval (tmin, tmax).
 * 32 bytes, 16-byte aligned.  tmax < tmin marks an inactive ray (a miss). */
typedef struct vsr_ray {
    float ox, oy, oz, tmin;
    float dx, dy, dz, tmax;
} vsr_ray;

/* A hit record (the paper's hit_record): distance, barycentrics (u weights
 * the second vertex, v the third) and the original triangle index.  A miss
 * has prim_id = VSR_MISS, t = +inf, u = v = 0.  16 bytes, 16-byte aligned. */
typedef struct vsr_hit {
    float t, u, v;
    uint32_t prim_id;
} vsr_hit;

typedef enum vsr_isect_kind {
    VSR_ISECT_NONE = 0,       /* no intersector: the default query overload */
    VSR_ISECT_DEFAULT = 1,    /* basic_intersector: forwards intersect() */
    VSR_ISECT_ALPHA_TEX = 2,  /* alpha mask: nearest texel alpha >= cutoff */
    VSR_ISECT_PROC_ALPHA = 3, /* sinf(f*uv.x) * sinf(f*uv.y) > 0 */
    VSR_ISECT_COUNT = 4,      /* bvh_costs: counts box and triangle tests */
    VSR_ISECT_CLIP = 5        /* clip box: intercepts node box tests too */
} vsr_isect_kind;

typedef enum vsr_dispatch {
    VSR_DISPATCH_STATIC = 0, /* intersector compiled into the kernel */
    VSR_DISPATCH_DYNAMIC = 1 /* run-time checked device function pointers */
} vsr_dispatch;

/* Intersector description.  Alpha intersectors read the triangle's texture
 * (geom_id) and interpolate its three texture coordinates with the hit's
 * barycentrics: uv = (1-u-v)*tc0 + u*tc1 + v*tc2.  Triangles whose geom_id is
 * VSR_NO_TEXTURE are opaque for both alpha intersectors.
 *
 * The clip box replaces both calls to intersect (Section 3.2: an intersector
 * may also overload intersect(ray, aabb) for the BVH's node boxes): a
 * candidate is accepted iff its hit point fmaf(t, d, o) (per component) lies
 * in the closed box [clip_lo, clip_hi], and a node box that does not overlap
 * the clip box counts as missed, so its subtree is skipped.  The answer is the
 * nearest hit inside the box.  Static dispatch; vsr_trace (one ray per thread
 * or persistent), vsr_trace_stats and vsr_trace_multi only. */
typedef struct vsr_intersector {
    int32_t kind;             /* vsr_isect_kind */
    int32_t dispatch;         /* vsr_dispatch */
    uint32_t alpha_cutoff_u8; /* 8-bit textures: accept iff alpha >= this */
    float alpha_cutoff_f;     /* float textures: accept iff alpha >= this */
    float proc_freq;          /* procedural frequency f (40 in the tests) */
    float clip_lo[3];         /* clip box (VSR_ISECT_CLIP), lo <= hi, finite */
    float clip_hi[3];
} vsr_intersector;

typedef enum vsr_query {
    VSR_CLOSEST = 0, /* nearest accepted candidate; equal t: lower prim id */
    VSR_ANY = 1      /* first accepted candidate in traversal order */
} vsr_query;

/* Launch configuration.  vsr_trace with params == NULL uses the
 * configuration vsr_trace_tune chose for the scene, intersector and query (or
 * tunes one on the call's own rays, see vsr_trace_tune); other entry points
 * take NULL as the defaults {128, 0, 16, 0, 0, 0, 0, 0, 0, 0, 0, 0}. */
typedef struct vsr_trace_params {
    uint32_t block_size;       /* threads per block, multiple of 32, 32..256 */
    uint32_t persistent;       /* 0: one ray per thread; 1: persistent warps
                                  (static or dynamic dispatch; vsr_trace,
                                  vsr_trace_multi, vsr_trace_instances,
                                  vsr_path_trace).  Each persistent launch
                                  claims rays from a counter of its own (8
                                  bytes from the stream-ordered allocator), so
                                  launches on one scene may overlap on
                                  different streams */
    uint32_t refill_threshold; /* persistent: refill idle lanes when fewer
                                  than this many of 32 are still active */
    uint32_t blocks_per_sm;    /* persistent: resident blocks per SM (0=auto) */
    uint32_t image_width;      /* 0: threads take rays in buffer order.  w > 0:
                                  the rays are a row-major image w pixels wide
                                  (the last row may be partial; widths above
                                  n act as n) and each warp
                                  takes a 4 x 8 pixel tile, so its rays are
                                  neighbours in both directions; rays and hits
                                  keep their layout.  Results are identical;
                                  coherent (camera) rays trace faster.  Not for
                                  batched launches. */
    uint32_t stack_regs;       /* traversal stack entries kept in registers
                                  (the rest spill to shared memory): 0, 1, 2,
                                  4 or 8 for vsr_trace and vsr_path_trace with
                                  static dispatch, 0, 2 or 4 for batches; the
                                  other queries keep the stack in shared
                                  memory and ignore it.  Results are
                                  identical for every value. */
    uint32_t watchdog_iterations; /* persistent launches and batches: outer-
                                  loop iterations a warp may run (0 = no
                                  limit).  A warp that runs out sets
                                  VSR_DEVERR_TIMEOUT in the scene's device
                                  error word, writes miss records for its
                                  rays in flight and stops: rays not yet
                                  traced keep whatever their hit records
                                  held. */
    uint32_t watchdog_ms;      /* persistent launches and batches: global-timer
                                  budget per warp, checked every 256
                                  iterations; 0 = 60000 ms, 0xFFFFFFFF = no
                                  limit.  Running out acts as above. */
    uint32_t reg_cap_blocks;   /* register budget of vsr_trace's kernels, for
                                  measurement: 0 = each kernel's own (static:
                                  none; dynamic: 3 blocks for closest hit, 4
                                  for any hit); 1 = none; 3 or 4 = compiled to
                                  fit that many 256-thread blocks per SM
                                  (static: one ray per thread with per-lane
                                  loops, stack_regs 0, intersectors default,
                                  alpha texture, procedural alpha and count;
                                  dynamic: every launch shape); 5 or 6
                                  likewise, static dispatch only.  Results are
                                  identical for every value. */
    uint32_t ray_order;        /* 0 = rays in the caller's order (or pixel
                                  tiles); 1 = coherence order: every launch
                                  first sorts the rays by a key of scene,
                                  origin (Morton code in the scene's root box)
                                  and direction (octahedral code), and threads
                                  (or a batch's claims) take them in sorted
                                  order, so a warp's lanes trace rays that
                                  start near each other and point the same
                                  way.  vsr_trace (image_width 0; scratch of
                                  20 bytes per ray plus histograms from the
                                  stream-ordered allocator) and batches (the
                                  scratch held by the batch); up to 2^28 rays.
                                  Results are identical; other entry points
                                  take 0. */
    uint32_t lockstep;         /* 1 = the warp runs the traversal in lock step:
                                  the node loop and the primitive loop repeat
                                  while any lane needs them and every pass ends
                                  in a warp vote, so lanes that diverge meet
                                  again at the next node.  Intersectors
                                  without counters (with dynamic dispatch:
                                  kinds without a box callback): a lane that
                                  holds a leaf keeps descending toward its
                                  next leaf while other lanes are still
                                  looking (any hit; closest hit with stack_regs
                                  0, where what the held leaf's hit culls is
                                  undone before the lane goes on).
                                  0 = each lane runs its own loops.  The same
                                  nodes and leaves are visited in the same
                                  order either way, so results are identical.
                                  vsr_trace and vsr_path_trace (static or
                                  dynamic dispatch; static: reg_cap_blocks 0),
                                  vsr_trace_multi (persistent 1) and batches;
                                  other entry points take 0. */
    uint32_t octant;           /* 1 = each warp first checks whether all its
                                  rays point into the same octant (the signs
                                  of dx, dy, dz); if so it runs a traversal
                                  compiled for that octant, whose node box
                                  test (Section 3.2, intersect(ray, aabb))
                                  reads the entry and exit plane of each axis
                                  directly instead of ordering the two planes
                                  with min/max: five ALU instructions per box
                                  instead of eleven.  Other warps, and scenes
                                  whose refitted boxes are not all finite
                                  with lo <= hi, run the generic test.  The
                                  outcome of every box test is the same, so
                                  results are identical.  Static dispatch,
                                  one ray per thread, per-lane loops
                                  (persistent 0, lockstep 0), stack_regs 0,
                                  reg_cap_blocks 0 or 1; vsr_trace,
                                  vsr_render and vsr_path_trace; other entry
                                  points take 0. */
} vsr_trace_params;

typedef struct vsr_scene vsr_scene;

/* ---------------------------------------------------------------- scene */

/*
 * Create a scene from indexed triangles (Section 3.1: basic_triangle<3,float>
 * primitives, texture coordinate lists and textures as in the alpha-mask
 * listing of Section 4).  All inputs are host pointers and are copied into
 * device memory owned by the scene, on the current CUDA device.
 *   verts   float32 [nverts*3]
 *   idx     uint32 [ntri*3]; every index < nverts
 *   uvs     float32 [ntri*6]: (u,v) of corner k of triangle p at 6p + 2k
 *   geom_id uint32 [ntri]: texture index < ntex, or VSR_NO_TEXTURE
 *   tex     [ntex] descriptors (may be NULL when ntex == 0)
 * Errors: VSR_ERR_ARG (null pointer, index or geom_id out of range, bad
 * texture), VSR_ERR_OOM, VSR_ERR_CUDA.  *out is NULL on failure.
 */
vsr_status vsr_scene_create_indexed(const float* verts, uint32_t nverts, const uint32_t* idx,
                                    const float* uvs, const uint32_t* geom_id, uint32_t ntri,
                                    const vsr_texture_desc* tex, uint32_t ntex,
                                    vsr_scene** out);

/* Same with three vertices per triangle: verts_xyz float32 [ntri*9]. */
vsr_status vsr_scene_create(const float* verts_xyz, const float* uvs, const uint32_t* geom_id,
                            uint32_t ntri, const vsr_texture_desc* tex, uint32_t ntex,
                            vsr_scene** out);

/* Free the scene and all device memory it owns (synchronises the device
 * first).  NULL is accepted. */
vsr_status vsr_scene_destroy(vsr_scene* scene);

/*
 * Load a serialised BVH (format in vsr_bvh.h) built over this scene's
 * triangles.  The blob is validated (magic, version, sizes, checksum, index
 * ranges, depth) and converted to the device layout: 32-byte nodes with
 * sibling pairs adjacent and 48-byte triangles (v0, e1 = v1 - v0,
 * e2 = v2 - v0) in leaf order.  Synchronous.  Errors: VSR_ERR_BLOB (invalid,
 * or num_prims != ntri), VSR_ERR_ARG, VSR_ERR_OOM, VSR_ERR_CUDA.
 */
vsr_status vsr_bvh_load(vsr_scene* scene, const void* blob, size_t bytes);

/* The library also exports the host builder and validator declared in
 * vsr_bvh.h (vsr_bvh_build, vsr_bvh_free, vsr_bvh_validate); vsr_bvh_load
 * runs vsr_bvh_validate before uploading. */

/* ---------------------------------------------------------------- trace */

/*
 * Trace n rays (Section 3.1 queries through the Section 3.2 traversal with
 * the intersector injected statically or dynamically).
 *   rays     device, vsr_ray [n], 16-byte aligned
 *   hits     device, vsr_hit [n], 16-byte aligned, caller-owned, written
 *   counters device uint32 [n*2] or NULL; only for VSR_ISECT_COUNT, which
 *            writes (box tests, triangle tests) per ray (bvh_costs)
 *   params   NULL: the configuration vsr_trace_tune chose for this scene,
 *            intersector kind, dispatch and query; if there is none, the
 *            first such call tunes one on its own rays in buffer order (as
 *            vsr_trace_tune with image_width 0: synchronous, the hits written
 *            several times, the last time with the result) and keeps it.  On
 *            a stream that is being captured the defaults apply instead.
 * Traversal order is fixed (root box tested once; at an inner node both
 * children are tested and, if both are hit, the child on the side of the
 * sign of the direction along the node's split axis is visited first; LIFO
 * stack), so any-hit results and counts are deterministic.
 * Errors: VSR_ERR_ARG, VSR_ERR_STATE (no BVH loaded), VSR_ERR_CUDA.
 */
vsr_status vsr_trace(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                     const vsr_intersector* isect, int32_t query, vsr_hit* hits,
                     uint32_t* counters, const vsr_trace_params* params, vsr_stream stream);

/*
 * Choose vsr_trace's launch configuration for (scene, intersector kind,
 * dispatch, query) by timing candidates on the caller's rays, keep it in the
 * scene for vsr_trace calls with params == NULL and return it in *out.
 * Candidates: one ray per thread with block 64, 128 or 256, 0, 1, 2, 4 or 8
 * stack entries in registers (static dispatch; dynamic: 0 entries) and
 * per-lane loops or lock step, starting from the default; then the fastest
 * of these in coherence order (ray_order 1, the sort timed with it); then
 * the persistent launch at the fastest configuration with per-lane loops and
 * in lock step, refill thresholds 1, 8, 16 and 24.  A candidate replaces the best only when at least 2%
 * faster.  The candidates take image_width (0: buffer order), except the
 * coherence-order one; all give the same hits, so only the time differs.
 * Synchronous (stream synchronised per candidate); hits is written several
 * times; counters are not written.  Not on a stream being captured
 * (VSR_ERR_STATE).  The configuration stays with the scene (vsr_scene_update
 * keeps it); a new call for the same key replaces it.
 * Errors as vsr_trace; VSR_ERR_ARG also for n == 0 or out == NULL.
 */
vsr_status vsr_trace_tune(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                          const vsr_intersector* isect, int32_t query, uint32_t image_width,
                          vsr_hit* hits, vsr_trace_params* out, vsr_stream stream);

/* The configuration vsr_trace uses with params == NULL for (scene,
 * intersector kind, dispatch, query), if one was tuned (VSR_ERR_STATE if
 * none).  Host only. */
vsr_status vsr_trace_tuned_params(vsr_scene* scene, const vsr_intersector* isect, int32_t query,
                                  vsr_trace_params* out);

/*
 * Multi-hit query: the first max_hits accepted hits of each ray in ascending
 * (t, prim) order -- the third visibility query of the library the paper
 * extends (Section 3.1), with the custom intersector injected exactly as for
 * closest-hit (Section 3.2).  The traversal is the closest-hit traversal whose
 * bound is the max_hits-th entry of a sorted buffer, so the intersector is
 * consulted for the candidates that would enter the buffer; max_hits == 1 is
 * the closest-hit query.
 *   hits      device vsr_hit [n * max_hits]: ray i's hits at i*max_hits + k,
 *             nearest first, then miss records (t = +inf, u = v = 0,
 *             prim = VSR_MISS)
 *   counters  as vsr_trace (COUNT intersector only), or NULL
 *   max_hits  1..16; static or dynamic dispatch (the callbacks as for
 *             vsr_trace)
 *   params    one ray per thread, or persistent warps (persistent 1, refill
 *             threshold, blocks per SM, watchdog as for vsr_trace) with
 *             per-lane loops or in lock step (lockstep 1 takes persistent
 *             1; speculation as for the closest-hit query, the buffer's
 *             last entry as the far limit); image_width allowed; stack in
 *             shared memory (stack_regs ignored).  Results are identical
 *             in every configuration.
 * Errors as vsr_trace.
 */
vsr_status vsr_trace_multi(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                           const vsr_intersector* isect, uint32_t max_hits, vsr_hit* hits,
                           uint32_t* counters, const vsr_trace_params* params,
                           vsr_stream stream);

/* ----------------------------------------------------------- path tracing */

/*
 * Diffuse path tracing on the closest-hit query with the intersector: a
 * workload of many incoherent segments through the same traversal (the paper
 * has no shading; its default kernels include a path tracer, Section 3.1).
 * Per path: a segment that misses returns throughput x sky; a hit multiplies
 * the throughput by the albedo (the colour of the nearest texel, the one the
 * alpha decision reads: RGBA8 / 255 or RGBA32F; `untextured` for untextured
 * triangles and u8 textures) and, while bounces remain, continues from
 * fmaf(t, d, o) over (eps, +inf) along the given local unit vector in the
 * face's tangent frame (face normal e1 x e2 turned against d; frame of Duff
 * et al. 2017); after `bounces` bounces the path returns 0.  FP32 with the
 * operation order of vsr_path_trace's kernels fixed (IEEE sqrt and division).
 *   rays      device vsr_ray [n], the primary segments
 *   dirs      device float32 [n * bounces * 3]: path i's bounce k at
 *             3 * (i * bounces + k), cosine-distributed for a diffuse surface
 *   radiance  device float32 [n * 3], written
 *   segments  device uint32 [n] or NULL: closest-hit queries path i made
 *   params    every segment's launch; image_width maps the primary
 *             segments to pixel tiles; persistent launches, lock step and
 *             the octant box test apply to each segment depth; ray_order 0
 * One closest-hit launch per segment depth plus one shading launch, on
 * `stream`.  After each bounce but the last, three small launches compact
 * the live paths (n < 2^32): the next segment's threads take the live paths
 * first, in index order, and the finished ones (inactive rays, dropped at
 * the root box test) after them; results do not depend on it.  Scratch
 * (n * 64 bytes plus 4 bytes per 256 paths) comes from the stream-ordered
 * allocator.  Errors as vsr_trace.
 */
typedef struct vsr_path_params {
    uint32_t bounces;      /* 0..64 */
    float eps;             /* tmin of bounce segments, finite, >= 0 */
    float sky[3];          /* finite */
    float untextured[3];   /* finite */
} vsr_path_params;
vsr_status vsr_path_trace(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                          const vsr_intersector* isect, const vsr_path_params* path,
                          const float* dirs, float* radiance, uint32_t* segments,
                          const vsr_trace_params* params, vsr_stream stream);

/* ------------------------------------------------------------- instancing */

/*
 * Instancing (Section 3.2: BVHs acting as compound primitives, where the
 * BVH stores BVHs as primitives and the custom intersector is passed on to
 * each BVH's own intersect).  An instance set is a top-level BVH whose leaves
 * hold instances; instance i shows mesh inst_mesh[i] (a scene with its BVH
 * loaded) through the world-to-object affine map W_i = world_to_object[12i ..
 * 12i+12) (row-major 3 x 4: rows (r0 r1 r2 | t)).  Rays are taken to object
 * space as o'_r = fmaf(W_r0, o.x, fmaf(W_r1, o.y, fmaf(W_r2, o.z, W_r3))),
 * d'_r = fmaf(W_r0, d.x, fmaf(W_r1, d.y, W_r2 * d.z)) with (tmin, tmax)
 * unchanged, so hit distances are in world units of the ray parameter.
 *   meshes      host array [nmeshes] of scenes with BVHs, on one device
 *   top_blob    a BVH blob over the instances' world-space boxes (primitive i
 *               is instance i; see vsr_bvh_build_boxes).  Each box must
 *               contain every world point whose object-space image lies in
 *               the mesh, or rays through the uncovered part miss.
 * The set copies the transforms and the meshes' device descriptors: the
 * meshes must outlive it, and neither vsr_bvh_load nor vsr_scene_update may
 * be called on them while it exists.
 * Errors: VSR_ERR_ARG (null, out of range, non-finite transform), VSR_ERR_BLOB
 * (invalid top-level blob or wrong instance count), VSR_ERR_STATE (a mesh
 * without BVH), VSR_ERR_OOM, VSR_ERR_CUDA.
 */
typedef struct vsr_instances vsr_instances;
vsr_status vsr_instances_create(vsr_scene* const* meshes, uint32_t nmeshes,
                                const uint32_t* inst_mesh, const float* world_to_object,
                                uint32_t ninst, const void* top_blob, size_t top_bytes,
                                vsr_instances** out);
vsr_status vsr_instances_destroy(vsr_instances* instances);

/*
 * Closest-hit or any-hit over an instance set with the intersector compiled
 * in (static dispatch) or reached through the callback tables (dynamic
 * dispatch; the callbacks see the mesh of the instance being traversed): the
 * top-level BVH is traversed while-while with the world-space ray (the same
 * order rule as a mesh), and at each instance the mesh's own traversal runs
 * with the object-space ray, continuing the running result.  Closest-hit
 * ties go to the lower instance id, then the lower primitive id.  Counters
 * (COUNT) include the top-level box tests.
 *   hits      device vsr_hit [n]: prim_id is the mesh's primitive id
 *   inst_ids  device uint32 [n] (VSR_MISS on a miss) or NULL
 *   params    one ray per thread, or persistent warps with per-lane loops
 *             (persistent 1, refill threshold, blocks per SM, watchdog as
 *             for vsr_trace; lockstep and ray_order 0); image_width
 *             allowed.  Results are identical in every configuration.
 * Errors as vsr_trace.  Traversal errors of the top level (and the watchdog's
 * VSR_DEVERR_TIMEOUT) go to the set's error word
 * (vsr_instances_device_error), those inside a mesh to the mesh's.
 */
vsr_status vsr_trace_instances(vsr_instances* instances, const vsr_ray* rays, uint64_t n,
                               const vsr_intersector* isect, int32_t query, vsr_hit* hits,
                               uint32_t* inst_ids, uint32_t* counters,
                               const vsr_trace_params* params, vsr_stream stream);

/* Read and clear the instance set's device error word (synchronous; bits as
 * vsr_get_device_error's 0, 1, 2 and 4). */
vsr_status vsr_instances_device_error(vsr_instances* instances, uint32_t* word);

/*
 * Measurement variant of vsr_trace with the static intersector: identical
 * hits, plus per-ray statistics stats device uint32 [n*4] = (box tests,
 * triangle tests, intersector consultations, texture look-ups), the last
 * being the consultations on triangles with a texture by an intersector that
 * reads texture coordinates (alpha texture, procedural alpha; 0 for the
 * others).  Used to count the bytes the traversal must fetch.  Errors as
 * vsr_trace.
 */
vsr_status vsr_trace_stats(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                           const vsr_intersector* isect, int32_t query, vsr_hit* hits,
                           uint32_t* stats, vsr_stream stream);

/*
 * Secondary rays toward a directional light from primary hit points: origin
 * o + t*d evaluated as fmaf(t, d, o) per component, direction light[3],
 * interval (eps, +inf).  A primary miss gives an inactive ray (tmin 0,
 * tmax -1, origin 0).  prim_rays/prim_hits/out: device [n].
 */
vsr_status vsr_make_shadow_rays(const vsr_ray* prim_rays, const vsr_hit* prim_hits, uint64_t n,
                                const float light[3], float eps, vsr_ray* out,
                                vsr_stream stream);

/*
 * Persistent-warp trace that allocates nothing.  The paper has no
 * counterpart: this entry point is for integrators.
 *
 * For callers that must not call cudaMalloc while they trace: for example an
 * application that hands all device memory to its own pool up front, or a
 * frame loop that cannot afford the synchronisation a fresh allocation can
 * bring.  Same arguments, results and errors as vsr_trace with
 * params->persistent = 1 (params may be NULL: block 128, refill 16; the
 * persistent flag is forced on; static dispatch only).
 *
 * The persistent kernel's only scratch -- the 64-bit counter from which warps
 * claim rays -- lives in a 256-byte array compiled into the library instead
 * of memory from cudaMalloc; every GPU that loads the library holds it until
 * the process exits.  The counter is cleared on `stream` before each launch.
 * All calls share the array: calls that overlap on the GPU race and must be
 * ordered (for example on one stream).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is kept per device together with
 * the id of the CUDA context it belongs to, and looked up again if that
 * context was replaced (for example after cudaDeviceReset).  n above
 * (2^31 - 2) * 32, the limit of one launch, is rejected with VSR_ERR_ARG.
 */
vsr_status vsr_trace_persistent_noalloc(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                                        const vsr_intersector* isect, int32_t query,
                                        vsr_hit* hits, uint32_t* counters,
                                        const vsr_trace_params* params, vsr_stream stream);

/* ---------------------------------------------------------------- batches */

/*
 * Many independent scenes, each with its own ray batch, traced in one
 * persistent launch (an extension of the paper's Section 3.1 queries: every
 * ray gets exactly the result vsr_trace would give it on its scene).  The
 * rays of all scenes form one index space; warps claim rays with one atomic
 * per warp and refill idle lanes, so batches of very uneven sizes share the
 * GPU without per-scene launches.
 *
 * vsr_batch_create records the scenes (each with a loaded BVH, all on one
 * device), the device ray and hit arrays (rays[k]/hits[k]: vsr_ray/vsr_hit
 * [n[k]], 16-byte aligned, caller-owned; n[k] may be 0), the intersector
 * (static dispatch; not the clip box) and the query, and builds the device
 * tables.  With params == NULL the launch configuration (block size, refill
 * threshold, blocks per SM, stack entries in registers, ray order) is chosen
 * by timing candidates on the batch itself at the first launch (with the
 * coherence order, the sort is part of every timed launch); results are cached per
 * workload shape in the process and, if the environment variable
 * VSR_TUNE_CACHE names a file, there too.  The shared-memory part of the
 * traversal stack is sized for the deepest BVH.  The persistent loop has the
 * watchdog of vsr_trace_params (a timeout is reported to every scene with a
 * ray in flight and to scene 0).
 *
 * vsr_batch_launch: the first call synchronises `stream`, tunes if needed,
 * runs the batch once and captures the launch (counter reset + kernel) in a
 * CUDA graph; every call then replays the graph on `stream`.  The recorded
 * pointers must stay valid for the batch's lifetime; the first launch writes
 * the hits more than once.  Errors: VSR_ERR_ARG, VSR_ERR_STATE (a scene
 * without BVH), VSR_ERR_OOM, VSR_ERR_CUDA.  nbatch is 1..65536.
 */
typedef struct vsr_batch vsr_batch;

vsr_status vsr_batch_create(vsr_scene* const* scenes, const vsr_ray* const* rays,
                            const uint64_t* n, vsr_hit* const* hits, uint32_t nbatch,
                            const vsr_intersector* isect, int32_t query,
                            const vsr_trace_params* params, vsr_batch** out);
vsr_status vsr_batch_launch(vsr_batch* batch, vsr_stream stream);
/* Launch configuration in use (the tuned one after the first launch). */
vsr_status vsr_batch_params(const vsr_batch* batch, vsr_trace_params* out);
/* Synchronises the device and frees the batch.  NULL is accepted. */
vsr_status vsr_batch_destroy(vsr_batch* batch);

/*
 * One-call form: the library keeps the last 8 batches keyed by every
 * argument and launches the matching one, creating (and tuning) it on first
 * use; make that first call outside any stream capture.
 */
vsr_status vsr_trace_batch(vsr_scene* const* scenes, const vsr_ray* const* rays,
                           const uint64_t* n, vsr_hit* const* hits, uint32_t nbatch,
                           const vsr_intersector* isect, int32_t query,
                           const vsr_trace_params* params, vsr_stream stream);

/* ---------------------------------------------------------------- gradients */

/*
 * Differentiable shading on the closest-hit query (an extension of the
 * paper's Section 3.1 queries; the paper has no gradients).  For a hit,
 *   c = albedo_rgb(uv) * max(0, n_f . light)
 * with uv the interpolated texture coordinate (as the alpha intersector uses
 * it), albedo the bilinear lookup of the triangle's texture (texel centres at
 * ((i + 0.5)/W, (j + 0.5)/H), clamp-to-edge indices; RGBA32F as stored,
 * RGBA8 divided by 255, u8 and untextured triangles albedo 1) and
 * n_f = normalize((v1 - v0) x (v2 - v0)) flipped to face the ray.  A miss
 * gives `background`.
 */
typedef struct vsr_shade_params {
    float light[3];      /* unit vector toward a directional light */
    float background[3]; /* colour of a miss */
    uint32_t grad_tex;   /* texture receiving texel gradients (RGBA32F), or
                            VSR_NO_TEXTURE */
    uint32_t reserved;   /* 0 */
} vsr_shade_params;

/*
 * Closest-hit trace with `isect` (static dispatch) and the shading above: the
 * trace kernels of vsr_trace write the hit records, then a shading pass reads
 * them.
 *   image device float32 [n*3], written; hits device vsr_hit [n] or NULL
 *         (NULL: the records go to n * 16 bytes of scratch from the
 *         stream-ordered allocator, freed on the stream).
 *   params NULL (the default configuration) or any vsr_trace configuration
 *         with ray_order 0.
 * Errors as vsr_trace.
 */
vsr_status vsr_render(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                      const vsr_intersector* isect, const vsr_shade_params* shade,
                      float* image, vsr_hit* hits, const vsr_trace_params* params,
                      vsr_stream stream);

/*
 * Adjoint of vsr_render at fixed visibility: every ray is traced again with
 * the same traversal (the same hit; no forward state is kept: the records go
 * to n * 16 bytes of stream-ordered scratch, freed on the stream) and dL/dc is
 * propagated to the vertices -- through the barycentrics u, v of the
 * Moller-Trumbore solve (dL/dv_k = -b_k M^-T (0, dL/du, dL/dv), M = [-d, e1,
 * e2], b = (1-u-v, u, v)) and through the face normal -- and to the texels of
 * texture shade->grad_tex through the bilinear weights.
 *   dL_dimage   device float32 [n*3]
 *   grad_verts  device float32 [nverts*3], accumulated (atomics: the
 *               summation order, hence the last bits, may vary between runs)
 *   grad_texels device float32 [w*h*4] of texture grad_tex (RGBA32F), or
 *               NULL; accumulated into the r, g, b channels
 * The scene must be unchanged since the forward render.  Errors as vsr_trace.
 */
vsr_status vsr_trace_backward(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                              const vsr_intersector* isect, const vsr_shade_params* shade,
                              const float* dL_dimage, float* grad_verts, float* grad_texels,
                              const vsr_trace_params* params, vsr_stream stream);

/*
 * The same adjoint from the hit records the forward render wrote
 * (vsr_render's `hits`): no traversal, one thread per ray.  The records are
 * the closest hits a re-trace finds, so the gradients are vsr_trace_backward's
 * (up to the order of the atomics).
 *   rays        device vsr_ray [n], the forward's rays (their directions
 *               enter the solve and the face orientation)
 *   hits        device vsr_hit [n] from vsr_render on the same rays, scene
 *               and intersector; a record whose primitive is out of range is
 *               skipped and sets device error bit VSR_DEVERR_HIT
 *   dL_dimage, grad_verts, grad_texels as vsr_trace_backward
 * The scene must be unchanged since the forward render.  Errors as vsr_trace.
 */
vsr_status vsr_render_backward_hits(vsr_scene* scene, const vsr_ray* rays, const vsr_hit* hits,
                                    uint64_t n, const vsr_shade_params* shade,
                                    const float* dL_dimage, float* grad_verts,
                                    float* grad_texels, vsr_stream stream);

/*
 * Ambient-occlusion shading on the closest-hit query:
 *   c = albedo_rgb(uv) * (1 - occluded / spp)      (background for a miss)
 * where the spp occlusion rays of pixel i are built exactly as
 * vsr_make_ao_rays builds them from the uniforms xi[i*spp + k] and traced
 * any-hit with the same intersector (static dispatch).  On `stream`: the
 * closest-hit trace into `hits` (at the configuration tuned for this scene,
 * intersector and the closest-hit query, with its pixel tiles if it has
 * them; else the default); the occlusion rays
 * and their any-hit records in n * spp * 48 bytes of scratch from the
 * stream-ordered allocator, traced at the configuration tuned for this
 * scene, intersector and the any-hit query (vsr_trace_tune; else the
 * default) and counted per pixel; the shading.  The counts do not depend on
 * the configuration.
 *   image     device float32 [n*3], written
 *   hits      device vsr_hit [n], written: the primary closest hits
 *   occlusion device float32 [n], written: occluded fraction (0 for a miss)
 *   xi        device float32 [n*spp*2]; spp 1..64
 * hits and occlusion are the state vsr_render_ao_backward needs.  Errors as
 * vsr_trace.
 */
vsr_status vsr_render_ao(vsr_scene* scene, const vsr_ray* rays, uint64_t n,
                         const vsr_intersector* isect, uint32_t spp, const float* xi,
                         float ao_tmax, float eps, const vsr_shade_params* shade, float* image,
                         vsr_hit* hits, float* occlusion, vsr_stream stream);

/*
 * Adjoint of vsr_render_ao with respect to the colour texels of texture
 * shade->grad_tex (RGBA32F) at fixed visibility, from the forward's hits and
 * occlusion (no traversal): dL/dc * (1 - occlusion) * bilinear weight is
 * accumulated into grad_texels [w*h*4] (r, g, b channels; atomics, so the
 * last bits may vary between runs).  The scene must be unchanged since the
 * forward.  A hit record whose primitive index is out of range is skipped
 * and sets bit 3 of the device error word.
 */
vsr_status vsr_render_ao_backward(vsr_scene* scene, const vsr_hit* hits, const float* occlusion,
                                  uint64_t n, const vsr_shade_params* shade,
                                  const float* dL_dimage, float* grad_texels, vsr_stream stream);

/*
 * Replace the scene's vertex positions and/or one texture's texels with
 * device data (same sizes as at creation; NULL leaves them unchanged).  After
 * a vertex update the triangle layout is rebuilt and the BVH boxes are refit
 * bottom-up (topology kept), so traces stay exact; traversal order and
 * bvh_costs counts then follow the refit boxes.  Synchronous.
 */
vsr_status vsr_scene_update(vsr_scene* scene, const float* verts, uint32_t tex_index,
                            const void* texels, vsr_stream stream);

/*
 * Ambient-occlusion rays from primary hits (a workload step; the paper has
 * no ray generation): spp rays per primary ray i, written at i*spp + k.
 * Origin fmaf(t, d, o); direction cosine-distributed about the face normal
 * turned against the primary direction, for the uniforms xi[i*spp + k] =
 * (x1, x2): sqrt(x1) cos(2 pi x2) t1 + sqrt(x1) sin(2 pi x2) t2 +
 * sqrt(1 - x1) n, with the tangent frame (t1, t2) of Duff et al. (2017,
 * "Building an orthonormal basis, revisited"); interval (eps, tmax).  A
 * primary miss gives inactive rays, and so does a hit record whose primitive
 * is out of range (device error bit 3).  FP32.
 *   prim_rays/prim_hits device [n]; xi device float32 [n*spp*2];
 *   out device vsr_ray [n*spp].  spp 1..64.
 */
vsr_status vsr_make_ao_rays(vsr_scene* scene, const vsr_ray* prim_rays, const vsr_hit* prim_hits,
                            uint64_t n, uint32_t spp, const float* xi, float tmax, float eps,
                            vsr_ray* out, vsr_stream stream);

/* ----------------------------------------------------------- measurement */

/* Read-bandwidth probe, the denominator of the memory roofline of the trace
 * kernels (whose node, triangle and texel fetches go through L1 and L2).  One
 * kernel launch on `stream` in which every thread of a full-occupancy grid
 * (SMs x resident 512-thread blocks) reads all of `buf` `reps` times with
 * 16-byte loads cached in L2 only; it writes nothing.  A buffer well inside
 * the L2 measures the L2 read rate, one far larger the HBM read rate: the
 * caller times the launch (bytes x reps read).
 *   buf    device memory of the current device, 16-byte aligned (not owned);
 *   bytes  a nonzero multiple of 16, within buf's allocation;
 *   reps   passes over the buffer, >= 1.
 * VSR_ERR_ARG on a null, unaligned, host or too-small buffer or a bad size;
 * VSR_ERR_CUDA if the launch fails.  Asynchronous. */
vsr_status vsr_read_probe(const void* buf, uint64_t bytes, uint32_t reps, vsr_stream stream);

/* L1 read probe, the denominator of the L1 level of the memory roofline.
 * One launch in which every block of a full-occupancy grid (SMs x resident
 * 512-thread blocks) reads all of `buf` `reps` times with 16-byte L1-cached
 * loads; the buffer is small enough to stay in every SM's L1, so after the
 * first pass the reads are L1 hits.  *bytes_read receives the bytes the
 * launch reads (blocks x bytes x reps); the caller times the launch.
 *   buf    device memory of the current device, 16-byte aligned (not owned);
 *   bytes  a nonzero multiple of 16, at most 65536, within buf's allocation;
 *   reps   passes, >= 1.
 * Errors as vsr_read_probe; VSR_ERR_ARG also for bytes above 65536 or a null
 * bytes_read.  Asynchronous. */
vsr_status vsr_read_probe_l1(const void* buf, uint64_t bytes, uint32_t reps,
                             uint64_t* bytes_read, vsr_stream stream);

/* ---------------------------------------------------------------- errors */

/* Message describing the last failure on the calling thread ("" if none). */
const char* vsr_last_error(void);

/* Read and clear the scene's device error word (synchronous).
 *   bit 0: a traversal stack overflowed;
 *   bit 1: a ray made more visits than the BVH has nodes (persistent and
 *          batched launches count every node, the others count leaves);
 *   bit 2: a render or backward kernel found a load whose address did not
 *          match its width and skipped it (vsr_last_error() names the line);
 *   bit 3: a caller-supplied hit record named a primitive out of range
 *          (skipped; vsr_make_ao_rays gives its rays inactive);
 *   bit 4 (VSR_DEVERR_TIMEOUT): a persistent or batched launch ran out of
 *          its watchdog budget (vsr_trace_params.watchdog_iterations,
 *          watchdog_ms); the launch's results are incomplete.  A batch
 *          reports it to every scene with a ray in flight and to scene 0.
 * Bits 0 and 1 end that ray as a miss; neither can happen with a validated
 * blob (each node is visited at most once per ray, and descent strictly
 * increases the node index).  These checks exist so that a corrupted
 * structure, a bad address or a loop that does not end gives an error
 * instead of a fault or a hung GPU. */
#define VSR_DEVERR_STACK 0x1u
#define VSR_DEVERR_STEPS 0x2u
#define VSR_DEVERR_ALIGN 0x4u
#define VSR_DEVERR_HIT 0x8u
#define VSR_DEVERR_TIMEOUT 0x10u
vsr_status vsr_get_device_error(vsr_scene* scene, uint32_t* word);

/* Library version, e.g. 100 for 0.1.0. */
int32_t vsr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VSR_H */
