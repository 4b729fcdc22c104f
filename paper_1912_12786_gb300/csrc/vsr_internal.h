// Host-side internals shared by the C-ABI translation unit and the kernel
// translation units of the GPU library.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "vsr_device.cuh"

namespace vsr {

struct LaunchArgs {
    DevScene sc;
    IsectParams ip;
    const float4* rays;
    unsigned long long n;
    RayMap map;  // thread -> ray (map.n == n)
    float4* hits;
    uint2* counters;  // COUNT intersector: (boxes, tris) per ray, may be null
    uint4* stats;     // measurement variant: (boxes, tris, cands, 0), may be null
    int query;
    uint32_t block;
    uint32_t persistent;
    uint32_t refill;
    uint32_t blocks_per_sm;
    unsigned long long* work;  // persistent: ray counter, zeroed before launch (null:
                               // the launch takes 8 bytes of stream-ordered scratch)
    const DevScene* dyn_user;  // dynamic dispatch: scene copy in device memory
    cudaStream_t stream;
    uint32_t stack_regs;       // traversal stack entries held in registers
    Watchdog wd;               // persistent: iteration and time budget
    uint32_t reg_cap;          // 0: each kernel's own register budget; 1, 3..6:
                               // __launch_bounds__(256, reg_cap) variants
    uint32_t lockstep = 0;     // 1: the warp runs the traversal in lock step
    uint32_t octant = 0;       // 1: box tests specialised to a warp's shared
                               // direction octant (k_trace_oct)
};

// Shading parameters of the differentiable render (device copy).
struct ShadeDev {
    float light[3];  // unit vector toward a directional light
    float bg[3];     // colour of a miss
    uint32_t grad_tex;
    uint32_t pad;
};

// Static injection: one instantiation per (query, intersector, stats,
// register-stack depth).
cudaError_t launch_static(const LaunchArgs& a, int kind, bool stats);
cudaError_t launch_static_octant(const LaunchArgs& a, int kind);
// Register-stack depths the static kernels are instantiated for.
bool stack_regs_supported(uint32_t k);
// The static one-ray-per-thread kernel under __launch_bounds__(256, 3..6)
// (trace_caps.cu): intersector kinds 1..4, stack in shared memory.
cudaError_t launch_static_capped(const LaunchArgs& a, int kind, uint32_t min_blocks);
// Dynamic injection: run-time checked function-pointer table.
cudaError_t launch_dynamic(const LaunchArgs& a, int kind);
// Grid of a persistent launch: SMs x resident blocks per SM (blocks_per_sm,
// or the occupancy of `kernel` at this block size and shared memory when 0);
// 0 on error.
int persistent_grid(uint32_t block, uint32_t blocks_per_sm, const void* kernel, size_t smem);
inline int persistent_grid(const LaunchArgs& a, const void* kernel, size_t smem) {
    return persistent_grid(a.block, a.blocks_per_sm, kernel, smem);
}

// Run `launch(counter)` with a persistent launch's ray counter, zeroed on
// `stream` first: `given` when not null, else 8 bytes of stream-ordered
// scratch freed on the stream after the launch, so persistent launches on
// different streams never share a counter.
template <class Launch>
cudaError_t with_ray_counter(unsigned long long* given, cudaStream_t stream, Launch&& launch) {
    unsigned long long* work = given;
    cudaError_t e = cudaSuccess;
    if (!work) {
        e = cudaMallocAsync(reinterpret_cast<void**>(&work), sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = launch(work);
    if (!given) {
        const cudaError_t f = cudaFreeAsync(work, stream);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

// Multi-hit query (trace_multi.cu): the first nh (1..16) accepted hits per
// ray in ascending (t, prim) order into a.hits [n * nh].
cudaError_t launch_multi(const LaunchArgs& a, int kind, const float* verts, const uint32_t* idx,
                         uint32_t nh, bool dynamic);
// Source line of the first misaligned access the multi-hit kernels skipped
// (0 if none), cleared after reading.
cudaError_t multi_align_error(unsigned* line);

// Instancing (trace_instances.cu): a top-level BVH whose leaves hold
// instances of meshes, each seen through a world-to-object affine map.
struct InstDev {
    const float4* nodes;     // top-level nodes, device layout as a mesh's
    const uint32_t* order;   // leaf slot -> instance id
    const float4* inst;      // 4 x float4 per instance: rows of W, {mesh id bits, 0, 0, 0}
    const DevScene* meshes;  // descriptors of the meshes (device copies)
    uint32_t* err;           // the instance set's device error word
    uint32_t ninst, root_ref, top_depth, max_leaves;
    float4 root_a, root_b;   // top-level root box
};

struct InstLaunch {
    InstDev is;
    IsectParams ip;
    const float4* rays;
    RayMap map;
    float4* hits;
    uint32_t* inst_ids;  // may be null
    uint2* counters;     // COUNT intersector, may be null
    uint32_t block;
    uint32_t stack_words;  // top-level depth + deepest mesh
    cudaStream_t stream;
    uint32_t persistent;     // 1: persistent warps (per-lane loops)
    uint32_t refill;         // persistent: refill threshold
    uint32_t blocks_per_sm;  // persistent: resident blocks per SM (0: occupancy)
    Watchdog wd;             // persistent: iteration and time budget
};
cudaError_t launch_instances(const InstLaunch& L, int kind, int query, bool dynamic);
// Source line of the first misaligned access the instanced kernels skipped
// (0 if none), cleared after reading.
cudaError_t instances_align_error(unsigned* line);

// Diffuse path tracing (path.cu): shading and the next segment per bounce.
struct PathDev {
    uint32_t bounces;
    float eps;
    float sky[3];
    float untex[3];
};
cudaError_t launch_path_init(const float4* rays, unsigned long long n, float4* work, float* f,
                             float* radiance, uint32_t* segments, cudaStream_t stream);
cudaError_t launch_path_bounce(const DevScene& sc, const PathDev& pd, const float* verts,
                               const uint32_t* idx, float4* work, const float4* hits, float* f,
                               const float* dirs, uint32_t k, unsigned long long n,
                               float* radiance, uint32_t* segments, cudaStream_t stream);
// Live-path compaction (path.cu): perm[0..n) becomes the path indices with
// the live paths first, in index order; counts holds path_compact_blocks(n)
// + 1 words of scratch.  n < 2^32.
uint32_t path_compact_blocks(unsigned long long n);
cudaError_t launch_path_compact(const float* f, unsigned long long n, uint32_t* counts,
                                uint32_t* perm, cudaStream_t stream);
// Source line of the first misaligned load the path kernels skipped (0 if
// none), cleared after reading.
cudaError_t path_align_error(unsigned* line);
cudaError_t launch_read_probe(const void* buf, unsigned long long bytes, uint32_t reps,
                              cudaStream_t stream);
cudaError_t launch_read_probe_l1(const void* buf, unsigned long long bytes, uint32_t reps,
                                 unsigned long long* bytes_read, cudaStream_t stream);

// Closest-hit render with diffuse shading, and its adjoint (render.cu).
// The render's shading pass from closest-hit records (the trace kernels
// write them first), one thread per ray.
cudaError_t launch_shade_hits(const DevScene& sc, const ShadeDev& sh, const float* verts,
                              const uint32_t* idx, const float4* rays, const float4* hits,
                              unsigned long long n, float* image, cudaStream_t stream);
// The adjoint from closest-hit records (no traversal), one thread per ray.
cudaError_t launch_render_backward_hits(const DevScene& sc, const ShadeDev& sh,
                                        const float* verts, const uint32_t* idx,
                                        const float4* rays, const float4* hits,
                                        unsigned long long n, const float* g, float* gv,
                                        float* gt, cudaStream_t stream);
// Source line of the first misaligned load a render kernel skipped (0 if
// none), cleared after reading.
cudaError_t render_align_error(unsigned* line);
// One scene of a batched launch: its descriptor and its ray and hit arrays.
struct BatchItem {
    DevScene sc;
    const float4* rays;
    float4* hits;
};

// A tile of the coherence sort (sort.cu): rays [start, start + count) of
// the index space, sorted by one block; its digit counts go to
// hist[hist_base + digit * stride].  A batch's tiles never straddle two
// scenes and each scene's tiles are laid out digit-major among themselves,
// so one scan of the counts sorts every scene's rays in place: scene s keeps
// slots [offsets[s], offsets[s+1]).
struct SortTile {
    uint32_t start, count, hist_base, stride;
};
constexpr uint32_t kSortTileRays = 4096;

struct BatchLaunch {
    const BatchItem* items;             // device [nbatch]
    const unsigned long long* offsets;  // device [nbatch + 1] ray prefix offsets
    uint32_t nbatch;
    IsectParams ip;
    unsigned long long total;
    unsigned long long* work;  // ray counter, zeroed before each launch
    uint32_t block, refill, blocks_per_sm, stack_max;
    uint32_t stack_regs;  // traversal stack entries held in registers
    Watchdog wd;          // iteration and time budget of the persistent loop
    uint32_t grid = 0;    // non-zero: launch exactly this grid, with no set-up calls
    uint32_t* sort_scratch = nullptr;  // non-null: trace in coherence order (sort.cu)
    const SortTile* sort_tiles = nullptr;  // device [sort_ntiles]
    const uint32_t* tile_scene = nullptr;  // device [sort_ntiles]: scene of each tile
    uint32_t sort_ntiles = 0;
    uint32_t lockstep = 0;             // 1: the warp runs the traversal in lock step
};

// Coherence order (sort.cu).  coherence_sort_tiles cuts a batch's rays into
// scene-aligned tiles (host); coherence_sort_words is the scratch, in 32-bit
// words, for n rays in ntiles tiles; at most coherence_sort_max_tiles tiles
// (uniform tiles: up to 2^28 rays in one scene).  The sorts leave in *perm
// (inside scratch) the ray indices in sorted order.
void coherence_sort_tiles(const unsigned long long* offsets, uint32_t nbatch,
                          std::vector<SortTile>* tiles, std::vector<uint32_t>* tile_scene);
size_t coherence_sort_words(uint32_t n, uint32_t ntiles);
uint32_t coherence_sort_max_tiles();
uint32_t coherence_sort_max_rays();
cudaError_t launch_coherence_sort(const BatchItem* items, const unsigned long long* offsets,
                                  const SortTile* tiles, const uint32_t* tile_scene,
                                  uint32_t ntiles, uint32_t n, uint32_t* scratch,
                                  uint32_t** perm, cudaStream_t stream);
// The same for the rays of one scene (vsr_trace with ray_order 1), in
// uniform tiles.
cudaError_t launch_coherence_sort_scene(const DevScene& sc, const float4* rays, uint32_t n,
                                        uint32_t* scratch, uint32_t** perm, cudaStream_t stream);

// Batched persistent trace over many scenes (batch.cu).
bool batch_stack_regs_supported(uint32_t k);
cudaError_t launch_batch(const BatchLaunch& b, int kind, int query, cudaStream_t stream);
// Grid that launch_batch uses for b (after its shared-memory attribute is set).
cudaError_t batch_grid(const BatchLaunch& b, int kind, int query, uint32_t* grid);

// Ambient-occlusion render and its texel adjoint (render.cu).
struct AoArgs {
    ShadeDev sh;
    const float* verts;
    const uint32_t* idx;
    uint32_t spp;
    const float2* xi;
    float tmax, eps;
    float4* hits;        // primary closest hits (written by the trace, read after)
    float* occ;          // occlusion counts (zeroed uint32), then occluded fractions
    float* image;        // forward
    const float* g;      // backward
    float* grad_texels;  // backward
};
// Image and occluded fractions from the hits and counts.
cudaError_t launch_ao_shade(const DevScene& sc, const AoArgs& ao, unsigned long long n,
                            cudaStream_t stream);
// Texel gradients from the saved hits and occluded fractions.
cudaError_t launch_ao_backward(const DevScene& sc, const AoArgs& ao, unsigned long long n,
                               cudaStream_t stream);

// Bottom-up refit over node lists grouped by level, deepest first
// (level_offsets is a host array of levels + 1 entries).  Any box that comes
// out non-finite or with lo > hi on some axis ORs 1 into *unordered (the
// caller zeroes it first).
cudaError_t launch_refit(float4* nodes, const uint32_t* level_nodes,
                         const uint32_t* level_offsets, uint32_t levels, const float* verts,
                         const uint32_t* idx, const uint32_t* order, uint32_t* unordered,
                         cudaStream_t stream);

}  // namespace vsr
