// Coherence order for batched launches: the rays of all scenes sorted by
// scene, then by a 32-bit key of origin and direction, and the batched kernel
// traces them in that order (claims take consecutive slots of the sorted
// order; each slot names a ray by its index in the batch's index space).
//
// Coherence key of a ray (32 bits):
//   high 12 bits   Morton code of the origin, quantised in its scene's root
//                  box (4 bits per axis, origin clamped to the box)
//   low 20 bits    the direction's octahedral coordinates, 10 bits each
// Camera rays of one scene share an origin and sort by direction; rays
// leaving surfaces sort by position, then direction.  (Measured on the
// batching workload with host-sorted rays: 12 origin + 20 direction bits gave
// the largest gain of the key widths tried; 12 + 12 half of it.)
//
// The sort is a least-significant-digit radix sort on 8-bit digits over
// (key, batch index) pairs: four passes on the coherence key, then the key is
// replaced by the ray's scene and one more pass per 8 bits of scene index
// (none for a single scene) restores scene-major order, keeping the
// coherence order inside each scene because every pass is stable.  Each
// pass: per-block digit histograms, an exclusive scan of them in digit-major
// order, and a stable scatter.  The scatter ranks a block's elements in
// shared memory -- each warp owns a contiguous sub-tile and walks it in
// order; lanes with the same digit find each other with __match_any_sync --
// places them digit by digit in a shared-memory copy of the tile, and writes
// that out so that each digit's run goes to consecutive addresses.  The
// order is a function of the rays alone, so it is the same on every launch.
// Results never depend on it: every ray is traced exactly as in buffer
// order.
#include "vsr_internal.h"

namespace vsr {

namespace {

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortPerThread = 16;
constexpr uint32_t kSortTile = kSortThreads * kSortPerThread;  // 4096 keys per block
constexpr uint32_t kWarps = kSortThreads / 32;
constexpr uint32_t kSubTile = kSortTile / kWarps;  // 512 keys per warp

__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // 10 bits -> every third bit
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint32_t quantise(float x, uint32_t bits) {
    const float c = fminf(fmaxf(x, 0.0f), 1.0f);
    const uint32_t n = 1u << bits;
    return min((uint32_t)(c * (float)n), n - 1u);
}

// Scene of batch index g: the largest s with offsets[s] <= g.
__device__ __forceinline__ uint32_t scene_of_index(const unsigned long long* __restrict__ offsets,
                                                   uint32_t nbatch, uint32_t g) {
    uint32_t lo = 0, hi = nbatch;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(offsets + mid) <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t coherence_key(float4 a, float4 b, float4 la, float4 hb) {
    constexpr uint32_t ob = 12u, db = 20u, pa = ob / 3u;
    const float ex = fmaxf(hb.x - la.x, 1e-30f), ey = fmaxf(hb.y - la.y, 1e-30f),
                ez = fmaxf(hb.z - la.z, 1e-30f);
    const uint32_t morton = spread3(quantise((a.x - la.x) / ex, pa)) |
                            (spread3(quantise((a.y - la.y) / ey, pa)) << 1) |
                            (spread3(quantise((a.z - la.z) / ez, pa)) << 2);
    // octahedral map of the direction onto [0, 1]^2
    const float l1 = fabsf(b.x) + fabsf(b.y) + fabsf(b.z);
    float ox = l1 > 0.0f ? b.x / l1 : 0.0f, oy = l1 > 0.0f ? b.y / l1 : 0.0f;
    if (b.z < 0.0f) {
        const float tx = (1.0f - fabsf(oy)) * (ox >= 0.0f ? 1.0f : -1.0f);
        const float ty = (1.0f - fabsf(ox)) * (oy >= 0.0f ? 1.0f : -1.0f);
        ox = tx;
        oy = ty;
    }
    constexpr uint32_t du = db / 2u, dv = db - du;
    const uint32_t dir = (quantise(0.5f * (ox + 1.0f), du) << dv) | quantise(0.5f * (oy + 1.0f), dv);
    return (morton << db) | dir;
}

__global__ void __launch_bounds__(256) k_ray_keys(const BatchItem* __restrict__ items,
                                                  const unsigned long long* __restrict__ offsets,
                                                  uint32_t nbatch, uint32_t n,
                                                  uint2* __restrict__ kv) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const uint32_t s = scene_of_index(offsets, nbatch, g);
    const unsigned long long ri = g - __ldg(offsets + s);
    const float4* rays = items[s].rays;
    const float4 a = __ldg(rays + 2 * ri), b = __ldg(rays + 2 * ri + 1);
    kv[g] = make_uint2(coherence_key(a, b, items[s].sc.root_a, items[s].sc.root_b), g);
}

// Coherence keys of one scene's rays (the scene by value: no device table).
__global__ void __launch_bounds__(256) k_ray_keys_scene(DevScene sc, const float4* __restrict__ rays,
                                                        uint32_t n, uint2* __restrict__ kv) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 a = __ldg(rays + 2ull * g), b = __ldg(rays + 2ull * g + 1);
    kv[g] = make_uint2(coherence_key(a, b, sc.root_a, sc.root_b), g);
}

// Replace every key by the scene of its ray, for the scene passes.
__global__ void __launch_bounds__(256) k_scene_keys(const unsigned long long* __restrict__ offsets,
                                                    uint32_t nbatch, uint32_t n,
                                                    uint2* __restrict__ kv) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    kv[i].x = scene_of_index(offsets, nbatch, kv[i].y);
}

// Per-block digit counts.  Lanes with equal digits add once per warp (keys of
// a block often share their high digits, which would otherwise serialise the
// shared-memory atomics on one counter).
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint2* __restrict__ kv,
                                                              uint32_t n, uint32_t shift,
                                                              uint32_t nblocks,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t base = blockIdx.x * kSortTile;
    for (uint32_t r = 0; r < kSortPerThread; ++r) {
        const uint32_t i = base + r * kSortThreads + threadIdx.x;
        const uint32_t d = i < n ? (__ldg(kv + i).x >> shift) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (d < 256u && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan, three launches: each block scans 2048 values and writes
// its total; one block scans the totals (up to 8192); every block adds its
// scanned total.
constexpr uint32_t kScanPer = 8;
constexpr uint32_t kScanBlock = 256 * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp,
                                                         uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = blockDim.x / 32u;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp ? s_warp[warp - 1] : 0u;
    *total = s_warp[blockDim.x / 32u - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(256) k_scan_blocks(uint32_t* __restrict__ data, uint32_t n,
                                                     uint32_t* __restrict__ totals) {
    __shared__ uint32_t s_warp[32];
    const uint32_t base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    uint32_t v[kScanPer], sum = 0;
    for (uint32_t k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? data[base + k] : 0u;
        sum += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, s_warp, &total);
    for (uint32_t k = 0; k < kScanPer; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_totals(uint32_t* __restrict__ totals, uint32_t n) {
    __shared__ uint32_t s_warp[32];
    const uint32_t base = threadIdx.x * kScanPer;
    uint32_t v[kScanPer], sum = 0;
    for (uint32_t k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? totals[base + k] : 0u;
        sum += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, s_warp, &total);
    for (uint32_t k = 0; k < kScanPer; ++k) {
        if (base + k < n) totals[base + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(256) k_scan_add(uint32_t* __restrict__ data, uint32_t n,
                                                  const uint32_t* __restrict__ totals) {
    const uint32_t add = totals[blockIdx.x];
    const uint32_t base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    for (uint32_t k = 0; k < kScanPer; ++k)
        if (base + k < n) data[base + k] += add;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint2* __restrict__ kv_in, uint2* __restrict__ kv_out, uint32_t n, uint32_t shift,
    uint32_t nblocks, const uint32_t* __restrict__ offsets) {
    __shared__ uint2 tile[kSortTile];       // the block's elements, grouped by digit
    __shared__ uint32_t wc[kWarps][256];    // per-warp digit counts, then positions
    __shared__ uint32_t dstart[256];        // block-local start of each digit's run
    __shared__ uint32_t gbase[256];         // global start of each digit's run
    __shared__ uint32_t s_warp[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wc[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t tile0 = blockIdx.x * kSortTile;
    const uint32_t in_block = min(kSortTile, n - tile0);
    const uint32_t sub = tile0 + warp * kSubTile;
    // per-warp digit counts of the warp's sub-tile
    for (uint32_t r = 0; r < kSubTile / 32; ++r) {
        const uint32_t i = sub + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (__ldg(kv_in + i).x >> shift) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // block-local layout: digit runs in digit order, inside a run the warps
    // in order
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
        uint32_t total;
        const uint32_t start = block_exclusive_scan(run, s_warp, &total);
        dstart[d] = start;
        gbase[d] = offsets[d * nblocks + blockIdx.x];
        for (uint32_t w = 0; w < kWarps; ++w) wc[w][d] += start;
    }
    __syncthreads();
    for (uint32_t r = 0; r < kSubTile / 32; ++r) {
        const uint32_t i = sub + r * 32 + lane;
        const bool ok = i < n;
        const uint2 e = ok ? __ldg(kv_in + i) : make_uint2(0u, 0u);
        const uint32_t d = ok ? (e.x >> shift) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (ok) {
            const uint32_t pos = wc[warp][d] + __popc(peers & lt);
            if (pos < in_block) tile[pos] = e;  // always true for consistent counts
        }
        __syncwarp();
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // write out: consecutive tile positions of one digit go to consecutive
    // global positions
    for (uint32_t k = threadIdx.x; k < in_block; k += kSortThreads) {
        const uint2 e = tile[k];
        const uint32_t d = (e.x >> shift) & 0xFFu;
        const uint32_t out = gbase[d] + (k - dstart[d]);
        if (out < n) kv_out[out] = e;  // always true for consistent histograms
    }
}

}  // namespace

// Scratch layout (32-bit words): two (key, index) arrays of n pairs, the
// permutation (n words), the digit histograms, the scan's block totals.
size_t coherence_sort_words(uint32_t n) {
    const size_t nblocks = (n + kSortTile - 1) / kSortTile;
    const size_t hist = 256 * nblocks;
    const size_t totals = (hist + kScanBlock - 1) / kScanBlock;
    return 5ull * n + hist + totals;
}

__global__ void __launch_bounds__(256) k_perm(const uint2* __restrict__ kv, uint32_t n,
                                              uint32_t* __restrict__ perm) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = kv[i].y;
}

uint32_t coherence_sort_max_rays() {
    // the histograms' scan takes up to 1024 x 8 block totals of 2048 values
    return (uint32_t)((1024ull * kScanPer * kScanBlock / 256ull) * kSortTile);
}

namespace {

// Radix passes over the (key, index) pairs in kv[*cur]: four on the coherence
// key, then, for batches, the key is replaced by the scene and one pass per
// 8 bits of scene index follows.  Leaves the batch indices in sorted order
// in `out`.
cudaError_t sort_pairs(uint2* kv[2], uint32_t n, uint32_t* out, uint32_t* hist,
                       uint32_t* totals, const unsigned long long* offsets, uint32_t nbatch,
                       cudaStream_t stream) {
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    const uint32_t hist_n = 256u * nblocks;
    const uint32_t ntot = (hist_n + kScanBlock - 1) / kScanBlock;
    if (ntot > 1024u * kScanPer) return cudaErrorInvalidValue;
    uint32_t scene_bits = 0;
    while ((1ull << scene_bits) < nbatch) ++scene_bits;
    cudaError_t e = cudaGetLastError();
    int cur = 0;
    auto pass = [&](uint32_t shift) {
        k_radix_hist<<<nblocks, kSortThreads, 0, stream>>>(kv[cur], n, shift, nblocks, hist);
        k_scan_blocks<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_scan_totals<<<1, 1024, 0, stream>>>(totals, ntot);
        k_scan_add<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_radix_scatter<<<nblocks, kSortThreads, 0, stream>>>(kv[cur], kv[cur ^ 1], n, shift,
                                                             nblocks, hist);
        e = cudaGetLastError();
        cur ^= 1;
    };
    for (uint32_t shift = 0; shift < 32 && e == cudaSuccess; shift += 8) pass(shift);
    if (scene_bits && e == cudaSuccess) {
        k_scene_keys<<<(n + 255) / 256, 256, 0, stream>>>(offsets, nbatch, n, kv[cur]);
        e = cudaGetLastError();
        for (uint32_t shift = 0; shift < scene_bits && e == cudaSuccess; shift += 8) pass(shift);
    }
    if (e == cudaSuccess) {
        k_perm<<<(n + 255) / 256, 256, 0, stream>>>(kv[cur], n, out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

cudaError_t launch_coherence_sort(const BatchItem* items, const unsigned long long* offsets,
                                  uint32_t nbatch, uint32_t n, uint32_t* scratch,
                                  uint32_t** perm, cudaStream_t stream) {
    *perm = scratch + 4ull * n;
    if (n == 0) return cudaSuccess;
    uint2* kv[2] = {reinterpret_cast<uint2*>(scratch),
                    reinterpret_cast<uint2*>(scratch + 2ull * n)};
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    uint32_t* hist = *perm + n;
    k_ray_keys<<<(n + 255) / 256, 256, 0, stream>>>(items, offsets, nbatch, n, kv[0]);
    return sort_pairs(kv, n, *perm, hist, hist + 256ull * nblocks, offsets, nbatch, stream);
}

cudaError_t launch_coherence_sort_scene(const DevScene& sc, const float4* rays, uint32_t n,
                                        uint32_t* scratch, uint32_t** perm,
                                        cudaStream_t stream) {
    *perm = scratch + 4ull * n;
    if (n == 0) return cudaSuccess;
    uint2* kv[2] = {reinterpret_cast<uint2*>(scratch),
                    reinterpret_cast<uint2*>(scratch + 2ull * n)};
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    uint32_t* hist = *perm + n;
    k_ray_keys_scene<<<(n + 255) / 256, 256, 0, stream>>>(sc, rays, n, kv[0]);
    return sort_pairs(kv, n, *perm, hist, hist + 256ull * nblocks, nullptr, 1u, stream);
}

}  // namespace vsr
