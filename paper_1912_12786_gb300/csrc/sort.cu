// Coherence order: the rays sorted by a 32-bit key of origin and direction,
// each scene's rays among themselves, and the trace kernels take them in
// that order (slot k of the ray map names the ray perm[k]).
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
// (key, ray index) pairs, four passes.  The rays are cut into tiles of up to
// 4096 that never straddle two scenes (SortTile).  Each pass: per-tile digit
// counts, one exclusive scan of all counts -- laid out scene by scene, each
// scene's digit-major -- and a stable scatter.  Because a scene's counts
// follow all earlier scenes' counts in the scan, every scene's rays are
// sorted within the scene's own slot range, with no pass over scene indices.
// The scatter ranks a tile in shared memory: each warp owns a contiguous
// sub-tile, holds its 16 pairs per lane in registers and walks them in
// order; lanes with the same digit find each other with eight ballots, one
// per digit bit (ALU work; a match instruction per pair saturated the
// memory-input pipe).
// The pairs are placed digit by digit in a shared-memory copy of the tile,
// which is written out so that each digit's run goes to consecutive
// addresses.  The order is a function of the rays alone, so it is the same
// on every launch.  Results never depend on it: every ray is traced exactly
// as in buffer order.
#include "vsr_internal.h"

namespace vsr {

namespace {

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortPerThread = kSortTileRays / kSortThreads;  // 16
constexpr uint32_t kWarps = kSortThreads / 32;
constexpr uint32_t kSubTile = kSortTileRays / kWarps;  // 512 pairs per warp
constexpr uint32_t kPerLane = kSubTile / 32;           // 16 pairs per lane

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

// The lanes of the warp holding a pair (`valid`) whose 8-bit digit equals
// this lane's: the intersection, over the digit's bits, of the lanes that
// agree on that bit.  Called by all 32 lanes.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid) {
    uint32_t m = __ballot_sync(kFullMask, valid);
#pragma unroll
    for (uint32_t b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t v = __ballot_sync(kFullMask, bit);
        m &= bit ? v : ~v;
    }
    return m;
}

// Tile b: from the table, or (table null) uniform tiles of one segment.
__device__ __forceinline__ SortTile tile_of(const SortTile* __restrict__ tiles, uint32_t b,
                                            uint32_t n, uint32_t ntiles) {
    if (tiles) return tiles[b];
    SortTile t;
    t.start = b * kSortTileRays;
    t.count = min(kSortTileRays, n - t.start);
    t.hist_base = b;
    t.stride = ntiles;
    return t;
}

// Keys of a batch: one block per tile, so the tile's scene is known.
__global__ void __launch_bounds__(kSortThreads) k_ray_keys(
    const BatchItem* __restrict__ items, const unsigned long long* __restrict__ offsets,
    const SortTile* __restrict__ tiles, const uint32_t* __restrict__ tile_scene,
    uint2* __restrict__ kv) {
    const SortTile t = tiles[blockIdx.x];
    const uint32_t s = tile_scene[blockIdx.x];
    const float4* rays = items[s].rays;
    const float4 la = items[s].sc.root_a, hb = items[s].sc.root_b;
    const unsigned long long lo = offsets[s];
    for (uint32_t k = threadIdx.x; k < t.count; k += kSortThreads) {
        const uint32_t g = t.start + k;
        const unsigned long long ri = g - lo;
        const float4 a = __ldg(rays + 2 * ri), b = __ldg(rays + 2 * ri + 1);
        kv[g] = make_uint2(coherence_key(a, b, la, hb), g);
    }
}

// Coherence keys of one scene's rays (the scene by value: no device table).
__global__ void __launch_bounds__(256) k_ray_keys_scene(DevScene sc, const float4* __restrict__ rays,
                                                        uint32_t n, uint2* __restrict__ kv) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 a = __ldg(rays + 2ull * g), b = __ldg(rays + 2ull * g + 1);
    kv[g] = make_uint2(coherence_key(a, b, sc.root_a, sc.root_b), g);
}

// Per-tile digit counts.  A lane loads all its keys first (16 independent
// loads in flight), then adds each to a shared-memory counter.  (Adding once
// per group of equal digits found by ballots, as the scatter ranks them,
// saves the shared atomics that collide on common high digits but costs
// more ALU work than it saves: measured 0.2 ms slower per batch sort.)
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint2* __restrict__ kv,
                                                              const SortTile* __restrict__ tiles,
                                                              uint32_t n, uint32_t ntiles,
                                                              uint32_t shift,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    const SortTile t = tile_of(tiles, blockIdx.x, n, ntiles);
    uint32_t d[kSortPerThread];
#pragma unroll
    for (uint32_t r = 0; r < kSortPerThread; ++r) {
        const uint32_t k = r * kSortThreads + threadIdx.x;
        d[r] = k < t.count ? (__ldg(&kv[t.start + k].x) >> shift) & 0xFFu : 256u;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kSortPerThread; ++r) {
        if (d[r] < 256u) atomicAdd(&h[d[r]], 1u);
    }
    __syncthreads();
    hist[t.hist_base + threadIdx.x * t.stride] = h[threadIdx.x];
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
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = blockDim.x / 32u;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullMask, w, o);
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

// Stable scatter of one tile.  Lane `lane` of warp w holds the pairs at tile
// positions w * 512 + r * 32 + lane (r = 0..15) in registers from the single
// load to the placement in shared memory.
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(
    const uint2* __restrict__ kv_in, uint2* __restrict__ kv_out,
    const SortTile* __restrict__ tiles, uint32_t n, uint32_t ntiles, uint32_t shift,
    const uint32_t* __restrict__ offsets) {
    __shared__ uint2 tile[kSortTileRays];   // the tile's pairs, grouped by digit
    __shared__ uint32_t wc[kWarps][256];    // per-warp digit counts, then positions
    __shared__ uint32_t dstart[256];        // tile-local start of each digit's run
    __shared__ uint32_t gbase[256];         // global start of each digit's run
    __shared__ uint32_t s_warp[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wc[0][0])[k] = 0u;
    const SortTile t = tile_of(tiles, blockIdx.x, n, ntiles);
    const uint32_t sub = warp * kSubTile;
    uint2 e[kPerLane];
#pragma unroll
    for (uint32_t r = 0; r < kPerLane; ++r) {
        const uint32_t k = sub + r * 32 + lane;
        e[r] = k < t.count ? __ldg(kv_in + t.start + k) : make_uint2(0u, 0u);
    }
    __syncthreads();
    // per-warp digit counts of the warp's sub-tile (digit 256: no pair)
    uint32_t peers[kPerLane];
#pragma unroll
    for (uint32_t r = 0; r < kPerLane; ++r) {
        const bool ok = sub + r * 32 + lane < t.count;
        const uint32_t d = (e[r].x >> shift) & 0xFFu;
        peers[r] = digit_peers(d, ok);
        if (ok && lane == (uint32_t)(__ffs(peers[r]) - 1)) wc[warp][d] += __popc(peers[r]);
        __syncwarp();
    }
    __syncthreads();
    // tile-local layout: digit runs in digit order, inside a run the warps
    // in order
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
        uint32_t total;
        const uint32_t start = block_exclusive_scan(run, s_warp, &total);
        dstart[d] = start;
        gbase[d] = offsets[t.hist_base + d * t.stride];
        for (uint32_t w = 0; w < kWarps; ++w) wc[w][d] += start;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kPerLane; ++r) {
        const bool ok = sub + r * 32 + lane < t.count;
        const uint32_t d = (e[r].x >> shift) & 0xFFu;
        if (ok) {
            const uint32_t pos = wc[warp][d] + __popc(peers[r] & lt);
            if (pos < t.count) tile[pos] = e[r];  // always true for consistent counts
        }
        __syncwarp();
        if (ok && lane == (uint32_t)(__ffs(peers[r]) - 1)) wc[warp][d] += __popc(peers[r]);
        __syncwarp();
    }
    __syncthreads();
    // write out: consecutive tile positions of one digit go to consecutive
    // global positions
    for (uint32_t k = threadIdx.x; k < t.count; k += kSortThreads) {
        const uint2 x = tile[k];
        const uint32_t d = (x.x >> shift) & 0xFFu;
        const uint32_t out = gbase[d] + (k - dstart[d]);
        if (out < n) kv_out[out] = x;  // always true for consistent counts
    }
}

__global__ void __launch_bounds__(256) k_perm(const uint2* __restrict__ kv, uint32_t n,
                                              uint32_t* __restrict__ perm) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = kv[i].y;
}

// Four radix passes over the (key, index) pairs in kv[0]; leaves the ray
// indices in sorted order in `out`.
cudaError_t sort_pairs(uint2* kv[2], uint32_t n, const SortTile* tiles, uint32_t ntiles,
                       uint32_t* out, uint32_t* hist, uint32_t* totals, cudaStream_t stream) {
    const uint32_t hist_n = 256u * ntiles;
    const uint32_t ntot = (hist_n + kScanBlock - 1) / kScanBlock;
    if (ntiles > coherence_sort_max_tiles() || ntot > 1024u * kScanPer)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaGetLastError();
    int cur = 0;
    for (uint32_t shift = 0; shift < 32 && e == cudaSuccess; shift += 8) {
        k_radix_hist<<<ntiles, kSortThreads, 0, stream>>>(kv[cur], tiles, n, ntiles, shift, hist);
        k_scan_blocks<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_scan_totals<<<1, 1024, 0, stream>>>(totals, ntot);
        k_scan_add<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_radix_scatter<<<ntiles, kSortThreads, 0, stream>>>(kv[cur], kv[cur ^ 1], tiles, n,
                                                             ntiles, shift, hist);
        e = cudaGetLastError();
        cur ^= 1;
    }
    if (e == cudaSuccess) {
        k_perm<<<(n + 255) / 256, 256, 0, stream>>>(kv[cur], n, out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

void coherence_sort_tiles(const unsigned long long* offsets, uint32_t nbatch,
                          std::vector<SortTile>* tiles, std::vector<uint32_t>* tile_scene) {
    tiles->clear();
    tile_scene->clear();
    uint32_t first = 0;  // index of the scene's first tile
    for (uint32_t s = 0; s < nbatch; ++s) {
        const unsigned long long lo = offsets[s], cnt = offsets[s + 1] - lo;
        const uint32_t nt = (uint32_t)((cnt + kSortTileRays - 1) / kSortTileRays);
        for (uint32_t j = 0; j < nt; ++j) {
            const unsigned long long at = (unsigned long long)j * kSortTileRays;
            const unsigned long long c = cnt - at < kSortTileRays ? cnt - at : kSortTileRays;
            tiles->push_back(SortTile{(uint32_t)(lo + at), (uint32_t)c, 256u * first + j, nt});
            tile_scene->push_back(s);
        }
        first += nt;
    }
}

// Scratch layout (32-bit words): two (key, index) arrays of n pairs, the
// permutation (n words), the digit counts (256 per tile), the scan's block
// totals.
size_t coherence_sort_words(uint32_t n, uint32_t ntiles) {
    const size_t hist = 256ull * ntiles;
    const size_t totals = (hist + kScanBlock - 1) / kScanBlock;
    return 5ull * n + hist + totals;
}

uint32_t coherence_sort_max_tiles() {
    // the counts' scan takes up to 1024 x 8 block totals of 2048 values
    return (uint32_t)(1024ull * kScanPer * kScanBlock / 256ull);
}

uint32_t coherence_sort_max_rays() {
    return (uint32_t)((unsigned long long)coherence_sort_max_tiles() * kSortTileRays);
}

cudaError_t launch_coherence_sort(const BatchItem* items, const unsigned long long* offsets,
                                  const SortTile* tiles, const uint32_t* tile_scene,
                                  uint32_t ntiles, uint32_t n, uint32_t* scratch,
                                  uint32_t** perm, cudaStream_t stream) {
    *perm = scratch + 4ull * n;
    if (n == 0 || ntiles == 0) return cudaSuccess;
    uint2* kv[2] = {reinterpret_cast<uint2*>(scratch),
                    reinterpret_cast<uint2*>(scratch + 2ull * n)};
    uint32_t* hist = *perm + n;
    k_ray_keys<<<ntiles, kSortThreads, 0, stream>>>(items, offsets, tiles, tile_scene, kv[0]);
    return sort_pairs(kv, n, tiles, ntiles, *perm, hist, hist + 256ull * ntiles, stream);
}

cudaError_t launch_coherence_sort_scene(const DevScene& sc, const float4* rays, uint32_t n,
                                        uint32_t* scratch, uint32_t** perm,
                                        cudaStream_t stream) {
    *perm = scratch + 4ull * n;
    if (n == 0) return cudaSuccess;
    uint2* kv[2] = {reinterpret_cast<uint2*>(scratch),
                    reinterpret_cast<uint2*>(scratch + 2ull * n)};
    const uint32_t ntiles = (n + kSortTileRays - 1) / kSortTileRays;
    uint32_t* hist = *perm + n;
    k_ray_keys_scene<<<(n + 255) / 256, 256, 0, stream>>>(sc, rays, n, kv[0]);
    return sort_pairs(kv, n, nullptr, ntiles, *perm, hist, hist + 256ull * ntiles, stream);
}

}  // namespace vsr
