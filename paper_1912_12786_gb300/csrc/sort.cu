// Coherence order for batched launches: the rays of all scenes sorted by a
// 32-bit key, and the batched kernel traces them in that order (claims take
// consecutive slots of the sorted order; each slot names a ray by its index
// in the batch's index space).
//
// Key of the ray with batch index g in scene s:
//   bits 31 .. 32-sb      s (sb = bits to number the scenes), so every
//                         scene's rays stay contiguous and in scene order
//   next ob bits          Morton code of the origin, quantised in the scene's
//                         root box (ob/3 bits per axis, origin clamped to it)
//   low db bits           the direction's octahedral coordinates, quantised
//                         (ceil(db/2) and floor(db/2) bits)
// with ob the largest multiple of 3 at most half of the 32 - sb bits left,
// and db the rest.  Camera rays of one scene share an origin and sort by
// direction; rays leaving surfaces sort by position, then direction.
//
// The sort is a least-significant-digit radix sort on 8-bit digits, four
// passes over (key, index) pairs, each pass: per-block digit histograms, an
// exclusive scan of the histograms in digit-major order, and a stable
// scatter.  Stability within a block: each warp owns a contiguous sub-tile
// and walks it in order; lanes with the same digit find each other with
// __match_any_sync and take ranks by their position in the warp; per-warp
// running offsets in shared memory start from a scan across the block's
// warps.  The order is a function of the keys alone, so it is the same on
// every launch.  Results never depend on it: every ray is traced exactly as
// in buffer order.
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

__global__ void __launch_bounds__(256) k_ray_keys(const BatchItem* __restrict__ items,
                                                  const unsigned long long* __restrict__ offsets,
                                                  uint32_t nbatch, uint32_t scene_bits,
                                                  uint32_t n, uint32_t* __restrict__ keys,
                                                  uint32_t* __restrict__ vals) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint32_t lo = 0, hi = nbatch;  // largest s with offsets[s] <= g
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(offsets + mid) <= g)
            lo = mid;
        else
            hi = mid;
    }
    const uint32_t s = lo;
    const unsigned long long ri = g - __ldg(offsets + s);
    const float4* rays = items[s].rays;
    const float4 a = __ldg(rays + 2 * ri), b = __ldg(rays + 2 * ri + 1);
    const float4 la = items[s].sc.root_a, hb = items[s].sc.root_b;
    const uint32_t cb = 32u - scene_bits;
    const uint32_t ob = (cb / 2u) / 3u * 3u, db = cb - ob;
    const uint32_t pa = ob / 3u;
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
    const uint32_t du = (db + 1u) / 2u, dv = db / 2u;
    const uint32_t dir = (quantise(0.5f * (ox + 1.0f), du) << dv) | quantise(0.5f * (oy + 1.0f), dv);
    const uint32_t code = (morton << db) | dir;
    keys[g] = (scene_bits ? (s << cb) : 0u) | (cb >= 32u ? code : (code & ((1u << cb) - 1u)));
    vals[g] = g;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                              uint32_t n, uint32_t shift,
                                                              uint32_t nblocks,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
    for (uint32_t r = 0; r < kSortPerThread; ++r) {
        const uint32_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(__ldg(keys + i) >> shift) & 0xFFu], 1u);
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
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t n, uint32_t shift,
    uint32_t nblocks, const uint32_t* __restrict__ offsets) {
    __shared__ uint32_t wc[kWarps][256];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wc[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t sub = blockIdx.x * kSortTile + warp * kSubTile;
    // per-warp digit counts of the warp's sub-tile
    for (uint32_t r = 0; r < kSubTile / 32; ++r) {
        const uint32_t i = sub + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (__ldg(keys_in + i) >> shift) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per-warp starting offsets: the block's global offset of the digit plus
    // the counts of the earlier warps
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = offsets[d * nblocks + blockIdx.x];
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t t = wc[w][d];
            wc[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    for (uint32_t r = 0; r < kSubTile / 32; ++r) {
        const uint32_t i = sub + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t key = ok ? __ldg(keys_in + i) : 0u;
        const uint32_t d = ok ? (key >> shift) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (ok) {
            const uint32_t out = wc[warp][d] + __popc(peers & lt);
            if (out < n) {  // always true for consistent histograms
                keys_out[out] = key;
                vals_out[out] = __ldg(vals_in + i);
            }
        }
        __syncwarp();
        if (ok && lane == (uint32_t)(__ffs(peers) - 1)) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
}

}  // namespace

size_t coherence_sort_words(uint32_t n) {
    const size_t nblocks = (n + kSortTile - 1) / kSortTile;
    const size_t hist = 256 * nblocks;
    const size_t totals = (hist + kScanBlock - 1) / kScanBlock;
    return 4ull * n + hist + totals;
}

uint32_t coherence_sort_max_rays() {
    // the histograms' scan takes up to 1024 x 8 block totals of 2048 values
    return (uint32_t)((1024ull * kScanPer * kScanBlock / 256ull) * kSortTile);
}

cudaError_t launch_coherence_sort(const BatchItem* items, const unsigned long long* offsets,
                                  uint32_t nbatch, uint32_t n, uint32_t* scratch,
                                  uint32_t** perm, cudaStream_t stream) {
    if (n == 0) {
        *perm = scratch;
        return cudaSuccess;
    }
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    const uint32_t hist_n = 256u * nblocks;
    const uint32_t ntot = (hist_n + kScanBlock - 1) / kScanBlock;
    if (ntot > 1024u * kScanPer) return cudaErrorInvalidValue;
    uint32_t* keys[2] = {scratch, scratch + n};
    uint32_t* vals[2] = {scratch + 2ull * n, scratch + 3ull * n};
    uint32_t* hist = scratch + 4ull * n;
    uint32_t* totals = hist + hist_n;
    uint32_t scene_bits = 0;
    while ((1ull << scene_bits) < nbatch) ++scene_bits;
    k_ray_keys<<<(n + 255) / 256, 256, 0, stream>>>(items, offsets, nbatch, scene_bits, n,
                                                    keys[0], vals[0]);
    cudaError_t e = cudaGetLastError();
    int cur = 0;
    for (uint32_t shift = 0; shift < 32 && e == cudaSuccess; shift += 8) {
        k_radix_hist<<<nblocks, kSortThreads, 0, stream>>>(keys[cur], n, shift, nblocks, hist);
        k_scan_blocks<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_scan_totals<<<1, 1024, 0, stream>>>(totals, ntot);
        k_scan_add<<<ntot, 256, 0, stream>>>(hist, hist_n, totals);
        k_radix_scatter<<<nblocks, kSortThreads, 0, stream>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                             vals[cur ^ 1], n, shift, nblocks,
                                                             hist);
        e = cudaGetLastError();
        cur ^= 1;
    }
    *perm = vals[cur];
    return e;
}

}  // namespace vsr
