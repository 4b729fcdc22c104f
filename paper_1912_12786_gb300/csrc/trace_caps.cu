// Statically injected trace kernels under a register budget
// (k_trace_cap, trace_static.cuh): 3 or 4 resident 256-thread blocks per SM,
// the budgets of the callback kernel, so that the cost of reaching the
// intersector through function pointers can be measured with the register
// budget held equal; 5 and 6 blocks (at most 51 and 42 registers) to measure
// what occupancy buys the static kernel.  One ray per thread, stack in
// shared memory.
#include "trace_static.cuh"

namespace vsr {

namespace {

template <int Q, class H, int MINB>
cudaError_t cap_one(const LaunchArgs& a) {
    auto k = k_trace_cap<Q, H, MINB>;
    const size_t smem = (size_t)stack_words(a.sc.stack_depth, 0) * a.block * sizeof(uint32_t);
    cudaError_t e = detail::ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    const unsigned long long grid = (a.map.threads + a.block - 1) / a.block;
    k<<<(unsigned)grid, a.block, smem, a.stream>>>(a.sc, a.ip, a.rays, a.map, a.hits, a.counters);
    return cudaGetLastError();
}

template <int Q, int MINB>
cudaError_t cap_kind(const LaunchArgs& a, int kind) {
    switch (kind) {
        case 1: return cap_one<Q, IsectDefault, MINB>(a);
        case 2: return cap_one<Q, IsectAlphaTex, MINB>(a);
        case 3: return cap_one<Q, IsectProcAlpha, MINB>(a);
        case 4: return cap_one<Q, IsectCount, MINB>(a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_static_capped(const LaunchArgs& a, int kind, uint32_t min_blocks) {
    if (min_blocks == 3)
        return a.query == kClosest ? cap_kind<kClosest, 3>(a, kind) : cap_kind<kAny, 3>(a, kind);
    if (min_blocks == 4)
        return a.query == kClosest ? cap_kind<kClosest, 4>(a, kind) : cap_kind<kAny, 4>(a, kind);
    if (min_blocks == 5)
        return a.query == kClosest ? cap_kind<kClosest, 5>(a, kind) : cap_kind<kAny, 5>(a, kind);
    if (min_blocks == 6)
        return a.query == kClosest ? cap_kind<kClosest, 6>(a, kind) : cap_kind<kAny, 6>(a, kind);
    return cudaErrorInvalidValue;
}

}  // namespace vsr
