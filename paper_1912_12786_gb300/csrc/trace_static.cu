// Dispatch of the statically injected trace kernels (trace_static.cuh) over
// the register-stack depths, and the persistent grid size.  The kernels of
// each depth K are instantiated in trace_k<K>.cu.
#include "vsr_internal.h"

namespace vsr {

cudaError_t launch_static_k0(const LaunchArgs& a, int kind, bool stats);
cudaError_t launch_static_k1(const LaunchArgs& a, int kind, bool stats);
cudaError_t launch_static_k2(const LaunchArgs& a, int kind, bool stats);
cudaError_t launch_static_k4(const LaunchArgs& a, int kind, bool stats);
cudaError_t launch_static_k8(const LaunchArgs& a, int kind, bool stats);

bool stack_regs_supported(uint32_t k) { return k == 0 || k == 1 || k == 2 || k == 4 || k == 8; }

cudaError_t launch_static(const LaunchArgs& a, int kind, bool stats) {
    // the measurement variant keeps the stack in shared memory: the depth
    // changes neither the visiting order nor the counts
    if (stats) return launch_static_k0(a, kind, true);
    if (a.reg_cap >= 3) return launch_static_capped(a, kind, a.reg_cap);
    if (a.octant) return launch_static_octant(a, kind);
    switch (a.stack_regs) {
        case 0: return launch_static_k0(a, kind, false);
        case 1: return launch_static_k1(a, kind, false);
        case 2: return launch_static_k2(a, kind, false);
        case 4: return launch_static_k4(a, kind, false);
        case 8: return launch_static_k8(a, kind, false);
        default: return cudaErrorInvalidValue;
    }
}

int persistent_grid(uint32_t block, uint32_t blocks_per_sm, const void* kernel, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (blocks_per_sm) {
        per_sm = (int)blocks_per_sm;
    } else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)block, smem) !=
               cudaSuccess) {
        return 0;
    }
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

}  // namespace vsr
