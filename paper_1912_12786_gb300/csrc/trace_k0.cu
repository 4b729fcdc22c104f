// Statically injected trace kernels with 0 stack entries in registers
// (trace_static.cuh).
#include "trace_static.cuh"

namespace vsr {

cudaError_t launch_static_k0(const LaunchArgs& a, int kind, bool stats) {
    return detail::launch_static_k<0>(a, kind, stats);
}

}  // namespace vsr
