// Statically injected trace kernels with 2 stack entries in registers
// (trace_static.cuh).
#include "trace_static.cuh"

namespace vsr {

cudaError_t launch_static_k2(const LaunchArgs& a, int kind, bool stats) {
    return detail::launch_static_k<2>(a, kind, stats);
}

}  // namespace vsr
