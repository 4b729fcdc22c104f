// Statically injected trace kernels with 8 stack entries in registers
// (trace_static.cuh).
#include "trace_static.cuh"

namespace vsr {

cudaError_t launch_static_k8(const LaunchArgs& a, int kind, bool stats) {
    return detail::launch_static_k<8>(a, kind, stats);
}

}  // namespace vsr
