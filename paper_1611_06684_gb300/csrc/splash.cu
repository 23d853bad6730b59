// Blocked sweep of Section 5.4 (placeholder until the FFBS kernels land).
#include "common.cuh"

namespace mrfk {

cudaError_t launch_splash(const SweepArgs& a, int layout, cudaStream_t s) {
    (void)a; (void)layout; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace mrfk
