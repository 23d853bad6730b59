// Instantiations of the sweep half-step kernels for L in {12, 13, 14, 15, 16}.
#include "sweep_impl.cuh"

namespace mrfk {
MRF_INSTANTIATE_SWEEP(12)
MRF_INSTANTIATE_SWEEP(13)
MRF_INSTANTIATE_SWEEP(14)
MRF_INSTANTIATE_SWEEP(15)
MRF_INSTANTIATE_SWEEP(16)
}  // namespace mrfk
