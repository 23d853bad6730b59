// Instantiations of the sweep half-step kernels for L in {2, 3, 4, 5, 6}.
#include "sweep_impl.cuh"

namespace mrfk {
MRF_INSTANTIATE_SWEEP(2)
MRF_INSTANTIATE_SWEEP(3)
MRF_INSTANTIATE_SWEEP(4)
MRF_INSTANTIATE_SWEEP(5)
MRF_INSTANTIATE_SWEEP(6)
}  // namespace mrfk
