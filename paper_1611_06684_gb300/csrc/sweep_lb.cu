// Instantiations of the sweep half-step kernels for L in {7, 8, 9, 10, 11}.
#include "sweep_impl.cuh"

namespace mrfk {
MRF_INSTANTIATE_SWEEP(7)
MRF_INSTANTIATE_SWEEP(8)
MRF_INSTANTIATE_SWEEP(9)
MRF_INSTANTIATE_SWEEP(10)
MRF_INSTANTIATE_SWEEP(11)
}  // namespace mrfk
