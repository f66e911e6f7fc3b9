// kernels_f32.cu -- FP32 instantiation of the grid-team solver kernel (bulk of SCS_MIXED).
#include "kernels.cuh"

namespace sscs {
template const void* kgrid_ptr<float>();
}  // namespace sscs
