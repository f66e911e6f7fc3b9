// kernels_f32.cu -- FP32 instantiation of the solver kernels (the bulk of SCS_MIXED).
#include "kernels.cuh"

namespace sscs {
template const void* kgrid_ptr<float>();
template const void* kblock_ptr<float>();
template cudaError_t launch_block<float>(int, int, size_t, cudaStream_t, const Args<float>*, int, int*);
}  // namespace sscs
