// kernels_block_f32.cu -- FP32 instantiation of the block-team kernel.
#include "kernels.cuh"

namespace sscs {
template const void* kblock_ptr<float>();
template cudaError_t launch_block<float>(int, int, size_t, cudaStream_t, const Args<float>*, int, int*,
                                         const DevSettings&, int);
}  // namespace sscs
