// kernels_block_f64.cu -- FP64 instantiation of the block-team (one CTA per instance) kernel.
#include "kernels.cuh"

namespace sscs {
template const void* kblock_ptr<double>();
template cudaError_t launch_block<double>(int, int, size_t, cudaStream_t, const Args<double>*, int, int*);
}  // namespace sscs
