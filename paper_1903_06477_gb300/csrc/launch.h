// launch.h -- host-visible handles of the solver kernels, defined in the
// per-precision translation units.
#pragma once

#include <cuda_runtime.h>

#include "solver.cuh"

namespace sscs {

template <typename T>
const void* kgrid_ptr();
template <typename T>
const void* kblock_ptr();
template <typename T>
cudaError_t launch_block(int grid, int threads, size_t dyn, cudaStream_t st, const Args<T>* insts, int B, int* queue,
                         const DevSettings& S, int mode);
cudaError_t launch_f2d(const float* in, double* out, long long n, cudaStream_t st);
cudaError_t launch_batch_handoff(const Args<float>* a32, const Args<double>* a64, int B, int mem, int resume,
                                 cudaStream_t st);
cudaError_t launch_batch_pack(const Args<double>* a64, int B, const long long* off, double* packed, cudaStream_t st);

}  // namespace sscs
