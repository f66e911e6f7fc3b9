// kernels_f64.cu -- FP64 instantiation of the grid-team solver kernel.
#include "kernels.cuh"

namespace sscs {
template const void* kgrid_ptr<double>();

cudaError_t launch_f2d(const float* in, double* out, long long n, cudaStream_t st)
{
    const int blocks = (int)std::min<long long>(1024, (n + 255) / 256 > 0 ? (n + 255) / 256 : 1);
    k_convert<float, double><<<blocks, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}
}  // namespace sscs
