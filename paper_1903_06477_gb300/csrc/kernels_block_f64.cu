// kernels_block_f64.cu -- FP64 instantiation of the block-team (one CTA per instance) kernel.
#include "kernels.cuh"

namespace sscs {

// FP32 phase -> FP64 phase hand-over for a batch: one block per instance copies
// the FP32 iterate (already FP64 in u_out) to the FP64 warm start and widens
// the CG warm starts
__global__ void k_batch_handoff(const Args<float>* a32, const Args<double>* a64, int B)
{
    for (int i = blockIdx.x; i < B; i += gridDim.x) {
        const DevWork<float>& w32 = a32[i].W;
        const DevWork<double>& w64 = a64[i].W;
        const int n = a64[i].P.n, N = n + a64[i].P.m + 1;
        for (int j = threadIdx.x; j < N; j += blockDim.x) w64.warm[j] = w32.u_out[j];
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            w64.ws[0][j] = (double)w32.ws[0][j];
            w64.ws[1][j] = (double)w32.ws[1][j];
        }
    }
}

// packs every instance's x, y, s into one buffer at off[i] (n + 2m doubles each)
__global__ void k_batch_pack(const Args<double>* a64, int B, const long long* off, double* packed)
{
    for (int i = blockIdx.x; i < B; i += gridDim.x) {
        const DevWork<double>& w = a64[i].W;
        const int n = a64[i].P.n, m = a64[i].P.m;
        double* dst = packed + off[i];
        for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = w.x_out[j];
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            dst[n + j] = w.y_out[j];
            dst[n + m + j] = w.s_out[j];
        }
    }
}

template const void* kblock_ptr<double>();
template cudaError_t launch_block<double>(int, int, size_t, cudaStream_t, const Args<double>*, int, int*,
                                          const DevSettings&, int);

cudaError_t launch_batch_handoff(const Args<float>* a32, const Args<double>* a64, int B, cudaStream_t st)
{
    k_batch_handoff<<<std::min(B, 4096), 256, 0, st>>>(a32, a64, B);
    return cudaGetLastError();
}
cudaError_t launch_batch_pack(const Args<double>* a64, int B, const long long* off, double* packed, cudaStream_t st)
{
    k_batch_pack<<<std::min(B, 4096), 256, 0, st>>>(a64, B, off, packed);
    return cudaGetLastError();
}
}  // namespace sscs
