// kernels_block_f64.cu -- FP64 instantiation of the block-team (one CTA per instance) kernel.
#include "kernels.cuh"

namespace sscs {

// FP32 phase -> FP64 phase hand-over for a batch: one block per instance copies
// the FP32 iterate (already FP64 in u_out) to the FP64 warm start and widens
// the CG warm starts; with resume also the direction memory (mem columns of
// Z and Xi), the pending secant pair and their tau entries
__global__ void k_batch_handoff(const Args<float>* a32, const Args<double>* a64, int B, int mem, int resume)
{
    for (int i = blockIdx.x; i < B; i += gridDim.x) {
        const DevWork<float>& w32 = a32[i].W;
        const DevWork<double>& w64 = a64[i].W;
        const int n = a64[i].P.n, nm = n + a64[i].P.m, N = nm + 1;
        for (int j = threadIdx.x; j < N; j += blockDim.x) w64.warm[j] = w32.u_out[j];
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            w64.ws[0][j] = (double)w32.ws[0][j];
            w64.ws[1][j] = (double)w32.ws[1][j];
        }
        if (resume) {
            const long long cols = (long long)(mem > 0 ? mem : 1) * nm;
            for (long long j = threadIdx.x; j < cols; j += blockDim.x) {
                w64.Zv[j] = (double)w32.Zv[j];
                w64.Xv[j] = (double)w32.Xv[j];
                if (w32.Qv && w64.Qv) w64.Qv[j] = (double)w32.Qv[j];
            }
            for (int j = threadIdx.x; j < nm; j += blockDim.x) {
                w64.zp.v[j] = (double)w32.zp.v[j];
                w64.xip.v[j] = (double)w32.xip.v[j];
            }
            for (int j = threadIdx.x; j < (mem > 0 ? mem : 1); j += blockDim.x) {
                w64.Zt[j] = w32.Zt[j];
                w64.Xt[j] = w32.Xt[j];
                if (w32.Qt && w64.Qt) w64.Qt[j] = w32.Qt[j];
            }
            if (threadIdx.x == 0) {
                *w64.zp.t = *w32.zp.t;
                *w64.xip.t = *w32.xip.t;
            }
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

cudaError_t launch_batch_handoff(const Args<float>* a32, const Args<double>* a64, int B, int mem, int resume,
                                 cudaStream_t st)
{
    k_batch_handoff<<<std::min(B, 4096), 256, 0, st>>>(a32, a64, B, mem, resume);
    return cudaGetLastError();
}
cudaError_t launch_batch_pack(const Args<double>* a64, int B, const long long* off, double* packed, cudaStream_t st)
{
    k_batch_pack<<<std::min(B, 4096), 256, 0, st>>>(a64, B, off, packed);
    return cudaGetLastError();
}
}  // namespace sscs
