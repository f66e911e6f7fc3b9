// kernels.cuh -- the solver kernels (instantiated once per precision in
// kernels_f64.cu and kernels_f32.cu so the two compile in parallel).
#pragma once

#include "launch.h"
#include "solver.cuh"
#include <algorithm>

namespace sscs {

struct SmemFixed {
    unsigned long long mbar[2 * MAX_WARPS];
    unsigned ph[MAX_WARPS];
    double red[(MAX_WARPS + 1) * KMAX];
    double G[AAMAX * AAMAX];
    double L[AAMAX * AAMAX];
    double rhs[AAMAX];
    double t[AAMAX];
};

template <typename T>
__global__ void __launch_bounds__(1024) k_grid(const __grid_constant__ Args<T> a)
{
    __shared__ SmemFixed sf;
    extern __shared__ __align__(128) unsigned char dyn[];
    const bool tma = a.P.A.wbnd != nullptr;
    if (tma && (threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        mbar_init(smem_addr(&sf.mbar[2 * w]), 1);
        mbar_init(smem_addr(&sf.mbar[2 * w + 1]), 1);
        sf.ph[w] = 0;
        fence_mbar_init();
    }
    __syncthreads();
    GridTeam tm{sf.red, tma ? dyn : nullptr, sf.mbar, sf.ph, a.W.partials, a.W.bar, a.W.abort_flag, 0};
    run_mode<T>(tm, a.P, a.W, a.S, a.mode, a.slot, sf.G, sf.rhs, sf.L, sf.t, dyn);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_block(const Args<T>* insts, int B, int* queue, DevSettings S, int mode)
{
    __shared__ SmemFixed sf;
    __shared__ int sidx;
    extern __shared__ __align__(128) unsigned char dyn[];
    BlockTeam tm{sf.red, nullptr, sf.mbar, sf.ph, nullptr};
    for (;;) {
        if (threadIdx.x == 0) sidx = atomicAdd(queue, 1);
        __syncthreads();
        const int i = sidx;
        __syncthreads();
        if (i >= B) break;
        run_mode<T>(tm, insts[i].P, insts[i].W, S, mode, insts[i].slot, sf.G, sf.rhs, sf.L, sf.t, dyn);
        __syncthreads();
    }
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* in, Tout* out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (Tout)in[i];
}


template <typename T>
const void* kgrid_ptr() { return (const void*)k_grid<T>; }
template <typename T>
const void* kblock_ptr() { return (const void*)k_block<T>; }
template <typename T>
cudaError_t launch_block(int grid, int threads, size_t dyn, cudaStream_t st, const Args<T>* insts, int B, int* queue,
                         const DevSettings& S, int mode)
{
    k_block<T><<<grid, threads, dyn, st>>>(insts, B, queue, S, mode);
    return cudaGetLastError();
}

}  // namespace sscs
