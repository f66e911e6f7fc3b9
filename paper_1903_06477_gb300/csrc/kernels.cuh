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
    double red[(MAX_WARPS + 2) * KMAX];  // reduction rows, final sums, one row of broadcast slots
    double G[AAMAX * AAMAX];
    double L[AAMAX * AAMAX];
    double rhs[AAMAX];
    double t[AAMAX];
};

// One CTA per SM, at most GRID_THREADS threads: the bound gives every thread
// 128 registers, which the solver's device functions need to run without
// spilling to local memory.
template <typename T>
__global__ void __launch_bounds__(GRID_THREADS, 1) k_grid(const __grid_constant__ Args<T> a)
{
    __shared__ SmemFixed sf;
    extern __shared__ __align__(128) unsigned char dyn[];
    const bool tma = a.P.A.wbnd != nullptr;
    // mbarriers of the TMA-staged products: per-warp pairs for the sliced ELL
    // stream; for the column-blocked ring, "full" barriers (one arrival: the
    // producer's) at [0, CB_MAX_STAGES) and "empty" barriers (one arrival per
    // compute warp) at [CB_MAX_STAGES, 2 CB_MAX_STAGES)
    // (the FP32 copies the FP64 phase's refinement multiplies by count too)
    const bool cb = a.P.A.cb.ncb > 0 || a.P.AT.cb.ncb > 0 || a.W.ir.A.cb.ncb > 0 || a.W.ir.AT.cb.ncb > 0;
    for (int i = threadIdx.x; i < 2 * MAX_WARPS; i += blockDim.x) {
        const bool empty = cb && i >= CB_MAX_STAGES && i < 2 * CB_MAX_STAGES;
        mbar_init(smem_addr(&sf.mbar[i]), empty ? (blockDim.x >> 5) - 1 : 1);
        if (i < MAX_WARPS) sf.ph[i] = 0;
    }
    fence_mbar_init();
    __syncthreads();
    GridTeam tm{sf.red, tma ? dyn : nullptr, dyn, sf.mbar, sf.ph, a.W.partials, a.W.bar, a.W.abort_flag, 0, 0ull};
    run_mode<T>(tm, a.P, a.W, a.S, a.mode, a.slot, sf.G, sf.rhs, sf.L, sf.t, dyn);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_block(const Args<T>* insts, int B, int* queue, DevSettings S, int mode)
{
    __shared__ SmemFixed sf;
    __shared__ int sidx;
    extern __shared__ __align__(128) unsigned char dyn[];
    BlockTeam tm{sf.red, nullptr, sf.mbar, sf.ph, nullptr, sf.L};
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
