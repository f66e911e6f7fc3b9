// common.cuh -- small device helpers shared by the SuperSCS CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sscs {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int KMAX = 16;                       // max values in one team reduction
constexpr int MAX_WARPS = 32;                  // 1024 threads per block at most
constexpr unsigned long long BARRIER_TIMEOUT_NS = 10ull * 1000ull * 1000ull * 1000ull;  // 10 s

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    return x;
}
__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    return x;
}

// read-only (for the whole kernel) matrix data: use the non-coherent path
template <typename T>
__device__ __forceinline__ T ro(const T* p) { return __ldg(p); }

}  // namespace sscs
