// team.cuh -- the two execution "teams" the SuperSCS device solver runs on.
//
// The whole SuperMann loop (Algorithm 1 of the paper) runs inside one kernel.
// Its steps are data-parallel passes separated by team-wide barriers, and
// every scalar decision (K0/K1/K2, backtracking, CG stopping) is taken from
// team-wide reductions that every thread computes identically, so no host
// round trip is needed.
//
//   BlockTeam : one CTA solves one instance (small problems, batched solves).
//   GridTeam  : every CTA of a cooperative launch solves one large instance;
//               barriers are a generation-counting grid barrier whose waits
//               are bounded by a 10 s timer (on expiry an abort flag is set,
//               every later barrier returns at once and the solver exits).
//
// Reductions are deterministic: fixed per-thread order, fixed shuffle tree,
// fixed order over warps and over blocks.
#pragma once

#include "common.cuh"

namespace sscs {

// Sum K doubles over the block; result in every thread.  red: smem of (MAX_WARPS+1)*KMAX doubles.
template <int K>
__device__ __forceinline__ void block_partial(double (&v)[K], double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = warp_sum(v[k]);
        if (lane == 0) red[wid * KMAX + k] = x;
    }
    __syncthreads();
}

struct BlockTeam {
    double* red;
    unsigned char* stage;      // TMA staging (unused by this team: null)
    unsigned long long* mbar;  // per-warp mbarriers
    unsigned* ph;              // per-warp mbarrier phase bits
    int* abort_flag;
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
    __device__ __forceinline__ int block() const { return 0; }
    __device__ __forceinline__ int nblocks() const { return 1; }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    __device__ __forceinline__ bool aborted() const { return false; }
    template <int K>
    __device__ __forceinline__ void reduce(double (&v)[K])
    {
        block_partial<K>(v, red);
        const int nw = blockDim.x >> 5;
        if (threadIdx.x < K) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * KMAX + threadIdx.x];
            red[MAX_WARPS * KMAX + threadIdx.x] = s;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = red[MAX_WARPS * KMAX + k];
    }
};

struct GridTeam {
    double* red;          // shared memory
    unsigned char* stage;      // dynamic shared memory: per-warp TMA staging (null when off)
    unsigned long long* mbar;  // shared: 2 mbarriers per warp
    unsigned* ph;              // shared: phase bits per warp
    double* partials;     // global, [2][KMAX][gridDim.x]
    unsigned* bar;        // global, [0] arrival count, [1] generation
    int* abort_flag;      // global
    int parity;

    __device__ __forceinline__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int size() const { return gridDim.x * blockDim.x; }
    __device__ __forceinline__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
    __device__ __forceinline__ int block() const { return blockIdx.x; }
    __device__ __forceinline__ int nblocks() const { return gridDim.x; }
    __device__ __forceinline__ bool aborted() const { return *(volatile int*)abort_flag != 0; }

    __device__ void sync()
    {
        __syncthreads();
        if (threadIdx.x == 0) {
            volatile unsigned* vgen = bar + 1;
            if (*(volatile int*)abort_flag == 0) {
                unsigned gen = *vgen;
                __threadfence();
                unsigned prev = atomicAdd(bar, 1u);
                if (prev == gridDim.x - 1) {
                    atomicExch(bar, 0u);
                    __threadfence();
                    atomicAdd(bar + 1, 1u);
                } else {
                    unsigned long long t0 = gtimer();
                    unsigned ns = 16;
                    while (*vgen == gen) {
                        if (*(volatile int*)abort_flag != 0) break;
                        if (gtimer() - t0 > BARRIER_TIMEOUT_NS) {
                            atomicExch(abort_flag, 1);
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 128) ns <<= 1;
                    }
                }
                __threadfence();
            }
        }
        __syncthreads();
    }

    // Team-wide sum of K values.  Every block writes its partial, then arrives
    // at the grid barrier; the last block to arrive sums the partials in
    // block order, publishes the K results and only then releases the
    // barrier, so every block reads the same K numbers (deterministic).
    template <int K>
    __device__ void reduce(double (&v)[K])
    {
        __shared__ int s_last;
        block_partial<K>(v, red);
        const int nw = blockDim.x >> 5;
        const int B = gridDim.x;
        double* P = partials + (size_t)parity * KMAX * B;
        double* R = partials + (size_t)2 * KMAX * B + (size_t)parity * KMAX;
        if (threadIdx.x < K) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * KMAX + threadIdx.x];
            P[(size_t)threadIdx.x * B + blockIdx.x] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int last = 0;
            volatile unsigned* vgen = bar + 1;
            if (*(volatile int*)abort_flag == 0) {
                const unsigned gen = *vgen;
                __threadfence();
                const unsigned prev = atomicAdd(bar, 1u);
                if (prev == gridDim.x - 1) {
                    __threadfence();
                    last = 1;
                } else {
                    const unsigned long long t0 = gtimer();
                    unsigned ns = 16;
                    while (*vgen == gen) {
                        if (*(volatile int*)abort_flag != 0) break;
                        if (gtimer() - t0 > BARRIER_TIMEOUT_NS) {
                            atomicExch(abort_flag, 1);
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 64) ns <<= 1;
                    }
                    __threadfence();
                }
            }
            s_last = last;
        }
        __syncthreads();
        if (s_last) {
            // all threads of the last block: thread j loads block j's K partials
            double pv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) pv[k] = 0.0;
            for (int j = threadIdx.x; j < B; j += blockDim.x)
#pragma unroll
                for (int k = 0; k < K; ++k) pv[k] += __ldcg(P + (size_t)k * B + j);
            block_partial<K>(pv, red);
            if (threadIdx.x < K) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += red[w * KMAX + threadIdx.x];
                R[threadIdx.x] = s;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            }
        }
        if (threadIdx.x < K) red[MAX_WARPS * KMAX + threadIdx.x] = __ldcg(R + threadIdx.x);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = red[MAX_WARPS * KMAX + k];
        parity ^= 1;
    }
};

}  // namespace sscs
