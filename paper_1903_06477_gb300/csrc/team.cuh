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
//               barriers count arrivals on one 64-bit counter and their waits
//               are bounded by a 10 s timer (on expiry an abort flag is set,
//               every later barrier returns at once and the solver exits).
//
// Reductions are deterministic: fixed per-thread order, fixed shuffle tree,
// fixed order over warps and over blocks.
#pragma once

#include "common.cuh"

namespace sscs {

// Sum K doubles over the block; result in every thread.  red: smem of (MAX_WARPS+2)*KMAX doubles
// (the last row holds the broadcast slots of bcast()).
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

// The same sums with fewer FP64 instructions, used by the grid team (in the
// batch kernel, limited to 64 registers a thread, the larger code made the
// compiler outline the solver loop with more spills).
//
// Each warp's sum of value k is the butterfly tree of warp_sum (pairs of
// lanes l, l+16, then l, l+8, ..., l, l+1, as seen from lane 0), but the
// trees of several values share instructions: at the first level the lower
// half-warp adds the pairs of one value and the upper half those of the
// next, at the second level groups of 8 lanes take four values.  Every node
// of every tree is the same sum of the same two operands (addition is
// commutative), so the results are bitwise those of warp_sum, with about a
// third of the FP64 additions (6 instead of 20 for four values).
template <int K>
__device__ __forceinline__ void block_partial_packed(double (&v)[K], double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* row = red + wid * KMAX;
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
#pragma unroll
    for (int k = 0; k + 4 <= K; k += 4) {
        // level 16: lanes 0-15 value k (a) / k+2 (b), lanes 16-31 value k+1 (a) / k+3 (b)
        const double a = (hi16 ? v[k + 1] : v[k]) + __shfl_xor_sync(FULL_MASK, hi16 ? v[k] : v[k + 1], 16);
        const double b = (hi16 ? v[k + 3] : v[k + 2]) + __shfl_xor_sync(FULL_MASK, hi16 ? v[k + 2] : v[k + 3], 16);
        // level 8: lanes 0-7 value k, 8-15 value k+2, 16-23 value k+1, 24-31 value k+3
        double s = (hi8 ? b : a) + __shfl_xor_sync(FULL_MASK, hi8 ? a : b, 8);
        s += __shfl_xor_sync(FULL_MASK, s, 4);
        s += __shfl_xor_sync(FULL_MASK, s, 2);
        s += __shfl_xor_sync(FULL_MASK, s, 1);
        if ((lane & 7) == 0) row[k + ((lane >> 4) & 1) + ((lane >> 2) & 2)] = s;
    }
    constexpr int k2 = K - K % 4;
    if constexpr (K % 4 >= 2) {
        // two values: lanes 0-15 value k2, lanes 16-31 value k2+1
        double a = (hi16 ? v[k2 + 1] : v[k2]) + __shfl_xor_sync(FULL_MASK, hi16 ? v[k2] : v[k2 + 1], 16);
        a += __shfl_xor_sync(FULL_MASK, a, 8);
        a += __shfl_xor_sync(FULL_MASK, a, 4);
        a += __shfl_xor_sync(FULL_MASK, a, 2);
        a += __shfl_xor_sync(FULL_MASK, a, 1);
        if ((lane & 15) == 0) row[k2 + (lane >> 4)] = a;
    }
    if constexpr (K % 2 == 1) {
        const double x = warp_sum(v[K - 1]);
        if (lane == 0) row[K - 1] = x;
    }
    __syncthreads();
}

struct BlockTeam {
    static constexpr bool kGrid = false;
    double* red;
    unsigned char* stage;      // TMA staging (unused by this team: null)
    unsigned long long* mbar;  // per-warp mbarriers
    unsigned* ph;              // per-warp mbarrier phase bits
    int* abort_flag;
    double* scratch;           // AAMAX * AAMAX doubles of shared memory, free during linear solves
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
    __device__ __forceinline__ int block() const { return 0; }
    __device__ __forceinline__ int nblocks() const { return 1; }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    __device__ __forceinline__ bool aborted() const { return false; }
    // shared-memory slots through which one thread hands scalars to its CTA
    __device__ __forceinline__ double* bcast() const { return red + (MAX_WARPS + 1) * KMAX; }
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
    static constexpr bool kGrid = true;
    double* red;          // shared memory
    unsigned char* stage;      // dynamic shared memory: per-warp TMA staging (null when off)
    unsigned char* dsm;        // dynamic shared memory base (column-blocked products)
    unsigned long long* mbar;  // shared: 2 mbarriers per warp
    unsigned* ph;              // shared: phase bits per warp
    double* partials;     // global, [2][KMAX][gridDim.x]
    unsigned* bar;        // global, 16 bytes zeroed before the launch: [0..1] 64-bit arrival count
    int* abort_flag;      // global
    int parity;
    unsigned long long epoch;  // barriers passed so far (the same in every thread of the grid)

    __device__ __forceinline__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int size() const { return gridDim.x * blockDim.x; }
    __device__ __forceinline__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
    __device__ __forceinline__ int block() const { return blockIdx.x; }
    __device__ __forceinline__ int nblocks() const { return gridDim.x; }
    __device__ __forceinline__ bool aborted() const { return *(volatile int*)abort_flag != 0; }
    // shared-memory slots through which one thread hands scalars to its CTA
    __device__ __forceinline__ double* bcast() const { return red + (MAX_WARPS + 1) * KMAX; }

    // Grid barrier on one monotonically increasing 64-bit arrival count: the
    // e-th barrier is passed once the count reaches e * gridDim.x, so no
    // reset or separate release write is needed.  The wait is bounded.
    __device__ void sync()
    {
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long* cnt = reinterpret_cast<unsigned long long*>(bar);
            if (*(volatile int*)abort_flag == 0) {
                const unsigned long long target = (epoch + 1) * gridDim.x;
                __threadfence();
                const unsigned long long prev = atomicAdd(cnt, 1ull);
                if (prev + 1 < target) {
                    const unsigned long long t0 = gtimer();
                    unsigned ns = 8;
                    while (*(volatile unsigned long long*)cnt < target) {
                        if (*(volatile int*)abort_flag != 0) break;
                        if (gtimer() - t0 > BARRIER_TIMEOUT_NS) {
                            atomicExch(abort_flag, 1);
                            break;
                        }
                        __nanosleep(ns);
                        if (ns < 64) ns <<= 1;
                    }
                }
                __threadfence();
            }
        }
        ++epoch;
        __syncthreads();
    }

    // Team-wide sum of K values.  Every block writes its K partials, passes
    // the grid barrier, then reads all blocks' partials and sums them in
    // block order with the same fixed tree, so every block gets the same K
    // numbers (deterministic).  Partials are double-buffered: a block can
    // only overwrite a buffer after the next barrier, which every block
    // reaches only once it has read this one.
    template <int K>
    __device__ void reduce(double (&v)[K])
    {
        block_partial_packed<K>(v, red);
        const int nw = blockDim.x >> 5;
        const int B = gridDim.x;
        double* P = partials + (size_t)parity * KMAX * B;
        if (threadIdx.x < K) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * KMAX + threadIdx.x];
            P[(size_t)threadIdx.x * B + blockIdx.x] = s;
        }
        sync();
        double pv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) pv[k] = 0.0;
        for (int j = threadIdx.x; j < B; j += blockDim.x)
#pragma unroll
            for (int k = 0; k < K; ++k) pv[k] += __ldcg(P + (size_t)k * B + j);
        block_partial_packed<K>(pv, red);
        if (threadIdx.x < K) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * KMAX + threadIdx.x];
            red[MAX_WARPS * KMAX + threadIdx.x] = s;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = red[MAX_WARPS * KMAX + k];
        parity ^= 1;
    }
};

}  // namespace sscs
