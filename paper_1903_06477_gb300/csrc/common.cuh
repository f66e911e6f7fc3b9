// common.cuh -- small device helpers shared by the SuperSCS CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sscs {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int KMAX = 16;                       // max values in one team reduction
constexpr int MAX_WARPS = 32;                  // 1024 threads per block at most
constexpr int GRID_THREADS = 512;              // largest block of the grid team (one CTA per SM)
constexpr int CB_MAX_STAGES = 4;               // deepest copy ring of the column-blocked products
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

// Streamed matrix entries (read once per sparse product): no L1 allocation and
// an L2 evict-first policy, so L1 and L2 keep the gathered vector entries.
__device__ __forceinline__ unsigned long long evict_first_policy()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ld_stream(const float* a, unsigned long long pol)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* a, unsigned long long pol)
{
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_stream(const int* a, unsigned long long pol)
{
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ unsigned short ld_stream(const unsigned short* a, unsigned long long pol)
{
    unsigned short v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(pol));
    return v;
}

// ---- asynchronous global -> shared copies (cp.async, L2 only) ---------------
// 16-byte copy that bypasses L1, so it sees what other CTAs wrote before the
// last grid barrier.  dst (shared) and src (global) 16-byte aligned.
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// hint: pull [p, p + bytes) into L2 (p 16-byte aligned, bytes % 16 == 0)
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---- TMA bulk copies (cp.async.bulk) and mbarriers --------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared bulk copy completing on an mbarrier; dst/src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void tma_load_1d(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                            unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}
// same without an L2 cache policy
__device__ __forceinline__ void tma_load_1d_plain(unsigned dst, const void* src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// order this thread's earlier generic-proxy accesses (any state space) before its later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr unsigned long long MBAR_TIMEOUT_NS = 2ull * 1000ull * 1000ull * 1000ull;  // 2 s
// bounded wait: false (and *abort_flag set) if the phase did not complete in time
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int* abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > MBAR_TIMEOUT_NS) {
            if (abort_flag) atomicExch(abort_flag, 2);
            return false;
        }
    }
    return true;
}

}  // namespace sscs
