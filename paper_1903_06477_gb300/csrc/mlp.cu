// mlp.cu -- the learned warm start: a 3-layer MLP trained and evaluated
// entirely by the kernels in this file (see include/superscs_mlp.h).
//
// Every product is written as C = A B^T with both operands K-contiguous (the
// backward pass works on transposed copies made by a tiled transpose kernel)
// and runs on one of two BF16 kernels with FP32 accumulation: gemm_nt_tc
// (default), tcgen05.mma fed by TMA with the accumulator in tensor memory, or
// gemm_nt, the warp-level MMA (m16n8k16) on 128x128x32 tiles staged by cp.async.
#include <cuda.h>  // CUtensorMap and its enums (types only: the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/superscs.h"
#include "../../include/superscs_mlp.h"

namespace sscs {
void record_error(const char* msg);
}

namespace {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128, BN = 128, BK = 32, NTH = 256, SROW = BK + 8;  // 80-byte smem rows: ldmatrix conflict-free

struct Epi {
    const float* bias;  // per column, or null
    const bf16* mask;   // relu' mask (value > 0 keeps), row-major with ldm, or null
    int ldm;
    int relu;
    float* C32;         // FP32 output or null
    int ldc;
    bf16* C16;          // BF16 output or null
    int ldc16;
};

__device__ __forceinline__ unsigned sa(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

// 16-byte async copy with zero fill of the bytes past src_bytes
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(sa(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M x N] = A[M x K] * B[N x K]^T.  lda, ldb multiples of 8, A and B 16-byte
// aligned; tails in M, N and K are zero-filled on load and masked on store.
__global__ void __launch_bounds__(NTH) gemm_nt(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                               const bf16* __restrict__ Bm, int ldb, Epi e)
{
    __shared__ __align__(16) bf16 As[2][BM][SROW];
    __shared__ __align__(16) bf16 Bs[2][BN][SROW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, 64 x 32 each
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    auto load = [&](int st, int k0) {
        for (int c = tid; c < BM * (BK / 8); c += NTH) {
            const int r = c >> 2, kc = (c & 3) * 8;
            const int gk = k0 + kc;
            int gm = m0 + r;
            int bytes = (gm < M && gk < K) ? min(16, (K - gk) * 2) : 0;
            const bf16* src = bytes ? A + (size_t)gm * lda + gk : A;
            cp16(&As[st][r][kc], src, bytes);
            const int gn = n0 + r;
            bytes = (gn < N && gk < K) ? min(16, (K - gk) * 2) : 0;
            src = bytes ? Bm + (size_t)gn * ldb + gk : Bm;
            cp16(&Bs[st][r][kc], src, bytes);
        }
    };

    const int KT = (K + BK - 1) / BK;
    load(0, 0);
    cp_commit();
    for (int kt = 0; kt < KT; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < KT) {
            load(st ^ 1, (kt + 1) * BK);
            cp_commit();
            cp_wait1();
        } else {
            cp_wait0();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[4][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int row = wm * 64 + mi * 16 + (lane & 15);
                const int col = kk + (lane >> 4) * 8;
                ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], &As[st][row][col]);
            }
            unsigned bfr[4][2];
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                const int row = wn * 32 + nj * 8 + (lane & 7) + (lane >> 4) * 8;
                const int col = kk + ((lane >> 3) & 1) * 8;
                ldsm_x4(bfr[nj][0], bfr[nj][1], bfr[nj + 1][0], bfr[nj + 1][1], &Bs[st][row][col]);
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 64 + mi * 16 + g + h * 8;
                if (m >= M) continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int n = n0 + wn * 32 + ni * 8 + 2 * t + q;
                    if (n >= N) continue;
                    float v = acc[mi][ni][h * 2 + q];
                    if (e.bias) v += e.bias[n];
                    if (e.mask && !((float)e.mask[(size_t)m * e.ldm + n] > 0.f)) v = 0.f;
                    if (e.relu) v = fmaxf(v, 0.f);
                    if (e.C32) e.C32[(size_t)m * e.ldc + n] = v;
                    if (e.C16) e.C16[(size_t)m * e.ldc16 + n] = __float2bfloat16(v);
                }
            }
}

// ---------------------------------------------------------------------------
// The same product C = A B^T on the fifth-generation tensor cores.
//
// Operands arrive by TMA: a 2D tensor map per operand (K innermost, rows
// outer) copies 128-row x 64-column BF16 boxes into shared memory with the
// 128-byte swizzle, zero-filling whatever lies past M, N or K, so the kernel
// needs no tail logic.  A ring of TC_STAGES stages (one A and one B box each,
// 32 KB) is filled by one producer lane (warp 0) and drained by one MMA lane
// (warp 1), which issues the four 128 x 128 x 16 tcgen05.mma of a stage from
// shared-memory descriptors (K-major, 128-byte swizzle, 1024 bytes between
// 8-row groups; the 16-element K steps advance the start address by 32 bytes
// inside the swizzle atom) and commits them to the stage's "empty" barrier,
// which frees it for the producer.  The FP32 accumulator (128 lanes x 128
// columns) lives in tensor memory, allocated by warp 1; after the last stage
// a commit to the "done" barrier hands it to the four epilogue warps (2..5),
// which read their lane quarter (warp % 4) with tcgen05.ld, apply bias, ReLU
// mask and output conversion, and store.  With split-K (grid z > 1) each CTA
// takes a contiguous range of K blocks and writes its FP32 partial tile to a
// workspace that a second kernel sums in a fixed order (deterministic) before
// the same epilogue.  Every wait is bounded; on expiry *err is set (1; 2 if
// copies or MMAs in flight did not drain either) and the tile is not written.
// ---------------------------------------------------------------------------
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 4, TC_NTH = 192;
constexpr int TC_TILE = TC_BM * TC_BK * 2;                 // bytes of one operand box (16 KB)
constexpr int TC_SMEM = TC_STAGES * 2 * TC_TILE + 1024;    // + slack to align the ring to 1024 bytes
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;
// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_BN >> 3) << 17) |
                              ((unsigned)(TC_BM >> 4) << 24);

__device__ __forceinline__ unsigned long long tc_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool tc_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ bool tc_wait(unsigned bar, unsigned parity)
{
    if (tc_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tc_now();
    while (!tc_try_wait(bar, parity))
        if (tc_now() - t0 > TC_WAIT_NS) return false;
    return true;
}
// shared-memory matrix descriptor, K-major with the 128-byte swizzle: start
// >> 4 (bits 0-13), leading offset 16 bytes (unused by swizzled K-major
// layouts, bits 16-29), stride offset 1024 bytes between 8-row groups (bits
// 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 = 128 bytes (bits 61-63)
__device__ __forceinline__ unsigned long long tc_desc_sw128(unsigned addr)
{
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((unsigned long long)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void tc_mma(unsigned tmem, unsigned long long ad, unsigned long long bd, unsigned acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_tma_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// one output element through the epilogue (bias, ReLU mask, ReLU, FP32 and/or BF16 store)
__device__ __forceinline__ void epi_store(const Epi& e, int m, int n, float x)
{
    if (e.bias) x += e.bias[n];
    if (e.mask && !((float)e.mask[(size_t)m * e.ldm + n] > 0.f)) x = 0.f;
    if (e.relu) x = fmaxf(x, 0.f);
    if (e.C32) e.C32[(size_t)m * e.ldc + n] = x;
    if (e.C16) e.C16[(size_t)m * e.ldc16 + n] = __float2bfloat16(x);
}

__global__ void __launch_bounds__(TC_NTH, 1) gemm_nt_tc(const __grid_constant__ CUtensorMap ta,
                                                         const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                                                         int kb_per_split, Epi e, float* ws, int* err)
{
    extern __shared__ unsigned char tc_dyn[];
    __shared__ __align__(8) unsigned long long bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_done;
    __shared__ unsigned tmem_slot;
    __shared__ int fail_s, issued_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const int KB = (K + TC_BK - 1) / TC_BK;
    const int kb0 = blockIdx.z * kb_per_split, kb1 = min(KB, kb0 + kb_per_split);
    const int nk = max(kb1 - kb0, 0);
    // the ring starts at the first 1024-byte boundary (the swizzle pattern follows address bits)
    const unsigned ring = (sa(tc_dyn) + 1023u) & ~1023u;
    auto full = [&](int s) { return sa(&bar_full[s]); };
    auto empty = [&](int s) { return sa(&bar_empty[s]); };
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full(s)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty(s)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar_done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        issued_s = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_slot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_slot;
    if (warp == 0 && lane == 0) {
        // producer: one stage = one A box and one B box (rows m0.. / n0.., K block kb0 + i)
        asm volatile("prefetch.tensormap [%0];" ::"l"(&ta) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tb) : "memory");
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            if (i >= TC_STAGES && !tc_wait(empty(s), (unsigned)((i / TC_STAGES) - 1) & 1u)) {
                atomicExch(&fail_s, 1);
                break;
            }
            if (*(volatile int*)&fail_s) break;
            const unsigned a_s = ring + (unsigned)s * 2u * TC_TILE, b_s = a_s + TC_TILE;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(s)), "r"(2 * TC_TILE)
                         : "memory");
            const int kx = (kb0 + i) * TC_BK;  // a multiple of 64 elements: 128-byte aligned inner coordinate
            tc_tma_2d(a_s, &ta, kx, m0, full(s));
            tc_tma_2d(b_s, &tb, kx, n0, full(s));
            issued_s = i + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA lane
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            if (!tc_wait(full(s), (unsigned)(i / TC_STAGES) & 1u) || *(volatile int*)&fail_s) {
                atomicExch(&fail_s, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a_s = ring + (unsigned)s * 2u * TC_TILE, b_s = a_s + TC_TILE;
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j)
                tc_mma(tmem, tc_desc_sw128(a_s + (unsigned)j * 32u), tc_desc_sw128(b_s + (unsigned)j * 32u),
                       (i | j) != 0);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(s))
                         : "memory");
        }
        // completion of the last commit implies completion of every earlier MMA
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sa(&bar_done))
                     : "memory");
    } else if (warp >= 2) {
        // epilogue: wait for the accumulator, then lane quarter warp % 4 = rows m0 + 32 (warp % 4) + lane
        // the tcgen05.ld below is warp-collective: decide once per warp
        const bool ok = __all_sync(0xffffffffu, nk == 0 || tc_wait(sa(&bar_done), 0u));
        if (!ok && lane == 0) atomicExch(&fail_s, 1);
        const int failed = __shfl_sync(0xffffffffu, *(volatile int*)&fail_s, 0);
        if (ok && !failed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int q = warp & 3;
#pragma unroll 1
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                unsigned v[32];
                if (nk > 0) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
                        "%30, %31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int t = 0; t < 32; ++t) v[t] = 0u;
                }
                // stage the warp's 32 x 32 chunk (lane = row) in shared memory -- the ring is idle
                // once every MMA has completed -- then write it row by row, lane = column, so each
                // store instruction covers 32 consecutive elements of one row
                float* stg = reinterpret_cast<float*>(tc_dyn + (ring - sa(tc_dyn))) + (size_t)(warp - 2) * 32 * 33;
#pragma unroll
                for (int t = 0; t < 32; ++t) stg[lane * 33 + t] = __uint_as_float(v[t]);
                __syncwarp();
                const int n = n0 + c0 + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int mr = m0 + q * 32 + rr;
                    if (mr >= M || n >= N) continue;
                    const float x = stg[rr * 33 + lane];
                    if (ws)
                        ws[((size_t)blockIdx.z * M + mr) * N + n] = x;  // split-K partial tile of split z
                    else
                        epi_store(e, mr, n, x);
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (*(volatile int*)&fail_s && tid == 0) {
        // before the stages and the tensor memory are released, copies still in flight and
        // MMAs still in flight must finish: the producer reuses a stage only after its MMAs
        // consumed it, so only the last TC_STAGES issued copies can be pending (each completes
        // the phase (i / TC_STAGES) of its stage's "full" barrier), and the "done" commit,
        // made after the MMA lane's last issue, completes once every MMA has
        bool drained = true;
        const int issued = issued_s;
        for (int i = max(0, issued - TC_STAGES); i < issued; ++i)
            if (!tc_wait(full(i % TC_STAGES), (unsigned)(i / TC_STAGES) & 1u)) drained = false;
        if (!tc_wait(sa(&bar_done), 0u)) drained = false;
        atomicMax(err, drained ? 1 : 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// split-K: C = epilogue(sum over z of ws[z]) in a fixed order
__global__ void splitk_epilogue(const float* ws, int splits, int M, int N, Epi e)
{
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += ws[(size_t)z * total + i];
        epi_store(e, (int)(i / N), (int)(i % N), acc);
    }
}

// out (C x R, ld_out) = in (R x C, ld_in)^T, BF16, 32 x 32 tiles
__global__ void transpose_bf16(const bf16* in, int R, int C, int ld_in, bf16* out, int ld_out)
{
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = in[(size_t)r * ld_in + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * ld_out + r] = tile[threadIdx.x][i];
    }
}

// Xn (bf16, ld) = (X - mean) / std, X row-major B x d
__global__ void normalize_to_bf16(const float* X, int B, int d, const float* mean, const float* istd, bf16* out, int ld)
{
    const long long total = (long long)B * d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / d), c = (int)(i % d);
        out[(size_t)r * ld + c] = __float2bfloat16((X[i] - mean[c]) * istd[c]);
    }
}

// loss partials and dy = (y - (t - mean)/std) / (B d): dy32 (B x d), dy16 (ld16)
__global__ void loss_grad(const float* y, const float* tgt, int B, int d, const float* mean, const float* istd,
                          float* dy32, bf16* dy16, int ld16, double* part)
{
    const long long total = (long long)B * d;
    const float scale = 1.0f / (float)total;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / d), c = (int)(i % d);
        const float diff = y[i] - (tgt[i] - mean[c]) * istd[c];
        acc += (double)diff * diff;
        const float g = diff * scale;
        dy32[i] = g;
        dy16[(size_t)r * ld16 + c] = __float2bfloat16(g);
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void sum_partials(const double* part, int nb, double scale, double* out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t * scale;
    }
}

// db[c] = sum_r D[r][c]
__global__ void col_sums(const float* D, int B, int d, float* db)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d; c += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < B; ++r) s += D[(size_t)r * d + c];
        db[c] = s;
    }
}

// Adam on all parameters; refreshes the BF16 copies of the weight matrices
struct Seg {
    long long off, len;
    bf16* w16;  // BF16 copy or null for biases
    int cols;   // row length of the matrix
    int ld16;   // leading dimension of the BF16 copy
};
struct Segs {
    Seg s[6];
};
__global__ void adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1c, float b2c, Segs segs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
        p[i] = pi;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (segs.s[k].w16 && i >= segs.s[k].off && i < segs.s[k].off + segs.s[k].len) {
                const long long j = i - segs.s[k].off;
                segs.s[k].w16[(j / segs.s[k].cols) * segs.s[k].ld16 + j % segs.s[k].cols] = __float2bfloat16(pi);
            }
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
// uniform(-a, a) from a counter-based hash of (seed, index); zero outside [off, off+len) of weights
__global__ void init_uniform(float* p, long long off, long long len, float a, unsigned long long seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h = mix64(seed ^ mix64((unsigned long long)(off + i)));
        const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
        p[off + i] = (float)((2.0 * u - 1.0) * a);
    }
}

// out (rows x cols, ld) = in (rows x cols, packed)
__global__ void f32_to_bf16_2d(const float* in, long long rows, int cols, bf16* out, int ld)
{
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[(i / cols) * ld + i % cols] = __float2bfloat16(in[i]);
}

// Y = y * std + mean (output units)
__global__ void denormalize(const float* y, int B, int d, const float* mean, const float* stdv, float* Y)
{
    const long long total = (long long)B * d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % d);
        Y[i] = y[i] * stdv[c] + mean[c];
    }
}

// per-column mean and inverse std (two passes in FP64), std < 1e-6 -> 1
__global__ void col_stats(const float* X, long long rows, int d, float* mean, float* stdv, float* istd)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long r = 0; r < rows; ++r) s += X[(size_t)r * d + c];
        const double mu = s / (double)rows;
        double q = 0.0;
        for (long long r = 0; r < rows; ++r) {
            const double e = X[(size_t)r * d + c] - mu;
            q += e * e;
        }
        double sd = sqrt(q / (double)rows);
        if (!(sd >= 1e-6)) sd = 1.0;
        mean[c] = (float)mu;
        stdv[c] = (float)sd;
        istd[c] = (float)(1.0 / sd);
    }
}

__global__ void fill_f32(float* p, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}

int pad8(int x) { return (x + 7) & ~7; }
int grid1d(long long n, int th = 256) { return (int)std::max<long long>(1, std::min<long long>((n + th - 1) / th, 8192)); }

}  // namespace

struct scs_mlp {
    int din, dh, dout, maxB;
    int ldin, ldout;  // padded leading dimensions (multiples of 8)
    cudaStream_t st;
    long long np;
    long long oW1, ob1, oW2, ob2, oW3, ob3;
    float *p, *g, *m, *v;                // parameters, gradients, Adam moments
    bf16 *W1, *W2, *W3, *W2t, *W3t;      // BF16 copies (W2t: h x h, W3t: h x ldout)
    float *in_mean, *in_std, *in_istd, *out_mean, *out_std, *out_istd;
    bf16 *Xn, *Xnt, *h1, *h1t, *h2, *h2t, *dy16, *dyt, *dh2_16, *dh2t, *dh1_16, *dh1t;
    float *y, *dy32, *dh2_32, *dh1_32;
    double *part, *loss;
    int* err;  // set by a tensor-core GEMM whose bounded wait expired
    int step;
    int gemm_impl;  // SCS_MLP_GEMM_MMA or SCS_MLP_GEMM_TCGEN05
    int lastB;      // rows of the last batch that went through forward()
    float* ws;      // split-K partial tiles of the tensor-core GEMMs
    size_t ws_floats;
    char* arena;
};

static int mlp_err(const char* what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    sscs::record_error(buf);
    return SCS_ECUDA;
}
#define MCU(x)                                          \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return mlp_err(#x, e_); \
    } while (0)

// Set once a tensor-core GEMM reported that its MMAs did not drain before the
// tensor memory was released: that memory may since have been written behind
// another CTA's back, so no later GEMM of this process is trusted.
static std::atomic<bool> g_tc_fatal{false};
static const char* const TC_FATAL_MSG =
    "mlp: a tensor-core GEMM released tensor memory while its MMAs may still have been running; "
    "results of this CUDA context can no longer be trusted, every later GEMM call fails";

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// tensor map of a row-major BF16 operand (rows x K, row stride ld elements): boxes of
// TC_BM rows x TC_BK columns, 128-byte swizzle, zero fill past the extents
static int operand_map(CUtensorMap* map, const bf16* base, int rows, int K, int ld)
{
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) {
        sscs::record_error("mlp: cuTensorMapEncodeTiled is unavailable");
        return SCS_ECUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "mlp: cuTensorMapEncodeTiled failed (%d)", (int)r);
        sscs::record_error(buf);
        return SCS_ECUDA;
    }
    return SCS_OK;
}

static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return sms > 0 ? sms : 1;
}

// K splits for a tcgen05 product: when its 128 x 128 tiles would leave most SMs idle and
// K is deep, split K (at least 4 K blocks a split) as far as the workspace allows
static int tc_splits(int M, int N, int K, size_t ws_floats)
{
    const int tiles = ((M + TC_BM - 1) / TC_BM) * ((N + TC_BN - 1) / TC_BN);
    const int KB = (K + TC_BK - 1) / TC_BK;
    const int sms = device_sms();
    if (ws_floats == 0 || 2 * tiles > sms || KB < 8) return 1;
    int sp = std::min((sms + tiles - 1) / tiles, KB / 4);
    while (sp > 1 && (size_t)sp * M * N > ws_floats) --sp;
    if (sp < 2) return 1;
    const int per = (KB + sp - 1) / sp;
    return (KB + per - 1) / per;
}

static int launch_gemm(int impl, cudaStream_t st, int* err, int M, int N, int K, const bf16* A, int lda,
                       const bf16* B, int ldb, const Epi& e, float* ws = nullptr, size_t ws_floats = 0)
{
    if (g_tc_fatal) {
        sscs::record_error(TC_FATAL_MSG);
        return SCS_ECUDA;
    }
    if (impl == SCS_MLP_GEMM_TCGEN05) {
        CUtensorMap ta, tb;
        int rc;
        if ((rc = operand_map(&ta, A, M, K, lda)) || (rc = operand_map(&tb, B, N, K, ldb))) return rc;
        const int KB = (K + TC_BK - 1) / TC_BK;
        const int splits = tc_splits(M, N, K, ws_floats);
        const int per = (KB + splits - 1) / splits;
        // a per-device attribute: set before every launch (a host call of about a microsecond)
        MCU(cudaFuncSetAttribute(gemm_nt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, splits);
        gemm_nt_tc<<<grid, TC_NTH, TC_SMEM, st>>>(ta, tb, M, N, K, per, e, splits > 1 ? ws : nullptr, err);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) return mlp_err("gemm_nt_tc launch", ce);
        if (splits > 1) {
            const long long total = (long long)M * N;
            splitk_epilogue<<<(int)std::min<long long>(8192, (total + 255) / 256), 256, 0, st>>>(ws, splits, M, N, e);
            ce = cudaGetLastError();
            if (ce != cudaSuccess) return mlp_err("splitk_epilogue launch", ce);
        }
        return SCS_OK;
    }
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_nt<<<grid, NTH, 0, st>>>(M, N, K, A, lda, B, ldb, e);
    const cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? SCS_OK : mlp_err("gemm_nt launch", ce);
}
static int gemm(scs_mlp* n, int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, const Epi& e)
{
    return launch_gemm(n->gemm_impl, n->st, n->err, M, N, K, A, lda, B, ldb, e, n->ws, n->ws_floats);
}
// reads (and clears) the tensor-core GEMM's timeout flag; the stream must be synchronised
static int check_err_flag(scs_mlp* n)
{
    int h = 0;
    MCU(cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->st));
    MCU(cudaStreamSynchronize(n->st));
    if (h) {
        MCU(cudaMemsetAsync(n->err, 0, sizeof(int), n->st));
        if (h >= 2) g_tc_fatal = true;
        sscs::record_error(h >= 2 ? TC_FATAL_MSG : "mlp: a tensor-core GEMM wait timed out; its output tile was not written");
        return SCS_ECUDA;
    }
    return SCS_OK;
}
static void transpose(scs_mlp* n, const bf16* in, int R, int C, int ld_in, bf16* out, int ld_out)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    transpose_bf16<<<grid, block, 0, n->st>>>(in, R, C, ld_in, out, ld_out);
}
static Epi epi(const float* bias, const bf16* mask, int ldm, int relu, float* C32, int ldc, bf16* C16, int ldc16)
{
    Epi e;
    e.bias = bias;
    e.mask = mask;
    e.ldm = ldm;
    e.relu = relu;
    e.C32 = C32;
    e.ldc = ldc;
    e.C16 = C16;
    e.ldc16 = ldc16;
    return e;
}

extern "C" int scs_mlp_create(int32_t din, int32_t dh, int32_t dout, int32_t maxB, uint64_t seed, void* stream,
                              scs_mlp** out)
{
    if (!out || din <= 0 || dh <= 0 || dout <= 0 || maxB <= 0 || dh % 8 != 0) {
        sscs::record_error("scs_mlp_create: bad sizes (all positive, d_hidden a multiple of 8)");
        return SCS_EINVAL;
    }
    *out = nullptr;
    scs_mlp* n = new (std::nothrow) scs_mlp();
    if (!n) return SCS_ENOMEM;
    memset(n, 0, sizeof(*n));
    n->din = din;
    n->dh = dh;
    n->dout = dout;
    n->maxB = maxB;
    n->ldin = pad8(din);
    n->ldout = pad8(dout);
    n->gemm_impl = SCS_MLP_GEMM_TCGEN05;
    n->st = (cudaStream_t)stream;
    const int Bp = pad8(maxB);
    n->oW1 = 0;
    n->ob1 = n->oW1 + (long long)dh * din;
    n->oW2 = n->ob1 + dh;
    n->ob2 = n->oW2 + (long long)dh * dh;
    n->oW3 = n->ob2 + dh;
    n->ob3 = n->oW3 + (long long)dout * dh;
    n->np = n->ob3 + dout;
    // one arena
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> plan;
    auto take = [&](void** ptr, size_t bytes) { plan.push_back({ptr, bytes}); };
    take((void**)&n->p, sizeof(float) * n->np);
    take((void**)&n->g, sizeof(float) * n->np);
    take((void**)&n->m, sizeof(float) * n->np);
    take((void**)&n->v, sizeof(float) * n->np);
    take((void**)&n->W1, sizeof(bf16) * (size_t)dh * n->ldin);
    take((void**)&n->W2, sizeof(bf16) * (size_t)dh * dh);
    take((void**)&n->W3, sizeof(bf16) * (size_t)dout * dh);
    take((void**)&n->W2t, sizeof(bf16) * (size_t)dh * dh);
    take((void**)&n->W3t, sizeof(bf16) * (size_t)dh * n->ldout);
    take((void**)&n->in_mean, sizeof(float) * din);
    take((void**)&n->in_std, sizeof(float) * din);
    take((void**)&n->in_istd, sizeof(float) * din);
    take((void**)&n->out_mean, sizeof(float) * dout);
    take((void**)&n->out_std, sizeof(float) * dout);
    take((void**)&n->out_istd, sizeof(float) * dout);
    take((void**)&n->Xn, sizeof(bf16) * (size_t)maxB * n->ldin);
    take((void**)&n->Xnt, sizeof(bf16) * (size_t)din * Bp);
    take((void**)&n->h1, sizeof(bf16) * (size_t)maxB * dh);
    take((void**)&n->h1t, sizeof(bf16) * (size_t)dh * Bp);
    take((void**)&n->h2, sizeof(bf16) * (size_t)maxB * dh);
    take((void**)&n->h2t, sizeof(bf16) * (size_t)dh * Bp);
    take((void**)&n->dy16, sizeof(bf16) * (size_t)maxB * n->ldout);
    take((void**)&n->dyt, sizeof(bf16) * (size_t)dout * Bp);
    take((void**)&n->dh2_16, sizeof(bf16) * (size_t)maxB * dh);
    take((void**)&n->dh2t, sizeof(bf16) * (size_t)dh * Bp);
    take((void**)&n->dh1_16, sizeof(bf16) * (size_t)maxB * dh);
    take((void**)&n->dh1t, sizeof(bf16) * (size_t)dh * Bp);
    take((void**)&n->y, sizeof(float) * (size_t)maxB * dout);
    take((void**)&n->dy32, sizeof(float) * (size_t)maxB * dout);
    take((void**)&n->dh2_32, sizeof(float) * (size_t)maxB * dh);
    take((void**)&n->dh1_32, sizeof(float) * (size_t)maxB * dh);
    take((void**)&n->part, sizeof(double) * 8192);
    take((void**)&n->loss, sizeof(double) * 2);
    take((void**)&n->err, sizeof(int) * 4);
    // split-K workspace: up to 16 partial tiles of the widest batch-row product
    n->ws_floats = (size_t)16 * maxB * (size_t)std::max(std::max(dh, din), 128);
    take((void**)&n->ws, sizeof(float) * n->ws_floats);
    for (auto& pl : plan) off += (pl.second + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc((void**)&n->arena, off);
    if (e != cudaSuccess) {
        delete n;
        return mlp_err("cudaMalloc", e);
    }
    size_t o = 0;
    for (auto& pl : plan) {
        *pl.first = n->arena + o;
        o += (pl.second + 255) & ~size_t(255);
    }
    auto fail = [&](int rc) { scs_mlp_destroy(n); return rc; };
    if (cudaMemsetAsync(n->arena, 0, off, n->st) != cudaSuccess) return fail(mlp_err("memset", cudaGetLastError()));
    init_uniform<<<grid1d((long long)dh * din), 256, 0, n->st>>>(n->p, n->oW1, (long long)dh * din, 1.f / sqrtf((float)din), seed);
    init_uniform<<<grid1d((long long)dh * dh), 256, 0, n->st>>>(n->p, n->oW2, (long long)dh * dh, 1.f / sqrtf((float)dh), seed);
    init_uniform<<<grid1d((long long)dout * dh), 256, 0, n->st>>>(n->p, n->oW3, (long long)dout * dh, 1.f / sqrtf((float)dh), seed);
    fill_f32<<<grid1d(din), 256, 0, n->st>>>(n->in_std, din, 1.f);
    fill_f32<<<grid1d(din), 256, 0, n->st>>>(n->in_istd, din, 1.f);
    fill_f32<<<grid1d(dout), 256, 0, n->st>>>(n->out_std, dout, 1.f);
    fill_f32<<<grid1d(dout), 256, 0, n->st>>>(n->out_istd, dout, 1.f);
    int rc = scs_mlp_set_params(n, nullptr);
    if (rc) return fail(rc);
    *out = n;
    return SCS_OK;
}

// refresh the BF16 copies (and transposes) from the FP32 parameters
static int refresh_bf16(scs_mlp* n)
{
    f32_to_bf16_2d<<<grid1d((long long)n->dh * n->din), 256, 0, n->st>>>(n->p + n->oW1, n->dh, n->din, n->W1, n->ldin);
    f32_to_bf16_2d<<<grid1d((long long)n->dh * n->dh), 256, 0, n->st>>>(n->p + n->oW2, n->dh, n->dh, n->W2, n->dh);
    f32_to_bf16_2d<<<grid1d((long long)n->dout * n->dh), 256, 0, n->st>>>(n->p + n->oW3, n->dout, n->dh, n->W3, n->dh);
    transpose(n, n->W2, n->dh, n->dh, n->dh, n->W2t, n->dh);
    transpose(n, n->W3, n->dout, n->dh, n->dh, n->W3t, n->ldout);
    MCU(cudaGetLastError());
    return SCS_OK;
}

extern "C" int64_t scs_mlp_num_params(const scs_mlp* n) { return n ? n->np : 0; }

extern "C" int scs_mlp_get_params(scs_mlp* n, float* params)
{
    if (!n || !params) return SCS_EINVAL;
    MCU(cudaMemcpyAsync(params, n->p, sizeof(float) * n->np, cudaMemcpyDefault, n->st));
    MCU(cudaStreamSynchronize(n->st));
    return SCS_OK;
}

extern "C" int scs_mlp_set_params(scs_mlp* n, const float* params)
{
    if (!n) return SCS_EINVAL;
    if (params) MCU(cudaMemcpyAsync(n->p, params, sizeof(float) * n->np, cudaMemcpyDefault, n->st));
    int rc = refresh_bf16(n);
    if (rc) return rc;
    MCU(cudaStreamSynchronize(n->st));
    return SCS_OK;
}

extern "C" int scs_mlp_fit_normalization(scs_mlp* n, const float* X, const float* Y, int64_t rows)
{
    if (!n || !X || !Y || rows <= 0) return SCS_EINVAL;
    col_stats<<<grid1d(n->din, 128), 128, 0, n->st>>>(X, rows, n->din, n->in_mean, n->in_std, n->in_istd);
    col_stats<<<grid1d(n->dout, 128), 128, 0, n->st>>>(Y, rows, n->dout, n->out_mean, n->out_std, n->out_istd);
    MCU(cudaGetLastError());
    MCU(cudaStreamSynchronize(n->st));
    return SCS_OK;
}

static int forward(scs_mlp* n, const float* X, int B)
{
    int rc;
    n->lastB = B;
    normalize_to_bf16<<<grid1d((long long)B * n->din), 256, 0, n->st>>>(X, B, n->din, n->in_mean, n->in_istd, n->Xn, n->ldin);
    if ((rc = gemm(n, B, n->dh, n->din, n->Xn, n->ldin, n->W1, n->ldin,
                   epi(n->p + n->ob1, nullptr, 0, 1, nullptr, 0, n->h1, n->dh))))
        return rc;
    if ((rc = gemm(n, B, n->dh, n->dh, n->h1, n->dh, n->W2, n->dh,
                   epi(n->p + n->ob2, nullptr, 0, 1, nullptr, 0, n->h2, n->dh))))
        return rc;
    if ((rc = gemm(n, B, n->dout, n->dh, n->h2, n->dh, n->W3, n->dh,
                   epi(n->p + n->ob3, nullptr, 0, 0, n->y, n->dout, nullptr, 0))))
        return rc;
    return SCS_OK;
}

// loss and gradients into n->g; returns loss in *loss_host
static int backward(scs_mlp* n, const float* Y, int B, float* loss_host)
{
    const int Bp = pad8(B);
    const int nb = grid1d((long long)B * n->dout);
    int rc;
    loss_grad<<<nb, 256, 0, n->st>>>(n->y, Y, B, n->dout, n->out_mean, n->out_istd, n->dy32, n->dy16, n->ldout, n->part);
    sum_partials<<<1, 256, 0, n->st>>>(n->part, nb, 0.5 / ((double)B * n->dout), n->loss);
    transpose(n, n->dy16, B, n->dout, n->ldout, n->dyt, Bp);
    transpose(n, n->h2, B, n->dh, n->dh, n->h2t, Bp);
    transpose(n, n->h1, B, n->dh, n->dh, n->h1t, Bp);
    transpose(n, n->Xn, B, n->din, n->ldin, n->Xnt, Bp);
    // layer 3: gW3 = dy^T h2, gb3 = colsum(dy), dh2 = (dy W3) * [h2 > 0]
    if ((rc = gemm(n, n->dout, n->dh, B, n->dyt, Bp, n->h2t, Bp, epi(nullptr, nullptr, 0, 0, n->g + n->oW3, n->dh, nullptr, 0))))
        return rc;
    col_sums<<<grid1d(n->dout), 256, 0, n->st>>>(n->dy32, B, n->dout, n->g + n->ob3);
    if ((rc = gemm(n, B, n->dh, n->dout, n->dy16, n->ldout, n->W3t, n->ldout,
                   epi(nullptr, n->h2, n->dh, 0, n->dh2_32, n->dh, n->dh2_16, n->dh))))
        return rc;
    // layer 2
    transpose(n, n->dh2_16, B, n->dh, n->dh, n->dh2t, Bp);
    if ((rc = gemm(n, n->dh, n->dh, B, n->dh2t, Bp, n->h1t, Bp, epi(nullptr, nullptr, 0, 0, n->g + n->oW2, n->dh, nullptr, 0))))
        return rc;
    col_sums<<<grid1d(n->dh), 256, 0, n->st>>>(n->dh2_32, B, n->dh, n->g + n->ob2);
    if ((rc = gemm(n, B, n->dh, n->dh, n->dh2_16, n->dh, n->W2t, n->dh,
                   epi(nullptr, n->h1, n->dh, 0, n->dh1_32, n->dh, n->dh1_16, n->dh))))
        return rc;
    // layer 1
    transpose(n, n->dh1_16, B, n->dh, n->dh, n->dh1t, Bp);
    if ((rc = gemm(n, n->dh, n->din, B, n->dh1t, Bp, n->Xnt, Bp, epi(nullptr, nullptr, 0, 0, n->g + n->oW1, n->din, nullptr, 0))))
        return rc;
    col_sums<<<grid1d(n->dh), 256, 0, n->st>>>(n->dh1_32, B, n->dh, n->g + n->ob1);
    MCU(cudaGetLastError());
    if (loss_host) {
        double l = 0.0;
        MCU(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->st));
        MCU(cudaStreamSynchronize(n->st));
        *loss_host = (float)l;
        if ((rc = check_err_flag(n))) return rc;
    }
    return SCS_OK;
}

extern "C" int scs_mlp_forward(scs_mlp* n, const float* X, int32_t B, float* Y)
{
    if (!n || !X || !Y || B <= 0 || B > n->maxB) {
        sscs::record_error("scs_mlp_forward: bad arguments");
        return SCS_EINVAL;
    }
    int rc = forward(n, X, B);
    if (rc) return rc;
    denormalize<<<grid1d((long long)B * n->dout), 256, 0, n->st>>>(n->y, B, n->dout, n->out_mean, n->out_std, Y);
    MCU(cudaGetLastError());
    return SCS_OK;
}

extern "C" int scs_mlp_gradients(scs_mlp* n, const float* X, const float* Y, int32_t B, float* grad, float* loss)
{
    if (!n || !X || !Y || B <= 0 || B > n->maxB) {
        sscs::record_error("scs_mlp_gradients: bad arguments");
        return SCS_EINVAL;
    }
    int rc = forward(n, X, B);
    if (!rc) rc = backward(n, Y, B, loss);
    if (rc) return rc;
    if (grad) MCU(cudaMemcpyAsync(grad, n->g, sizeof(float) * n->np, cudaMemcpyDefault, n->st));
    MCU(cudaStreamSynchronize(n->st));
    return check_err_flag(n);
}

extern "C" int scs_mlp_train_step(scs_mlp* n, const float* X, const float* Y, int32_t B, float lr, float* loss)
{
    if (!n || !X || !Y || B <= 0 || B > n->maxB) {
        sscs::record_error("scs_mlp_train_step: bad arguments");
        return SCS_EINVAL;
    }
    int rc = forward(n, X, B);
    if (!rc) rc = backward(n, Y, B, loss);
    if (rc) return rc;
    n->step++;
    // bias corrections 1 - beta^t in FP64: in FP32, 1 - 0.999f^t loses five digits to cancellation
    const float b1c = (float)(1.0 - pow(0.9, (double)n->step)), b2c = (float)(1.0 - pow(0.999, (double)n->step));
    Segs segs;
    segs.s[0] = {n->oW1, (long long)n->dh * n->din, n->W1, n->din, n->ldin};
    segs.s[1] = {n->ob1, n->dh, nullptr, 1, 1};
    segs.s[2] = {n->oW2, (long long)n->dh * n->dh, n->W2, n->dh, n->dh};
    segs.s[3] = {n->ob2, n->dh, nullptr, 1, 1};
    segs.s[4] = {n->oW3, (long long)n->dout * n->dh, n->W3, n->dh, n->dh};
    segs.s[5] = {n->ob3, n->dout, nullptr, 1, 1};
    adam<<<grid1d(n->np), 256, 0, n->st>>>(n->p, n->g, n->m, n->v, n->np, lr, b1c, b2c, segs);
    transpose(n, n->W2, n->dh, n->dh, n->dh, n->W2t, n->dh);
    transpose(n, n->W3, n->dout, n->dh, n->dh, n->W3t, n->ldout);
    MCU(cudaGetLastError());
    return SCS_OK;
}

extern "C" int scs_mlp_set_gemm(scs_mlp* n, int32_t impl)
{
    if (!n || (impl != SCS_MLP_GEMM_MMA && impl != SCS_MLP_GEMM_TCGEN05)) {
        sscs::record_error("scs_mlp_set_gemm: bad arguments");
        return SCS_EINVAL;
    }
    n->gemm_impl = impl;
    return SCS_OK;
}

extern "C" int scs_mlp_gemm_nt(int32_t impl, int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                               const void* B, int32_t ldb, float* C, int32_t ldc, void* stream)
{
    // with K = 0 the operands are never read (C = 0) and may be null
    const bool aligned = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
    const bool operands_ok = K == 0 || (A && B && aligned);
    if ((impl != SCS_MLP_GEMM_MMA && impl != SCS_MLP_GEMM_TCGEN05) || M < 0 || N < 0 || K < 0 || !operands_ok ||
        !C || lda < K || ldb < K || lda % 8 || ldb % 8 || ldc < N) {
        sscs::record_error("scs_mlp_gemm_nt: bad arguments");
        return SCS_EINVAL;
    }
    if (M == 0 || N == 0) return SCS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (K == 0) {  // empty sum: no kernel reads the (possibly null) operands
        MCU(cudaMemset2DAsync(C, sizeof(float) * (size_t)ldc, 0, sizeof(float) * (size_t)N, (size_t)M, st));
        MCU(cudaStreamSynchronize(st));
        return SCS_OK;
    }
    int* err = nullptr;
    MCU(cudaMalloc((void**)&err, sizeof(int)));
    // the split-K workspace this product would use (tensor-core kernel only)
    float* ws = nullptr;
    size_t ws_floats = 0;
    if (impl == SCS_MLP_GEMM_TCGEN05) {
        const int sp = tc_splits(M, N, K, (size_t)1 << 40);
        if (sp > 1) {
            ws_floats = (size_t)sp * M * N;
            if (cudaMalloc((void**)&ws, sizeof(float) * ws_floats) != cudaSuccess) {
                cudaFree(err);
                return mlp_err("cudaMalloc", cudaGetLastError());
            }
        }
    }
    int rc = SCS_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) rc = mlp_err("memset", cudaGetLastError());
    if (!rc)
        rc = launch_gemm(impl, st, err, M, N, K, static_cast<const bf16*>(A), lda, static_cast<const bf16*>(B), ldb,
                         epi(nullptr, nullptr, 0, 0, C, ldc, nullptr, 0), ws, ws_floats);
    int h = 0;
    if (!rc && cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = mlp_err("copy", cudaGetLastError());
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = mlp_err("gemm", cudaGetLastError());
    cudaFree(err);
    if (ws) cudaFree(ws);
    if (!rc && h) {
        if (h >= 2) g_tc_fatal = true;
        sscs::record_error(h >= 2 ? TC_FATAL_MSG : "scs_mlp_gemm_nt: a tensor-core wait timed out");
        rc = SCS_ECUDA;
    }
    return rc;
}

extern "C" int scs_mlp_read(scs_mlp* n, int32_t what, void* out, int64_t* rows, int64_t* cols, int32_t* elem_bytes)
{
    if (!n) {
        sscs::record_error("scs_mlp_read: NULL network");
        return SCS_EINVAL;
    }
    const void* src = nullptr;
    long long r = 1, c = 0, ld = 0;
    int eb = 4;
    const long long B = n->lastB;
    switch (what) {
        case SCS_MLP_READ_PARAMS: src = n->p; c = n->np; break;
        case SCS_MLP_READ_GRAD: src = n->g; c = n->np; break;
        case SCS_MLP_READ_ADAM_M: src = n->m; c = n->np; break;
        case SCS_MLP_READ_ADAM_V: src = n->v; c = n->np; break;
        case SCS_MLP_READ_IN_MEAN: src = n->in_mean; c = n->din; break;
        case SCS_MLP_READ_IN_STD: src = n->in_std; c = n->din; break;
        case SCS_MLP_READ_OUT_MEAN: src = n->out_mean; c = n->dout; break;
        case SCS_MLP_READ_OUT_STD: src = n->out_std; c = n->dout; break;
        case SCS_MLP_READ_XN: src = n->Xn; r = B; c = n->din; ld = n->ldin; eb = 2; break;
        case SCS_MLP_READ_H1: src = n->h1; r = B; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_H2: src = n->h2; r = B; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_Y: src = n->y; r = B; c = n->dout; break;
        case SCS_MLP_READ_DY: src = n->dy32; r = B; c = n->dout; break;
        case SCS_MLP_READ_DY16: src = n->dy16; r = B; c = n->dout; ld = n->ldout; eb = 2; break;
        case SCS_MLP_READ_DH2: src = n->dh2_32; r = B; c = n->dh; break;
        case SCS_MLP_READ_DH2_16: src = n->dh2_16; r = B; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_DH1: src = n->dh1_32; r = B; c = n->dh; break;
        case SCS_MLP_READ_DH1_16: src = n->dh1_16; r = B; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_W1: src = n->W1; r = n->dh; c = n->din; ld = n->ldin; eb = 2; break;
        case SCS_MLP_READ_W2: src = n->W2; r = n->dh; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_W3: src = n->W3; r = n->dout; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_W2T: src = n->W2t; r = n->dh; c = n->dh; eb = 2; break;
        case SCS_MLP_READ_W3T: src = n->W3t; r = n->dh; c = n->dout; ld = n->ldout; eb = 2; break;
        default:
            sscs::record_error("scs_mlp_read: unknown buffer");
            return SCS_EINVAL;
    }
    if (ld == 0) ld = c;
    if (rows) *rows = r;
    if (cols) *cols = c;
    if (elem_bytes) *elem_bytes = eb;
    if (!out || r == 0 || c == 0) return SCS_OK;
    MCU(cudaMemcpy2DAsync(out, (size_t)c * eb, src, (size_t)ld * eb, (size_t)c * eb, (size_t)r, cudaMemcpyDefault,
                          n->st));
    MCU(cudaStreamSynchronize(n->st));
    return SCS_OK;
}

extern "C" void scs_mlp_destroy(scs_mlp* n)
{
    if (!n) return;
    if (n->arena) cudaFree(n->arena);
    delete n;
}
