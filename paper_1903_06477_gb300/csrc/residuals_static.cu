// residuals_static.cu -- an allocation-free way to evaluate the relative
// primal residual, dual residual and duality gap of a candidate (x, y, s).
//
// It computes the same three numbers as scs_residuals, but needs no scs_work
// and makes no device allocation: its only scratch (the vector A^T y and the
// per-block partial sums) lives in the file-scope array below, which every
// GPU that loads this library keeps until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/superscs.h"

namespace {

constexpr int RS_MAX_N = 1 << 20;  // largest n accepted (the A^T y part of the scratch)
constexpr int RS_BLOCKS = 1024;    // fixed grid of the two streaming kernels
// sums per block: |Ax+s-b|^2, <b,y>, |b|^2, skipped column indices, |A^T y+c|^2, <c,x>, |c|^2
constexpr int RS_VALS = 7;
constexpr int RS_THREADS = 256;
constexpr size_t RS_DOUBLES = (size_t)RS_MAX_N + (size_t)RS_VALS * RS_BLOCKS;
constexpr int RS_MAX_CONTEXTS = 64;

thread_local char rs_err[256];
std::mutex rs_mutex;
// device address of the scratch array per CUDA context, keyed by the
// context's process-unique ID (a context created after cudaDeviceReset gets
// a new ID, and its reloaded module a new address)
struct RsEntry {
    unsigned long long ctx_id;
    double* ptr;
};
RsEntry rs_cache[RS_MAX_CONTEXTS];
int rs_cache_len = 0;

}  // namespace

namespace sscs {
void record_error(const char* msg);  // sets the message scs_last_error(NULL) returns
}

static int rs_fail(int code)
{
    sscs::record_error(rs_err);
    return code;
}

// 8 MiB + 56 KiB of scratch per device: A^T y (RS_MAX_N doubles), then block partials.
static __device__ __align__(256) double g_rs_scratch[RS_DOUBLES];

__device__ __forceinline__ double rs_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sums K values over the block into part[k * RS_BLOCKS + blockIdx.x]
template <int K>
__device__ void rs_block_store(double (&v)[K], double* part, int off)
{
    __shared__ double red[RS_THREADS / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double s = rs_warp_sum(v[k]);
        if (lane == 0) red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < RS_THREADS / 32; ++w) s += red[w][threadIdx.x];
        part[(size_t)(off + threadIdx.x) * RS_BLOCKS + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(RS_THREADS) rs_zero(double* aty, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) aty[j] = 0.0;
}

// rows of A: primal residual terms, <b,y>, |b|^2, and A^T y scattered by
// atomics.  A column index outside [0, n) is skipped (it would read x or
// write the scratch out of bounds) and counted; a nonzero count makes every
// output NaN.
__global__ void __launch_bounds__(RS_THREADS) rs_rows(int m, int n, const int64_t* Ap, const int32_t* Ai,
                                                      const double* Ax, const double* b, const double* x,
                                                      const double* y, const double* s, double* aty, double* part)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double ax = 0.0;
        const double yi = y[i];
        for (int64_t k = Ap[i]; k < Ap[i + 1]; ++k) {
            const int j = Ai[k];
            if ((unsigned)j >= (unsigned)n) {
                v[3] += 1.0;
                continue;
            }
            ax += Ax[k] * x[j];
            atomicAdd(aty + j, Ax[k] * yi);
        }
        const double bi = b[i];
        const double e = ax + s[i] - bi;
        v[0] += e * e;
        v[1] += bi * yi;
        v[2] += bi * bi;
    }
    rs_block_store<4>(v, part, 0);
}

// columns: dual residual terms, <c,x>, |c|^2
__global__ void __launch_bounds__(RS_THREADS) rs_cols(int n, const double* c, const double* x, const double* aty,
                                                      double* part)
{
    double v[3] = {0.0, 0.0, 0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double cj = c[j];
        const double g = aty[j] + cj;
        v[0] += g * g;
        v[1] += cj * x[j];
        v[2] += cj * cj;
    }
    rs_block_store<3>(v, part, 4);
}

// one block: fixed-order sums of the partials, then the three ratios of Sec. 4.3
__global__ void __launch_bounds__(RS_THREADS) rs_final(const double* part, double* out)
{
    __shared__ double tot[RS_VALS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < RS_VALS; k += RS_THREADS / 32) {
        double s = 0.0;
        for (int j = lane; j < RS_BLOCKS; j += 32) s += part[(size_t)k * RS_BLOCKS + j];
        s = rs_warp_sum(s);
        if (lane == 0) tot[k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nb = sqrt(tot[2]), nc = sqrt(tot[6]);
        const double cx = tot[5], by = tot[1];
        const bool bad = tot[3] != 0.0;  // column indices outside [0, n) were skipped
        out[0] = bad ? NAN : sqrt(tot[0]) / (1.0 + nb);
        out[1] = bad ? NAN : sqrt(tot[4]) / (1.0 + nc);
        out[2] = bad ? NAN : fabs(cx + by) / (1.0 + fabs(cx) + fabs(by));
    }
}

// Device address of the static scratch in the current CUDA context (the
// host-side name of the array is only a stand-in, not a device address).  It
// is looked up with cudaGetSymbolAddress once per context -- normally once
// per device, on the first call with that device current -- and cached under
// the context's process-unique ID, so a call after cudaDeviceReset (a new
// primary context, the module reloaded) looks it up again instead of using a
// stale address.
typedef int (*rs_ctx_get_current_fn)(void** ctx);
typedef int (*rs_ctx_get_id_fn)(void* ctx, unsigned long long* id);

static int rs_context_id(unsigned long long* id)
{
    static rs_ctx_get_current_fn get_current = nullptr;
    static rs_ctx_get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        const cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        const cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e1 == cudaSuccess && e2 == cudaSuccess && q1 == cudaDriverEntryPointSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = (rs_ctx_get_current_fn)f1;
            get_id = (rs_ctx_get_id_fn)f2;
        }
    });
    if (!get_current || !get_id) {
        snprintf(rs_err, sizeof rs_err, "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
        return rs_fail(SCS_ECUDA);
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) {
        // no context is current yet: make the current device's primary context current
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess || get_current(&ctx) != 0 || !ctx) {
            snprintf(rs_err, sizeof rs_err, "no current CUDA context");
            return rs_fail(SCS_ECUDA);
        }
    }
    if (get_id(ctx, id) != 0) {
        snprintf(rs_err, sizeof rs_err, "cuCtxGetId failed");
        return rs_fail(SCS_ECUDA);
    }
    return SCS_OK;
}

static int rs_scratch(double** out)
{
    unsigned long long id = 0;
    int rc = rs_context_id(&id);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(rs_mutex);
    for (int k = 0; k < rs_cache_len; ++k)
        if (rs_cache[k].ctx_id == id) {
            *out = rs_cache[k].ptr;
            return SCS_OK;
        }
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_rs_scratch);
    if (e != cudaSuccess || !p) {
        snprintf(rs_err, sizeof rs_err, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        return rs_fail(SCS_ECUDA);
    }
    // a full table keeps its oldest entries; later contexts look the address up on every call
    if (rs_cache_len < RS_MAX_CONTEXTS) rs_cache[rs_cache_len++] = RsEntry{id, p};
    *out = p;
    return SCS_OK;
}

extern "C" int scs_residuals_noalloc(int32_t m, int32_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                                     const double* b, const double* c, const double* x, const double* y,
                                     const double* s, double* out, void* cuda_stream)
{
    if (m <= 0 || n <= 0) {
        snprintf(rs_err, sizeof rs_err, "m and n must be positive (m=%d n=%d)", m, n);
        return rs_fail(SCS_EINVAL);
    }
    if (n > RS_MAX_N) {
        snprintf(rs_err, sizeof rs_err, "n = %d exceeds the static scratch limit of %d columns", n, RS_MAX_N);
        return rs_fail(SCS_EINVAL);
    }
    if (!Ap || !Ai || !Ax || !b || !c || !x || !y || !s || !out) {
        snprintf(rs_err, sizeof rs_err, "NULL argument");
        return rs_fail(SCS_EINVAL);
    }
    double* scratch = nullptr;
    int rc = rs_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* aty = scratch;
    double* part = scratch + RS_MAX_N;
    rs_zero<<<RS_BLOCKS, RS_THREADS, 0, st>>>(aty, n);
    rs_rows<<<RS_BLOCKS, RS_THREADS, 0, st>>>(m, n, Ap, Ai, Ax, b, x, y, s, aty, part);
    rs_cols<<<RS_BLOCKS, RS_THREADS, 0, st>>>(n, c, x, aty, part);
    rs_final<<<1, RS_THREADS, 0, st>>>(part, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(rs_err, sizeof rs_err, "kernel launch failed: %s", cudaGetErrorString(e));
        return rs_fail(SCS_ECUDA);
    }
    return SCS_OK;
}
