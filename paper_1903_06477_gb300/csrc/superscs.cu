// superscs.cu -- host side of the C ABI declared in include/superscs.h:
// validation, the CSR transpose of A built once at setup, one device arena
// per problem (or per batch), and the launches of the device-resident solver.
//
// Launch shapes
//   GridTeam : one cooperative launch of (SMs x resident blocks) CTAs that
//              runs the whole of Algorithm 1 for one large instance.
//   BlockTeam: persistent CTAs that take instances from an atomic queue
//              (largest first) and run Algorithm 1 on each.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/superscs.h"
#include "solver.cuh"
#include "cb_layout.h"

using namespace sscs;

#include "launch.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static void set_err(char* dst, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    if (dst != g_err) memcpy(g_err, dst, 512);
}

namespace sscs {
void record_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace sscs

#define CU(call, errbuf)                                                                                    \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) {                                                                            \
            set_err(errbuf, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);    \
            return SCS_ECUDA;                                                                               \
        }                                                                                                   \
    } while (0)

// ---------------------------------------------------------------------------
// host problem preparation
// ---------------------------------------------------------------------------
struct HostProb {
    int n = 0, m = 0;
    long long nnz = 0;
    std::vector<int> Ap, Ai, Tp, Ti;
    std::vector<double> Ax, Tx, b, c;
    int f = 0, l = 0;
    std::vector<int> q, s, q_off, s_off;
    int ep = 0, ed = 0, e_off = 0;  // exponential cones and the row offset of the first
    double nb = 0, nc = 0;
    int vecA = 32, vecT = 32;
    struct Sell {
        int rows = 0, V = 1, nslices = 0;
        std::vector<int> ptr, col, perm;
        std::vector<double> val;
        std::vector<int> wbnd;  // per-warp slice ranges for the TMA-staged product (grid team)
    } SA, ST;
    // column-blocked copies for the grid team (layout of Cblk in solver.cuh),
    // one per matrix and bulk precision (the block width depends on it)
    using Cb = CbLayout;
    Cb cA64, cAT64, cA32, cAT32;
};

// nnz-balanced contiguous slice ranges for W warps: warp w owns [b[w], b[w+1])
static void warp_bounds(HostProb::Sell& S, int W)
{
    S.wbnd.assign(W + 1, 0);
    const long long total = S.ptr.back();
    for (int w = 0; w <= W; ++w) {
        const long long target = total * w / W;
        S.wbnd[w] = (int)(std::lower_bound(S.ptr.begin(), S.ptr.end(), target) - S.ptr.begin());
        if (S.wbnd[w] > S.nslices) S.wbnd[w] = S.nslices;
    }
    S.wbnd[W] = S.nslices;
}

// Sliced ELL (SELL-H-sigma) from CSR: rows sorted by length (descending,
// stable) inside windows of sigma rows, H = 32 / V rows per slice, slice
// width = longest row rounded up to a multiple of V; padding has value 0 and
// repeats the row's last column (or 0 for an empty row).
static void build_sell(int rows, const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<double>& vx,
                       int V, HostProb::Sell& S)
{
    const int H = 32 / V;
    const int sigma = 4096;
    S.rows = rows;
    S.V = V;
    S.nslices = (rows + H - 1) / H;
    std::vector<int> order(rows);
    std::iota(order.begin(), order.end(), 0);
    for (int w0 = 0; w0 < rows; w0 += sigma) {
        const int w1 = std::min(rows, w0 + sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1,
                         [&](int a, int b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
    }
    S.perm.assign((size_t)S.nslices * H, -1);
    for (int i = 0; i < rows; ++i) S.perm[i] = order[i];
    S.ptr.assign(S.nslices + 1, 0);
    for (int s = 0; s < S.nslices; ++s) {
        int w = 0;
        for (int r = 0; r < H; ++r) {
            const int pos = s * H + r;
            if (pos < rows) w = std::max(w, rp[order[pos] + 1] - rp[order[pos]]);
        }
        w = (w + V - 1) / V * V;
        S.ptr[s + 1] = S.ptr[s] + w * H;
    }
    const size_t tot = (size_t)S.ptr[S.nslices];
    S.col.assign(tot, 0);
    S.val.assign(tot, 0.0);
    for (int s = 0; s < S.nslices; ++s) {
        const int w = (S.ptr[s + 1] - S.ptr[s]) / H;
        for (int r = 0; r < H; ++r) {
            const int pos = s * H + r;
            if (pos >= rows) continue;
            const int row = order[pos];
            const int b = rp[row], len = rp[row + 1] - b;
            const int padc = len > 0 ? ci[b + len - 1] : 0;
            for (int j = 0; j < w; ++j) {
                const size_t idx = (size_t)S.ptr[s] + (size_t)j * H + r;
                if (j < len) {
                    S.col[idx] = ci[b + j];
                    S.val[idx] = vx[b + j];
                } else {
                    S.col[idx] = padc;
                }
            }
        }
    }
}

// Host-side check of the column-blocked layout (see superscs.h): build it,
// verify its invariants and replay the product exactly as the segment loop
// walks it, in FP64, against the CSR product.
extern "C" int scs_cb_layout_check(int32_t rows, int32_t cols, const int64_t* Ap, const int32_t* Ai,
                                   const double* Ax, int32_t ctas, int32_t compute_warps, int32_t elem_bytes,
                                   int32_t vectors, int64_t smem_bytes, const double* x, double* y, int64_t* stats)
{
    if (rows <= 0 || cols <= 0 || !Ap || !Ai || !Ax || !x || !y || !stats || ctas < 1 || compute_warps < 1 ||
        (elem_bytes != 4 && elem_bytes != 8) || (vectors != 1 && vectors != 2) || smem_bytes < 4096)
        return SCS_EINVAL;
    if (Ap[0] != 0 || Ap[rows] >= (1ll << 31)) return SCS_EINVAL;
    std::vector<int> rp(rows + 1), ci(Ap[rows]);
    std::vector<double> vx(Ax, Ax + Ap[rows]);
    for (int i = 0; i <= rows; ++i) rp[i] = (int)Ap[i];
    for (long long e = 0; e < Ap[rows]; ++e) {
        if (Ai[e] < 0 || Ai[e] >= cols) return SCS_EINVAL;
        ci[e] = Ai[e];
    }
    HostProb::Cb C;
    plan_cb(rows, cols, rp, ci, vx, ctas, compute_warps, elem_bytes, vectors, (size_t)smem_bytes, true, C);
    for (int k = 0; k < 8; ++k) stats[k] = 0;
    if (C.ncb == 0) return SCS_OK;  // the layout does not fit: the solver would use sliced ELL
    long long bad = 0;
    auto req = [&](bool c) { if (!c) ++bad; };
    const int E = 16 / elem_bytes, H = 32 / C.V, S = C.S, nw = compute_warps;
    req(C.cw % 4 == 0 && C.cw <= 65536 && (long long)C.ncb * C.cw >= cols && (long long)(C.ncb - 1) * C.cw < cols);
    req(C.dyn() <= (size_t)smem_bytes);
    req((size_t)C.stage_off >= (size_t)2 * vectors * C.acc_rows * elem_bytes && C.stage_off % 16 == 0);
    req(C.ms % 4 == 0 && C.stage_bytes % 16 == 0 && C.off_x % 16 == 0 && C.off_col % 16 == 0 && C.off_val % 16 == 0);
    req(C.off_x >= 4 * C.ms && C.off_col > C.off_x && C.off_val > C.off_col && C.stage_bytes > C.off_val);
    req((int)C.rbnd.size() == ctas + 1 && C.rbnd[0] == 0 && C.rbnd[ctas] == rows);
    for (int k = 0; k < C.ncb; ++k) {
        const int len = std::min(C.cw, cols - k * C.cw);
        for (int mis = 0; mis < E; ++mis) req(((mis + len + E - 1) / E) * 16 <= C.off_col - C.off_x);
    }
    std::fill(y, y + rows, 0.0);
    long long prev_end = 0;
    std::vector<double> acc;
    std::vector<char> seen;
    for (int b = 0; b < ctas; ++b) {
        const int r0 = C.rbnd[b], R = C.rbnd[b + 1] - r0;
        req(R >= 0 && R <= C.acc_rows);
        acc.assign(std::max(R, 1), 0.0);
        for (int k = 0; k < C.ncb; ++k) {
            const int len = std::min(C.cw, cols - k * C.cw);
            const int* mt = C.meta.data() + ((size_t)b * C.ncb + k) * C.ms;
            const int e0 = mt[0], e1 = mt[1], ns = mt[4];
            req(e0 == prev_end && e1 >= e0 && e0 % 32 == 0 && e1 % 32 == 0);
            req((long long)(e1 - e0) * 2 <= C.off_val - C.off_col &&
                (long long)(e1 - e0) * elem_bytes <= C.stage_bytes - C.off_val);
            const int* m2 = C.meta.data() + ((size_t)b * C.ncb + (k + S) % C.ncb) * C.ms;
            req(mt[2] == m2[0] && mt[3] == m2[1]);
            req(cb_meta_words(nw, ns, H) <= C.ms);
            prev_end = e1;
            const int* wl = mt + 5;
            const int* st = wl + nw + 1;
            const uint16_t* sr = (const uint16_t*)(st + ns + 1);
            req(wl[0] == 0 && wl[nw] == ns && st[0] == 0 && (long long)st[ns] * 32 == e1 - e0);
            seen.assign(std::max(R, 1), 0);
            for (int w = 0; w < nw; ++w) {
                req(wl[w] <= wl[w + 1]);
                for (int sl = wl[w]; sl < wl[w + 1]; ++sl) {
                    req(st[sl + 1] > st[sl]);
                    double a[32] = {};
                    for (int t = st[sl]; t < st[sl + 1]; ++t)
                        for (int lane = 0; lane < 32; ++lane) {
                            const size_t idx = (size_t)e0 + 32 * (size_t)t + lane;
                            const int c = C.col[idx];
                            req(c < len);
                            a[lane] += C.val[idx] * x[(size_t)k * C.cw + c];
                        }
                    for (int r = 0; r < H; ++r) {
                        double sum = 0;
                        for (int q = 0; q < C.V; ++q) sum += a[q * H + r];
                        const int rw = sr[sl * H + r];
                        if (rw == 0xFFFF) {
                            req(sum == 0.0);
                            continue;
                        }
                        req(rw < R && !seen[rw]);
                        if (rw < R) {
                            seen[rw] = 1;
                            acc[rw] += sum;
                        }
                    }
                }
            }
        }
        for (int lr = 0; lr < R; ++lr) y[r0 + lr] = acc[lr];
    }
    req(prev_end == (long long)C.col.size());
    stats[0] = bad;
    stats[1] = C.ncb;
    stats[2] = C.cw;
    stats[3] = C.V;
    stats[4] = (int64_t)C.col.size();
    stats[5] = (int64_t)C.dyn();
    stats[6] = C.S;
    stats[7] = C.ms;
    return SCS_OK;
}

// Host-side check of the tiled layout (see superscs.h): build it, verify its
// invariants and replay the product as the tile passes (row sums per tile)
// and the second pass (partials added in block order) compute it, in FP64.
extern "C" int scs_tile_layout_check(int32_t rows, int32_t cols, const int64_t* Ap, const int32_t* Ai,
                                     const double* Ax, int32_t ctas, int32_t compute_warps, int32_t elem_bytes,
                                     int32_t vectors, int64_t smem_bytes, const double* x, double* y, int64_t* stats)
{
    if (rows <= 0 || cols <= 0 || !Ap || !Ai || !Ax || !x || !y || !stats || ctas < 1 || compute_warps < 1 ||
        (elem_bytes != 4 && elem_bytes != 8) || (vectors != 1 && vectors != 2) || smem_bytes < 4096)
        return SCS_EINVAL;
    if (Ap[0] != 0 || Ap[rows] >= (1ll << 31)) return SCS_EINVAL;
    std::vector<int> rp(rows + 1), ci(Ap[rows]);
    std::vector<double> vx(Ax, Ax + Ap[rows]);
    for (int i = 0; i <= rows; ++i) rp[i] = (int)Ap[i];
    for (long long e = 0; e < Ap[rows]; ++e) {
        if (Ai[e] < 0 || Ai[e] >= cols) return SCS_EINVAL;
        ci[e] = Ai[e];
    }
    HostProb::Cb C;
    plan_tile(rows, cols, rp, ci, vx, ctas, compute_warps, elem_bytes, vectors, (size_t)smem_bytes, true, C);
    for (int k = 0; k < 8; ++k) stats[k] = 0;
    if (C.ncb == 0) return SCS_OK;  // no split fits: the solver would use another layout
    long long bad = 0;
    auto req = [&](bool c) { if (!c) ++bad; };
    const int E = 16 / elem_bytes, H = 32 / C.V, S = C.S, nw = compute_warps, Cn = C.ncb, R = C.R;
    req(C.tile == 1 && R * Cn <= ctas && R >= 1 && C.rows == rows && C.nv == vectors);
    req(C.part_elems() == (size_t)2 * vectors * Cn * rows);
    req(C.cw % 4 == 0 && C.cw <= 65536 && (long long)Cn * C.cw >= cols && (long long)(Cn - 1) * C.cw < cols);
    req(C.dyn() <= (size_t)smem_bytes);
    req(C.off_x % 16 == 0 && C.off_x >= C.acc_rows * elem_bytes && C.stage_off % 16 == 0);
    req((long long)C.stage_off - C.off_x >= (long long)((C.cw + 2 * E - 1) / E) * 16);
    req(C.ms % 4 == 0 && C.stage_bytes % 16 == 0 && C.off_col % 16 == 0 && C.off_val % 16 == 0);
    req(C.off_col >= 4 * C.ms && C.off_val >= C.off_col && C.stage_bytes >= C.off_val);
    req((int)C.rbnd.size() == R + 1 && C.rbnd[0] == 0 && C.rbnd[R] == rows);
    req((int)C.cbeg.size() == R * Cn + 1 && C.cbeg[0] == 0 && (size_t)C.cbeg[R * Cn] * C.ms == C.meta.size());
    // part[k][row], as the tile passes leave it (rows a tile does not reach stay 0)
    std::vector<double> part((size_t)Cn * rows, 0.0);
    long long prev_end = 0;
    std::vector<double> acc;
    std::vector<char> seen;
    for (int r = 0; r < R; ++r) {
        const int r0 = C.rbnd[r], Rr = C.rbnd[r + 1] - r0;
        req(Rr >= 0 && Rr <= C.acc_rows && Rr < 0xFFFF);
        for (int k = 0; k < Cn; ++k) {
            const int g = r * Cn + k;
            const int len = std::min(C.cw, cols - k * C.cw);
            acc.assign(std::max(Rr, 1), 0.0);
            seen.assign(std::max(Rr, 1), 0);
            req(C.cbeg[g + 1] >= C.cbeg[g]);
            for (int j = C.cbeg[g]; j < C.cbeg[g + 1]; ++j) {
                const int* mt = C.meta.data() + (size_t)j * C.ms;
                const int e0 = mt[0], e1 = mt[1], ns = mt[4];
                req(e0 == prev_end && e1 >= e0 && e0 % 32 == 0 && e1 % 32 == 0);
                req((long long)(e1 - e0) * 2 <= C.off_val - C.off_col &&
                    (long long)(e1 - e0) * elem_bytes <= C.stage_bytes - C.off_val);
                if (j + S < C.cbeg[g + 1]) {
                    const int* m2 = C.meta.data() + (size_t)(j + S) * C.ms;
                    req(mt[2] == m2[0] && mt[3] == m2[1]);
                }
                req(cb_meta_words(nw, ns, H) <= C.ms);
                prev_end = e1;
                const int* wl = mt + 5;
                const int* st = wl + nw + 1;
                const uint16_t* sr = (const uint16_t*)(st + ns + 1);
                req(wl[0] == 0 && wl[nw] == ns && st[0] == 0 && (long long)st[ns] * 32 == e1 - e0);
                for (int w = 0; w < nw; ++w) {
                    req(wl[w] <= wl[w + 1]);
                    for (int sl = wl[w]; sl < wl[w + 1]; ++sl) {
                        req(st[sl + 1] > st[sl]);
                        double a[32] = {};
                        for (int t = st[sl]; t < st[sl + 1]; ++t)
                            for (int lane = 0; lane < 32; ++lane) {
                                const size_t idx = (size_t)e0 + 32 * (size_t)t + lane;
                                const int c = C.col[idx];
                                req(c < len);
                                a[lane] += C.val[idx] * x[(size_t)k * C.cw + std::min(c, len - 1)];
                            }
                        for (int rr = 0; rr < H; ++rr) {
                            double sum = 0;
                            for (int q = 0; q < C.V; ++q) sum += a[q * H + rr];
                            const int rw = sr[sl * H + rr];
                            if (rw == 0xFFFF) {
                                req(sum == 0.0);
                                continue;
                            }
                            // every row of a tile lies in one slice: its sum is stored, not added
                            req(rw < Rr && !seen[rw]);
                            if (rw < Rr) {
                                seen[rw] = 1;
                                acc[rw] = sum;
                            }
                        }
                    }
                }
            }
            for (int lr = 0; lr < Rr; ++lr) part[(size_t)k * rows + r0 + lr] = acc[lr];
        }
    }
    req(prev_end == (long long)C.col.size());
    for (int i = 0; i < rows; ++i) {
        double s = 0;
        for (int k = 0; k < Cn; ++k) s += part[(size_t)k * rows + i];
        y[i] = s;
    }
    stats[0] = bad;
    stats[1] = Cn;
    stats[2] = R;
    stats[3] = C.V;
    stats[4] = (int64_t)C.col.size();
    stats[5] = (int64_t)C.dyn();
    stats[6] = C.cbeg[R * Cn];
    stats[7] = C.ms;
    return SCS_OK;
}

static int pick_lanes(long long nnz, int rows)
{
    const double avg = rows > 0 ? (double)nnz / rows : 0.0;
    int v = 1;
    while (v < 32 && 2.0 * v * 8.0 <= avg) v <<= 1;  // about 8 or more elements per lane
    return v;
}

static void finish_layouts(HostProb& H, bool sell_A, bool sell_T);

// Validate and copy the problem, build the CSR of A^T.  Unless keep_csr, also
// build the sliced layouts and drop the CSR copies (finish_layouts).
static int prepare(const scs_data* d, const scs_cone* k, HostProb& H, char* err, bool keep_csr = false)
{
    if (!d || !k) { set_err(err, "data and cone must not be NULL"); return SCS_EINVAL; }
    if (d->m <= 0 || d->n <= 0) { set_err(err, "m and n must be positive (m=%d n=%d)", d->m, d->n); return SCS_EINVAL; }
    if (!d->Ap || !d->Ai || !d->Ax || !d->b || !d->c) { set_err(err, "data arrays must not be NULL"); return SCS_EINVAL; }
    const int m = d->m, n = d->n;
    if (d->Ap[0] != 0) { set_err(err, "Ap[0] must be 0"); return SCS_EINVAL; }
    for (int i = 0; i < m; ++i)
        if (d->Ap[i + 1] < d->Ap[i]) { set_err(err, "Ap is not nondecreasing at row %d", i); return SCS_EINVAL; }
    const long long nnz = d->Ap[m];
    if (nnz >= (1ll << 31)) { set_err(err, "nnz = %lld is not below 2^31", nnz); return SCS_EINVAL; }
    if (k->f < 0 || k->l < 0 || k->nq < 0 || k->ns < 0 || k->ep < 0 || k->ed < 0) { set_err(err, "negative cone counts"); return SCS_EINVAL; }
    if ((k->nq > 0 && !k->q) || (k->ns > 0 && !k->s)) { set_err(err, "cone arrays must not be NULL"); return SCS_EINVAL; }
    long long rows = (long long)k->f + k->l;
    H.q_off.assign(1, 0);
    for (int i = 0; i < k->nq; ++i) {
        if (k->q[i] < 1) { set_err(err, "SOC %d has dimension %d < 1", i, k->q[i]); return SCS_EINVAL; }
        H.q.push_back(k->q[i]);
    }
    for (int i = 0; i < k->ns; ++i) {
        if (k->s[i] < 1 || k->s[i] > PSD_BIG_MAX) {
            set_err(err, "PSD block %d has order %d outside 1..%d", i, k->s[i], PSD_BIG_MAX);
            return SCS_EINVAL;
        }
        H.s.push_back(k->s[i]);
    }
    long long o = (long long)k->f + k->l;
    for (int i = 0; i < k->nq; ++i) { o += k->q[i]; }
    for (int i = 0; i < k->ns; ++i) { o += (long long)k->s[i] * (k->s[i] + 1) / 2; }
    const long long e_off = o;
    o += 3LL * k->ep + 3LL * k->ed;
    rows = o;
    if (rows != m) { set_err(err, "cone rows (%lld) do not sum to m (%d)", rows, m); return SCS_EINVAL; }
    H.n = n;
    H.m = m;
    H.nnz = nnz;
    H.f = k->f;
    H.l = k->l;
    H.ep = k->ep;
    H.ed = k->ed;
    H.e_off = (int)e_off;
    long long qo = (long long)k->f + k->l;
    for (int i = 0; i < k->nq; ++i) { H.q_off.push_back(0); }
    H.q_off[0] = (int)qo;
    for (int i = 0; i < k->nq; ++i) H.q_off[i + 1] = H.q_off[i] + k->q[i];
    long long so = qo;
    for (int i = 0; i < k->nq; ++i) so += k->q[i];
    for (int i = 0; i < k->ns; ++i) {
        H.s_off.push_back((int)so);
        so += (long long)k->s[i] * (k->s[i] + 1) / 2;
    }
    H.Ap.resize(m + 1);
    for (int i = 0; i <= m; ++i) H.Ap[i] = (int)d->Ap[i];
    H.Ai.assign(d->Ai, d->Ai + nnz);
    H.Ax.assign(d->Ax, d->Ax + nnz);
    for (long long e = 0; e < nnz; ++e) {
        if (H.Ai[e] < 0 || H.Ai[e] >= n) { set_err(err, "column index %d out of range at %lld", H.Ai[e], e); return SCS_EINVAL; }
        if (!std::isfinite(H.Ax[e])) { set_err(err, "non-finite A value at %lld", e); return SCS_EINVAL; }
    }
    H.b.assign(d->b, d->b + m);
    H.c.assign(d->c, d->c + n);
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(H.b[i])) { set_err(err, "non-finite b[%d]", i); return SCS_EINVAL; }
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(H.c[j])) { set_err(err, "non-finite c[%d]", j); return SCS_EINVAL; }
    // CSR of A^T: counting sort by column, rows ascending inside each column
    H.Tp.assign(n + 1, 0);
    for (long long e = 0; e < nnz; ++e) H.Tp[H.Ai[e] + 1]++;
    for (int j = 0; j < n; ++j) H.Tp[j + 1] += H.Tp[j];
    H.Ti.resize(nnz);
    H.Tx.resize(nnz);
    std::vector<int> pos(H.Tp.begin(), H.Tp.end() - 1);
    for (int i = 0; i < m; ++i)
        for (int e = H.Ap[i]; e < H.Ap[i + 1]; ++e) {
            const int j = H.Ai[e];
            H.Ti[pos[j]] = i;
            H.Tx[pos[j]] = H.Ax[e];
            pos[j]++;
        }
    double s = 0;
    for (int i = 0; i < m; ++i) s += H.b[i] * H.b[i];
    H.nb = std::sqrt(s);
    s = 0;
    for (int j = 0; j < n; ++j) s += H.c[j] * H.c[j];
    H.nc = std::sqrt(s);
    H.vecA = pick_lanes(nnz, m);
    H.vecT = pick_lanes(nnz, n);
    if (keep_csr) return SCS_OK;
    finish_layouts(H, true, true);
    if ((long long)H.SA.ptr.back() >= (1ll << 31) || (long long)H.ST.ptr.back() >= (1ll << 31)) {
        set_err(err, "padded matrix too large");
        return SCS_EINVAL;
    }
    return SCS_OK;
}

// Build the sliced ELL copies that are needed (an empty one, with no slices,
// stands for a matrix that only runs column-blocked) and drop the CSR copies.
static void finish_layouts(HostProb& H, bool sell_A, bool sell_T)
{
    auto empty = [](int rows, HostProb::Sell& S) {
        S = HostProb::Sell();
        S.rows = rows;
        S.ptr.assign(1, 0);
    };
    if (sell_A) build_sell(H.m, H.Ap, H.Ai, H.Ax, H.vecA, H.SA); else empty(H.m, H.SA);
    if (sell_T) build_sell(H.n, H.Tp, H.Ti, H.Tx, H.vecT, H.ST); else empty(H.n, H.ST);
    std::vector<int>().swap(H.Ap);
    std::vector<int>().swap(H.Ai);
    std::vector<int>().swap(H.Tp);
    std::vector<int>().swap(H.Ti);
    std::vector<double>().swap(H.Ax);
    std::vector<double>().swap(H.Tx);
}

constexpr int DIRECT_MAX_N = 4096;  // largest n factored densely by the direct linear solves

static int check_settings(const scs_settings* S, char* err)
{
    if (!S) { set_err(err, "settings must not be NULL"); return SCS_EINVAL; }
    if (S->direction < 0 || S->direction > 3) { set_err(err, "bad direction %d", S->direction); return SCS_EINVAL; }
    if ((S->direction == SCS_DIR_AA || S->direction == SCS_DIR_AA_QR) && (S->mem < 0 || S->mem > AAMAX)) { set_err(err, "AA mem must be in 0..%d", AAMAX); return SCS_EINVAL; }
    if (S->direction == SCS_DIR_RB && (S->mem < 0 || S->mem > MAXMEM)) { set_err(err, "RB mem must be in 0..%d", MAXMEM); return SCS_EINVAL; }
    if (!(S->eps > 0) || S->max_iters < 0 || S->ls_max < 0 || S->cg_max < 0) { set_err(err, "bad tolerances or caps"); return SCS_EINVAL; }
    if (!(S->lambda > 0 && S->lambda < 2)) { set_err(err, "lambda must lie in (0,2)"); return SCS_EINVAL; }
    if (!(S->sigma > 0 && S->sigma < 1)) { set_err(err, "sigma must lie in (0,1)"); return SCS_EINVAL; }
    if (S->precision != SCS_FP64 && S->precision != SCS_MIXED) { set_err(err, "bad precision"); return SCS_EINVAL; }
    if (S->threads != 0 && (S->threads < 32 || S->threads > 1024 || S->threads % 32)) { set_err(err, "threads must be a multiple of 32 in 32..1024"); return SCS_EINVAL; }
    if (!(S->psd_recheck_tol >= 0)) { set_err(err, "psd_recheck_tol must be >= 0"); return SCS_EINVAL; }
    if (S->spmv_path < 0 || S->spmv_path > 4) { set_err(err, "spmv_path must be in 0..4"); return SCS_EINVAL; }
    return SCS_OK;
}

// ---------------------------------------------------------------------------
// device arena
// ---------------------------------------------------------------------------
struct Arena {
    size_t off = 0;
    char* base = nullptr;
    template <typename X>
    X* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        X* p = (X*)(base + off);
        off += sizeof(X) * std::max<size_t>(count, 1);
        return p;
    }
};

// layout of one instance's data and work in precision T; base == nullptr only measures
template <typename T>
static void lay_out(Arena& A, const HostProb& H, int mem, bool qr, bool direct, int max_blocks, DevProb<T>& P,
                    DevWork<T>& W,
                    const int* shared_idx /* index arrays shared with another precision or null */,
                    DevState* st_ext = nullptr)
{
    const int n = H.n, m = H.m, nm = n + m;
    const long long nnz = H.nnz;
    P.n = n;
    P.m = m;
    auto lay_sell = [&](const HostProb::Sell& hs, Sell<T>& ds) {
        ds.rows = hs.rows;
        ds.V = hs.V;
        ds.nslices = hs.nslices;
        ds.l1 = hs.val.size() * (sizeof(int) + sizeof(T)) <= 48 * 1024 ? 1 : 0;
        if (shared_idx == nullptr) {
            ds.ptr = A.take<int>(hs.ptr.size());
            ds.col = A.take<int>(hs.col.size());
            ds.perm = A.take<int>(hs.perm.size());
            ds.wbnd = hs.wbnd.empty() ? nullptr : A.take<int>(hs.wbnd.size());
        }
        ds.val = A.take<T>(hs.val.size());
    };
    lay_sell(H.SA, P.A);
    lay_sell(H.ST, P.AT);
    auto lay_cb = [&](const HostProb::Cb& hc, Cblk<T>& dc) {
        dc = Cblk<T>{};
        if (hc.ncb == 0) return;
        dc.ncb = hc.ncb;
        dc.cw = hc.cw;
        dc.cols = hc.cols;
        dc.nw = hc.nw;
        dc.V = hc.V;
        dc.acc_rows = hc.acc_rows;
        dc.ms = hc.ms;
        dc.S = hc.S;
        dc.stage_off = hc.stage_off;
        dc.stage_bytes = hc.stage_bytes;
        dc.off_x = hc.off_x;
        dc.off_col = hc.off_col;
        dc.off_val = hc.off_val;
        dc.rbnd = A.take<int>(hc.rbnd.size());
        dc.meta = A.take<int>(hc.meta.size());
        dc.col = A.take<unsigned short>(hc.col.size());
        dc.val = A.take<T>(hc.val.size());
        dc.tile = hc.tile;
        dc.R = hc.R;
        dc.rows = hc.rows;
        dc.nv = hc.nv;
        dc.cbeg = hc.tile ? A.take<int>(hc.cbeg.size()) : nullptr;
        dc.part = hc.tile ? A.take<T>(hc.part_elems()) : nullptr;
    };
    lay_cb(sizeof(T) == 8 ? H.cA64 : H.cA32, P.A.cb);
    lay_cb(sizeof(T) == 8 ? H.cAT64 : H.cAT32, P.AT.cb);
    if (shared_idx == nullptr) {
        P.q_off = A.take<int>(H.q_off.size());
        P.s_dim = A.take<int>(H.s.size());
        P.s_off = A.take<int>(H.s_off.size());
    }
    P.b = A.take<T>(m);
    P.c = A.take<T>(n);
    P.nb = H.nb;
    P.nc = H.nc;
    P.f = H.f;
    P.l = H.l;
    P.nq = (int)H.q.size();
    P.ns = (int)H.s.size();
    P.ep = H.ep;
    P.ed = H.ed;
    P.e_off = H.e_off;
    // global Jacobi workspaces of the PSD blocks above PSD_MAX (their offsets are uploaded with the problem)
    size_t big = 0;
    for (int d : H.s)
        if (d > PSD_MAX) big += psd_big_bytes<T>(d);
    P.big_off = H.s.empty() ? nullptr : A.take<long long>(H.s.size());
    P.psd_big = big ? A.take<unsigned char>(big) : nullptr;
    // warm-start eigenvectors of every PSD block (offsets uploaded with the problem, flags zeroed with the arena)
    size_t vbytes = 0;
    for (int d : H.s) vbytes += psd_v_bytes<T>(d);
    P.v_off = H.s.empty() ? nullptr : A.take<long long>(H.s.size());
    W.psd_v = vbytes ? A.take<unsigned char>(vbytes) : nullptr;
    W.psd_vok = H.s.empty() ? nullptr : A.take<int>(H.s.size());
    double* taus = A.take<double>(16);
    HV<T>* hvs[] = {&W.u, &W.ut, &W.ub, &W.Ru, &W.d, &W.dt, &W.wb, &W.Rw, &W.zp, &W.xip, &W.zt};
    for (int i = 0; i < 11; ++i) {
        hvs[i]->v = A.take<T>(nm);
        hvs[i]->t = taus + i;
    }
    W.g = A.take<T>(nm);
    W.ws[0] = A.take<T>(n);
    W.ws[1] = A.take<T>(n);
    W.cr = A.take<T>(n);
    W.cp = A.take<T>(n);
    W.cq = A.take<T>(n);
    W.tn = A.take<T>(n);
    W.tm = A.take<T>(m);
    W.py = A.take<T>(m);
    const int mm = std::max(mem, 1);
    W.Zv = A.take<T>((size_t)mm * nm);
    W.Xv = A.take<T>((size_t)mm * nm);
    W.Zt = A.take<double>(mm);
    W.Xt = A.take<double>(mm);
    W.Qv = qr ? A.take<T>((size_t)mm * nm) : nullptr;
    W.Qt = qr ? A.take<double>(mm) : nullptr;
    W.io_in = A.take<double>(nm + 1);
    W.io_out = A.take<double>(nm + 1);
    W.io_out2 = A.take<double>(nm + 1);
    W.warm = A.take<double>(nm + 1);
    W.x_out = A.take<double>(n);
    W.y_out = A.take<double>(m);
    W.s_out = A.take<double>(m);
    W.u_out = A.take<double>(nm + 1);
    W.partials = A.take<double>((size_t)2 * KMAX * std::max(max_blocks, 1) + 2 * KMAX);
    W.bar = A.take<unsigned>(4);
    W.abort_flag = A.take<int>(4);
    W.st = st_ext ? st_ext : A.take<DevState>(1);
    W.res = A.take<Resume>(1);
    W.ir = IrBufs{};
    W.chol = direct ? A.take<T>((size_t)n * n) : nullptr;
    W.chol_fail = A.take<int>(4);
}

// The FP64 phase of SCS_MIXED reads the FP32 phase's loop state (one shared
// record) and refines its linear solves with the FP32 copy of A and the FP32
// phase's CG vectors, which are idle by then.
static void link_phases(const DevProb<float>& P32, DevWork<float>& W32, DevWork<double>& W64)
{
    W32.res = W64.res;
    W64.ir = IrBufs{P32.A, P32.AT, W32.cr, W32.cp, W32.cq, W32.tn, W32.tm};
}

// Widens the FP32 phase's direction memory (mem columns of Z and Xi), the
// pending secant pair and their FP64 tau entries into the FP64 work.
static cudaError_t widen_memory(const DevWork<float>& W32, const DevWork<double>& W64, int mem, int nm, cudaStream_t st)
{
    const long long cols = (long long)std::max(mem, 1) * nm;
    cudaError_t e;
    if ((e = launch_f2d(W32.Zv, W64.Zv, cols, st)) != cudaSuccess) return e;
    if ((e = launch_f2d(W32.Xv, W64.Xv, cols, st)) != cudaSuccess) return e;
    if (W32.Qv && W64.Qv) {
        if ((e = launch_f2d(W32.Qv, W64.Qv, cols, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(W64.Qt, W32.Qt, sizeof(double) * std::max(mem, 1), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
    }
    if ((e = launch_f2d(W32.zp.v, W64.zp.v, nm, st)) != cudaSuccess) return e;
    if ((e = launch_f2d(W32.xip.v, W64.xip.v, nm, st)) != cudaSuccess) return e;
    const size_t tb = sizeof(double) * std::max(mem, 1);
    if ((e = cudaMemcpyAsync(W64.Zt, W32.Zt, tb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(W64.Xt, W32.Xt, tb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(W64.zp.t, W32.zp.t, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    return cudaMemcpyAsync(W64.xip.t, W32.xip.t, sizeof(double), cudaMemcpyDeviceToDevice, st);
}

template <typename T>
static int upload(const HostProb& H, const DevProb<T>& P, bool idx, cudaStream_t st, char* err, bool matrix = true)
{
    auto put_i = [&](const std::vector<int>& v, const int* dst) -> int {
        if (!v.empty()) CU(cudaMemcpyAsync((void*)dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, st), err);
        return SCS_OK;
    };
    std::vector<T> tmp;
    auto put_t = [&](const std::vector<double>& v, const T* dst) -> int {
        if (v.empty()) return SCS_OK;
        if (sizeof(T) == sizeof(double)) {
            CU(cudaMemcpyAsync((void*)dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, st), err);
        } else {
            tmp.resize(v.size());
            for (size_t i = 0; i < v.size(); ++i) tmp[i] = (T)v[i];
            CU(cudaMemcpyAsync((void*)dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice, st), err);
            CU(cudaStreamSynchronize(st), err);  // tmp is reused
        }
        return SCS_OK;
    };
    auto put_u16 = [&](const std::vector<uint16_t>& v, const unsigned short* dst) -> int {
        if (!v.empty()) CU(cudaMemcpyAsync((void*)dst, v.data(), 2 * v.size(), cudaMemcpyHostToDevice, st), err);
        return SCS_OK;
    };
    // byte offsets of the PSD blocks' global Jacobi workspaces (-1: decomposed in shared memory)
    // and of their warm-start eigenvectors
    auto put_big = [&]() -> int {
        if (H.s.empty()) return SCS_OK;
        std::vector<long long> off(H.s.size(), -1), voff(H.s.size(), 0);
        long long o = 0, ov = 0;
        for (size_t k = 0; k < H.s.size(); ++k) {
            if (H.s[k] > PSD_MAX) {
                off[k] = o;
                o += (long long)psd_big_bytes<T>(H.s[k]);
            }
            voff[k] = ov;
            ov += (long long)psd_v_bytes<T>(H.s[k]);
        }
        CU(cudaMemcpyAsync((void*)P.big_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st),
           err);
        CU(cudaMemcpyAsync((void*)P.v_off, voff.data(), sizeof(long long) * voff.size(), cudaMemcpyHostToDevice, st),
           err);
        CU(cudaStreamSynchronize(st), err);  // off and voff are locals
        return SCS_OK;
    };
    auto put_cb = [&](const HostProb::Cb& hc, const Cblk<T>& dc) -> int {
        if (hc.ncb == 0) return SCS_OK;
        int r;
        if ((r = put_i(hc.rbnd, dc.rbnd)) || (r = put_i(hc.meta, dc.meta)) || (r = put_u16(hc.col, dc.col)) ||
            (r = put_t(hc.val, dc.val)) || (hc.tile && (r = put_i(hc.cbeg, dc.cbeg))))
            return r;
        return SCS_OK;
    };
    int rc;
    if ((rc = put_big())) return rc;
    if (!matrix) {
        if ((rc = put_t(H.b, P.b)) || (rc = put_t(H.c, P.c))) return rc;
        CU(cudaStreamSynchronize(st), err);
        return SCS_OK;
    }
    if ((rc = put_cb(sizeof(T) == 8 ? H.cA64 : H.cA32, P.A.cb)) ||
        (rc = put_cb(sizeof(T) == 8 ? H.cAT64 : H.cAT32, P.AT.cb)))
        return rc;
    if (idx) {
        if ((rc = put_i(H.SA.ptr, P.A.ptr)) || (rc = put_i(H.SA.col, P.A.col)) || (rc = put_i(H.SA.perm, P.A.perm)) ||
            (rc = put_i(H.ST.ptr, P.AT.ptr)) || (rc = put_i(H.ST.col, P.AT.col)) || (rc = put_i(H.ST.perm, P.AT.perm)) ||
            (rc = put_i(H.SA.wbnd, P.A.wbnd)) || (rc = put_i(H.ST.wbnd, P.AT.wbnd)) ||
            (rc = put_i(H.q_off, P.q_off)) || (rc = put_i(H.s, P.s_dim)) || (rc = put_i(H.s_off, P.s_off)))
            return rc;
    }
    if ((rc = put_t(H.SA.val, P.A.val)) || (rc = put_t(H.ST.val, P.AT.val)) || (rc = put_t(H.b, P.b)) ||
        (rc = put_t(H.c, P.c)))
        return rc;
    CU(cudaStreamSynchronize(st), err);
    return SCS_OK;
}

static DevSettings dev_settings(const scs_settings* S)
{
    DevSettings D;
    D.direction = S->direction;
    D.mem = S->mem;
    D.eps = S->eps;
    D.c0 = S->c0;
    D.c1 = S->c1;
    D.q = S->q;
    D.sigma = S->sigma;
    D.lambda = S->lambda;
    D.thetabar = S->thetabar;
    D.max_iters = S->max_iters;
    D.ls_max = S->ls_max;
    D.cg_max = S->cg_max;
    D.check_every = S->check_every;
    D.cg_rtol = S->cg_rtol;
    D.aa_reg = S->aa_reg;
    D.time_limit_ns = S->time_limit_s > 0 ? S->time_limit_s * 1e9 : 0.0;
    D.stall_iters = 0;
    D.use_warm = 0;
    D.switch_kkt = 0.0;
    D.cg_adapt = S->cg_adapt;
    D.keep_ws = 0;
    D.warm_fallback = S->warm_fallback;
    D.save_state = 0;
    D.resume = 0;
    D.refine = 0;
    D.stall_after_tau = S->mixed_stall_after_tau;
    D.psd_tol = S->psd_recheck_tol;
    return D;
}

struct DevInfo {
    int team = SCS_TEAM_GRID;
    int threads = 512;
    int grid = 0;
    int sms = 0;
    size_t dyn64 = 0, dyn32 = 0;
    bool maxl1 = false;  // grid of one CTA per SM without dynamic shared memory: prefer L1
};

template <typename T>
static size_t dyn_smem(const HostProb& H, int threads, bool tma)
{
    const size_t psd = H.s.empty() ? 0 : psd_smem_bytes<T>();
    const size_t stage = tma ? (size_t)(threads / 32) * 2 * tma_stage_bytes<T>() : 0;
    return std::max(psd, stage);
}

template <typename T>
static int config_kernels(size_t dyn, char* err)
{
    if (dyn > 48 * 1024) {
        CU(cudaFuncSetAttribute(kgrid_ptr<T>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn), err);
        CU(cudaFuncSetAttribute(kblock_ptr<T>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn), err);
    }
    return SCS_OK;
}

template <typename T>
static int launch(const DevInfo& D, size_t dyn, const Args<T>& a, Args<T>* dev_args, int* queue, cudaStream_t st,
                  char* err)
{
    const int team = D.team, threads = D.threads, grid = D.grid;
    if (team == SCS_TEAM_GRID) {
        // Sliced-ELL products are bound by their random gathers: with one CTA
        // per SM and no dynamic shared memory, give the rest of the SM's 256 KB
        // to L1 so more of the gathered vector stays on chip.  (A per-kernel
        // attribute of this process, so it is set before every launch.)
        CU(cudaFuncSetAttribute(kgrid_ptr<T>(), cudaFuncAttributePreferredSharedMemoryCarveout,
                                D.maxl1 && dyn == 0 ? (int)cudaSharedmemCarveoutMaxL1
                                                    : (int)cudaSharedmemCarveoutDefault),
           err);
        CU(cudaMemsetAsync(a.W.bar, 0, 4 * sizeof(unsigned), st), err);
        CU(cudaMemsetAsync(a.W.abort_flag, 0, 4 * sizeof(int), st), err);
        void* kargs[] = {(void*)&a};
        CU(cudaLaunchCooperativeKernel(kgrid_ptr<T>(), dim3(grid), dim3(threads), kargs, dyn, st), err);
    } else {
        CU(cudaMemcpyAsync(dev_args, &a, sizeof(Args<T>), cudaMemcpyHostToDevice, st), err);
        CU(cudaMemsetAsync(queue, 0, sizeof(int), st), err);
        CU(launch_block<T>(1, threads, dyn, st, dev_args, 1, queue, a.S, a.mode), err);
    }
    return SCS_OK;
}

// ---------------------------------------------------------------------------
// scs_work
// ---------------------------------------------------------------------------
struct scs_work {
    HostProb H;
    scs_settings S;
    cudaStream_t stream = nullptr;
    DevInfo D;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    DevProb<double> P64;
    DevWork<double> W64;
    DevProb<float> P32;
    DevWork<float> W32;
    bool has32 = false;
    Args<double>* dargs64 = nullptr;
    Args<float>* dargs32 = nullptr;
    int* queue = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    char err[512];
    double setup_s = 0;
};

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" int scs_default_settings(scs_settings* o)
{
    if (!o) return SCS_EINVAL;
    memset(o, 0, sizeof(*o));
    o->direction = SCS_DIR_AA;
    o->mem = 10;
    o->eps = 1e-5;
    o->c0 = 0.99;
    o->c1 = 0.99;
    o->q = 0.99;
    o->sigma = 1e-2;
    o->lambda = 1.0;
    o->thetabar = 0.1;
    o->max_iters = 10000;
    o->ls_max = 20;
    o->cg_max = 1000;
    o->check_every = 1;
    o->cg_rtol = 1e-10;
    o->time_limit_s = 0;
    o->precision = SCS_FP64;
    o->aa_reg = 1e-10;
    o->team = SCS_TEAM_AUTO;
    o->threads = 0;
    o->mixed_cg_rtol = 1e-6;
    o->mixed_stall = 50;
    o->mixed_max_iters = 10000;
    o->mixed_switch = 0.0;
    o->cg_adapt = 0.0;
    o->spmv_path = 0;
    o->warm_fallback = 0;
    o->mixed_resume = 1;
    o->mixed_refine = 1;
    o->linsys_direct = 0;
    o->mixed_stall_after_tau = 1;
    o->psd_recheck_tol = 1e-4;
    return SCS_OK;
}

template <typename T>
static Args<T> make_args(const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S, int mode, int slot = 0)
{
    Args<T> a;
    a.P = P;
    a.W = W;
    a.S = S;
    a.mode = mode;
    a.slot = slot;
    return a;
}

template <typename T>
static int run_setup_g(scs_work* w, const DevProb<T>& P, const DevWork<T>& W, Args<T>* dargs, size_t dyn)
{
    DevSettings S = dev_settings(&w->S);
    S.cg_max = std::max(10 * w->S.cg_max, 10000);
    S.cg_rtol = std::min(w->S.cg_rtol, sizeof(T) == 8 ? 1e-12 : 1e-7);
    Args<T> a = make_args(P, W, S, MODE_SETUP);
    return launch<T>(w->D, dyn, a, dargs, w->queue, w->stream, w->err);
}

extern "C" int scs_setup(const scs_data* data, const scs_cone* cone, const scs_settings* settings, void* cuda_stream,
                         scs_work** out)
{
    if (!out) { set_err(g_err, "out must not be NULL"); return SCS_EINVAL; }
    *out = nullptr;
    const double t0 = now_s();
    scs_work* w = new (std::nothrow) scs_work();
    if (!w) { set_err(g_err, "host allocation failed"); return SCS_ENOMEM; }
    w->err[0] = 0;
    int rc = check_settings(settings, w->err);
    if (!rc) rc = prepare(data, cone, w->H, w->err, true);
    if (rc) { memcpy(g_err, w->err, 512); delete w; return rc; }
    w->S = *settings;
    w->stream = (cudaStream_t)cuda_stream;
    const HostProb& H = w->H;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) { set_err(g_err, "no CUDA device: %s", cudaGetErrorString(ce)); delete w; return SCS_ECUDA; }
    cudaDeviceGetAttribute(&w->D.sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const long long work_size = H.nnz + (long long)H.n + H.m;
    int team = settings->team;
    if (team == SCS_TEAM_AUTO) team = (work_size < 150000 || !coop) ? SCS_TEAM_BLOCK : SCS_TEAM_GRID;
    if (team == SCS_TEAM_GRID && !coop) { set_err(w->err, "device lacks cooperative launch"); memcpy(g_err, w->err, 512); delete w; return SCS_ECUDA; }
    w->D.team = team;
    w->D.threads = settings->threads ? settings->threads : (team == SCS_TEAM_GRID ? GRID_THREADS : 256);
    if (team == SCS_TEAM_GRID && w->D.threads > GRID_THREADS) {
        set_err(w->err, "the grid team runs at most %d threads per block (got %d)", GRID_THREADS, w->D.threads);
        memcpy(g_err, w->err, 512);
        delete w;
        return SCS_EINVAL;
    }
    w->has32 = settings->precision == SCS_MIXED;
    // the TMA-staged stream only on request: on the gather-bound products it
    // measured no faster than direct streaming loads
    const bool tma = team == SCS_TEAM_GRID && settings->spmv_path == 2;
    // column-blocked products for the grid team (one CTA per SM): built here,
    // where the grid and the block size are known
    bool cb = false;
    if (team == SCS_TEAM_GRID && (settings->spmv_path == 0 || settings->spmv_path >= 3)) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa64{}, fa32{};
        cudaFuncGetAttributes(&fa64, kgrid_ptr<double>());
        cudaFuncGetAttributes(&fa32, kgrid_ptr<float>());
        const size_t stat = std::max(fa64.sharedSizeBytes, fa32.sharedSizeBytes);
        if ((size_t)optin > stat + 2048) {
            const size_t dyn_max = ((size_t)optin - stat - 1024) & ~size_t(15);
            const int G = w->D.sms, nw = w->D.threads / 32 - 1;  // compute warps; the last warp copies
            const bool force = settings->spmv_path >= 3;
            const bool tiles = settings->spmv_path == 4;
            HostProb& Hm = w->H;
            // tiles on request where a split fits, else the column-blocked layout (each on its own host thread)
            auto plan = [&](bool transposed, int esize, int nv, HostProb::Cb& L) {
                const int rows = transposed ? Hm.n : Hm.m, cols = transposed ? Hm.m : Hm.n;
                const auto& rp = transposed ? Hm.Tp : Hm.Ap;
                const auto& ci = transposed ? Hm.Ti : Hm.Ai;
                const auto& vx = transposed ? Hm.Tx : Hm.Ax;
                if (tiles) plan_tile(rows, cols, rp, ci, vx, G, nw, esize, nv, dyn_max, true, L);
                if (L.ncb == 0) plan_cb(rows, cols, rp, ci, vx, G, nw, esize, nv, dyn_max, force, L);
            };
            std::vector<std::thread> th;
            th.emplace_back([&] { plan(false, 8, 1, Hm.cA64); });
            th.emplace_back([&] { plan(true, 8, 2, Hm.cAT64); });
            if (w->has32) {
                th.emplace_back([&] { plan(false, 4, 1, Hm.cA32); });
                th.emplace_back([&] { plan(true, 4, 2, Hm.cAT32); });
            }
            for (auto& t : th) t.join();
            cb = H.cA64.ncb || H.cAT64.ncb || H.cA32.ncb || H.cAT32.ncb;
        }
    }
    finish_layouts(w->H, !(H.cA64.ncb && (!w->has32 || H.cA32.ncb)), !(H.cAT64.ncb && (!w->has32 || H.cAT32.ncb)));
    if ((long long)H.SA.ptr.back() >= (1ll << 31) || (long long)H.ST.ptr.back() >= (1ll << 31)) {
        set_err(w->err, "padded matrix too large");
        memcpy(g_err, w->err, 512);
        delete w;
        return SCS_EINVAL;
    }
    w->D.dyn64 = std::max({dyn_smem<double>(H, w->D.threads, tma), H.cA64.dyn(), H.cAT64.dyn()});
    w->D.dyn32 = w->has32 ? std::max({dyn_smem<float>(H, w->D.threads, tma), H.cA32.dyn(), H.cAT32.dyn()}) : 0;
    // the FP64 phase of SCS_MIXED also runs FP32 products (refinement corrections)
    if (w->has32) w->D.dyn64 = std::max(w->D.dyn64, w->D.dyn32);
    int rc2 = config_kernels<double>(w->D.dyn64, w->err);
    if (!rc2 && w->has32) rc2 = config_kernels<float>(w->D.dyn32, w->err);
    if (rc2) { memcpy(g_err, w->err, 512); delete w; return rc2; }
    if (team == SCS_TEAM_GRID) {
        int nb64 = 0, nb32 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb64, kgrid_ptr<double>(), w->D.threads, w->D.dyn64);
        int nb = nb64;
        if (w->has32) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb32, kgrid_ptr<float>(), w->D.threads, w->D.dyn32);
            nb = std::min(nb64, nb32);
        }
        if (nb < 1) { set_err(w->err, "solver kernel cannot be resident with %d threads", w->D.threads); memcpy(g_err, w->err, 512); delete w; return SCS_ECUDA; }
        // the column-blocked layout was cut for exactly one CTA per SM
        w->D.grid = w->D.sms * (cb ? 1 : std::min(nb, 4));
        w->D.maxl1 = !cb && std::min(nb, 4) == 1;
        if (tma) {
            warp_bounds(w->H.SA, w->D.grid * (w->D.threads / 32));
            warp_bounds(w->H.ST, w->D.grid * (w->D.threads / 32));
        }
    } else {
        w->D.grid = 1;
    }
    // measure and allocate one arena
    Arena A;
    DevProb<double> P64{};
    DevWork<double> W64{};
    DevProb<float> P32{};
    DevWork<float> W32{};
    const int mem = std::max(settings->mem, 1);
    const bool qr = settings->direction == SCS_DIR_AA_QR;
    // direct solves: one CTA per instance only (the factor is formed and used by one CTA)
    const bool direct = settings->linsys_direct && team == SCS_TEAM_BLOCK && H.n <= DIRECT_MAX_N;
    lay_out<double>(A, H, mem, qr, direct, w->D.grid, P64, W64, nullptr);
    if (w->has32) lay_out<float>(A, H, mem, qr, direct, w->D.grid, P32, W32, (const int*)1);
    size_t bytes = A.off + sizeof(Args<double>) + sizeof(Args<float>) + 1024;
    ce = cudaMalloc((void**)&w->arena, bytes);
    if (ce != cudaSuccess) { set_err(w->err, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(ce)); memcpy(g_err, w->err, 512); delete w; return SCS_ENOMEM; }
    w->arena_bytes = bytes;
    A.off = 0;
    A.base = w->arena;
    lay_out<double>(A, H, mem, qr, direct, w->D.grid, w->P64, w->W64, nullptr);
    if (w->has32) {
        lay_out<float>(A, H, mem, qr, direct, w->D.grid, w->P32, w->W32, (const int*)1);
        w->P32.A.ptr = w->P64.A.ptr;
        w->P32.A.col = w->P64.A.col;
        w->P32.A.perm = w->P64.A.perm;
        w->P32.AT.ptr = w->P64.AT.ptr;
        w->P32.AT.col = w->P64.AT.col;
        w->P32.AT.perm = w->P64.AT.perm;
        w->P32.A.wbnd = w->P64.A.wbnd;
        w->P32.AT.wbnd = w->P64.AT.wbnd;
        w->P32.q_off = w->P64.q_off;
        w->P32.s_dim = w->P64.s_dim;
        w->P32.s_off = w->P64.s_off;
        link_phases(w->P32, w->W32, w->W64);
    }
    w->dargs64 = A.take<Args<double>>(1);
    w->dargs32 = A.take<Args<float>>(1);
    w->queue = A.take<int>(4);
    if (A.off > bytes) { set_err(w->err, "arena overflow"); memcpy(g_err, w->err, 512); scs_finish(w); return SCS_ECUDA; }
    auto fail = [&](int r) { memcpy(g_err, w->err, 512); scs_finish(w); return r; };
    if (cudaMemsetAsync(w->arena, 0, bytes, w->stream) != cudaSuccess) { set_err(w->err, "memset failed"); return fail(SCS_ECUDA); }
    if ((rc = upload<double>(H, w->P64, true, w->stream, w->err))) return fail(rc);
    if (w->has32 && (rc = upload<float>(H, w->P32, false, w->stream, w->err))) return fail(rc);
    if (direct) {
        // factor I + A^T A in each precision before g is solved with it
        DevSettings SF = dev_settings(settings);
        if ((rc = launch<double>(w->D, w->D.dyn64, make_args(w->P64, w->W64, SF, MODE_FACTOR), w->dargs64, w->queue,
                                 w->stream, w->err)))
            return fail(rc);
        if (w->has32 && (rc = launch<float>(w->D, w->D.dyn32, make_args(w->P32, w->W32, SF, MODE_FACTOR), w->dargs32,
                                            w->queue, w->stream, w->err)))
            return fail(rc);
    }
    if ((rc = run_setup_g<double>(w, w->P64, w->W64, w->dargs64, w->D.dyn64))) return fail(rc);
    if (w->has32 && (rc = run_setup_g<float>(w, w->P32, w->W32, w->dargs32, w->D.dyn32))) return fail(rc);
    if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
        set_err(w->err, "setup kernels failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SCS_ECUDA);
    }
    int abort_flag = 0;
    cudaMemcpy(&abort_flag, w->W64.abort_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (abort_flag) { set_err(w->err, "device barrier timed out in setup"); return fail(SCS_ETIMEOUT); }
    if (direct) {
        int f64 = 0, f32 = 0;
        cudaMemcpy(&f64, w->W64.chol_fail, sizeof(int), cudaMemcpyDeviceToHost);
        if (w->has32) cudaMemcpy(&f32, w->W32.chol_fail, sizeof(int), cudaMemcpyDeviceToHost);
        if (f64 || f32) { set_err(w->err, "Cholesky factorisation of I + A^T A met a non-positive pivot"); return fail(SCS_EINVAL); }
    }
    for (auto& e : w->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { set_err(w->err, "cudaEventCreate failed"); return fail(SCS_ECUDA); }
    w->setup_s = now_s() - t0;
    *out = w;
    return SCS_OK;
}

extern "C" void scs_finish(scs_work* w)
{
    if (!w) return;
    for (auto& e : w->ev)
        if (e) cudaEventDestroy(e);
    if (w->arena) cudaFree(w->arena);
    delete w;
}

extern "C" const char* scs_last_error(const scs_work* w) { return w ? w->err : g_err; }

static void fill_info(scs_info* info, const DevState& s)
{
    info->warm_fallback_taken = s.fallback;
    info->status = s.status;
    info->iters = s.iters;
    info->k0 = s.k0;
    info->k1 = s.k1;
    info->k2 = s.k2;
    info->backtracks = s.backtracks;
    info->cg_iters = s.cg_iters;
    info->pr = s.pr;
    info->dr = s.dr;
    info->gap = s.gap;
    info->ic = s.ic;
    info->uc = s.uc;
    info->pobj = s.pobj;
    info->dobj = s.dobj;
    info->mat_passes_ir = s.mat_passes_ir;
    info->cg_iters_ir = s.cg_iters_ir;
    info->ir_sweeps = s.ir_sweeps;
    for (int k = 0; k < 5; ++k) info->part_s[0][k] = s.part_ns[k] * 1e-9;
}

extern "C" int scs_solve(scs_work* w, double* x, double* y, double* s, scs_info* info)
{
    if (!w) { set_err(g_err, "work is NULL"); return SCS_EINVAL; }
    const double t0 = now_s();
    const HostProb& H = w->H;
    const int N = H.n + H.m + 1;
    int rc;
    DevSettings S = dev_settings(&w->S);
    if (w->S.warm == 1) {
        if (!w->S.warm_u) { set_err(w->err, "warm = 1 needs warm_u"); return SCS_EINVAL; }
        CU(cudaMemcpyAsync(w->W64.warm, w->S.warm_u, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
        S.use_warm = 1;
    } else if (w->S.warm == 2) {
        S.use_warm = 1;  // set by scs_set_warm
    }
    DevState st32{};
    if (w->has32) {
        DevSettings S32 = S;
        S32.cg_rtol = w->S.mixed_cg_rtol > 0 ? w->S.mixed_cg_rtol : 1e-6;
        S32.stall_iters = w->S.mixed_stall;
        S32.switch_kkt = w->S.mixed_switch;
        S32.max_iters = w->S.mixed_max_iters > 0 ? std::min(w->S.mixed_max_iters, w->S.max_iters) : w->S.max_iters;
        S32.save_state = w->S.mixed_resume ? 1 : 0;
        if (S.use_warm) CU(cudaMemcpyAsync(w->W32.warm, w->W64.warm, sizeof(double) * N, cudaMemcpyDeviceToDevice, w->stream), w->err);
        Args<float> a32 = make_args(w->P32, w->W32, S32, MODE_SOLVE);
        CU(cudaEventRecord(w->ev[2], w->stream), w->err);
        if ((rc = launch<float>(w->D, w->D.dyn32, a32, w->dargs32, w->queue, w->stream, w->err))) return rc;
        CU(cudaEventRecord(w->ev[3], w->stream), w->err);
        // FP64 phase starts from the FP32 iterate and CG warm starts
        CU(cudaMemcpyAsync(w->W64.warm, w->W32.u_out, sizeof(double) * N, cudaMemcpyDeviceToDevice, w->stream), w->err);
        for (int k = 0; k < 2; ++k) {
            CU(launch_f2d(w->W32.ws[k], w->W64.ws[k], H.n, w->stream), w->err);
        }
        if (w->S.mixed_resume) CU(widen_memory(w->W32, w->W64, w->S.mem, H.n + H.m, w->stream), w->err);
        S.use_warm = 1;
        S.keep_ws = 1;
        S.warm_fallback = 0;
        S.resume = w->S.mixed_resume ? 1 : 0;
        S.refine = w->S.mixed_refine ? 1 : 0;
        CU(cudaMemcpyAsync(&st32, w->W32.st, sizeof(DevState), cudaMemcpyDeviceToHost, w->stream), w->err);
    }
    Args<double> a = make_args(w->P64, w->W64, S, MODE_SOLVE);
    CU(cudaEventRecord(w->ev[0], w->stream), w->err);
    if ((rc = launch<double>(w->D, w->D.dyn64, a, w->dargs64, w->queue, w->stream, w->err))) return rc;
    CU(cudaEventRecord(w->ev[1], w->stream), w->err);
    DevState st{};
    int abort_flag = 0;
    CU(cudaMemcpyAsync(&st, w->W64.st, sizeof(DevState), cudaMemcpyDeviceToHost, w->stream), w->err);
    CU(cudaMemcpyAsync(&abort_flag, w->W64.abort_flag, sizeof(int), cudaMemcpyDeviceToHost, w->stream), w->err);
    if (x) CU(cudaMemcpyAsync(x, w->W64.x_out, sizeof(double) * H.n, cudaMemcpyDefault, w->stream), w->err);
    if (y) CU(cudaMemcpyAsync(y, w->W64.y_out, sizeof(double) * H.m, cudaMemcpyDefault, w->stream), w->err);
    if (s) CU(cudaMemcpyAsync(s, w->W64.s_out, sizeof(double) * H.m, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    int abort32 = 0;
    if (w->has32) CU(cudaMemcpy(&abort32, w->W32.abort_flag, sizeof(int), cudaMemcpyDeviceToHost), w->err);
    if (info) {
        memset(info, 0, sizeof(*info));
        fill_info(info, st);
        if (w->has32) {
            info->warm_fallback_taken |= st32.fallback;
            info->iters += st32.iters;
            info->iters_fp32 = st32.iters;
            info->kkt_fp32 = std::max(st32.pr, std::max(st32.dr, st32.gap));
            info->k0 += st32.k0;
            info->k1 += st32.k1;
            info->k2 += st32.k2;
            info->backtracks += st32.backtracks;
            info->cg_iters += st32.cg_iters;
        }
        info->setup_s = w->setup_s;
        info->solve_s = now_s() - t0;
        info->device_error = abort_flag | abort32;
        info->threads_per_block = w->D.threads;
        info->team = w->D.team;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w->ev[0], w->ev[1]) == cudaSuccess) info->kernel_s[0] = ms * 1e-3;
        cudaGetLastError();
        info->mat_passes[0] = st.mat_passes;
        if (w->has32) {
            if (cudaEventElapsedTime(&ms, w->ev[2], w->ev[3]) == cudaSuccess) info->kernel_s[1] = ms * 1e-3;
            cudaGetLastError();  // a failed timing query must not surface in a later error check
            info->mat_passes[1] = st32.mat_passes;
            info->cg_iters_fp32 = st32.cg_iters;
            info->psd_resid_fp32 = st32.psd_resid;
            info->psd_redo_fp32 = st32.psd_redo;
            for (int k = 0; k < 5; ++k) info->part_s[1][k] = st32.part_ns[k] * 1e-9;
        }
    }
    if (abort_flag || abort32) { set_err(w->err, "device barrier timed out"); return SCS_ETIMEOUT; }
    return SCS_OK;
}

extern "C" int scs_get_u(scs_work* w, double* u)
{
    if (!w || !u) { set_err(w ? w->err : g_err, "NULL argument"); return SCS_EINVAL; }
    const int N = w->H.n + w->H.m + 1;
    CU(cudaMemcpyAsync(u, w->W64.u_out, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

extern "C" int scs_set_warm(scs_work* w, const double* u)
{
    if (!w) { set_err(g_err, "work is NULL"); return SCS_EINVAL; }
    if (!u) {
        w->S.warm = 0;
        w->S.warm_u = nullptr;
        return SCS_OK;
    }
    const int N = w->H.n + w->H.m + 1;
    CU(cudaMemcpyAsync(w->W64.warm, u, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    w->S.warm = 2;  // already on the device
    w->S.warm_u = nullptr;
    return SCS_OK;
}

extern "C" int scs_update_bc(scs_work* w, const double* b, const double* c)
{
    if (!w) { set_err(g_err, "work is NULL"); return SCS_EINVAL; }
    HostProb& H = w->H;
    if (b) {
        for (int i = 0; i < H.m; ++i)
            if (!std::isfinite(b[i])) { set_err(w->err, "non-finite b[%d]", i); return SCS_EINVAL; }
        H.b.assign(b, b + H.m);
    }
    if (c) {
        for (int j = 0; j < H.n; ++j)
            if (!std::isfinite(c[j])) { set_err(w->err, "non-finite c[%d]", j); return SCS_EINVAL; }
        H.c.assign(c, c + H.n);
    }
    double s2 = 0;
    for (double v : H.b) s2 += v * v;
    H.nb = std::sqrt(s2);
    s2 = 0;
    for (double v : H.c) s2 += v * v;
    H.nc = std::sqrt(s2);
    w->P64.nb = w->P32.nb = H.nb;
    w->P64.nc = w->P32.nc = H.nc;
    int rc;
    CU(cudaMemcpyAsync((void*)w->P64.b, H.b.data(), sizeof(double) * H.m, cudaMemcpyHostToDevice, w->stream), w->err);
    CU(cudaMemcpyAsync((void*)w->P64.c, H.c.data(), sizeof(double) * H.n, cudaMemcpyHostToDevice, w->stream), w->err);
    CU(cudaMemsetAsync(w->W64.ws[0], 0, sizeof(double) * H.n, w->stream), w->err);
    if ((rc = run_setup_g<double>(w, w->P64, w->W64, w->dargs64, w->D.dyn64))) return rc;
    if (w->has32) {
        std::vector<float> tb(H.b.begin(), H.b.end()), tc(H.c.begin(), H.c.end());
        CU(cudaMemcpyAsync((void*)w->P32.b, tb.data(), sizeof(float) * H.m, cudaMemcpyHostToDevice, w->stream), w->err);
        CU(cudaMemcpyAsync((void*)w->P32.c, tc.data(), sizeof(float) * H.n, cudaMemcpyHostToDevice, w->stream), w->err);
        CU(cudaMemsetAsync(w->W32.ws[0], 0, sizeof(float) * H.n, w->stream), w->err);
        if ((rc = run_setup_g<float>(w, w->P32, w->W32, w->dargs32, w->D.dyn32))) return rc;
        CU(cudaStreamSynchronize(w->stream), w->err);
    }
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

static int single_op(scs_work* w, int mode, int slot, const double* in, double* out, double* out2)
{
    if (!w || !in) { set_err(w ? w->err : g_err, "NULL argument"); return SCS_EINVAL; }
    const int N = w->H.n + w->H.m + 1;
    CU(cudaMemcpyAsync(w->W64.io_in, in, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    DevSettings S = dev_settings(&w->S);
    Args<double> a = make_args(w->P64, w->W64, S, mode, slot);
    int rc = launch<double>(w->D, w->D.dyn64, a, w->dargs64, w->queue, w->stream, w->err);
    if (rc) return rc;
    if (out) CU(cudaMemcpyAsync(out, w->W64.io_out, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    if (out2) CU(cudaMemcpyAsync(out2, w->W64.io_out2, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

extern "C" int scs_project_cone_prec(scs_work* w, int32_t precision, const double* v, double* out, double* stats)
{
    if (!w || !v || !out) { set_err(w ? w->err : g_err, "NULL argument"); return SCS_EINVAL; }
    if (precision == SCS_FP64) {
        const int rc = single_op(w, MODE_PROJECT, 0, v, out, nullptr);
        if (rc == SCS_OK && stats) {
            const double z[2] = {0.0, 0.0};
            CU(cudaMemcpy(stats, z, sizeof z, cudaMemcpyDefault), w->err);
        }
        return rc;
    }
    if (precision != SCS_MIXED) { set_err(w->err, "bad precision"); return SCS_EINVAL; }
    if (!w->has32) { set_err(w->err, "work was not set up with SCS_MIXED"); return SCS_EINVAL; }
    const int N = w->H.n + w->H.m + 1;
    CU(cudaMemcpyAsync(w->W32.io_in, v, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    DevSettings S = dev_settings(&w->S);
    Args<float> a = make_args(w->P32, w->W32, S, MODE_PROJECT, 0);
    int rc = launch<float>(w->D, w->D.dyn32, a, w->dargs32, w->queue, w->stream, w->err);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, w->W32.io_out, sizeof(double) * N, cudaMemcpyDefault, w->stream), w->err);
    DevState st;
    CU(cudaMemcpyAsync(&st, w->W32.st, sizeof st, cudaMemcpyDeviceToHost, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    if (stats) {
        const double s2[2] = {st.psd_resid, (double)st.psd_redo};
        CU(cudaMemcpy(stats, s2, sizeof s2, cudaMemcpyDefault), w->err);
    }
    return SCS_OK;
}

extern "C" int scs_profile(scs_work* w, int32_t precision, int32_t reps, double* ns)
{
    if (!w || !ns || reps < 1) { set_err(w ? w->err : g_err, "bad arguments"); return SCS_EINVAL; }
    DevSettings S = dev_settings(&w->S);
    int rc;
    if (precision == SCS_MIXED) {
        if (!w->has32) { set_err(w->err, "work was not set up with SCS_MIXED"); return SCS_EINVAL; }
        Args<float> a = make_args(w->P32, w->W32, S, MODE_PROFILE, reps);
        if ((rc = launch<float>(w->D, w->D.dyn32, a, w->dargs32, w->queue, w->stream, w->err))) return rc;
        CU(cudaMemcpyAsync(ns, w->W32.io_out, 5 * sizeof(double), cudaMemcpyDefault, w->stream), w->err);
    } else {
        Args<double> a = make_args(w->P64, w->W64, S, MODE_PROFILE, reps);
        if ((rc = launch<double>(w->D, w->D.dyn64, a, w->dargs64, w->queue, w->stream, w->err))) return rc;
        CU(cudaMemcpyAsync(ns, w->W64.io_out, 5 * sizeof(double), cudaMemcpyDefault, w->stream), w->err);
    }
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

extern "C" int scs_spmv(scs_work* w, int32_t precision, int32_t op, const double* in, const double* in2, double* out,
                        double* out2)
{
    if (!w || !in || !out || op < 0 || op > 2 || (op == 2 && (!in2 || !out2))) {
        set_err(w ? w->err : g_err, "bad arguments");
        return SCS_EINVAL;
    }
    if (precision != SCS_FP64 && precision != SCS_MIXED) { set_err(w->err, "bad precision"); return SCS_EINVAL; }
    if (precision == SCS_MIXED && !w->has32) { set_err(w->err, "work was not set up with SCS_MIXED"); return SCS_EINVAL; }
    const int n = w->H.n, m = w->H.m;
    const int nin = op == 0 ? n : m, nout = op == 0 ? m : n;
    double* io_in = precision == SCS_MIXED ? w->W32.io_in : w->W64.io_in;
    double* io_out = precision == SCS_MIXED ? w->W32.io_out : w->W64.io_out;
    double* io_out2 = precision == SCS_MIXED ? w->W32.io_out2 : w->W64.io_out2;
    CU(cudaMemcpyAsync(io_in, in, sizeof(double) * nin, cudaMemcpyDefault, w->stream), w->err);
    if (op == 2) CU(cudaMemcpyAsync(io_out2, in2, sizeof(double) * m, cudaMemcpyDefault, w->stream), w->err);
    DevSettings S = dev_settings(&w->S);
    int rc;
    if (precision == SCS_MIXED) {
        Args<float> a = make_args(w->P32, w->W32, S, MODE_SPMV, op);
        rc = launch<float>(w->D, w->D.dyn32, a, w->dargs32, w->queue, w->stream, w->err);
    } else {
        Args<double> a = make_args(w->P64, w->W64, S, MODE_SPMV, op);
        rc = launch<double>(w->D, w->D.dyn64, a, w->dargs64, w->queue, w->stream, w->err);
    }
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, io_out, sizeof(double) * nout, cudaMemcpyDefault, w->stream), w->err);
    if (op == 2) CU(cudaMemcpyAsync(out2, io_out2, sizeof(double) * nout, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

extern "C" int scs_residuals(scs_work* w, const double* x, const double* y, const double* s, double* out)
{
    if (!w || !x || !y || !s || !out) { set_err(w ? w->err : g_err, "NULL argument"); return SCS_EINVAL; }
    const int n = w->H.n, m = w->H.m;
    CU(cudaMemcpyAsync(w->W64.io_in, x, sizeof(double) * n, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaMemcpyAsync(w->W64.io_in + n, y, sizeof(double) * m, cudaMemcpyDefault, w->stream), w->err);
    CU(cudaMemcpyAsync(w->W64.io_out2, s, sizeof(double) * m, cudaMemcpyDefault, w->stream), w->err);
    DevSettings S = dev_settings(&w->S);
    Args<double> a = make_args(w->P64, w->W64, S, MODE_RESID);
    int rc = launch<double>(w->D, w->D.dyn64, a, w->dargs64, w->queue, w->stream, w->err);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, w->W64.io_out, 3 * sizeof(double), cudaMemcpyDefault, w->stream), w->err);
    CU(cudaStreamSynchronize(w->stream), w->err);
    return SCS_OK;
}

extern "C" int scs_linsys(scs_work* w, const double* r, double* out, int32_t slot)
{
    if (!w || slot < 0 || slot > 3) { set_err(w ? w->err : g_err, "bad arguments"); return SCS_EINVAL; }
    if ((slot & 2) && !w->has32) { set_err(w->err, "refinement needs a work set up with SCS_MIXED"); return SCS_EINVAL; }
    return single_op(w, MODE_LINSYS, slot, r, out, nullptr);
}
extern "C" int scs_project_cone(scs_work* w, const double* v, double* out)
{
    return single_op(w, MODE_PROJECT, 0, v, out, nullptr);
}
extern "C" int scs_apply_T(scs_work* w, const double* u, double* Tu, double* Ru)
{
    return single_op(w, MODE_APPLY_T, 0, u, Tu, Ru);
}

// ---------------------------------------------------------------------------
// batches: one arena, one descriptor per instance (uploaded once), persistent
// CTAs taking instances from a queue; states and outputs are gathered into
// contiguous buffers so a batch solve needs a fixed number of launches and
// copies whatever B is.
// ---------------------------------------------------------------------------
struct scs_batch {
    int B = 0;
    std::vector<HostProb> H;
    std::vector<int> order;  // queue position -> instance
    scs_settings S;
    cudaStream_t stream = nullptr;
    // the device work of one batch solve, captured once and replayed
    cudaStream_t gstream = nullptr;   // capture stream (the caller's stream cannot be captured when it is the legacy default)
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t gev = nullptr;        // orders the graph after the caller's stream
    int graph_warm = -1;              // use_warm the graph was captured with
    char* arena = nullptr;
    int threads = 256, grid = 1, sms = 1;
    bool autotuned = false;
    bool has32 = false;
    bool shared = false;  // all instances share instance 0's matrix arrays
    bool use_warm = false;
    size_t dyn64 = 0, dyn32 = 0;
    std::vector<Args<double>> a64;
    std::vector<Args<float>> a32;
    Args<double>* d64 = nullptr;
    Args<float>* d32 = nullptr;
    DevState* st64 = nullptr;  // B contiguous states (queue order)
    DevState* st32 = nullptr;
    long long* off = nullptr;  // packed output offsets (queue order)
    double* packed = nullptr;  // n + 2m doubles per instance
    std::vector<long long> hoff;
    long long packed_len = 0;
    double* hpacked = nullptr;  // pinned host staging
    DevState* hst = nullptr;    // pinned host staging (2B states)
    int* queue = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_all[2] = {nullptr, nullptr};  // around the whole solve, on the stream it runs on
    char err[512];
    double setup_s = 0;
    double tune_ms[4] = {0, 0, 0, 0};
};

static int occupancy_grid(const void* fn, int threads, size_t dyn, int sms, int B)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, dyn);
    return std::max(1, std::min(B, sms * std::max(nb, 1)));
}

template <typename T>
static DevSettings batch_settings(const scs_batch* b, bool first_phase_of_mixed)
{
    DevSettings S = dev_settings(&b->S);
    if (first_phase_of_mixed) {
        S.cg_rtol = b->S.mixed_cg_rtol > 0 ? b->S.mixed_cg_rtol : 1e-6;
        S.stall_iters = b->S.mixed_stall;
        S.switch_kkt = b->S.mixed_switch;
        S.max_iters = b->S.mixed_max_iters > 0 ? std::min(b->S.mixed_max_iters, b->S.max_iters) : b->S.max_iters;
        S.save_state = b->S.mixed_resume ? 1 : 0;
    }
    return S;
}

// Autotuner: time the first solve phase on an evenly spaced sample of the
// (size-sorted) instances for 128, 256, 512 and 1024 threads per CTA and keep
// the fastest; the sample's results are discarded (the real solve overwrites
// them).
template <typename T>
static int autotune(scs_batch* b, const std::vector<Args<T>>& host_args, size_t dyn, const DevSettings& S,
                    Args<T>* scratch_args)
{
    const int cand[4] = {128, 256, 512, 1024};
    // The sample must keep every candidate's resident CTAs busy for two waves:
    // with only a couple of instances per SM, large CTAs look fast (each
    // instance gets more threads) although the whole batch runs best with more,
    // smaller CTAs in flight.
    const void* fn = sizeof(T) == 8 ? kblock_ptr<double>() : kblock_ptr<float>();
    int resident = 1;
    for (int c = 0; c < 4; ++c) resident = std::max(resident, occupancy_grid(fn, cand[c], dyn, b->sms, b->B));
    const int nsamp = std::min(b->B, std::max(2 * b->sms, 2 * resident));
    std::vector<Args<T>> samp(nsamp);
    for (int i = 0; i < nsamp; ++i) samp[i] = host_args[(size_t)i * b->B / nsamp];
    CU(cudaMemcpyAsync(scratch_args, samp.data(), sizeof(Args<T>) * nsamp, cudaMemcpyHostToDevice, b->stream), b->err);
    float best = 1e30f;
    for (int c = 0; c < 4; ++c) {
        const int grid = occupancy_grid(fn, cand[c], dyn, b->sms, nsamp);
        CU(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream), b->err);
        CU(cudaEventRecord(b->ev[0], b->stream), b->err);
        CU(launch_block<T>(grid, cand[c], dyn, b->stream, scratch_args, nsamp, b->queue, S, MODE_SOLVE), b->err);
        CU(cudaEventRecord(b->ev[1], b->stream), b->err);
        CU(cudaEventSynchronize(b->ev[1]), b->err);
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]), b->err);
        b->tune_ms[c] = ms;
        if (ms < best) {
            best = ms;
            b->threads = cand[c];
        }
    }
    b->autotuned = true;
    return SCS_OK;
}

static int batch_finish_setup(scs_batch* b, const scs_settings* settings, scs_batch** out, double t0);

extern "C" int scs_batch_setup(int32_t B, const scs_data* const* data, const scs_cone* const* cones,
                               const scs_settings* settings, void* cuda_stream, scs_batch** out)
{
    if (!out) { set_err(g_err, "out must not be NULL"); return SCS_EINVAL; }
    *out = nullptr;
    if (B <= 0 || !data || !cones) { set_err(g_err, "bad batch arguments"); return SCS_EINVAL; }
    const double t0 = now_s();
    scs_batch* b = new (std::nothrow) scs_batch();
    if (!b) return SCS_ENOMEM;
    b->err[0] = 0;
    int rc = check_settings(settings, b->err);
    if (rc) { memcpy(g_err, b->err, 512); delete b; return rc; }
    b->B = B;
    b->S = *settings;
    b->stream = (cudaStream_t)cuda_stream;
    b->H.resize(B);
    for (int i = 0; i < B; ++i) {
        if ((rc = prepare(data[i], cones[i], b->H[i], b->err))) {
            char tmp[512];
            snprintf(tmp, sizeof tmp, "instance %d: %.480s", i, b->err);
            memcpy(b->err, tmp, 512);
            memcpy(g_err, b->err, 512);
            delete b;
            return rc;
        }
    }
    return batch_finish_setup(b, settings, out, t0);
}

// common part of the batch setups once every b->H[i] is prepared
static int batch_finish_setup(scs_batch* b, const scs_settings* settings, scs_batch** out, double t0)
{
    const int B = b->B;
    int rc = 0;
    b->order.resize(B);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return b->H[x].nnz + b->H[x].n + b->H[x].m > b->H[y].nnz + b->H[y].n + b->H[y].m;
    });
    b->has32 = settings->precision == SCS_MIXED;
    bool any_psd = false;
    for (auto& h : b->H) any_psd |= !h.s.empty();
    b->dyn64 = any_psd ? psd_smem_bytes<double>() : 0;
    b->dyn32 = any_psd && b->has32 ? psd_smem_bytes<float>() : 0;
    if (b->has32) b->dyn64 = std::max(b->dyn64, b->dyn32);
    if ((rc = config_kernels<double>(b->dyn64, b->err)) || (b->has32 && (rc = config_kernels<float>(b->dyn32, b->err)))) {
        memcpy(g_err, b->err, 512);
        delete b;
        return rc;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    const int mem = std::max(settings->mem, 1);
    const bool qr = settings->direction == SCS_DIR_AA_QR;
    const bool direct = settings->linsys_direct != 0;
    b->hoff.resize(B + 1, 0);
    for (int qi = 0; qi < B; ++qi) {
        const HostProb& h = b->H[b->order[qi]];
        b->hoff[qi + 1] = b->hoff[qi] + h.n + 2LL * h.m;
    }
    b->packed_len = b->hoff[B];
    Arena A;
    b->a64.resize(B);
    if (b->has32) b->a32.resize(B);
    auto lay_all = [&](bool real) {
        DevState* st64 = A.take<DevState>(B);
        DevState* st32 = A.take<DevState>(B);
        for (int qi = 0; qi < B; ++qi) {
            const HostProb& h = b->H[b->order[qi]];
            lay_out<double>(A, h, mem, qr, direct && h.n <= DIRECT_MAX_N, 1, b->a64[qi].P, b->a64[qi].W, nullptr, real ? st64 + qi : nullptr);
            b->a64[qi].slot = 0;
            if (real && b->shared && qi > 0) {
                b->a64[qi].P.A = b->a64[0].P.A;
                b->a64[qi].P.AT = b->a64[0].P.AT;
                b->a64[qi].P.q_off = b->a64[0].P.q_off;
                b->a64[qi].P.s_dim = b->a64[0].P.s_dim;
                b->a64[qi].P.s_off = b->a64[0].P.s_off;
            }
            if (b->has32) {
                lay_out<float>(A, h, mem, qr, direct && h.n <= DIRECT_MAX_N, 1, b->a32[qi].P, b->a32[qi].W, (const int*)1, real ? st32 + qi : nullptr);
                b->a32[qi].slot = 0;
                if (real) {
                    DevProb<float>& p = b->a32[qi].P;
                    const DevProb<double>& q = b->a64[qi].P;
                    p.A.ptr = q.A.ptr; p.A.col = q.A.col; p.A.perm = q.A.perm; p.A.wbnd = q.A.wbnd;
                    p.AT.ptr = q.AT.ptr; p.AT.col = q.AT.col; p.AT.perm = q.AT.perm; p.AT.wbnd = q.AT.wbnd;
                    p.q_off = q.q_off; p.s_dim = q.s_dim; p.s_off = q.s_off;
                    if (b->shared && qi > 0) {
                        p.A.val = b->a32[0].P.A.val;
                        p.AT.val = b->a32[0].P.AT.val;
                    }
                    link_phases(p, b->a32[qi].W, b->a64[qi].W);
                }
            }
        }
        if (real) {
            b->st64 = st64;
            b->st32 = st32;
        }
        Args<double>* d64 = A.take<Args<double>>(B);
        Args<float>* d32 = A.take<Args<float>>(B);
        Args<double>* t64 = A.take<Args<double>>(B);  // the autotuner's sample: at most B instances
        Args<float>* t32 = A.take<Args<float>>(B);
        long long* off = A.take<long long>(B + 1);
        double* packed = A.take<double>(b->packed_len);
        int* queue = A.take<int>(4);
        if (real) {
            b->d64 = d64;
            b->d32 = d32;
            b->off = off;
            b->packed = packed;
            b->queue = queue;
        }
        return std::make_pair(t64, t32);
    };
    lay_all(false);
    const size_t bytes = A.off + 1024;
    if (cudaMalloc((void**)&b->arena, bytes) != cudaSuccess) {
        set_err(b->err, "cudaMalloc(%zu) failed", bytes);
        memcpy(g_err, b->err, 512);
        delete b;
        return SCS_ENOMEM;
    }
    auto fail = [&](int r) { memcpy(g_err, b->err, 512); scs_batch_finish(b); return r; };
    if (cudaMallocHost((void**)&b->hpacked, sizeof(double) * std::max<long long>(b->packed_len, 1)) != cudaSuccess ||
        cudaMallocHost((void**)&b->hst, sizeof(DevState) * 2 * B) != cudaSuccess) {
        set_err(b->err, "cudaMallocHost failed");
        return fail(SCS_ENOMEM);
    }
    for (auto& e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { set_err(b->err, "cudaEventCreate failed"); return fail(SCS_ECUDA); }
    for (auto& e : b->ev_all)
        if (cudaEventCreate(&e) != cudaSuccess) { set_err(b->err, "cudaEventCreate failed"); return fail(SCS_ECUDA); }
    A.off = 0;
    A.base = b->arena;
    auto tune_args = lay_all(true);
    if (cudaMemsetAsync(b->arena, 0, bytes, b->stream) != cudaSuccess) { set_err(b->err, "memset failed"); return fail(SCS_ECUDA); }
    for (int qi = 0; qi < B; ++qi) {
        const HostProb& h = b->H[b->order[qi]];
        const bool mat = !b->shared || qi == 0;
        if ((rc = upload<double>(h, b->a64[qi].P, true, b->stream, b->err, mat))) return fail(rc);
        if (b->has32 && (rc = upload<float>(h, b->a32[qi].P, false, b->stream, b->err, mat))) return fail(rc);
    }
    if (cudaMemcpyAsync(b->off, b->hoff.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d64, b->a64.data(), sizeof(Args<double>) * B, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        (b->has32 && cudaMemcpyAsync(b->d32, b->a32.data(), sizeof(Args<float>) * B, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)) {
        set_err(b->err, "descriptor upload failed");
        return fail(SCS_ECUDA);
    }
    DevSettings S = dev_settings(settings);
    S.cg_max = std::max(10 * settings->cg_max, 10000);
    DevSettings S64 = S, S32 = S;
    S64.cg_rtol = std::min(settings->cg_rtol, 1e-12);
    S32.cg_rtol = std::min(settings->cg_rtol, 1e-7);
    // setup (g = M^{-1}(c, b)) with a provisional shape
    b->threads = settings->threads ? settings->threads : 256;
    b->grid = occupancy_grid(kblock_ptr<double>(), b->threads, b->dyn64, b->sms, B);
    if (direct) {
        // factor I + A^T A of every instance (n <= DIRECT_MAX_N) in each precision before g is solved with it
        CU(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream), b->err);
        CU(launch_block<double>(b->grid, b->threads, b->dyn64, b->stream, b->d64, B, b->queue, S64, MODE_FACTOR), b->err);
        if (b->has32) {
            const int g32 = occupancy_grid(kblock_ptr<float>(), b->threads, b->dyn32, b->sms, B);
            CU(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream), b->err);
            CU(launch_block<float>(g32, b->threads, b->dyn32, b->stream, b->d32, B, b->queue, S32, MODE_FACTOR), b->err);
        }
    }
    CU(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream), b->err);
    CU(launch_block<double>(b->grid, b->threads, b->dyn64, b->stream, b->d64, B, b->queue, S64, MODE_SETUP), b->err);
    if (b->has32) {
        const int g32 = occupancy_grid(kblock_ptr<float>(), b->threads, b->dyn32, b->sms, B);
        CU(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream), b->err);
        CU(launch_block<float>(g32, b->threads, b->dyn32, b->stream, b->d32, B, b->queue, S32, MODE_SETUP), b->err);
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        set_err(b->err, "batch setup kernels failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SCS_ECUDA);
    }
    if (!settings->threads && B >= 64) {
        if (b->has32) rc = autotune<float>(b, b->a32, b->dyn32, batch_settings<float>(b, true), tune_args.second);
        else rc = autotune<double>(b, b->a64, b->dyn64, batch_settings<double>(b, false), tune_args.first);
        if (rc) return fail(rc);
    }
    b->setup_s = now_s() - t0;
    *out = b;
    return SCS_OK;
}

extern "C" int scs_batch_setup_shared(int32_t B, const scs_data* data, const scs_cone* cone, const double* const* bv,
                                      const double* const* cv, const scs_settings* settings, void* cuda_stream,
                                      scs_batch** out)
{
    if (!out) { set_err(g_err, "out must not be NULL"); return SCS_EINVAL; }
    *out = nullptr;
    if (B <= 0 || !data || !cone || !bv || !cv) { set_err(g_err, "bad batch arguments"); return SCS_EINVAL; }
    const double t0 = now_s();
    scs_batch* b = new (std::nothrow) scs_batch();
    if (!b) return SCS_ENOMEM;
    b->err[0] = 0;
    int rc = check_settings(settings, b->err);
    if (rc) { memcpy(g_err, b->err, 512); delete b; return rc; }
    b->B = B;
    b->S = *settings;
    b->stream = (cudaStream_t)cuda_stream;
    b->shared = true;
    b->H.resize(B);
    if ((rc = prepare(data, cone, b->H[0], b->err))) { memcpy(g_err, b->err, 512); delete b; return rc; }
    for (int i = 0; i < B; ++i) {
        HostProb& h = b->H[i];
        if (i > 0) {  // light copy: sizes and cones; the matrix stays with instance 0
            const HostProb& h0 = b->H[0];
            h.n = h0.n; h.m = h0.m; h.nnz = h0.nnz; h.f = h0.f; h.l = h0.l;
            h.ep = h0.ep; h.ed = h0.ed; h.e_off = h0.e_off;
            h.q = h0.q; h.s = h0.s; h.q_off = h0.q_off; h.s_off = h0.s_off; h.vecA = h0.vecA; h.vecT = h0.vecT;
            h.SA.rows = h0.SA.rows; h.SA.V = h0.SA.V; h.SA.nslices = h0.SA.nslices;
            h.ST.rows = h0.ST.rows; h.ST.V = h0.ST.V; h.ST.nslices = h0.ST.nslices;
        }
        if (!bv[i] || !cv[i]) { set_err(b->err, "instance %d: NULL b or c", i); memcpy(g_err, b->err, 512); delete b; return SCS_EINVAL; }
        h.b.assign(bv[i], bv[i] + h.m);
        h.c.assign(cv[i], cv[i] + h.n);
        double sb = 0, sc = 0;
        for (double v : h.b) { if (!std::isfinite(v)) { set_err(b->err, "instance %d: non-finite b", i); memcpy(g_err, b->err, 512); delete b; return SCS_EINVAL; } sb += v * v; }
        for (double v : h.c) { if (!std::isfinite(v)) { set_err(b->err, "instance %d: non-finite c", i); memcpy(g_err, b->err, 512); delete b; return SCS_EINVAL; } sc += v * v; }
        h.nb = std::sqrt(sb);
        h.nc = std::sqrt(sc);
    }
    return batch_finish_setup(b, settings, out, t0);
}

extern "C" int scs_batch_set_warm(scs_batch* b, const double* const* u)
{
    if (!b) { set_err(g_err, "batch is NULL"); return SCS_EINVAL; }
    if (!u) { b->use_warm = false; return SCS_OK; }
    for (int qi = 0; qi < b->B; ++qi) {
        const int i = b->order[qi];
        const HostProb& h = b->H[i];
        const size_t N = (size_t)h.n + h.m + 1;
        if (!u[i]) { set_err(b->err, "instance %d: NULL warm start", i); return SCS_EINVAL; }
        CU(cudaMemcpyAsync(b->a64[qi].W.warm, u[i], sizeof(double) * N, cudaMemcpyDefault, b->stream), b->err);
        if (b->has32) CU(cudaMemcpyAsync(b->a32[qi].W.warm, u[i], sizeof(double) * N, cudaMemcpyDefault, b->stream), b->err);
    }
    CU(cudaStreamSynchronize(b->stream), b->err);
    b->use_warm = true;
    return SCS_OK;
}

extern "C" void scs_batch_finish(scs_batch* b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->gev) cudaEventDestroy(b->gev);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : b->ev_all)
        if (e) cudaEventDestroy(e);
    if (b->hpacked) cudaFreeHost(b->hpacked);
    if (b->hst) cudaFreeHost(b->hst);
    if (b->arena) cudaFree(b->arena);
    delete b;
}

// The device work of one batch solve, enqueued on st: FP32 phase (SCS_MIXED),
// hand-over, FP64 phase, packing of the outputs, copies of outputs and
// states to the pinned host staging buffers.  No synchronisation, so it can
// be captured in a CUDA graph.
static int batch_enqueue(scs_batch* b, cudaStream_t st, int g32, int g64, bool capturing)
{
    const int B = b->B;
    // timing events: inside a capture they must be external record nodes so
    // they can be read after the graph runs
    auto rec = [&](cudaEvent_t e) {
        return capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
    };
    if (b->has32) {
        DevSettings S32 = batch_settings<float>(b, true);
        S32.use_warm = b->use_warm ? 1 : 0;
        CU(cudaMemsetAsync(b->queue, 0, sizeof(int), st), b->err);
        CU(rec(b->ev[2]), b->err);
        CU(launch_block<float>(g32, b->threads, b->dyn32, st, b->d32, B, b->queue, S32, MODE_SOLVE), b->err);
        CU(rec(b->ev[3]), b->err);
        CU(launch_batch_handoff(b->d32, b->d64, B, b->S.mem, b->S.mixed_resume ? 1 : 0, st), b->err);
    }
    DevSettings S = batch_settings<double>(b, false);
    if (b->has32) {
        S.use_warm = 1;
        S.keep_ws = 1;
        S.warm_fallback = 0;
        S.resume = b->S.mixed_resume ? 1 : 0;
        S.refine = b->S.mixed_refine ? 1 : 0;
    } else {
        S.use_warm = b->use_warm ? 1 : 0;
    }
    CU(cudaMemsetAsync(b->queue, 0, sizeof(int), st), b->err);
    CU(rec(b->ev[0]), b->err);
    CU(launch_block<double>(g64, b->threads, b->dyn64, st, b->d64, B, b->queue, S, MODE_SOLVE), b->err);
    CU(rec(b->ev[1]), b->err);
    CU(launch_batch_pack(b->d64, B, b->off, b->packed, st), b->err);
    CU(cudaMemcpyAsync(b->hpacked, b->packed, sizeof(double) * b->packed_len, cudaMemcpyDeviceToHost, st), b->err);
    CU(cudaMemcpyAsync(b->hst, b->st64, sizeof(DevState) * B, cudaMemcpyDeviceToHost, st), b->err);
    if (b->has32) CU(cudaMemcpyAsync(b->hst + B, b->st32, sizeof(DevState) * B, cudaMemcpyDeviceToHost, st), b->err);
    return SCS_OK;
}

// Capture batch_enqueue into a CUDA graph on the batch's private capture
// stream (again whenever the warm-start mode changes, which changes the
// kernels' parameters).  Returns non-zero if capture is unavailable; the
// caller then enqueues directly.
static int batch_graph(scs_batch* b, int g32, int g64)
{
    const int warm = b->use_warm ? 1 : 0;
    if (b->gexec && b->graph_warm == warm) return SCS_OK;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if ((!b->gstream && cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess) ||
        (!b->gev && cudaEventCreateWithFlags(&b->gev, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        return SCS_ECUDA;
    }
    if (cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SCS_ECUDA;
    }
    const int rc = batch_enqueue(b, b->gstream, g32, g64, true);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->gstream, &g);
    if (rc || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return SCS_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        b->gexec = nullptr;
        cudaGetLastError();
        return SCS_ECUDA;
    }
    b->graph_warm = warm;
    return SCS_OK;
}

extern "C" int scs_batch_solve(scs_batch* b, double* const* x, double* const* y, double* const* s, scs_info* infos)
{
    if (!b) { set_err(g_err, "batch is NULL"); return SCS_EINVAL; }
    const double t0 = now_s();
    const int B = b->B;
    float ms32 = 0.f, ms64 = 0.f;
    const int g32 = b->has32 ? occupancy_grid(kblock_ptr<float>(), b->threads, b->dyn32, b->sms, B) : 0;
    const int g64 = occupancy_grid(kblock_ptr<double>(), b->threads, b->dyn64, b->sms, B);
    b->grid = g64;
    // One graph launch replays the whole batch solve.  The graph runs on the
    // batch's capture stream, ordered after the caller's stream by an event.
    if (batch_graph(b, g32, g64) == SCS_OK) {
        CU(cudaEventRecord(b->gev, b->stream), b->err);
        CU(cudaStreamWaitEvent(b->gstream, b->gev, 0), b->err);
        CU(cudaEventRecord(b->ev_all[0], b->gstream), b->err);
        CU(cudaGraphLaunch(b->gexec, b->gstream), b->err);
        CU(cudaEventRecord(b->ev_all[1], b->gstream), b->err);
        CU(cudaStreamSynchronize(b->gstream), b->err);
    } else {
        CU(cudaEventRecord(b->ev_all[0], b->stream), b->err);
        int rc = batch_enqueue(b, b->stream, g32, g64, false);
        if (rc) return rc;
        CU(cudaEventRecord(b->ev_all[1], b->stream), b->err);
    }
    CU(cudaStreamSynchronize(b->stream), b->err);
    float ms_all = 0.f;
    if (cudaEventElapsedTime(&ms_all, b->ev_all[0], b->ev_all[1]) != cudaSuccess) ms_all = 0.f;
    if (cudaEventElapsedTime(&ms64, b->ev[0], b->ev[1]) != cudaSuccess) ms64 = 0.f;
    if (b->has32 && cudaEventElapsedTime(&ms32, b->ev[2], b->ev[3]) != cudaSuccess) ms32 = 0.f;
    cudaGetLastError();  // a failed timing query must not surface in a later error check
    for (int qi = 0; qi < B; ++qi) {
        const int i = b->order[qi];
        const HostProb& h = b->H[i];
        const double* src = b->hpacked + b->hoff[qi];
        if (x && x[i]) memcpy(x[i], src, sizeof(double) * h.n);
        if (y && y[i]) memcpy(y[i], src + h.n, sizeof(double) * h.m);
        if (s && s[i]) memcpy(s[i], src + h.n + h.m, sizeof(double) * h.m);
    }
    const double el = now_s() - t0;
    if (infos) {
        for (int qi = 0; qi < B; ++qi) {
            const int i = b->order[qi];
            scs_info* info = &infos[i];
            memset(info, 0, sizeof(*info));
            fill_info(info, b->hst[qi]);
            info->mat_passes[0] = b->hst[qi].mat_passes;
            info->kernel_s[0] = ms64 * 1e-3;
            if (b->has32) {
                const DevState& t = b->hst[B + qi];
                info->warm_fallback_taken |= t.fallback;
                info->iters += t.iters;
                info->iters_fp32 = t.iters;
                info->kkt_fp32 = std::max(t.pr, std::max(t.dr, t.gap));
                info->k0 += t.k0;
                info->k1 += t.k1;
                info->k2 += t.k2;
                info->backtracks += t.backtracks;
                info->cg_iters += t.cg_iters;
                info->cg_iters_fp32 = t.cg_iters;
                info->mat_passes[1] = t.mat_passes;
                info->psd_resid_fp32 = t.psd_resid;
                info->psd_redo_fp32 = t.psd_redo;
                info->kernel_s[1] = ms32 * 1e-3;
            }
            info->setup_s = b->setup_s;
            info->solve_s = el;
            info->batch_device_s = ms_all * 1e-3;
            info->threads_per_block = b->threads;
            info->team = SCS_TEAM_BLOCK;
        }
    }
    return SCS_OK;
}

extern "C" int scs_solve_batch(int32_t B, const scs_data* const* data, const scs_cone* const* cones,
                               const scs_settings* settings, void* cuda_stream, double* const* x, double* const* y,
                               double* const* s, scs_info* infos)
{
    scs_batch* b = nullptr;
    int rc = scs_batch_setup(B, data, cones, settings, cuda_stream, &b);
    if (rc) return rc;
    rc = scs_batch_solve(b, x, y, s, infos);
    scs_batch_finish(b);
    return rc;
}
