// solver.cuh -- device-resident SuperSCS (Sopasakis, Menounou, Patrinos,
// arXiv 1903.06477), generic over the bulk precision T (double or float)
// and over the execution team (one CTA, or every CTA of a cooperative grid).
//
// Structure of one outer iteration (Algorithm 1):
//   termination test (Sec. 4.3)       2 SpMVs + 1 reduction
//   direction d (Sec. 4.4, AA or RB)   passes over the N x mem buffers
//   d~ = (I+Q)^{-1} d                  CG on I + A^T A (Sec. 4.1)
//   K0 | line search with K1/K2        fused projection + residual passes
// HSDE vectors keep their tau entry in FP64 whatever T is.
#pragma once

#include "common.cuh"
#include "team.cuh"

namespace sscs {

constexpr int MAXMEM = 64;   // direction memory cap (RB)
constexpr int AAMAX = 32;    // Anderson memory cap (Gram matrix kept in shared memory)
constexpr int PSD_MAX = 64;  // largest PSD order decomposed in shared memory
constexpr int PSD_LD = PSD_MAX + 1;  // row stride bound of a block's matrices in shared memory
constexpr int PSD_BIG_MAX = 1024;    // largest PSD order (orders above PSD_MAX use a global-memory workspace)

enum Mode { MODE_SETUP = 0, MODE_SOLVE = 1, MODE_LINSYS = 2, MODE_PROJECT = 3, MODE_APPLY_T = 4, MODE_PROFILE = 5,
            MODE_RESID = 6, MODE_SPMV = 7, MODE_FACTOR = 8 };
enum { ST_SOLVED = 1, ST_INFEASIBLE = -1, ST_UNBOUNDED = -2, ST_MAX_ITERS = -3, ST_TIME_LIMIT = -4,
       ST_NUMERICAL = -5, ST_STALLED = -6 };

template <typename T>
struct HV {  // HSDE vector: (chi, psi) bulk of n+m entries in T, tau in FP64
    T* v;
    double* t;
};

struct DevSettings {
    int direction, mem;
    double eps, c0, c1, q, sigma, lambda, thetabar;
    int max_iters, ls_max, cg_max, check_every;
    double cg_rtol, aa_reg;
    double time_limit_ns;  // <= 0: none
    int stall_iters;       // > 0: stop when ||Ru|| has not dropped 10% below its best for this many iterations
    int use_warm;
    double switch_kkt;     // > 0: stop (hand over) once max(pr,dr,gap) <= switch_kkt
    double cg_adapt;       // > 0: CG inside the loop also stops at ||res|| <= cg_adapt ||Ru||
    int keep_ws;           // 1: keep the CG warm starts found in ws (handed over by the FP32 phase)
    int warm_fallback;     // > 0 with a warm start: restart cold if ||Ru|| is not below the cold
                           // start's ||Ru0|| after this many iterations
    int save_state;        // 1: write the loop state to W.res when the solve ends (FP32 phase of SCS_MIXED)
    int resume;            // 1: continue from the loop state in W.res instead of starting Algorithm 1 afresh
    int stall_after_tau;   // 1: the stall count starts only once tau_ > 0 (FP32 phase of SCS_MIXED)
    int refine;            // 1 (FP64 data only): linear systems by iterative refinement, FP64 residuals
                           // and FP32 CG corrections on the FP32 copy of A (W.ir)
    double psd_tol;        // FP32 eigensolves: a PSD block whose FP64-evaluated relative eigen-residual
                           // exceeds this is decomposed again in FP64
};

// State of Algorithm 1 at the end of the FP32 phase of SCS_MIXED, so that the
// FP64 phase continues the same iteration (direction memory, the K0/K1
// references eta, eta0, r_safe and the outer index nu) instead of restarting.
struct Resume {
    int valid, count, have_pair, nu;
    long long inserted;
    double eta, eta0, r_safe, nz2;
    double G[AAMAX * AAMAX];  // AA Gram matrix of the stored pairs
};

struct DevState {
    int status, iters, k0, k1, k2, backtracks;
    long long cg_iters;
    double pr, dr, gap, ic, uc, pobj, dobj, nRu, hg;
    int setup_cg, pad;
    long long mat_passes;  // SpMV passes over A or A^T
    double psd_resid;      // largest ||X V - V L||_F / ||X||_F of the FP32 eigensolves, in FP64
    int fallback;          // 1 if the warm start was abandoned for the cold start
    int pad2;
    long long mat_passes_ir;  // FP32 passes of the refinement corrections (FP64 phase)
    long long cg_iters_ir;    // FP32 CG iterations of the refinement corrections (FP64 phase)
    long long ir_sweeps;      // refinement sweeps (FP32 correction solves)
    // device time (globaltimer, read by the leader thread between team barriers) of the parts of
    // Algorithm 1: [0] termination tests, [1] directions, [2] linear solves (all of minv / its
    // refinement variant), [3] the CG loops inside them, [4] everything else (K0 steps, line
    // searches, projections, updates)
    double part_ns[5];
    long long psd_redo;    // PSD blocks of the FP32 phase decomposed again in FP64 (eigen-residual above psd_tol)
};

// Column-blocked sliced ELL, the grid team's layout for large matrices.  CTA b
// owns the contiguous rows [rbnd[b], rbnd[b+1]); the columns are cut into ncb
// blocks of cw.  A "segment" is one (CTA, column block) pair: the CTA's rows
// that have entries in the block, sorted by their count there (descending),
// packed as slices of H = 32 / V rows with element j of slice row r at
// step (slice start + j / V), lane (j % V) * H + r, 32 entries per step, and
// its column stored as a 16-bit offset inside the block (padding: value 0,
// offset 0).  The slices of a segment are dealt to the CTA's warps (largest
// first to the least-loaded warp) and stored warp by warp.  The entries of
// segment g = b * ncb + k are contiguous, [E0, E1) of col / val.
//
// Each segment has ms 32-bit words of metadata at meta + g * ms:
//   [0] E0   [1] E1   [2], [3] E0, E1 of the CTA's segment (k + S) mod ncb
//   [4] ns: slices    [5 .. 5+nw] first slice of each warp (nw+1 values)
//   [6+nw .. 6+nw+ns] slice start steps from E0 (ns+1 values)
//   then ns * H 16-bit row indices inside the CTA's range (0xFFFF: none),
//   two per word, low half first.
//
// The product streams segments through a ring of S shared-memory stages,
// warp-specialised: the CTA's last warp is the producer, which copies a
// segment's metadata, its slice of the multiplied vector and its entries with
// bulk (TMA) copies completing on the stage's "full" mbarrier as soon as the
// stage's "empty" mbarrier says every compute warp is done with it; the
// other nw warps compute, so the random reads of the vector and the matrix
// stream are all shared-memory reads.  The rows of one segment are distinct,
// and the partial sums are double-buffered by segment parity: a compute warp
// starts segment j once segment j-2 is finished by every warp (its "empty"
// barrier), so warps may run one segment apart without two of them ever
// updating the same sum, and each sum is accumulated in a fixed order
// (deterministic).  CTA b visits the column blocks in the order b, b+1, ...
// (mod ncb), so at any moment the CTAs read different slices of the vector.
// The CTA adds its two partial-sum buffers after the last block.
template <typename T>
struct Cblk {
    int ncb;          // column blocks (0: layout absent)
    int cw;           // columns per block (multiple of 4)
    int cols;         // columns of the matrix
    int nw;           // compute warps per CTA (the CTA has nw + 1 warps)
    int V;            // lanes per row
    int acc_rows;     // partial-sum entries per buffer (largest row range); 2 buffers per vector
    int ms;           // metadata words per segment (multiple of 4)
    int S;            // stages in the copy ring (2..CB_MAX_STAGES)
    int stage_off;    // byte offset of stage 0 in dynamic shared memory
    int stage_bytes;  // bytes per stage (multiple of 16)
    int off_x, off_col, off_val;  // byte offsets inside a stage (tiles: off_x = the vector slice's offset
                                  // in dynamic shared memory, after the tile's row sums)
    const int* rbnd;
    const int* meta;
    const unsigned short* col;
    const T* val;
    // two-dimensional tiles (tile = 1; layout in cb_layout.h): R row blocks of
    // rbnd, ncb column blocks, tile g = r * ncb + k on CTA g with chunks
    // [cbeg[g], cbeg[g+1]) of meta; part holds two buffers of nv x ncb x rows
    // partial sums
    int tile, R, rows, nv;
    const int* cbeg;
    T* part;
};

// Sliced ELL with row sorting (SELL-H-sigma) and V lanes per row, H = 32 / V
// rows per slice: element j of the slice's row r sits at ptr[s] + j*H + r,
// so lane q*H + r of a warp reads element t*V + q of row r at
// ptr[s] + 32 t + lane -- every load of a warp is one coalesced 32-element
// segment, and each lane streams its own run of independent loads.
template <typename T>
struct Sell {
    int rows, V, nslices;
    const int* ptr;    // nslices + 1 offsets (multiples of 32)
    const int* col;    // padded column indices
    const T* val;      // padded values (0 in padding)
    const int* perm;   // sorted position -> original row (nslices * H entries, -1 past the end)
    const int* wbnd;   // grid team only: warp w owns slices [wbnd[w], wbnd[w+1]) (nnz-balanced), else null
    Cblk<T> cb;        // grid team only: column-blocked copy (cb.ncb > 0), used instead of the above
    int l1;            // block team: the padded matrix is small enough (48 KB) to keep in L1 across products
};

constexpr int TMA_CH = 8;  // t-steps (of 32 elements) per staged chunk
template <typename T>
__host__ __device__ constexpr int tma_stage_bytes()
{
    return TMA_CH * 32 * (4 + (int)sizeof(T));
}

template <typename T>
struct DevProb {
    int n, m;
    Sell<T> A;   // A   (m rows)
    Sell<T> AT;  // A^T (n rows)
    const T *b, *c;
    double nb, nc;
    int f, l, nq, ns;
    const int* q_off;  // nq+1 row offsets of the SOCs inside s
    const int* s_dim;  // ns PSD orders
    const int* s_off;  // ns row offsets of the PSD blocks inside s
    int ep, ed;        // primal / dual exponential cones (3 rows each)
    int e_off;         // row offset of the first exponential cone inside s
    // PSD blocks above PSD_MAX: the Jacobi workspace of block k starts at psd_big + big_off[k]
    // bytes (laid out by psd_big_ws below; big_off[k] < 0 for blocks decomposed in shared memory)
    unsigned char* psd_big;
    const long long* big_off;
    const long long* v_off;  // byte offset of each PSD block's warm-start eigenvectors in DevWork::psd_v
};

// Iterative refinement of the FP64 linear solves (SCS_MIXED, FP64 phase): the
// FP32 copies of A and A^T and FP32 vectors for the correction solves.
struct IrBufs {
    Sell<float> A, AT;
    float *r, *p, *q, *x;  // n
    float* tm;             // m
};

template <typename T>
struct DevWork {
    IrBufs ir;
    Resume* res;  // loop state handed from the FP32 to the FP64 phase (SCS_MIXED)
    T* chol;      // direct solves: n x n row-major, lower triangle = Cholesky factor of I + A^T A (else null)
    int* chol_fail;  // set by MODE_FACTOR if a pivot was not positive (the factor is then not used)
    HV<T> u, ut, ub, Ru, d, dt, wb, Rw, zp, xip, zt;
    T* g;       // n+m: g = M^{-1}(c, b)
    T* ws[2];   // CG warm starts (n) for the u~ and d~ systems
    T *cr, *cp, *cq, *tn;  // n
    T *tm, *py;            // m
    T* Zv;
    double* Zt;  // mem columns (AA: z^i; RB: z^i)
    T* Xv;
    double* Xt;  // mem columns (AA: xi^i; RB: z~^i)
    T* Qv;
    double* Qt;  // AA with QR: mem orthonormal columns, Xi (oldest first) = Q R
    double *io_in, *io_out, *io_out2;      // N-vectors of the single-operator entries
    double* warm;                          // N: warm start (FP64)
    double *x_out, *y_out, *s_out, *u_out; // results (FP64)
    unsigned char* psd_v;  // PSD blocks: eigenvectors of the last converged decomposition (warm starts)
    int* psd_vok;          // per PSD block: 0 if psd_v holds nothing, else warm-start generations
    double* partials;      // [2][KMAX][blocks] block partials, then [2][KMAX] results
    unsigned* bar;
    int* abort_flag;
    DevState* st;
};

template <typename T>
struct Args {
    DevProb<T> P;
    DevWork<T> W;
    DevSettings S;
    int mode;
    int slot;
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// ---------------------------------------------------------------------------
// sparse products on the sliced-ELL layout: warps of the team take slices in
// turn; xf(c) supplies the gathered vector entry, epi(row, sum) consumes the
// row result (only lanes q = 0 call it)
// ---------------------------------------------------------------------------
// Matrix entries of the sliced-ELL products: streamed past L1 (evict-first in
// L2), except for a block-team instance small enough to stay in L1 across the
// products of its solve (Sell::l1), whose entries are cached there.
template <typename V>
__device__ __forceinline__ V ldm(const V* p, unsigned long long pol, bool l1)
{
    return l1 ? ro(p) : ld_stream(p, pol);
}

template <typename T, class Team, class XF, class Epi>
__device__ __forceinline__ void sell_v(const Team& tm, const Sell<T>& S, XF& xf, Epi& epi)
{
    const int H = 32 / S.V;
    const int lane = threadIdx.x & 31;
    const int nw = tm.size() >> 5;
    const unsigned long long pol = evict_first_policy();
    const bool l1 = !Team::kGrid && S.l1;
    for (int s = tm.rank() >> 5; s < S.nslices; s += nw) {
        const int p0 = ro(S.ptr + s);
        const int tc = (ro(S.ptr + s + 1) - p0) >> 5;
        const int* cp = S.col + p0 + lane;
        const T* vp = S.val + p0 + lane;
        T a0 = 0, a1 = 0;
        int t = 0;
        for (; t + 4 <= tc; t += 4) {
            const int c0 = ldm(cp + 32 * t, pol, l1), c1 = ldm(cp + 32 * (t + 1), pol, l1),
                      c2 = ldm(cp + 32 * (t + 2), pol, l1), c3 = ldm(cp + 32 * (t + 3), pol, l1);
            const T v0 = ldm(vp + 32 * t, pol, l1), v1 = ldm(vp + 32 * (t + 1), pol, l1),
                    v2 = ldm(vp + 32 * (t + 2), pol, l1), v3 = ldm(vp + 32 * (t + 3), pol, l1);
            const T x0 = xf(c0), x1 = xf(c1), x2 = xf(c2), x3 = xf(c3);
            a0 = fmaT(v0, x0, a0);
            a1 = fmaT(v1, x1, a1);
            a0 = fmaT(v2, x2, a0);
            a1 = fmaT(v3, x3, a1);
        }
        for (; t < tc; ++t) a0 += ldm(vp + 32 * t, pol, l1) * xf(ldm(cp + 32 * t, pol, l1));
        T acc = a0 + a1;
        for (int o = H; o < 32; o <<= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
        const int pos = s * H + lane;
        if (lane < H && pos < S.rows) epi(ro(S.perm + pos), acc);
    }
}

template <typename T, class Team, class XF1, class XF2, class Epi>
__device__ __forceinline__ void sell2_v(const Team& tm, const Sell<T>& S, XF1& xf1, XF2& xf2, Epi& epi)
{
    const int H = 32 / S.V;
    const int lane = threadIdx.x & 31;
    const int nw = tm.size() >> 5;
    const unsigned long long pol = evict_first_policy();
    const bool l1 = !Team::kGrid && S.l1;
    for (int s = tm.rank() >> 5; s < S.nslices; s += nw) {
        const int p0 = ro(S.ptr + s);
        const int tc = (ro(S.ptr + s + 1) - p0) >> 5;
        const int* cp = S.col + p0 + lane;
        const T* vp = S.val + p0 + lane;
        T a1 = 0, a2 = 0, b1 = 0, b2 = 0;
        int t = 0;
        for (; t + 2 <= tc; t += 2) {
            const int c0 = ldm(cp + 32 * t, pol, l1), c1 = ldm(cp + 32 * (t + 1), pol, l1);
            const T v0 = ldm(vp + 32 * t, pol, l1), v1 = ldm(vp + 32 * (t + 1), pol, l1);
            a1 += v0 * xf1(c0);
            a2 += v0 * xf2(c0);
            b1 += v1 * xf1(c1);
            b2 += v1 * xf2(c1);
        }
        if (t < tc) {
            const int c0 = ldm(cp + 32 * t, pol, l1);
            const T v0 = ldm(vp + 32 * t, pol, l1);
            a1 += v0 * xf1(c0);
            a2 += v0 * xf2(c0);
        }
        a1 += b1;
        a2 += b2;
        for (int o = H; o < 32; o <<= 1) {
            a1 += __shfl_xor_sync(FULL_MASK, a1, o);
            a2 += __shfl_xor_sync(FULL_MASK, a2, o);
        }
        const int pos = s * H + lane;
        if (lane < H && pos < S.rows) epi(ro(S.perm + pos), a1, a2);
    }
}

// Sparse product with the matrix stream staged through shared memory by TMA
// bulk copies: each warp owns a contiguous, nnz-balanced run of slices,
// copies it in chunks of TMA_CH t-steps into a two-stage buffer (one
// mbarrier per stage) and computes chunk k while chunk k+1 is in flight, so
// the HBM stream never waits on the gathers.  Waits are bounded: on timeout
// the abort flag is set, the warp waits (bounded) for its other copy and
// leaves the product unfinished.
template <typename T, class Team, class XF, class Epi>
__device__ __forceinline__ void sell_tma(const Team& tm, const Sell<T>& S, XF& xf, Epi& epi)
{
    const int H = 32 / S.V;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = tm.rank() >> 5;
    const int s0 = ro(S.wbnd + gw), s1 = ro(S.wbnd + gw + 1);
    if (s0 >= s1) return;
    const int e0 = ro(S.ptr + s0);
    const int total_t = (ro(S.ptr + s1) - e0) >> 5;
    constexpr int SB = tma_stage_bytes<T>();
    unsigned char* wbuf = tm.stage + (size_t)wib * 2 * SB;
    const unsigned bar0 = smem_addr(&tm.mbar[2 * wib]), bar1 = smem_addr(&tm.mbar[2 * wib + 1]);
    unsigned ph = tm.ph[wib];
    const unsigned long long pol = evict_first_policy();
    const int nch = (total_t + TMA_CH - 1) / TMA_CH;
    auto issue = [&](int k) {
        const int t_lo = k * TMA_CH;
        const int nt = min(TMA_CH, total_t - t_lo);
        unsigned char* dst = wbuf + (k & 1) * SB;
        const unsigned bar = (k & 1) ? bar1 : bar0;
        const unsigned bc = (unsigned)nt * 32u * 4u, bv = (unsigned)nt * 32u * (unsigned)sizeof(T);
        fence_proxy_async();
        mbar_expect_tx(bar, bc + bv);
        tma_load_1d(smem_addr(dst), S.col + e0 + 32 * t_lo, bc, bar, pol);
        tma_load_1d(smem_addr(dst + TMA_CH * 32 * 4), S.val + e0 + 32 * t_lo, bv, bar, pol);
    };
    auto finalize = [&](int sl, T a) {
        for (int o = H; o < 32; o <<= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
        const int pos = sl * H + lane;
        if (lane < H && pos < S.rows) epi(ro(S.perm + pos), a);
    };
    if (nch > 0 && lane == 0) issue(0);
    int cur = s0;
    int bound = (ro(S.ptr + cur + 1) - e0) >> 5;
    T acc = 0;
    for (int k = 0; k < nch; ++k) {
        const bool more = k + 1 < nch;
        if (more) {
            __syncwarp();
            if (lane == 0) issue(k + 1);
        }
        const unsigned bar = (k & 1) ? bar1 : bar0;
        bool ok = mbar_wait(bar, (ph >> (k & 1)) & 1u, tm.abort_flag);
        ok = __all_sync(FULL_MASK, ok);
        ph ^= 1u << (k & 1);
        if (!ok) {
            if (more) {
                const unsigned obar = (k & 1) ? bar0 : bar1;
                mbar_wait(obar, (ph >> ((k + 1) & 1)) & 1u, nullptr);
                ph ^= 1u << ((k + 1) & 1);
            }
            if (lane == 0) tm.ph[wib] = ph;
            __syncwarp();
            return;
        }
        const int t_lo = k * TMA_CH;
        const int nt = min(TMA_CH, total_t - t_lo);
        const int* sc = (const int*)(wbuf + (k & 1) * SB);
        const T* sv = (const T*)(wbuf + (k & 1) * SB + TMA_CH * 32 * 4);
        int cs[TMA_CH];
        T vs[TMA_CH], xs[TMA_CH];
#pragma unroll
        for (int t = 0; t < TMA_CH; ++t) {
            cs[t] = t < nt ? sc[t * 32 + lane] : 0;
            vs[t] = t < nt ? sv[t * 32 + lane] : T(0);
        }
#pragma unroll
        for (int t = 0; t < TMA_CH; ++t) xs[t] = xf(cs[t]);
#pragma unroll
        for (int t = 0; t < TMA_CH; ++t) {
            if (t < nt) {
                const int tg = t_lo + t;
                while (tg == bound) {
                    finalize(cur, acc);
                    acc = 0;
                    ++cur;
                    bound = (ro(S.ptr + cur + 1) - e0) >> 5;
                }
                acc = fmaT(vs[t], xs[t], acc);
            }
        }
    }
    while (cur < s1) {
        finalize(cur, acc);
        acc = 0;
        ++cur;
    }
    if (lane == 0) tm.ph[wib] = ph;
    __syncwarp();
}

// ---------------------------------------------------------------------------
// column-blocked product (grid team): y = M x (NV = 1) or M x1, M x2 (NV = 2)
// ---------------------------------------------------------------------------

// One segment from its stage: compute warp w runs its slices (matrix
// entries, the vector slice and the metadata all in shared memory); row sums
// are reduced over the V = 32 / H lanes of a row and added to acc (rows of a
// segment are distinct, so plain read-modify-writes do not race).  Operands
// are byte offsets into the dynamic shared memory, indexed through the
// shared array itself so the loads are 32-bit-addressed shared loads and the
// hot loop touches no local memory.
template <typename T>
__device__ __forceinline__ void cb_segment(int nw, int H, unsigned mt_off, unsigned xs_off, unsigned col_off,
                                           unsigned val_off, unsigned acc_off)
{
    extern __shared__ __align__(128) unsigned char cb_sm[];
    const int* mt = (const int*)(cb_sm + mt_off);
    const T* xs = (const T*)(cb_sm + xs_off);
    const unsigned short* scol = (const unsigned short*)(cb_sm + col_off);
    const T* sval = (const T*)(cb_sm + val_off);
    T* acc = (T*)(cb_sm + acc_off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ns = mt[4];
    const int* wl = mt + 5;
    const int* st = wl + nw + 1;
    const unsigned short* sr = (const unsigned short*)(st + ns + 1);
    const int s_hi = wl[w + 1];
    int s0 = wl[w];
    if constexpr (sizeof(T) == 4) {
        // FP32, two slices at a time: their steps interleave four by four, so a warp keeps
        // eight independent offset -> gather -> FMA chains in flight instead of four (the
        // slices are short: about six steps at the benchmark's row lengths)
        for (; s0 + 1 < s_hi; s0 += 2) {
            int ta = st[s0];
            const int ta1 = st[s0 + 1];
            int tb = ta1;
            const int tb1 = st[s0 + 2];
            T a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
            for (; ta < ta1 || tb < tb1; ta += 4, tb += 4) {
                const bool p0 = ta < ta1, p1 = ta + 1 < ta1, p2 = ta + 2 < ta1, p3 = ta + 3 < ta1;
                const bool q0 = tb < tb1, q1 = tb + 1 < tb1, q2 = tb + 2 < tb1, q3 = tb + 3 < tb1;
                const int c0 = p0 ? (int)scol[ta * 32 + lane] : 0;
                const int c1 = p1 ? (int)scol[ta * 32 + 32 + lane] : 0;
                const int c2 = p2 ? (int)scol[ta * 32 + 64 + lane] : 0;
                const int c3 = p3 ? (int)scol[ta * 32 + 96 + lane] : 0;
                const int d0 = q0 ? (int)scol[tb * 32 + lane] : 0;
                const int d1 = q1 ? (int)scol[tb * 32 + 32 + lane] : 0;
                const int d2 = q2 ? (int)scol[tb * 32 + 64 + lane] : 0;
                const int d3 = q3 ? (int)scol[tb * 32 + 96 + lane] : 0;
                const T v0 = p0 ? sval[ta * 32 + lane] : T(0);
                const T v1 = p1 ? sval[ta * 32 + 32 + lane] : T(0);
                const T v2 = p2 ? sval[ta * 32 + 64 + lane] : T(0);
                const T v3 = p3 ? sval[ta * 32 + 96 + lane] : T(0);
                const T u0 = q0 ? sval[tb * 32 + lane] : T(0);
                const T u1 = q1 ? sval[tb * 32 + 32 + lane] : T(0);
                const T u2 = q2 ? sval[tb * 32 + 64 + lane] : T(0);
                const T u3 = q3 ? sval[tb * 32 + 96 + lane] : T(0);
                a0 = fmaT(v0, xs[c0], a0);
                a1 = fmaT(v1, xs[c1], a1);
                a2 = fmaT(v2, xs[c2], a2);
                a3 = fmaT(v3, xs[c3], a3);
                b0 = fmaT(u0, xs[d0], b0);
                b1 = fmaT(u1, xs[d1], b1);
                b2 = fmaT(u2, xs[d2], b2);
                b3 = fmaT(u3, xs[d3], b3);
            }
            T a = (a0 + a2) + (a1 + a3), b = (b0 + b2) + (b1 + b3);
            for (int o = H; o < 32; o <<= 1) {
                a += __shfl_xor_sync(FULL_MASK, a, o);
                b += __shfl_xor_sync(FULL_MASK, b, o);
            }
            if (lane < H) {
                const int ra = sr[s0 * H + lane], rb = sr[(s0 + 1) * H + lane];
                if (ra != 0xFFFF) acc[ra] += a;
                if (rb != 0xFFFF) acc[rb] += b;
            }
        }
    }
    for (int s = s0; s < s_hi; ++s) {
        const int t1 = st[s + 1];
        int t = st[s];
        T a0 = 0, a1 = 0;
        if constexpr (sizeof(T) == 4) {
            // FP32: four steps per trip, the tail predicated (offset 0, value 0)
            T a2 = 0, a3 = 0;
            for (; t < t1; t += 4) {
                const bool o1 = t + 1 < t1, o2 = t + 2 < t1, o3 = t + 3 < t1;
                const int c0 = scol[t * 32 + lane];
                const int c1 = o1 ? (int)scol[t * 32 + 32 + lane] : 0;
                const int c2 = o2 ? (int)scol[t * 32 + 64 + lane] : 0;
                const int c3 = o3 ? (int)scol[t * 32 + 96 + lane] : 0;
                const T v0 = sval[t * 32 + lane];
                const T v1 = o1 ? sval[t * 32 + 32 + lane] : T(0);
                const T v2 = o2 ? sval[t * 32 + 64 + lane] : T(0);
                const T v3 = o3 ? sval[t * 32 + 96 + lane] : T(0);
                a0 = fmaT(v0, xs[c0], a0);
                a1 = fmaT(v1, xs[c1], a1);
                a2 = fmaT(v2, xs[c2], a2);
                a3 = fmaT(v3, xs[c3], a3);
            }
            a0 += a2;
            a1 += a3;
        } else {
            for (; t + 2 <= t1; t += 2) {
                const int c0 = scol[t * 32 + lane], c1 = scol[t * 32 + 32 + lane];
                const T v0 = sval[t * 32 + lane], v1 = sval[t * 32 + 32 + lane];
                a0 = fmaT(v0, xs[c0], a0);
                a1 = fmaT(v1, xs[c1], a1);
            }
            if (t < t1) a0 = fmaT(sval[t * 32 + lane], xs[scol[t * 32 + lane]], a0);
        }
        T a = a0 + a1;
        for (int o = H; o < 32; o <<= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
        if (lane < H) {
            const int r = sr[s * H + lane];
            if (r != 0xFFFF) acc[r] += a;
        }
    }
}

// acc[0, R) + acc[acc_rows, acc_rows + R) = (rows of this CTA's range) . x
// over all column blocks (even segments into the first buffer, odd into the
// second), through the ring of S stages: full barriers tm.mbar[0..S-1], empty
// barriers tm.mbar[CB_MAX_STAGES + s]; tm.ph[s] counts the stage's past uses,
// so use u of this pass waits on parity (ph[s] + u) & 1.  Every field the
// loops need is read once into registers (the structs live in local memory,
// which misses the small L1 left beside the stages).  Returns false if a wait
// ran out of time (the abort flag is then set and the copies still in
// flight are waited for, bounded, before returning).
template <typename T>
__device__ bool cb_pass(const GridTeam& tm, const Cblk<T>& C, const T* x, T* acc, unsigned long long pol)
{
    constexpr int E = 16 / (int)sizeof(T);
    const int S = C.S, ncb = C.ncb, nw = C.nw, H = 32 / C.V, ms = C.ms, cw = C.cw, cols = C.cols;
    const int off_x = C.off_x, off_col = C.off_col, off_val = C.off_val, ar = C.acc_rows;
    const int* meta = C.meta;
    const unsigned short* gcol = C.col;
    const T* gval = C.val;
    unsigned char* const tm_dsm = tm.dsm;
    unsigned char* st0 = tm_dsm + C.stage_off;
    const unsigned acc_off = (unsigned)((unsigned char*)acc - tm_dsm);
    const int stage_bytes = C.stage_bytes;
    unsigned long long* mbar = tm.mbar;
    unsigned* ph = tm.ph;
    int* abort_flag = tm.abort_flag;
    const int g0 = blockIdx.x * ncb;
    const int k0 = blockIdx.x % ncb;  // first column block of this CTA
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mis = (int)(((uintptr_t)x & 15) / sizeof(T));
    auto stage = [=](int s) { return st0 + (size_t)s * stage_bytes; };
    auto full = [=](int s) { return smem_addr(&mbar[s]); };
    auto empty = [=](int s) { return smem_addr(&mbar[CB_MAX_STAGES + s]); };
    auto blk = [=](int j) { return (k0 + j) % ncb; };  // column block of the j-th segment visited
    __syncthreads();  // stages free, acc zeroed, ph current
    bool ok = true;
    int issued = 0;
    if (w == nw) {
        // producer warp: lane 0 issues every copy
        if (lane == 0) {
            auto issue = [=](int j, int e0, int e1) {
                const int s = j % S, k = blk(j);
                unsigned char* d = stage(s);
                const int len = min(cw, cols - k * cw);
                const unsigned xb = (unsigned)((mis + len + E - 1) / E) * 16u;
                const unsigned ne = (unsigned)(e1 - e0);
                const unsigned mb = (unsigned)ms * 4u;
                mbar_expect_tx(full(s), mb + xb + ne * (2u + (unsigned)sizeof(T)));
                tma_load_1d_plain(smem_addr(d), meta + (size_t)(g0 + k) * ms, mb, full(s));
                tma_load_1d_plain(smem_addr(d + off_x), x + (size_t)k * cw - mis, xb, full(s));
                if (ne) {
                    tma_load_1d(smem_addr(d + off_col), gcol + e0, ne * 2u, full(s), pol);
                    tma_load_1d(smem_addr(d + off_val), gval + e0, ne * (unsigned)sizeof(T), full(s), pol);
                }
            };
            // x was written by generic stores (other CTAs, before the last
            // grid barrier) and is read here by the async proxy
            fence_proxy_async_all();
            const int npro = min(S, ncb);
            int e0a = 0, e1a = 0, e0b = 0, e1b = 0, e0c = 0, e1c = 0, e0d = 0, e1d = 0;
            e0a = ro(meta + (size_t)(g0 + blk(0)) * ms);
            e1a = ro(meta + (size_t)(g0 + blk(0)) * ms + 1);
            if (npro > 1) {
                e0b = ro(meta + (size_t)(g0 + blk(1)) * ms);
                e1b = ro(meta + (size_t)(g0 + blk(1)) * ms + 1);
            }
            if (npro > 2) {
                e0c = ro(meta + (size_t)(g0 + blk(2)) * ms);
                e1c = ro(meta + (size_t)(g0 + blk(2)) * ms + 1);
            }
            if (npro > 3) {
                e0d = ro(meta + (size_t)(g0 + blk(3)) * ms);
                e1d = ro(meta + (size_t)(g0 + blk(3)) * ms + 1);
            }
            issue(0, e0a, e1a);
            if (npro > 1) issue(1, e0b, e1b);
            if (npro > 2) issue(2, e0c, e1c);
            if (npro > 3) issue(3, e0d, e1d);
            issued = npro;
            for (int j = S; j < ncb; ++j) {
                const int s = j % S;
                if (!mbar_wait(empty(s), (ph[s] + j / S - 1) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                // the stage's header names the segment visited S after its own
                const int* h = (const int*)stage(s);
                const int ne0 = h[2], ne1 = h[3];
                fence_proxy_async();  // the stage was read through the generic proxy
                issue(j, ne0, ne1);
                issued = j + 1;
            }
        }
    } else {
        for (int j = 0; j < ncb; ++j) {
            const int s = j % S;
            if (!mbar_wait(full(s), (ph[s] + j / S) & 1u, abort_flag)) {
                ok = false;
                break;
            }
            if (j >= 2) {  // every warp is done with segment j-2 (same partial-sum buffer)
                const int s2 = (j - 2) % S;
                if (!mbar_wait(empty(s2), (ph[s2] + (j - 2) / S) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
            }
            const unsigned so = (unsigned)(stage(s) - tm_dsm);
            cb_segment<T>(nw, H, so, so + off_x + mis * (unsigned)sizeof(T), so + off_col, so + off_val,
                          acc_off + (unsigned)((j & 1) * ar * (int)sizeof(T)));
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
        }
    }
    const bool all_ok = __syncthreads_and(ok);
    if (!all_ok && w == nw && lane == 0) {
        // copies of the last S issued segments may still be in flight
        for (int j = max(0, issued - S); j < issued; ++j) mbar_wait(full(j % S), (ph[j % S] + j / S) & 1u, nullptr);
    }
    __syncthreads();  // everyone has read ph for this pass
    if (threadIdx.x == 0 && all_ok)
        for (int s = 0; s < S; ++s) ph[s] += (unsigned)((ncb - s + S - 1) / S);
    return all_ok;
}

// The product: one pass per multiplied vector (NV = 2: x1 into acc1, then x2
// into acc2), then epi(row, sum) (or epi(row, sum1, sum2)) for every row of
// the CTA's range.
template <typename T, int NV, class Epi>
__device__ void cb_spmv(const GridTeam& tm, const Cblk<T>& C, const T* x1, const T* x2, Epi& epi)
{
    const int b = blockIdx.x;
    const int r0 = ro(C.rbnd + b), R = ro(C.rbnd + b + 1) - r0;
    const int ar = C.acc_rows;
    T* acc1 = (T*)tm.dsm;      // two buffers of ar
    T* acc2 = acc1 + 2 * ar;   // two more for the second vector
    const unsigned long long pol = evict_first_policy();
    __syncthreads();  // shared memory is free (earlier users done)
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        acc1[r] = 0;
        acc1[ar + r] = 0;
        if constexpr (NV == 2) {
            acc2[r] = 0;
            acc2[ar + r] = 0;
        }
    }
    if (!cb_pass<T>(tm, C, x1, acc1, pol)) return;
    if constexpr (NV == 2) {
        if (!cb_pass<T>(tm, C, x2, acc2, pol)) return;
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        if constexpr (NV == 1)
            epi(r0 + r, acc1[r] + acc1[ar + r]);
        else
            epi(r0 + r, acc1[r] + acc1[ar + r], acc2[r] + acc2[ar + r]);
    }
}

// ---------------------------------------------------------------------------
// two-dimensional tiled product (grid team): y = M x (NV = 1) or M x1, M x2
// ---------------------------------------------------------------------------

// One chunk from its stage: compute warp w runs its slices against the
// resident vector slice xs; each row's sum (reduced over its V lanes) is
// final and is stored to the tile's row array at the start of dynamic shared
// memory (every row of a tile lies in exactly one slice, so the stores never
// meet).
template <typename T>
__device__ __forceinline__ void tile_chunk(int nw, int H, unsigned mt_off, unsigned xs_off, unsigned col_off,
                                           unsigned val_off)
{
    extern __shared__ __align__(128) unsigned char cb_sm[];
    const int* mt = (const int*)(cb_sm + mt_off);
    const T* xs = (const T*)(cb_sm + xs_off);
    const unsigned short* scol = (const unsigned short*)(cb_sm + col_off);
    const T* sval = (const T*)(cb_sm + val_off);
    T* acc = (T*)cb_sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ns = mt[4];
    const int* wl = mt + 5;
    const int* st = wl + nw + 1;
    const unsigned short* sr = (const unsigned short*)(st + ns + 1);
    const int s_hi = wl[w + 1];
    for (int s = wl[w]; s < s_hi; ++s) {
        const int t1 = st[s + 1];
        int t = st[s];
        T a0 = 0, a1 = 0;
        if constexpr (sizeof(T) == 4) {
            // four steps per trip, the tail predicated (offset 0, value 0)
            T a2 = 0, a3 = 0;
            for (; t < t1; t += 4) {
                const bool o1 = t + 1 < t1, o2 = t + 2 < t1, o3 = t + 3 < t1;
                const int c0 = scol[t * 32 + lane];
                const int c1 = o1 ? (int)scol[t * 32 + 32 + lane] : 0;
                const int c2 = o2 ? (int)scol[t * 32 + 64 + lane] : 0;
                const int c3 = o3 ? (int)scol[t * 32 + 96 + lane] : 0;
                const T v0 = sval[t * 32 + lane];
                const T v1 = o1 ? sval[t * 32 + 32 + lane] : T(0);
                const T v2 = o2 ? sval[t * 32 + 64 + lane] : T(0);
                const T v3 = o3 ? sval[t * 32 + 96 + lane] : T(0);
                a0 = fmaT(v0, xs[c0], a0);
                a1 = fmaT(v1, xs[c1], a1);
                a2 = fmaT(v2, xs[c2], a2);
                a3 = fmaT(v3, xs[c3], a3);
            }
            a0 += a2;
            a1 += a3;
        } else {
            for (; t + 2 <= t1; t += 2) {
                const int c0 = scol[t * 32 + lane], c1 = scol[t * 32 + 32 + lane];
                const T v0 = sval[t * 32 + lane], v1 = sval[t * 32 + 32 + lane];
                a0 = fmaT(v0, xs[c0], a0);
                a1 = fmaT(v1, xs[c1], a1);
            }
            if (t < t1) a0 = fmaT(sval[t * 32 + lane], xs[scol[t * 32 + lane]], a0);
        }
        T a = a0 + a1;
        for (int o = H; o < 32; o <<= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
        if (lane < H) {
            const int r = sr[s * H + lane];
            if (r != 0xFFFF) acc[r] = a;
        }
    }
}

// This CTA's tile of M x: the vector slice is copied once (completing on
// mbarrier 2 CB_MAX_STAGES, its uses counted in ph[CB_MAX_STAGES]), the
// chunks stream through the ring of S stages as the column-blocked segments
// do (full barriers tm.mbar[0..S-1], empty barriers tm.mbar[CB_MAX_STAGES +
// s]), the row sums collect in shared memory and go to part[k][rows of the
// block] at the end.  Returns false if a wait ran out of time (the abort
// flag is then set and the copies still in flight are waited for, bounded,
// before returning).
template <typename T>
__device__ bool tile_pass(const GridTeam& tm, const Cblk<T>& C, const T* x, T* part, unsigned long long pol)
{
    constexpr int E = 16 / (int)sizeof(T);
    const int S = C.S, ncb = C.ncb, nw = C.nw, H = 32 / C.V, ms = C.ms, cw = C.cw, cols = C.cols, rows = C.rows;
    const int off_col = C.off_col, off_val = C.off_val, stage_bytes = C.stage_bytes, off_x = C.off_x;
    const int* meta = C.meta;
    const unsigned short* gcol = C.col;
    const T* gval = C.val;
    unsigned char* const dsm = tm.dsm;
    unsigned char* st0 = dsm + C.stage_off;
    unsigned long long* mbar = tm.mbar;
    unsigned* ph = tm.ph;
    int* abort_flag = tm.abort_flag;
    const int g = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (g >= C.R * ncb) return true;  // no tile on this CTA (uniform in the CTA)
    const int r = g / ncb, k = g % ncb;
    const int r0 = ro(C.rbnd + r), Rr = ro(C.rbnd + r + 1) - r0;
    const int c0 = ro(C.cbeg + g), nch = ro(C.cbeg + g + 1) - c0;
    const int mis = (int)(((uintptr_t)x & 15) / sizeof(T));
    T* acc = (T*)dsm;
    auto stage = [=](int s) { return st0 + (size_t)s * stage_bytes; };
    auto full = [=](int s) { return smem_addr(&mbar[s]); };
    auto empty = [=](int s) { return smem_addr(&mbar[CB_MAX_STAGES + s]); };
    const unsigned xbar = smem_addr(&mbar[2 * CB_MAX_STAGES]);
    __syncthreads();  // shared memory free (earlier users done), ph current
    for (int i = threadIdx.x; i < Rr; i += blockDim.x) acc[i] = 0;
    __syncthreads();  // the row sums are zero before any warp stores one
    bool ok = true;
    int issued = 0;
    if (nch > 0) {
        if (w == nw) {
            // producer warp: lane 0 issues every copy
            if (lane == 0) {
                auto issue = [=](int j, int e0, int e1) {
                    const int s = j % S;
                    unsigned char* d = stage(s);
                    const unsigned ne = (unsigned)(e1 - e0);
                    const unsigned mb = (unsigned)ms * 4u;
                    mbar_expect_tx(full(s), mb + ne * (2u + (unsigned)sizeof(T)));
                    tma_load_1d_plain(smem_addr(d), meta + (size_t)(c0 + j) * ms, mb, full(s));
                    if (ne) {
                        tma_load_1d(smem_addr(d + off_col), gcol + e0, ne * 2u, full(s), pol);
                        tma_load_1d(smem_addr(d + off_val), gval + e0, ne * (unsigned)sizeof(T), full(s), pol);
                    }
                };
                // x was written by generic stores (other CTAs, before the last
                // grid barrier) and is read here by the async proxy
                fence_proxy_async_all();
                const int len = min(cw, cols - k * cw);
                const unsigned xb = (unsigned)((mis + len + E - 1) / E) * 16u;
                mbar_expect_tx(xbar, xb);
                tma_load_1d_plain(smem_addr(dsm + off_x), x + (size_t)k * cw - mis, xb, xbar);
                const int npro = min(S, nch);
                for (int j = 0; j < npro; ++j)
                    issue(j, ro(meta + (size_t)(c0 + j) * ms), ro(meta + (size_t)(c0 + j) * ms + 1));
                issued = npro;
                for (int j = S; j < nch; ++j) {
                    const int s = j % S;
                    if (!mbar_wait(empty(s), (ph[s] + j / S - 1) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    // the stage's header names the chunk S after its own
                    const int* h = (const int*)stage(s);
                    const int ne0 = h[2], ne1 = h[3];
                    fence_proxy_async();  // the stage was read through the generic proxy
                    issue(j, ne0, ne1);
                    issued = j + 1;
                }
            }
        } else {
            if (!mbar_wait(xbar, ph[CB_MAX_STAGES] & 1u, abort_flag)) ok = false;
            for (int j = 0; ok && j < nch; ++j) {
                const int s = j % S;
                if (!mbar_wait(full(s), (ph[s] + j / S) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const unsigned so = (unsigned)(stage(s) - dsm);
                tile_chunk<T>(nw, H, so, (unsigned)off_x + mis * (unsigned)sizeof(T), so + off_col, so + off_val);
                __syncwarp();
                if (lane == 0) mbar_arrive(empty(s));
            }
        }
    }
    const bool all_ok = __syncthreads_and(ok);
    if (!all_ok && w == nw && lane == 0 && nch > 0) {
        // the slice copy and the copies of the last S issued chunks may still be in flight
        mbar_wait(xbar, ph[CB_MAX_STAGES] & 1u, nullptr);
        for (int j = max(0, issued - S); j < issued; ++j) mbar_wait(full(j % S), (ph[j % S] + j / S) & 1u, nullptr);
    }
    __syncthreads();  // everyone has read ph for this pass
    if (threadIdx.x == 0 && nch > 0) {
        for (int s = 0; s < S; ++s) ph[s] += (unsigned)((nch - s + S - 1) / S);
        ph[CB_MAX_STAGES] += 1u;
    }
    if (!all_ok) return false;
    T* out = part + (size_t)k * rows + r0;
    for (int i = threadIdx.x; i < Rr; i += blockDim.x) out[i] = acc[i];
    return true;
}

// The tiled product: one tile pass per vector into its partial sums, a grid
// barrier, then epi(row, sum) (or epi(row, sum1, sum2)) for every row, the
// sum over the column blocks taken in block order (deterministic), rows dealt
// like the team's vector loops.  The partial sums alternate between two
// buffers by the parity of the barrier count at entry: the next product of
// this matrix either starts one barrier later (the other buffer) or after a
// barrier that every CTA reaches only once it has read this one.
template <typename T, int NV, class Epi>
__device__ void tile_spmv(GridTeam& tm, const Cblk<T>& C, const T* x1, const T* x2, Epi& epi)
{
    const unsigned long long pol = evict_first_policy();
    const int rows = C.rows, ncb = C.ncb;
    T* part = C.part + (size_t)(tm.epoch & 1ull) * C.nv * ncb * rows;
    if (!tile_pass<T>(tm, C, x1, part, pol)) return;
    if constexpr (NV == 2) {
        if (!tile_pass<T>(tm, C, x2, part + (size_t)ncb * rows, pol)) return;
    }
    tm.sync();
    for (int i = tm.rank(); i < rows; i += tm.size()) {
        T s1 = 0;
        for (int k = 0; k < ncb; ++k) s1 += part[(size_t)k * rows + i];
        if constexpr (NV == 1) {
            epi(i, s1);
        } else {
            T s2 = 0;
            for (int k = 0; k < ncb; ++k) s2 += part[(size_t)(ncb + k) * rows + i];
            epi(i, s1, s2);
        }
    }
}

template <typename T, class Team, class XF, class Epi>
__device__ __forceinline__ void spmv_f(const Team& tm, const Sell<T>& S, XF xf, Epi epi)
{
    if (S.wbnd != nullptr && tm.stage != nullptr)
        sell_tma(tm, S, xf, epi);
    else
        sell_v(tm, S, xf, epi);
}

template <typename T, class Team, class Epi>
__device__ __forceinline__ void spmv(Team& tm, const Sell<T>& S, const T* x, Epi epi)
{
    if constexpr (Team::kGrid) {
        if (S.cb.ncb > 0) {
            if (S.cb.tile)
                tile_spmv<T, 1>(tm, S.cb, x, x, epi);
            else
                cb_spmv<T, 1>(tm, S.cb, x, x, epi);
            return;
        }
    }
    auto f = [x](int c) { return x[c]; };
    spmv_f(tm, S, f, epi);
}

template <typename T, class Team, class Epi>
__device__ __forceinline__ void spmv2(Team& tm, const Sell<T>& S, const T* x1, const T* x2, Epi epi)
{
    if constexpr (Team::kGrid) {
        if (S.cb.ncb > 0) {
            if (S.cb.tile)
                tile_spmv<T, 2>(tm, S.cb, x1, x2, epi);
            else
                cb_spmv<T, 2>(tm, S.cb, x1, x2, epi);
            return;
        }
    }
    auto f1 = [x1](int c) { return x1[c]; };
    auto f2 = [x2](int c) { return x2[c]; };
    sell2_v(tm, S, f1, f2, epi);
}

// ---------------------------------------------------------------------------
// CG on (I + A^T A) x = rhs from the residual r = rhs - (I + A^T A) x of the
// start x, rr = ||r||^2 (already reduced), stopping at ||r|| <= tol or after
// cg_max iterations.  One reduction per iteration: <p,q>, <r,q>, <q,q> are
// reduced together, ||r - alpha q||^2 = rr - 2 alpha <r,q> + alpha^2 <q,q>
// gives beta, and x, r, p are updated in one pass; the exact ||r||^2 of the
// updated r rides along with the next reduction and replaces the recurrence
// value before it is used for alpha.  Returns the iterations.
// ---------------------------------------------------------------------------
template <typename T>
struct CgBufs {
    T *r, *p, *q;  // n
    T* tm;         // m
};

template <typename T, class Team>
__device__ int cg_loop(Team& tm, const Sell<T>& A, const Sell<T>& AT, int n, CgBufs<T> b, T* x, double rr,
                       double tol, int cg_max)
{
    T* p = b.p;
    T* q = b.q;
    T* r = b.r;
    T* tmv = b.tm;
    for (int j = tm.rank(); j < n; j += tm.size()) p[j] = r[j];
    tm.sync();
    int it = 0;
    T rr_part = 0;
    bool have_part = false;
    while (it < cg_max) {
        if (tm.aborted()) break;
        spmv(tm, A, p, [&](int i, T s) { tmv[i] = s; });
        tm.sync();
        T pq = 0, rq = 0, qq = 0;
        spmv(tm, AT, tmv, [&](int j, T s) {
            const T qj = p[j] + s;
            q[j] = qj;
            pq += p[j] * qj;
            rq += r[j] * qj;
            qq += qj * qj;
        });
        double red[4] = {(double)pq, (double)rq, (double)qq, (double)rr_part};
        tm.reduce(red);
        ++it;
        // The scalar step (two FP64 divisions, a square root) is evaluated by
        // one thread per CTA and handed to the others through shared memory:
        // the FP64 pipe is a small fraction of the FP32 one, and every thread
        // of every warp evaluating it costs more than the extra CTA barrier.
        // The values are the same bits either way (rr lives in thread 0).
        double* bc = tm.bcast();
        if (threadIdx.x == 0) {
            if (have_part) rr = red[3];
            const double alpha = rr / red[0];
            double rr_new = rr - 2.0 * alpha * red[1] + alpha * alpha * red[2];
            if (rr_new < 0.0) rr_new = 0.0;
            reinterpret_cast<T*>(bc)[0] = (T)alpha;
            reinterpret_cast<T*>(bc)[1] = (T)(rr_new / rr);
            reinterpret_cast<int*>(bc + 2)[0] = (!(sqrt(rr_new) > tol) || it >= cg_max) ? 1 : 0;
            rr = rr_new;
        }
        __syncthreads();
        const T ta = reinterpret_cast<const T*>(bc)[0];
        const T tb = reinterpret_cast<const T*>(bc)[1];
        const bool done = reinterpret_cast<const int*>(bc + 2)[0] != 0;
        rr_part = 0;
        if (done) {
            for (int j = tm.rank(); j < n; j += tm.size()) x[j] += ta * p[j];
        } else {
            for (int j = tm.rank(); j < n; j += tm.size()) {
                const T pj = p[j];
                x[j] += ta * pj;
                const T rj = r[j] - ta * q[j];
                r[j] = rj;
                p[j] = rj + tb * pj;
                rr_part += rj * rj;
            }
        }
        have_part = true;
        tm.sync();
        if (done) break;
    }
    return it;
}

// ---------------------------------------------------------------------------
// Direct solves of (I + A^T A) x = b (the "direct" alternative Sec. 4.1 names
// beside CG), for one CTA per instance: the matrix is formed column by column
// as e_j + A^T (A e_j) with the solver's own sparse products, factored
// L L^T in place (right-looking, one column per step), and each solve is a
// forward and a backward substitution in blocks of 32: warp 0 solves the
// 32 x 32 diagonal block with shuffles, then the whole CTA updates the rows
// outside it (two CTA barriers per block).
// ---------------------------------------------------------------------------
constexpr int CHOL_B = 32;

template <typename T, class Team>
__device__ void chol_factor(Team& tm, const DevProb<T>& P, const DevWork<T>& W)
{
    const int n = P.n;
    T* L = W.chol;
    T* ej = W.cp;
    T* y = W.tm;
    for (int j = 0; j < n; ++j) {
        for (int i = tm.rank(); i < n; i += tm.size()) ej[i] = i == j ? T(1) : T(0);
        tm.sync();
        spmv(tm, P.A, ej, [&](int i, T v) { y[i] = v; });
        tm.sync();
        spmv(tm, P.AT, y, [&](int i, T v) {
            if (i >= j) L[(size_t)i * n + j] = v + (i == j ? T(1) : T(0));
        });
        tm.sync();
    }
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const T djj = L[(size_t)j * n + j];
            if (!(djj > T(0))) bad = 1;
            L[(size_t)j * n + j] = djj > T(0) ? sqrt(djj) : T(1);
        }
        __syncthreads();
        const T d = L[(size_t)j * n + j];
        for (int i = j + 1 + tm.rank(); i < n; i += tm.size()) L[(size_t)i * n + j] /= d;
        __syncthreads();
        const int r = n - j - 1;
        for (long long idx = tm.rank(); idx < (long long)r * r; idx += tm.size()) {
            const int ii = j + 1 + (int)(idx / r), kk = j + 1 + (int)(idx % r);
            if (kk <= ii) L[(size_t)ii * n + kk] -= L[(size_t)ii * n + j] * L[(size_t)kk * n + j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) atomicExch(W.chol_fail, 1);
    __syncthreads();
}

// b (n, in place) <- (L L^T)^{-1} b.  dg: CHOL_B x CHOL_B values of shared
// memory for the diagonal block, loaded by the whole CTA with coalesced reads
// before warp 0 solves it; element (r, c) sits at r CHOL_B + (c xor r), so the
// lanes of a warp reading one column, or one row, hit distinct banks.  zb:
// CHOL_B values of shared memory.
template <typename T, class Team>
__device__ void chol_solve(Team& tm, const T* L, int n, T* b, T* dg, T* zb)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto D = [&](int r, int c) -> T& { return dg[r * CHOL_B + (c ^ r)]; };
    auto load_diag = [&](int jb, int w) {
        __syncthreads();  // the previous block's readers are done
        for (int idx = threadIdx.x; idx < w * CHOL_B; idx += blockDim.x) {
            const int r = idx / CHOL_B, c = idx % CHOL_B;
            D(r, c) = c < w ? L[(size_t)(jb + r) * n + jb + c] : T(0);
        }
        __syncthreads();
    };
    // forward: L z = b
    for (int jb = 0; jb < n; jb += CHOL_B) {
        const int w = min(CHOL_B, n - jb);
        load_diag(jb, w);
        if (warp == 0) {
            T v = lane < w ? b[jb + lane] : T(0);
            for (int c = 0; c < w; ++c) {
                const T zc = __shfl_sync(FULL_MASK, v, c) / D(c, c);
                if (lane == c) v = zc;
                if (lane > c && lane < w) v -= D(lane, c) * zc;
            }
            if (lane < w) {
                b[jb + lane] = v;
                zb[lane] = v;
            }
        }
        __syncthreads();
        for (int i = jb + w + tm.rank(); i < n; i += tm.size()) {
            T acc = b[i];
            const T* row = L + (size_t)i * n + jb;
            for (int c = 0; c < w; ++c) acc -= row[c] * zb[c];
            b[i] = acc;
        }
        __syncthreads();
    }
    // backward: L^T x = z
    for (int jb = ((n - 1) / CHOL_B) * CHOL_B; jb >= 0; jb -= CHOL_B) {
        const int w = min(CHOL_B, n - jb);
        load_diag(jb, w);
        if (warp == 0) {
            T v = lane < w ? b[jb + lane] : T(0);
            for (int c = w - 1; c >= 0; --c) {
                const T xc = __shfl_sync(FULL_MASK, v, c) / D(c, c);
                if (lane == c) v = xc;
                if (lane < c) v -= D(c, lane) * xc;
            }
            if (lane < w) {
                b[jb + lane] = v;
                zb[lane] = v;
            }
        }
        __syncthreads();
        for (int k = tm.rank(); k < jb; k += tm.size()) {
            T acc = b[k];
            for (int c = 0; c < w; ++c) acc -= L[(size_t)(jb + c) * n + k] * zb[c];
            b[k] = acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// M^{-1}(a, e) for M = [I A^T; -A I]: x = (I + A^T A)^{-1}(a - A^T e) by CG
// warm-started from x (in place), y = e + A x written to W.py.  Returns the CG
// iterations; htp = <c, x> + <b, y>.  CG stops when ||res|| <= rtol ||rhs||.
// (Block elimination of the linear-system step of Eq. drs; Sec. 4.1 names CG.)
// ---------------------------------------------------------------------------
template <typename T, class Team>
__device__ __forceinline__ bool direct_available(const Team&, const DevWork<T>& W)
{
    if constexpr (Team::kGrid) return false;
    else return W.chol != nullptr;
}

template <typename T, class Team>
__device__ int minv(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const T* a, const T* e, T* x, double rtol,
                    int cg_max, double& htp, double atol = 0.0)
{
    const int n = P.n;
    T* tmv = W.tm;
    T* r = W.cr;
    spmv(tm, P.A, x, [&](int i, T s) { tmv[i] = s; });
    tm.sync();
    T acc_b = 0, acc_r = 0;
    spmv2(tm, P.AT, e, tmv, [&](int j, T s1, T s2) {
        const T rhs = a[j] - s1;
        const T res = rhs - x[j] - s2;
        r[j] = res;
        acc_b += rhs * rhs;
        acc_r += res * res;
    });
    double red2[2] = {(double)acc_b, (double)acc_r};
    tm.reduce(red2);
    const double rhs2 = red2[0];
    const double rr = red2[1];
    const double tol = fmax(rtol * sqrt(rhs2), atol);
    int it = 0;
    if (rhs2 == 0.0) {
        for (int j = tm.rank(); j < n; j += tm.size()) x[j] = 0;
        tm.sync();
    } else if (direct_available(tm, W)) {
        // direct: x <- x + (L L^T)^{-1} r, the residual of the warm start solved exactly
        if constexpr (!Team::kGrid) {
            // shared scratch of the CTA: the AA direction's Cholesky array (idle during a linear
            // solve) for the diagonal block, the reduction rows for the block's solution
            chol_solve<T>(tm, W.chol, n, r, reinterpret_cast<T*>(tm.scratch), reinterpret_cast<T*>(tm.red));
        }
        for (int j = tm.rank(); j < n; j += tm.size()) x[j] += r[j];
        tm.sync();
    } else if (sqrt(rr) > tol) {
        const unsigned long long tc0 = tm.leader() ? gtimer() : 0ull;
        it = cg_loop<T>(tm, P.A, P.AT, n, CgBufs<T>{r, W.cp, W.cq, tmv}, x, rr, tol, cg_max);
        if (tm.leader()) W.st->part_ns[3] += (double)(gtimer() - tc0);
    }
    T hb = 0, hc = 0;
    T* py = W.py;
    spmv(tm, P.A, x, [&](int i, T s) {
        const T yi = e[i] + s;
        py[i] = yi;
        hb += ro(P.b + i) * yi;
    });
    for (int j = tm.rank(); j < n; j += tm.size()) hc += ro(P.c + j) * x[j];
    double red4[2] = {(double)hb, (double)hc};
    tm.reduce(red4);
    htp = red4[0] + red4[1];
    if (tm.leader()) W.st->mat_passes += 3 + 2 * it;
    return it;
}

// The same M^{-1}(a, e) in FP64 by iterative refinement (SCS_MIXED, FP64
// phase): the residual r = rhs - (I + A^T A) x is formed in FP64 with the FP64
// matrix, the correction solves (I + A^T A) dx = r / ||r|| in FP32 with the
// FP32 copy of A by the same CG from dx = 0, and x += ||r|| dx in FP64; then
// the FP64 residual is formed again, until ||r|| <= tol.  Where the requested
// accuracy relative to ||r|| is looser than IR_VERIFY (the solves inside the
// loop under cg_adapt) one correction is taken without the checking residual:
// its FP32 rounding (about 1e-7 of ||r|| times the growth of the products) is
// far below what was asked.  Each correction is asked for at most IR_FLOOR
// relative accuracy, about what FP32 CG reaches reliably.  Returns the FP32
// CG iterations.
constexpr double IR_VERIFY = 1e-3;
constexpr double IR_FLOOR = 1e-5;
constexpr int IR_MAX_SWEEPS = 6;

template <class Team>
__device__ int minv_ir(Team& tm, const DevProb<double>& P, const DevWork<double>& W, const double* a,
                       const double* e, double* x, double rtol, int cg_max, double& htp, double atol)
{
    const int n = P.n;
    double* tmv = W.tm;
    double* r = W.cr;
    double* rhs = W.tn;
    const IrBufs& ir = W.ir;
    spmv(tm, P.A, x, [&](int i, double s) { tmv[i] = s; });
    tm.sync();
    double acc_b = 0, acc_r = 0;
    spmv2(tm, P.AT, e, tmv, [&](int j, double s1, double s2) {
        const double rh = a[j] - s1;
        const double res = rh - x[j] - s2;
        rhs[j] = rh;
        r[j] = res;
        acc_b += rh * rh;
        acc_r += res * res;
    });
    double red2[2] = {acc_b, acc_r};
    tm.reduce(red2);
    const double rhs2 = red2[0];
    double rr = red2[1];
    const double tol = fmax(rtol * sqrt(rhs2), atol);
    long long passes64 = 3, passes32 = 0, sweeps = 0;
    int it = 0;
    if (rhs2 == 0.0) {
        for (int j = tm.rank(); j < n; j += tm.size()) x[j] = 0;
        tm.sync();
    } else {
        for (int sw = 0; sw < IR_MAX_SWEEPS && sqrt(rr) > tol && it < cg_max && !tm.aborted(); ++sw) {
            const double nr = sqrt(rr);
            const double want = tol / nr;  // relative accuracy asked of this correction
            // the scaled residual in FP32, the correction from zero
            float acc32 = 0.f;
            const double inv = 1.0 / nr;
            for (int j = tm.rank(); j < n; j += tm.size()) {
                const float rj = (float)(r[j] * inv);
                ir.r[j] = rj;
                ir.x[j] = 0.f;
                acc32 += rj * rj;
            }
            double red3[1] = {(double)acc32};
            tm.reduce(red3);
            const unsigned long long tc0 = tm.leader() ? gtimer() : 0ull;
            const int k = cg_loop<float>(tm, ir.A, ir.AT, n, CgBufs<float>{ir.r, ir.p, ir.q, ir.tm}, ir.x, red3[0],
                                         fmax(want, IR_FLOOR) * sqrt(red3[0]), cg_max - it);
            if (tm.leader()) W.st->part_ns[3] += (double)(gtimer() - tc0);
            it += k;
            passes32 += 2 * k;
            ++sweeps;
            if (want >= IR_VERIFY) {
                for (int j = tm.rank(); j < n; j += tm.size()) x[j] += nr * (double)ir.x[j];
                tm.sync();
                break;
            }
            for (int j = tm.rank(); j < n; j += tm.size()) x[j] += nr * (double)ir.x[j];
            tm.sync();
            // FP64 residual of the corrected x
            spmv(tm, P.A, x, [&](int i, double s) { tmv[i] = s; });
            tm.sync();
            double acc = 0;
            spmv(tm, P.AT, tmv, [&](int j, double s) {
                const double res = rhs[j] - x[j] - s;
                r[j] = res;
                acc += res * res;
            });
            double red4[1] = {acc};
            tm.reduce(red4);
            rr = red4[0];
            passes64 += 2;
        }
    }
    double hb = 0, hc = 0;
    double* py = W.py;
    spmv(tm, P.A, x, [&](int i, double s) {
        const double yi = e[i] + s;
        py[i] = yi;
        hb += ro(P.b + i) * yi;
    });
    for (int j = tm.rank(); j < n; j += tm.size()) hc += ro(P.c + j) * x[j];
    double red5[2] = {hb, hc};
    tm.reduce(red5);
    htp = red5[0] + red5[1];
    if (tm.leader()) {
        W.st->mat_passes += passes64 + 1;
        W.st->mat_passes_ir += passes32;
        W.st->cg_iters_ir += it;
        W.st->ir_sweeps += sweeps;
    }
    return it;
}

// out = (I+Q)^{-1} r via tau = (r_tau + h^T M^{-1} r) / (1 + h^T g), (x,y) = M^{-1} r - tau g.
// r and out must not share storage of the bulk part.
template <typename T, class Team>
__device__ int linsys(Team& tm, const DevProb<T>& P, const DevWork<T>& W, HV<T> r, HV<T> out, int slot,
                      double rtol, int cg_max, double hg, double atol = 0.0, bool refine = false)
{
    const int n = P.n, m = P.m;
    const double rtau = *r.t;
    T* x = W.ws[slot];
    double htp;
    int it;
    const unsigned long long tl0 = tm.leader() ? gtimer() : 0ull;
    if constexpr (sizeof(T) == sizeof(double)) {
        it = refine ? minv_ir(tm, P, W, r.v, r.v + n, x, rtol, cg_max, htp, atol)
                    : minv(tm, P, W, r.v, r.v + n, x, rtol, cg_max, htp, atol);
    } else {
        it = minv(tm, P, W, r.v, r.v + n, x, rtol, cg_max, htp, atol);
    }
    const double tau = (rtau + htp) / (1.0 + hg);
    const T tt = (T)tau;
    for (int i = tm.rank(); i < n; i += tm.size()) out.v[i] = x[i] - tt * W.g[i];
    for (int i = tm.rank(); i < m; i += tm.size()) out.v[n + i] = W.py[i] - tt * W.g[n + i];
    if (tm.leader()) *out.t = tau;
    tm.sync();
    if (tm.leader()) W.st->part_ns[2] += (double)(gtimer() - tl0);
    return it;
}

// ---------------------------------------------------------------------------
// Projection on C = R^n x K* x R_+ fused with the DRS residual (Eq. drs):
// for each element the op supplies (w, w~), the pass forms v = 2 w~ - w,
// projects it (identity on chi and zero-cone rows, max(0,.) on the orthant,
// closed form per SOC with one warp per cone, eigen-decomposition per PSD
// block with one CTA per block) and hands (w, w~, w_) back to the op.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int svec_index(int d, int i, int j)  // i >= j
{
    return j * d - j * (j - 1) / 2 + (i - j);
}

__device__ __forceinline__ double block_sum(double x, double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Parallel two-sided Jacobi (round-robin pairing, d/2 disjoint rotations per
// round) on the dp x dp matrix X in shared memory; V receives the
// eigenvectors as columns.  Rotation formula as in the textbook cyclic method.
// v_init: V already holds an orthogonal start basis (the rotations are
// accumulated onto it), else it starts as the identity.  Returns true if the
// off-diagonal mass fell below tol2 times the total within max_sweeps (the
// same value in every thread).
template <typename T>
__device__ bool jacobi_block(T* X, T* V, int dp, int ld, int* pp, int* qq, T* cs, T* sn, double* red, double tol2,
                             int max_sweeps, bool v_init = false)
{
    // X and V are dp x dp with row stride ld = dp + 1 (odd): a warp walking a
    // column touches 32 different banks
    const int tid = threadIdx.x, nt = blockDim.x;
    if (!v_init)
        for (int idx = tid; idx < dp * dp; idx += nt) {
            const int i = idx / dp, j = idx % dp;
            V[i * ld + j] = (i == j) ? T(1) : T(0);
        }
    double total = 0.0;
    for (int idx = tid; idx < dp * dp; idx += nt) {
        const T x = X[(idx / dp) * ld + idx % dp];
        total += (double)x * (double)x;
    }
    __syncthreads();
    total = block_sum(total, red);
    const int half = dp / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int idx = tid; idx < dp * dp; idx += nt) {
            const int i = idx / dp, j = idx % dp;
            if (i != j) off += (double)X[i * ld + j] * (double)X[i * ld + j];
        }
        off = block_sum(off, red);
        if (off <= tol2 * total || off == 0.0) return true;
        for (int rnd = 0; rnd < dp - 1; ++rnd) {
            for (int k = tid; k < half; k += nt) {
                int a, b;
                if (k == 0) {
                    a = rnd;
                    b = dp - 1;
                } else {
                    a = (rnd + k) % (dp - 1);
                    b = (rnd - k + dp - 1) % (dp - 1);
                }
                const int p = a < b ? a : b, qd = a < b ? b : a;
                const T apq = X[p * ld + qd];
                T c = 1, s = 0;
                if (apq != T(0)) {
                    const T theta = (X[qd * ld + qd] - X[p * ld + p]) / (T(2) * apq);
                    const T at = theta < T(0) ? -theta : theta;
                    T t;
                    if (at > T(1e18))
                        t = T(0.5) / theta;
                    else
                        t = (theta >= T(0) ? T(1) : T(-1)) / (at + sqrt(theta * theta + T(1)));
                    c = T(1) / sqrt(t * t + T(1));
                    s = t * c;
                }
                pp[k] = p;
                qq[k] = qd;
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // columns: X <- X J and V <- V J
            for (int idx = tid; idx < half * dp; idx += nt) {
                const int k = idx / dp, i = idx % dp;
                const int p = pp[k], qd = qq[k];
                const T c = cs[k], s = sn[k];
                const T xp = X[i * ld + p], xq = X[i * ld + qd];
                X[i * ld + p] = c * xp - s * xq;
                X[i * ld + qd] = s * xp + c * xq;
                const T vp = V[i * ld + p], vq = V[i * ld + qd];
                V[i * ld + p] = c * vp - s * vq;
                V[i * ld + qd] = s * vp + c * vq;
            }
            __syncthreads();
            // rows: X <- J^T X
            for (int idx = tid; idx < half * dp; idx += nt) {
                const int k = idx / dp, j = idx % dp;
                const int p = pp[k], qd = qq[k];
                const T c = cs[k], s = sn[k];
                const T xp = X[p * ld + j], xq = X[qd * ld + j];
                X[p * ld + j] = c * xp - s * xq;
                X[qd * ld + j] = s * xp + c * xq;
            }
            __syncthreads();
        }
    }
    return false;
}

// ---------------------------------------------------------------------------
// Exponential cone K = cl{(x1, x2, x3) : x1 >= x2 exp(x3 / x2), x2 > 0}
// (Sec. 2, cone (v)), one cone per thread, in FP64 whatever T is.  With
// (r, s, t) = (x3, x2, x1): a point inside K is kept, a point of the polar
// cone -K* goes to 0, a point with r <= 0 and s <= 0 goes to the face
// (r, 0, max(t, 0)).  Any other point projects on the boundary: either on the
// face {s = 0, r <= 0, t >= 0}, whose nearest point is (min(r,0), 0,
// max(t,0)), or on a ray c (rho, 1, e^rho), c > 0, where the distance is
// stationary in rho, i.e. where
//   F(rho) = r (1 + (1-rho) e^{2rho}) - s (rho + e^{2rho}) + t e^rho (rho^2 - rho + 1)
// vanishes.  The sign changes of F (evaluated as F e^{-2rho} for rho > 0)
// are found on a grid of step 1/4 over [-60, 60] (its roots lie at least
// about 3 apart) and by doubling brackets outside it, each root is bisected
// to full precision, and the nearest of the candidates (origin, face point,
// ray points) is returned.  The dual cone K* = cl{y3 < 0, -y3 exp(y2/y3) <= e y1}
// is projected through Moreau's decomposition, Pi_{K*}(v) = v + Pi_K(-v).
// ---------------------------------------------------------------------------
// F for rho <= 0 given e = e^rho, and for rho > 0 given em = e^-rho (scaled by e^-2rho)
static __device__ __forceinline__ double expc_Fn(double rho, double e, double r, double s, double t)
{
    const double e2 = e * e;
    return r * (1.0 + (1.0 - rho) * e2) - s * (rho + e2) + t * e * (rho * rho - rho + 1.0);
}
static __device__ __forceinline__ double expc_Fp(double rho, double em, double r, double s, double t)
{
    const double em2 = em * em;
    return r * ((1.0 - rho) + em2) - s * (rho * em2 + 1.0) + t * em * (rho * rho - rho + 1.0);
}
static __device__ __forceinline__ double expc_F(double rho, double r, double s, double t)
{
    return rho <= 0.0 ? expc_Fn(rho, exp(rho), r, s, t) : expc_Fp(rho, exp(-rho), r, s, t);
}

// Root of F in [lo, hi] (a sign change) to adjacent doubles: regula falsi with the
// Illinois modification (the retained end's value is halved when the same end is
// kept twice), a bisection step every fourth iteration so the bracket at least halves
// that often.  Converges in a dozen evaluations where bisection needs about sixty.
static __device__ double expc_root(double lo, double hi, double flo, double r, double s, double t)
{
    // both ends exactly (the grid's values carry the incremental exponentials' roundings)
    flo = expc_F(lo, r, s, t);
    if (flo == 0.0) return lo;
    double fhi = expc_F(hi, r, s, t);
    if (fhi == 0.0) return hi;
    int kept = 0;  // -1: lo kept last time, +1: hi kept last time
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double x = mid;
        if ((it & 3) != 3) {
            const double sec = (lo * fhi - hi * flo) / (fhi - flo);
            if (sec > lo && sec < hi) x = sec;
        }
        const double fx = expc_F(x, r, s, t);
        if (fx == 0.0) return x;
        if ((fx > 0.0) == (flo > 0.0)) {
            lo = x;
            flo = fx;
            if (kept == 1) fhi *= 0.5;
            kept = 1;
        } else {
            hi = x;
            fhi = fx;
            if (kept == -1) flo *= 0.5;
            kept = -1;
        }
    }
    return 0.5 * (lo + hi);
}

// candidate on the ray of slope rho: the ray's nearest point to (r, s, t) if it lies on the open ray
static __device__ void expc_try_ray(double rho, double r, double s, double t, double& br, double& bs, double& bt, double& bd)
{
    double a0, a1, a2;  // the ray direction scaled by 1 / max(1, e^rho)
    if (rho <= 0.0) {
        a0 = rho;
        a1 = 1.0;
        a2 = exp(rho);
    } else {
        const double em = exp(-rho);
        a0 = rho * em;
        a1 = em;
        a2 = 1.0;
    }
    const double c = (r * a0 + s * a1 + t * a2) / (a0 * a0 + a1 * a1 + a2 * a2);
    if (!(c > 0.0)) return;
    const double pr = c * a0, ps = c * a1, pt = c * a2;
    const double d = (r - pr) * (r - pr) + (s - ps) * (s - ps) + (t - pt) * (t - pt);
    if (d < bd) {
        bd = d;
        br = pr;
        bs = ps;
        bt = pt;
    }
}

// x = (x1, x2, x3) <- Pi_K(x)
static __device__ void expc_project(double& x1, double& x2, double& x3)
{
    const double r = x3, s = x2, t = x1;
    if (s > 0.0 ? s * exp(r / s) <= t : (s == 0.0 && r <= 0.0 && t >= 0.0)) return;  // in K
    if (r > 0.0 ? r * exp(s / r) <= -2.718281828459045 * t : (r == 0.0 && s <= 0.0 && t <= 0.0)) {
        x1 = x2 = x3 = 0.0;  // in the polar cone
        return;
    }
    if (r <= 0.0 && s <= 0.0) {
        x1 = t > 0.0 ? t : 0.0;
        x2 = 0.0;
        return;
    }
    double br = 0.0, bs = 0.0, bt = 0.0, bd = r * r + s * s + t * t;  // the origin
    {
        const double fr = fmin(r, 0.0), ft = fmax(t, 0.0);
        const double d = (r - fr) * (r - fr) + s * s + (t - ft) * (t - ft);
        if (d < bd) {
            bd = d;
            br = fr;
            bs = 0.0;
            bt = ft;
        }
    }
    // outside the grid F is dominated by its linear part: at most one sign change on each side
    for (int side = 0; side < 2; ++side) {
        double a = side == 0 ? -60.0 : 60.0;
        double fa = expc_F(a, r, s, t);
        for (int k = 0; k < 1100; ++k) {
            const double b = 2.0 * a;
            if (!isfinite(b)) break;
            const double fb = expc_F(b, r, s, t);
            if (fb != 0.0 && (fb > 0.0) != (fa > 0.0)) {
                const double rho = side == 0 ? expc_root(b, a, fb, r, s, t) : expc_root(a, b, fa, r, s, t);
                expc_try_ray(rho, r, s, t, br, bs, bt, bd);
                break;
            }
            a = b;
            fa = fb;
        }
    }
    // the grid: e^rho (rho <= 0) and e^-rho (rho > 0) advance by a factor e^(+-1/4) per step and
    // are evaluated afresh every 16 steps, so the scan takes one exp in 16; the roots are refined
    // with exact evaluations
    const double up = exp(0.25), down = exp(-0.25);
    double xa = -60.0, ea = exp(-60.0), fa = expc_Fn(xa, ea, r, s, t);
    double emb = 0.0;
    for (int k = 1; k <= 480; ++k) {
        const double xb = -60.0 + 0.25 * k;
        double fb;
        if (k <= 240) {
            ea = (k & 15) == 0 ? exp(xb) : ea * up;
            fb = expc_Fn(xb, ea, r, s, t);
        } else {
            emb = (k & 15) == 0 || k == 241 ? exp(-xb) : emb * down;
            fb = expc_Fp(xb, emb, r, s, t);
        }
        if (fb == 0.0) expc_try_ray(xb, r, s, t, br, bs, bt, bd);
        else if (fa != 0.0 && (fb > 0.0) != (fa > 0.0))
            expc_try_ray(expc_root(xa, xb, fa, r, s, t), r, s, t, br, bs, bt, bd);
        xa = xb;
        fa = fb;
    }
    x1 = bt;
    x2 = bs;
    x3 = br;
}

template <typename T>
struct PsdSmem {
    T* X;
    T* V;
    int* pp;
    int* qq;
    T* cs;
    T* sn;
    T* lam;
    double* red;
    double* X0;  // FP32 eigensolves only: the input matrix in FP64 for the residual recheck
};

template <typename T>
__host__ __device__ constexpr size_t psd_smem_bytes()
{
    return sizeof(T) * (2 * PSD_MAX * PSD_LD + 3 * PSD_MAX) + sizeof(int) * PSD_MAX + 64 * sizeof(double) +
           (sizeof(T) == 4 ? sizeof(double) * PSD_MAX * PSD_LD : 0);
}

// Workspace of one PSD block of order d > PSD_MAX in global memory, with the
// relative layout of the shared-memory one (X and V adjacent, then cs, sn,
// lam, pp, qq and, for FP32, X0), so that the FP64 redo's overlays hold:
// the FP64 eigenvectors over X and V, the FP64 cosines over cs and sn, the
// FP64 sines over lam.
template <typename T>
__host__ __device__ constexpr size_t psd_big_bytes(int d)
{
    const size_t dp = (size_t)(d + (d & 1)), ld = dp + 1;
    const size_t b = sizeof(T) * (2 * dp * ld + 2 * dp) + sizeof(int) * dp + (sizeof(T) == 4 ? 8 * dp * ld : 0);
    return (b + 15) & ~size_t(15);
}

// warm-start eigenvectors of one PSD block: dp x (dp + 1) elements, 16-byte aligned
template <typename T>
__host__ __device__ constexpr size_t psd_v_bytes(int d)
{
    const size_t dp = (size_t)(d + (d & 1));
    return (sizeof(T) * dp * (dp + 1) + 15) & ~size_t(15);
}

template <typename T>
__device__ PsdSmem<T> psd_big_ws(unsigned char* base, int d, double* red)
{
    const int dp = d + (d & 1), ld = dp + 1, half = dp / 2;
    PsdSmem<T> s;
    s.X = (T*)base;
    s.V = s.X + (size_t)dp * ld;
    s.cs = s.V + (size_t)dp * ld;
    s.sn = s.cs + half;
    s.lam = s.sn + half;
    s.red = red;
    s.pp = (int*)(s.lam + dp);
    s.qq = s.pp + half;
    s.X0 = sizeof(T) == 4 ? (double*)(s.qq + half) : nullptr;
    return s;
}

template <typename T>
__device__ PsdSmem<T> psd_smem(unsigned char* base)
{
    PsdSmem<T> s;
    s.X = (T*)base;
    s.V = s.X + PSD_MAX * PSD_LD;
    s.cs = s.V + PSD_MAX * PSD_LD;
    s.sn = s.cs + PSD_MAX / 2;
    s.lam = s.sn + PSD_MAX / 2;
    s.red = (double*)(s.lam + 2 * PSD_MAX);
    s.pp = (int*)(s.red + 32);
    s.qq = s.pp + PSD_MAX / 2;
    s.X0 = sizeof(T) == 4 ? (double*)(s.qq + PSD_MAX / 2) : nullptr;
    return s;
}

// Where the FP32 eigensolves report to: the largest relative eigen-residual
// (FP64-evaluated), the count of blocks decomposed again in FP64, and the
// bound above which that happens.
struct PsdCheck {
    double* resid;
    long long* redo;
    double tol;
    // warm starts: block k's eigenvectors of its last converged decomposition are kept at
    // vbase + voff[k] bytes (dp x (dp+1) elements of the bulk type); vok[k] = 0: none, else the
    // number of decompositions since the last cold one
    unsigned char* vbase;
    const long long* voff;
    int* vok;
};

// FP64 Jacobi of the block whose FP64 copy X0 is in shared memory (FP32
// eigensolves only).  The FP32 X and V are dead by now: the FP64
// eigenvectors overlay them (2 PSD_MAX x PSD_LD floats = PSD_MAX x PSD_LD
// doubles), the rotation cosines and sines the FP32 cs / sn and lam arrays.
// X0 leaves with the eigenvalues on its diagonal, V64 with the eigenvectors.
static __device__ __noinline__ void psd_redo_fp64(PsdSmem<float>& sm, int dp, int ld)
{
    double* V64 = reinterpret_cast<double*>(sm.X);
    double* cs64 = reinterpret_cast<double*>(sm.cs);
    double* sn64 = reinterpret_cast<double*>(sm.lam);
    __syncthreads();
    jacobi_block<double>(sm.X0, V64, dp, ld, sm.pp, sm.qq, cs64, sn64, sm.red, 1e-26, 20);
}

template <typename T, class Team, class Op>
__device__ void project_pass(Team& tm, const DevProb<T>& P, Op& op, unsigned char* psd_base,
                             PsdCheck ck = PsdCheck{nullptr, nullptr, 0.0})
{
    const int n = P.n;
    const int lin = n + P.f + P.l;
    const int fz = n + P.f;
    for (int i = tm.rank(); i < lin; i += tm.size()) {
        T w, wt;
        op.load(i, w, wt);
        const T v = T(2) * wt - w;
        const T wb = (i >= fz) ? (v > T(0) ? v : T(0)) : v;
        op.store(i, w, wt, wb);
    }
    // second-order cones, t last: one warp per cone
    const int lane = threadIdx.x & 31;
    const int nw = tm.size() >> 5;
    for (int k = tm.rank() >> 5; k < P.nq; k += nw) {
        const int o = n + ro(P.q_off + k);
        const int dim = ro(P.q_off + k + 1) - ro(P.q_off + k);
        T ss = 0;
        for (int j = lane; j < dim - 1; j += 32) {
            T w, wt;
            op.load(o + j, w, wt);
            const T v = T(2) * wt - w;
            ss += v * v;
        }
        T wT, wtT;
        op.load(o + dim - 1, wT, wtT);
        const T tv = T(2) * wtT - wT;
        const double nx = sqrt((double)warp_sum(ss));
        const double t = (double)tv;
        int mode;
        double a = 0.0, tb = 0.0;
        if (nx <= t) mode = 0;
        else if (nx <= -t) mode = 1;
        else {
            mode = 2;
            a = (nx + t) / (2.0 * nx);
            tb = a * nx;
        }
        for (int j = lane; j < dim - 1; j += 32) {
            T w, wt;
            op.load(o + j, w, wt);
            const T v = T(2) * wt - w;
            const T wb = mode == 0 ? v : (mode == 1 ? T(0) : (T)(a * (double)v));
            op.store(o + j, w, wt, wb);
        }
        if (lane == 0) op.store(o + dim - 1, wT, wtT, mode == 0 ? tv : (mode == 1 ? T(0) : (T)tb));
        __syncwarp();
    }
    // PSD blocks: one CTA per block, Jacobi eigen-decomposition in shared memory
    // (orders above PSD_MAX: in the block's workspace in global memory)
    if (P.ns > 0) {
        const PsdSmem<T> sm_small = psd_smem<T>(psd_base);
        for (int k = tm.block(); k < P.ns; k += tm.nblocks()) {
            const int d = ro(P.s_dim + k);
            const int o = n + ro(P.s_off + k);
            const int dp = d + (d & 1);
            const int ld = dp + 1;  // odd row stride: column walks are free of bank conflicts
            PsdSmem<T> sm = d > PSD_MAX ? psd_big_ws<T>(P.psd_big + ro(P.big_off + k), d, sm_small.red) : sm_small;
            const double isq2 = 0.70710678118654752440;
            __syncthreads();
            for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x) {
                const int i = idx / dp, j = idx % dp;
                T val = 0;
                if (i < d && j < d) {
                    const int ii = i > j ? i : j, jj = i > j ? j : i;
                    T w, wt;
                    op.load(o + svec_index(d, ii, jj), w, wt);
                    const T v = T(2) * wt - w;
                    val = (ii == jj) ? v : (T)((double)v * isq2);
                }
                sm.X[i * ld + j] = val;
                if constexpr (sizeof(T) == 4) sm.X0[i * ld + j] = (double)val;
            }
            __syncthreads();
            const double tol2 = sizeof(T) == 8 ? 1e-26 : 1e-11;
            // Warm start: successive projections of a block see nearby matrices, so the
            // eigenvectors Vp of the last converged decomposition nearly diagonalise this one.
            // X <- Vp^T X Vp (symmetrised) and V <- Vp, then the sweeps accumulate onto V:
            // the same eigenpairs, found in a few sweeps instead of a dozen.  vok[k] counts the
            // generations since the last cold start; V loses orthogonality by a few roundings
            // per generation, so every PSD_WARM_GEN-th decomposition starts cold again.
            constexpr int PSD_WARM_GEN = sizeof(T) == 4 ? 16 : 64;
            T* Vp = ck.vbase ? reinterpret_cast<T*>(ck.vbase + ro(ck.voff + k)) : nullptr;
            const int gen = Vp ? *(volatile const int*)(ck.vok + k) : 0;
            const bool warm = gen > 0 && gen < PSD_WARM_GEN;
            if (warm) {
                for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x) {  // V <- X Vp
                    const int i = idx / dp, j = idx % dp;
                    T s = 0;
                    for (int l = 0; l < dp; ++l) s = fmaT(sm.X[i * ld + l], Vp[l * ld + j], s);
                    sm.V[i * ld + j] = s;
                }
                __syncthreads();
                for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x) {  // X <- Vp^T V
                    const int i = idx / dp, j = idx % dp;
                    T s = 0;
                    for (int l = 0; l < dp; ++l) s = fmaT(Vp[l * ld + i], sm.V[l * ld + j], s);
                    sm.X[i * ld + j] = s;
                }
                __syncthreads();
                for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x) {
                    const int i = idx / dp, j = idx % dp;
                    if (i < j) {
                        const T a = T(0.5) * (sm.X[i * ld + j] + sm.X[j * ld + i]);
                        sm.X[i * ld + j] = a;
                        sm.X[j * ld + i] = a;
                    }
                    sm.V[i * ld + j] = Vp[i * ld + j];
                }
                __syncthreads();
            }
            const bool conv = jacobi_block<T>(sm.X, sm.V, dp, ld, sm.pp, sm.qq, sm.cs, sm.sn, sm.red, tol2,
                                              d > PSD_MAX ? 30 : (sizeof(T) == 8 ? 20 : 15), warm);
            if (Vp) {
                if (conv)
                    for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x)
                        Vp[(idx / dp) * ld + idx % dp] = sm.V[(idx / dp) * ld + idx % dp];
                if (threadIdx.x == 0) ck.vok[k] = conv ? (warm ? gen + 1 : 1) : 0;
            }
            if constexpr (sizeof(T) == 4) {
                // FP64 recheck of the FP32 eigenpairs: ||X V - V diag(l)||_F / ||X||_F
                double r2 = 0.0, x2 = 0.0;
                for (int idx = threadIdx.x; idx < dp * dp; idx += blockDim.x) {
                    const int i = idx / dp, k = idx % dp;
                    double acc = -(double)sm.V[i * ld + k] * (double)sm.X[k * ld + k];
                    for (int j = 0; j < dp; ++j) acc += sm.X0[i * ld + j] * (double)sm.V[j * ld + k];
                    r2 += acc * acc;
                    x2 += sm.X0[i * ld + k] * sm.X0[i * ld + k];
                }
                r2 = block_sum(r2, sm.red);
                x2 = block_sum(x2, sm.red);
                // block_sum hands every thread the same sums, so the decision
                // to decompose the block again in FP64 is uniform in the CTA
                const double rel = x2 > 0.0 ? sqrt(r2 / x2) : 0.0;
                if (threadIdx.x == 0 && ck.resid)
                    atomicMax((unsigned long long*)ck.resid, (unsigned long long)__double_as_longlong(rel));
                if (rel > ck.tol && ck.redo) {
                    psd_redo_fp64(sm, dp, ld);
                    if (threadIdx.x == 0) {
                        atomicAdd((unsigned long long*)ck.redo, 1ull);
                        if (Vp) ck.vok[k] = 0;  // the FP32 eigenvectors were not good enough to start from
                    }
                    const double* V64 = reinterpret_cast<const double*>(sm.X);
                    for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
                        const int i = idx / d, j = idx % d;
                        if (i < j) continue;
                        double s = 0.0;
                        for (int kk = 0; kk < dp; ++kk) {
                            const double l = sm.X0[kk * ld + kk];
                            if (l > 0.0) s += V64[i * ld + kk] * l * V64[j * ld + kk];
                        }
                        const int e = o + svec_index(d, i, j);
                        T w, wt;
                        op.load(e, w, wt);
                        op.store(e, w, wt, (T)(i == j ? s : s * 1.41421356237309504880));
                    }
                    __syncthreads();
                    continue;
                }
            }
            for (int i = threadIdx.x; i < dp; i += blockDim.x) {
                const T l = sm.X[i * ld + i];
                sm.lam[i] = l > T(0) ? l : T(0);
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
                const int i = idx / d, j = idx % d;
                if (i < j) continue;
                T s = 0;
                for (int kk = 0; kk < dp; ++kk) s += sm.V[i * ld + kk] * sm.lam[kk] * sm.V[j * ld + kk];
                const int e = o + svec_index(d, i, j);
                T w, wt;
                op.load(e, w, wt);
                op.store(e, w, wt, i == j ? s : (T)((double)s * 1.41421356237309504880));
            }
            __syncthreads();
        }
    }
    // exponential cones, one per thread: the psi part lies in K*, so a primal
    // block projects on the dual cone (Moreau: v + Pi_K(-v)) and a dual block on K
    for (int k = tm.rank(); k < P.ep + P.ed; k += tm.size()) {
        const int o = n + P.e_off + 3 * k;
        T w[3], wt[3];
        double v[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            op.load(o + j, w[j], wt[j]);
            v[j] = 2.0 * (double)wt[j] - (double)w[j];
        }
        if (k < P.ep) {
            double m1 = -v[0], m2 = -v[1], m3 = -v[2];
            expc_project(m1, m2, m3);
            v[0] += m1;
            v[1] += m2;
            v[2] += m3;
        } else {
            expc_project(v[0], v[1], v[2]);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) op.store(o + j, w[j], wt[j], (T)v[j]);
    }
    if (tm.leader()) {
        double w, wt;
        op.load_tau(w, wt);
        const double v = 2.0 * wt - w;
        op.store_tau(w, wt, v > 0.0 ? v : 0.0);
    }
}

// ---- ops of the projection pass ----
// residual at (u, u~): u_ = Pi(2u~ - u), R = u~ - u_;  acc0 = ||R||^2
template <typename T>
struct OpResidual {
    HV<T> u, ut, ub, R;
    T acc0;
    __device__ void load(int i, T& w, T& wt) const { w = u.v[i]; wt = ut.v[i]; }
    __device__ void store(int i, T, T wt, T wb)
    {
        ub.v[i] = wb;
        const T r = wt - wb;
        R.v[i] = r;
        acc0 += r * r;
    }
    __device__ void load_tau(double& w, double& wt) const { w = *u.t; wt = *ut.t; }
    __device__ void store_tau(double, double wt, double wb)
    {
        *ub.t = wb;
        const double r = wt - wb;
        *R.t = r;
        acc0 += (T)(r * r);
    }
};

// K0 (blind step): u <- u + d, u~ <- u~ + d~, then the residual of the new
// point; secant pair z = d, xi = R_new - R_old; acc0 = ||R_new||^2, acc1 = ||d||^2
template <typename T>
struct OpK0 {
    HV<T> u, ut, ub, Ru, d, dt, zp, xip;
    T acc0, acc1;
    __device__ void load(int i, T& w, T& wt) const { w = u.v[i] + d.v[i]; wt = ut.v[i] + dt.v[i]; }
    __device__ void store(int i, T w, T wt, T wb)
    {
        const T di = d.v[i];
        u.v[i] = w;
        ut.v[i] = wt;
        ub.v[i] = wb;
        const T r = wt - wb;
        xip.v[i] = r - Ru.v[i];
        zp.v[i] = di;
        Ru.v[i] = r;
        acc0 += r * r;
        acc1 += di * di;
    }
    __device__ void load_tau(double& w, double& wt) const { w = *u.t + *d.t; wt = *ut.t + *dt.t; }
    __device__ void store_tau(double w, double wt, double wb)
    {
        const double di = *d.t;
        *u.t = w;
        *ut.t = wt;
        *ub.t = wb;
        const double r = wt - wb;
        *xip.t = r - *Ru.t;
        *zp.t = di;
        *Ru.t = r;
        acc0 += (T)(r * r);
        acc1 += (T)(di * di);
    }
};

// line-search trial at w = u + alpha d, w~ = u~ + alpha d~ (linearity trick,
// Sec. 4.2): stores w_ and Rw; acc0 = ||Rw||^2, acc1 = <Rw, Rw - alpha d>
template <typename T>
struct OpTrial {
    HV<T> u, ut, d, dt, wb, Rw;
    double alpha;
    T acc0, acc1;
    __device__ void load(int i, T& w, T& wt) const
    {
        const T a = (T)alpha;
        w = u.v[i] + a * d.v[i];
        wt = ut.v[i] + a * dt.v[i];
    }
    __device__ void store(int i, T, T wt, T wbv)
    {
        wb.v[i] = wbv;
        const T r = wt - wbv;
        Rw.v[i] = r;
        acc0 += r * r;
        acc1 += r * (r - (T)alpha * d.v[i]);
    }
    __device__ void load_tau(double& w, double& wt) const
    {
        w = *u.t + alpha * *d.t;
        wt = *ut.t + alpha * *dt.t;
    }
    __device__ void store_tau(double, double wt, double wbv)
    {
        *wb.t = wbv;
        const double r = wt - wbv;
        *Rw.t = r;
        acc0 += (T)(r * r);
        acc1 += (T)(r * (r - alpha * *d.t));
    }
};

// plain projection: v -> Pi_C(v) (as w = -v, w~ = 0)
template <typename T>
struct OpProject {
    const T* vin;
    const double* tin;
    T* out;
    double* tout;
    __device__ void load(int i, T& w, T& wt) const { w = -vin[i]; wt = 0; }
    __device__ void store(int i, T, T, T wb) { out[i] = wb; }
    __device__ void load_tau(double& w, double& wt) const { w = -*tin; wt = 0.0; }
    __device__ void store_tau(double, double, double wb) { *tout = wb; }
};

// ---------------------------------------------------------------------------
// elementwise helpers on HSDE vectors
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Termination (Sec. 4.3) on (u, u~, u_).  Returns a status (0 = continue).
// Certificates use the reading ic = ||b|| ||A^T psi_|| / (-<b, psi_>) and
// uc = ||c|| ||A chi_ + sigma_|| / (-<c, chi_>) on unscaled vectors.
// ---------------------------------------------------------------------------
struct TermOut {
    double pr, dr, gap, ic, uc, pobj, dobj, bpsi, cchi;
    bool time_up;
};

template <typename T, class Team>
__device__ int termination(Team& tm, const DevProb<T>& P, const DevWork<T>& W, double eps, double deadline_ns,
                           TermOut& o)
{
    const int n = P.n, m = P.m;
    const T* chib = W.ub.v;
    const T* psib = W.ub.v + n;
    const T* psit = W.ut.v + n;
    const T* psi = W.u.v + n;
    const double taub = *W.ub.t;
    T* tmv = W.tm;
    T* tnv = W.tn;
    spmv(tm, P.A, chib, [&](int i, T s) { tmv[i] = s; });
    spmv(tm, P.AT, psib, [&](int j, T s) { tnv[j] = s; });
    tm.sync();
    if (tm.leader()) W.st->mat_passes += 2;
    const bool pos = taub > 0.0;
    const T inv = pos ? (T)(1.0 / taub) : T(0);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
    for (int i = tm.rank(); i < m; i += tm.size()) {
        const T sig = psib[i] - T(2) * psit[i] + psi[i];
        const T bi = ro(P.b + i);
        if (pos) {
            const T e = tmv[i] * inv + sig * inv - bi;
            a0 += e * e;
        }
        const T f = tmv[i] + sig;
        a4 += f * f;
        a3 += bi * psib[i];
    }
    for (int j = tm.rank(); j < n; j += tm.size()) {
        const T cj = ro(P.c + j);
        if (pos) {
            const T gq = tnv[j] * inv + cj;
            a1 += gq * gq;
        }
        a2 += cj * chib[j];
        a5 += tnv[j] * tnv[j];
    }
    double tflag = 0.0;
    if (tm.leader() && deadline_ns > 0.0 && (double)gtimer() > deadline_ns) tflag = 1.0;
    double red[7] = {(double)a0, (double)a1, (double)a2, (double)a3, (double)a4, (double)a5, tflag};
    tm.reduce(red);
    o.time_up = red[6] > 0.0;
    o.cchi = red[2];
    o.bpsi = red[3];
    o.pr = o.dr = o.gap = INFINITY;
    o.pobj = o.dobj = NAN;
    int status = 0;
    if (pos) {
        o.pr = sqrt(red[0]) / (1.0 + P.nb);
        o.dr = sqrt(red[1]) / (1.0 + P.nc);
        const double cx = red[2] / taub, by = red[3] / taub;
        o.gap = fabs(cx + by) / (1.0 + fabs(cx) + fabs(by));
        o.pobj = cx;
        o.dobj = -by;
        if (o.pr <= eps && o.dr <= eps && o.gap <= eps) status = ST_SOLVED;
    }
    o.ic = red[3] < 0.0 ? P.nb * sqrt(red[5]) / (-red[3]) : INFINITY;
    o.uc = red[2] < 0.0 ? P.nc * sqrt(red[4]) / (-red[2]) : INFINITY;
    if (!status) {
        if (o.ic < eps) status = ST_INFEASIBLE;
        else if (o.uc < eps) status = ST_UNBOUNDED;
    }
    return status;
}

// ---------------------------------------------------------------------------
// directions (Sec. 4.4)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ HV<T> col(T* base, double* tb, int k, int nm)
{
    return HV<T>{base + (size_t)k * nm, tb + k};
}

// small dense Cholesky solve by warp 0 of every block (k <= 32):
// (G + reg I) t = rhs with reg raised tenfold up to 8 times; false on failure
static __device__ bool small_chol(const double* G, const double* rhs, double* L, double* t, int k, double reg0)
{
    __shared__ int ok_s;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        bool ok = false;
        double reg = reg0;
        for (int attempt = 0; attempt < 8 && !ok; ++attempt, reg *= 10.0) {
            ok = true;
            for (int j = 0; j < k; ++j) {
                double s = (lane < j) ? L[j * AAMAX + lane] * L[j * AAMAX + lane] : 0.0;
                s = warp_sum(s);
                const double dj = G[j * AAMAX + j] + reg - s;
                if (!(dj > 0.0)) {
                    ok = false;
                    break;
                }
                const double ljj = sqrt(dj);
                if (lane > j && lane < k) {
                    double e = G[lane * AAMAX + j];
                    for (int p = 0; p < j; ++p) e -= L[lane * AAMAX + p] * L[j * AAMAX + p];
                    L[lane * AAMAX + j] = e / ljj;
                }
                if (lane == 0) L[j * AAMAX + j] = ljj;
                __syncwarp();
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (ok) {
                for (int i = 0; i < k; ++i) {
                    double e = rhs[i];
                    for (int p = 0; p < i; ++p) e -= L[i * AAMAX + p] * t[p];
                    t[i] = e / L[i * AAMAX + i];
                }
                for (int i = k - 1; i >= 0; --i) {
                    double e = t[i];
                    for (int p = i + 1; p < k; ++p) e -= L[p * AAMAX + i] * t[p];
                    t[i] = e / L[i * AAMAX + i];
                }
            }
            ok_s = ok ? 1 : 0;
        }
    }
    __syncthreads();
    return ok_s != 0;
}

struct DirState {
    int count;     // stored pairs
    long long inserted;
};

// Anderson's acceleration: d = -Ru - (Z - Xi) t, t = argmin ||Xi t - Ru|| by
// regularised normal equations; ring buffer of the last mem pairs.
template <typename T, class Team>
__device__ void aa_direction(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S,
                             bool have_pair, double nz2, DirState& ds, double* G, double* sm_rhs, double* sm_L,
                             double* sm_t)
{
    const int nm = P.n + P.m;
    const int mem = S.mem;
    if (have_pair && mem > 0 && nz2 > 0.0) {
        const int slot = (int)(ds.inserted % mem);
        HV<T> Zs = col(W.Zv, W.Zt, slot, nm), Xs = col(W.Xv, W.Xt, slot, nm);
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            Zs.v[i] = W.zp.v[i];
            Xs.v[i] = W.xip.v[i];
        }
        if (tm.leader()) {
            *Zs.t = *W.zp.t;
            *Xs.t = *W.xip.t;
        }
        ds.inserted++;
        if (ds.count < mem) ds.count++;
        tm.sync();
        // new Gram row: <xi_slot, xi_j> for all stored j, in chunks of 8
        for (int j0 = 0; j0 < ds.count; j0 += 8) {
            T a[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = 0;
            for (int i = tm.rank(); i < nm; i += tm.size()) {
                const T xs = Xs.v[i];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (j0 + q < ds.count) a[q] += xs * W.Xv[(size_t)(j0 + q) * nm + i];
            }
            double red[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) red[q] = (double)a[q];
            if (tm.leader()) {
                const double xt = *Xs.t;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (j0 + q < ds.count) red[q] += xt * W.Xt[j0 + q];
            }
            tm.reduce(red);
            if (threadIdx.x == 0) {
                for (int q = 0; q < 8 && j0 + q < ds.count; ++q) {
                    G[slot * AAMAX + j0 + q] = red[q];
                    G[(j0 + q) * AAMAX + slot] = red[q];
                }
            }
        }
    }
    const int k = ds.count;
    if (k == 0) {
        for (int i = tm.rank(); i < nm; i += tm.size()) W.d.v[i] = -W.Ru.v[i];
        if (tm.leader()) *W.d.t = -*W.Ru.t;
        tm.sync();
        return;
    }
    // rhs_j = <xi_j, Ru>
    for (int j0 = 0; j0 < k; j0 += 8) {
        T a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 0;
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            const T r = W.Ru.v[i];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < k) a[q] += r * W.Xv[(size_t)(j0 + q) * nm + i];
        }
        double red[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) red[q] = (double)a[q];
        if (tm.leader()) {
            const double rt = *W.Ru.t;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < k) red[q] += rt * W.Xt[j0 + q];
        }
        tm.reduce(red);
        if (threadIdx.x == 0)
            for (int q = 0; q < 8 && j0 + q < k; ++q) sm_rhs[j0 + q] = red[q];
    }
    __syncthreads();
    double tr = 0.0;
    for (int j = 0; j < k; ++j) tr += G[j * AAMAX + j];
    bool ok = false;
    if (tr > 0.0) ok = small_chol(G, sm_rhs, sm_L, sm_t, k, S.aa_reg * tr / k);
    // d = -Ru - sum_j t_j (Z_j - Xi_j)
    for (int i = tm.rank(); i < nm; i += tm.size()) {
        T di = -W.Ru.v[i];
        if (ok)
            for (int j = 0; j < k; ++j) di -= (T)sm_t[j] * (W.Zv[(size_t)j * nm + i] - W.Xv[(size_t)j * nm + i]);
        W.d.v[i] = di;
    }
    if (tm.leader()) {
        double di = -*W.Ru.t;
        if (ok)
            for (int j = 0; j < k; ++j) di -= sm_t[j] * (W.Zt[j] - W.Xt[j]);
        *W.d.t = di;
    }
    tm.sync();
}

// Anderson's acceleration with the least squares min ||Xi t - Ru|| solved
// through Xi = Q R (Sec. 4.4: an updated QR factorisation in place of the
// normal equations).  Q's columns are kept oldest first in W.Qv/W.Qt, R
// (upper triangular, row stride AAMAX) in the CTA's shared array G; Z and Xi
// stay in their ring slots (the oldest pair at (inserted - count) mod mem).
//  - a full window drops its oldest pair: R without its first column is upper
//    Hessenberg; Givens rotations (j, j+1), j = 0..k-2, restore the triangle
//    (computed by thread 0 of every CTA from identical data) and one pass
//    applies them to Q's columns, carrying column j+1 in a register;
//  - a new pair enters by two rounds of classical Gram-Schmidt (dots in
//    chunks of 8 per reduction); a remainder below 1e-14 ||xi|| is rank
//    deficient and the pair is not stored;
//  - t solves R t = Q^T Ru, d = -Ru - sum_j t_j (Z_j - Xi_j).
template <typename T, class Team>
__device__ void aa_qr_direction(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S,
                                bool have_pair, double nz2, DirState& ds, double* R, double* sm_h, double* sm_cs,
                                double* sm_t)
{
    const int nm = P.n + P.m;
    const int mem = S.mem;
    auto qcol = [&](int j) { return W.Qv + (size_t)j * nm; };
    auto slot_of = [&](int j) { return (int)((ds.inserted - ds.count + j) % mem); };  // ring slot of pair j
    if (have_pair && mem > 0 && nz2 > 0.0) {
        if (ds.count == mem) {
            const int k = ds.count;
            if (threadIdx.x == 0) {
                for (int j = 0; j + 1 < k; ++j) {
                    const double a = R[j * AAMAX + j + 1], b = R[(j + 1) * AAMAX + j + 1];
                    const double h = hypot(a, b);
                    const double c = h > 0.0 ? a / h : 1.0, sn = h > 0.0 ? b / h : 0.0;
                    for (int col = j + 1; col < k; ++col) {
                        const double x = R[j * AAMAX + col], y = R[(j + 1) * AAMAX + col];
                        R[j * AAMAX + col] = c * x + sn * y;
                        R[(j + 1) * AAMAX + col] = -sn * x + c * y;
                    }
                    sm_cs[2 * j] = c;
                    sm_cs[2 * j + 1] = sn;
                }
                for (int r = 0; r + 1 < k; ++r)
                    for (int col = 0; col + 1 < k; ++col) R[r * AAMAX + col] = col >= r ? R[r * AAMAX + col + 1] : 0.0;
                for (int col = 0; col < k; ++col) R[(k - 1) * AAMAX + col] = 0.0;
            }
            __syncthreads();
            for (int i = tm.rank(); i < nm; i += tm.size()) {
                T x = qcol(0)[i];
                for (int j = 0; j + 1 < k; ++j) {
                    const T y = qcol(j + 1)[i];
                    const T c = (T)sm_cs[2 * j], sn = (T)sm_cs[2 * j + 1];
                    qcol(j)[i] = c * x + sn * y;
                    x = -sn * x + c * y;
                }
            }
            if (tm.leader()) {
                double x = W.Qt[0];
                for (int j = 0; j + 1 < k; ++j) {
                    const double y = W.Qt[j + 1];
                    W.Qt[j] = sm_cs[2 * j] * x + sm_cs[2 * j + 1] * y;
                    x = -sm_cs[2 * j + 1] * x + sm_cs[2 * j] * y;
                }
            }
            ds.count = k - 1;
            tm.sync();
        }
        // append xi: the new column k of Q is built in place
        const int k = ds.count;
        const T* xi = W.xip.v;
        const double xit = *W.xip.t;
        T* w = qcol(k);
        double nxi2 = 0.0;
        for (int round = 0; round < 2; ++round) {
            const T* src = round == 0 ? xi : w;
            const double srct = round == 0 ? xit : W.Qt[k];
            // h_j = <q_j, src>, chunks of 8 (the first chunk of round 0 also reduces ||xi||^2)
            for (int j0 = 0; j0 < (k > 0 ? k : 1); j0 += 8) {
                T a[8];
                T x2 = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = 0;
                for (int i = tm.rank(); i < nm; i += tm.size()) {
                    const T v = src[i];
                    if (round == 0 && j0 == 0) x2 += v * v;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (j0 + q < k) a[q] += qcol(j0 + q)[i] * v;
                }
                double red[9];
#pragma unroll
                for (int q = 0; q < 8; ++q) red[q] = (double)a[q];
                red[8] = (double)x2;
                if (tm.leader()) {
                    if (round == 0 && j0 == 0) red[8] += srct * srct;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (j0 + q < k) red[q] += W.Qt[j0 + q] * srct;
                }
                tm.reduce(red);
                if (round == 0 && j0 == 0) nxi2 = red[8];
                if (threadIdx.x == 0)
                    for (int q = 0; q < 8 && j0 + q < k; ++q) sm_h[j0 + q] = red[q];
            }
            __syncthreads();
            // w = src - Q h (and ||w||^2 after the second round); R's new column accumulates h
            T ww = 0;
            for (int i = tm.rank(); i < nm; i += tm.size()) {
                T v = src[i];
                for (int j = 0; j < k; ++j) v -= (T)sm_h[j] * qcol(j)[i];
                w[i] = v;
                ww += v * v;
            }
            double red2[1] = {(double)ww};
            if (tm.leader()) {
                double v = srct;
                for (int j = 0; j < k; ++j) v -= sm_h[j] * W.Qt[j];
                W.Qt[k] = v;
                red2[0] += v * v;
            }
            tm.reduce(red2);
            if (threadIdx.x == 0)
                for (int j = 0; j < k; ++j) R[j * AAMAX + k] = (round == 0 ? 0.0 : R[j * AAMAX + k]) + sm_h[j];
            if (round == 1 && threadIdx.x == 0) sm_t[0] = red2[0];  // ||w||^2 after the second round
            __syncthreads();
        }
        const double rkk = sqrt(sm_t[0]);
        if (rkk > 1e-14 * sqrt(nxi2)) {
            const T inv = (T)(1.0 / rkk);
            const int slot = (int)(ds.inserted % mem);
            HV<T> Zs = col(W.Zv, W.Zt, slot, nm), Xs = col(W.Xv, W.Xt, slot, nm);
            for (int i = tm.rank(); i < nm; i += tm.size()) {
                w[i] *= inv;
                Zs.v[i] = W.zp.v[i];
                Xs.v[i] = xi[i];
            }
            if (tm.leader()) {
                W.Qt[k] /= rkk;
                *Zs.t = *W.zp.t;
                *Xs.t = xit;
            }
            if (threadIdx.x == 0) R[k * AAMAX + k] = rkk;
            ds.inserted++;
            ds.count++;
        }
        tm.sync();
    }
    const int k = ds.count;
    if (k == 0) {
        for (int i = tm.rank(); i < nm; i += tm.size()) W.d.v[i] = -W.Ru.v[i];
        if (tm.leader()) *W.d.t = -*W.Ru.t;
        tm.sync();
        return;
    }
    // Q^T Ru, then R t = Q^T Ru by back substitution (thread 0 of every CTA)
    for (int j0 = 0; j0 < k; j0 += 8) {
        T a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 0;
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            const T r = W.Ru.v[i];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < k) a[q] += qcol(j0 + q)[i] * r;
        }
        double red[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) red[q] = (double)a[q];
        if (tm.leader()) {
            const double rt = *W.Ru.t;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + q < k) red[q] += W.Qt[j0 + q] * rt;
        }
        tm.reduce(red);
        if (threadIdx.x == 0)
            for (int q = 0; q < 8 && j0 + q < k; ++q) sm_t[j0 + q] = red[q];
    }
    if (threadIdx.x == 0)
        for (int j = k - 1; j >= 0; --j) {
            double e = sm_t[j];
            for (int p = j + 1; p < k; ++p) e -= R[j * AAMAX + p] * sm_t[p];
            sm_t[j] = e / R[j * AAMAX + j];
        }
    __syncthreads();
    for (int i = tm.rank(); i < nm; i += tm.size()) {
        T di = -W.Ru.v[i];
        for (int j = 0; j < k; ++j) {
            const size_t o = (size_t)slot_of(j) * nm + i;
            di -= (T)sm_t[j] * (W.Zv[o] - W.Xv[o]);
        }
        W.d.v[i] = di;
    }
    if (tm.leader()) {
        double di = -*W.Ru.t;
        for (int j = 0; j < k; ++j) di -= sm_t[j] * (W.Zt[slot_of(j)] - W.Xt[slot_of(j)]);
        *W.d.t = di;
    }
    tm.sync();
}

// Restarted Broyden, Algorithm 2 (readings: m' = stored pairs; restart when
// m' = mem empties the buffers without storing the current pair; the
// denominator of z~ is <z, H xi~>; sgn(0) = 1).
template <typename T, class Team>
__device__ void rb_direction(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S,
                             bool have_pair, double nz2, DirState& ds)
{
    const int nm = P.n + P.m;
    HV<T> d = W.d, zt = W.zt, Ru = W.Ru, z = W.zp, xi = W.xip;
    if (!have_pair || !(nz2 > 0.0)) {
        for (int i = tm.rank(); i < nm; i += tm.size()) d.v[i] = -Ru.v[i];
        if (tm.leader()) *d.t = -*Ru.t;
        tm.sync();
        return;
    }
    const int cnt = ds.count;
    // pass 0: d = -Ru, zt = xi; dots with the first stored z (or with z when none)
    {
        const T* z0 = cnt > 0 ? W.Zv : z.v;
        const double z0t = cnt > 0 ? W.Zt[0] : *z.t;
        T a = 0, b = 0;
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            const T di = -Ru.v[i], zi = xi.v[i];
            d.v[i] = di;
            zt.v[i] = zi;
            a += z0[i] * zi;
            b += z0[i] * di;
        }
        double red[2] = {(double)a, (double)b};
        if (tm.leader()) {
            *d.t = -*Ru.t;
            *zt.t = *xi.t;
            red[0] += z0t * *xi.t;
            red[1] += z0t * (-*Ru.t);
        }
        tm.reduce(red);
        double ca = red[0], cb = red[1];
        // stored pairs: zt += <z^k, zt> z~^k ; d += <z^k, d> z~^k, dots for the next pair fused
        for (int k = 0; k < cnt; ++k) {
            const T* zk1 = (k + 1 < cnt) ? W.Zv + (size_t)(k + 1) * nm : z.v;
            const double zk1t = (k + 1 < cnt) ? W.Zt[k + 1] : *z.t;
            const T* ztk = W.Xv + (size_t)k * nm;
            const T ta = (T)ca, tb = (T)cb;
            T a2 = 0, b2 = 0;
            for (int i = tm.rank(); i < nm; i += tm.size()) {
                const T zti = zt.v[i] + ta * ztk[i];
                const T di = d.v[i] + tb * ztk[i];
                zt.v[i] = zti;
                d.v[i] = di;
                a2 += zk1[i] * zti;
                b2 += zk1[i] * di;
            }
            double red2[2] = {(double)a2, (double)b2};
            if (tm.leader()) {
                const double zti = *zt.t + ca * W.Xt[k];
                const double di = *d.t + cb * W.Xt[k];
                *zt.t = zti;
                *d.t = di;
                red2[0] += zk1t * zti;
                red2[1] += zk1t * di;
            }
            tm.reduce(red2);
            ca = red2[0];
            cb = red2[1];
        }
        // now ca = <z, H xi>, cb = <z, H(-r)>
        const double gamma = ca / nz2;
        const double sg = gamma >= 0.0 ? 1.0 : -1.0;
        const double theta = fabs(gamma) >= S.thetabar ? 1.0 : (1.0 - sg * S.thetabar) / (1.0 - gamma);
        // z~ = (z - ((1-theta) z + theta H xi)) / <z, (1-theta) z + theta H xi>
        const double den = (1.0 - theta) * nz2 + theta * ca;
        const bool store = cnt < S.mem;
        T* ztn = W.Xv + (size_t)cnt * nm;  // used only when storing
        T* zsn = W.Zv + (size_t)cnt * nm;
        const T f1 = (T)(theta / den);
        const T tcb = (T)cb;
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            const T zi = z.v[i];
            const T zn = f1 * (zi - zt.v[i]);
            d.v[i] += tcb * zn;
            if (store) {
                ztn[i] = zn;
                zsn[i] = zi;
            }
        }
        if (tm.leader()) {
            const double zi = *z.t;
            const double zn = (theta / den) * (zi - *zt.t);
            *d.t += cb * zn;
            if (store) {
                W.Xt[cnt] = zn;
                W.Zt[cnt] = zi;
            }
        }
        tm.sync();
        ds.count = store ? cnt + 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// outputs (Sec. 3.1 recovery rules)
// ---------------------------------------------------------------------------
template <typename T, class Team>
__device__ void write_outputs(Team& tm, const DevProb<T>& P, const DevWork<T>& W, int status, const TermOut& o)
{
    const int n = P.n, m = P.m;
    const double taub = *W.ub.t;
    const T* chib = W.ub.v;
    const T* psib = W.ub.v + n;
    for (int i = tm.rank(); i < m; i += tm.size()) {
        const double sig = (double)psib[i] - 2.0 * (double)W.ut.v[n + i] + (double)W.u.v[n + i];
        double yv, sv;
        if (status == ST_INFEASIBLE) {
            yv = (double)psib[i] / (-o.bpsi);
            sv = NAN;
        } else if (status == ST_UNBOUNDED) {
            yv = NAN;
            sv = sig / (-o.cchi);
        } else if (taub > 0.0) {
            yv = (double)psib[i] / taub;
            sv = sig / taub;
        } else {
            yv = NAN;
            sv = NAN;
        }
        W.y_out[i] = yv;
        W.s_out[i] = sv;
    }
    for (int j = tm.rank(); j < n; j += tm.size()) {
        double xv;
        if (status == ST_INFEASIBLE) xv = NAN;
        else if (status == ST_UNBOUNDED) xv = (double)chib[j] / (-o.cchi);
        else if (taub > 0.0) xv = (double)chib[j] / taub;
        else xv = NAN;
        W.x_out[j] = xv;
    }
    for (int i = tm.rank(); i < n + m; i += tm.size()) W.u_out[i] = (double)W.u.v[i];
    if (tm.leader()) W.u_out[n + m] = *W.u.t;
}

// ---------------------------------------------------------------------------
// Algorithm 1 with the linearity trick (Sec. 4.2).  Readings where the paper
// is silent: u0 = (0,0,1) unless warm; q^nu with nu the outer index; at most
// ls_max halvings, then alpha = 0 (the KM step); ||Rw|| = 0 is accepted as
// K1; secant pair z = w - u, xi = Rw - Ru of the last evaluated w; after K2
// the new u~ is solved from the new u; termination before the direction.
// ---------------------------------------------------------------------------
// Returns 1 (and writes no result) when a warm start is abandoned for the
// cold start; the caller then runs it again cold with the counts carried over.
template <typename T, class Team>
__device__ int superscs(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S, double* G,
                        double* sm_rhs, double* sm_L, double* sm_t, unsigned char* psd, bool use_warm,
                        int iter_base, long long cg_base, int& iters_out, long long& cg_out)
{
    const int n = P.n, m = P.m, nm = n + m;
    const double hg = W.st->hg;
    long long cg_total = cg_base;
    int k0 = 0, k1 = 0, k2 = 0, bt = 0;
    const double deadline = S.time_limit_ns > 0.0 ? (double)gtimer() + S.time_limit_ns : 0.0;
    // CG warm starts from zero unless the previous phase handed them over
    if (!S.keep_ws)
        for (int i = tm.rank(); i < n; i += tm.size()) {
            W.ws[0][i] = T(0);
            W.ws[1][i] = T(0);
        }
    // the PSD eigensolves' warm starts live within one solve: a solve neither depends on nor
    // profits from an earlier one (the flags are read after the next team barrier)
    if (W.psd_vok)
        for (int k = tm.rank(); k < P.ns; k += tm.size()) W.psd_vok[k] = 0;
    if (tm.leader() && iter_base == 0) {
        W.st->mat_passes = 0;
        W.st->mat_passes_ir = 0;
        W.st->cg_iters_ir = 0;
        W.st->ir_sweeps = 0;
        for (int k = 0; k < 5; ++k) W.st->part_ns[k] = 0.0;
        W.st->psd_resid = 0.0;
        W.st->psd_redo = 0;
        W.st->fallback = 0;
    }
    // residual of the cold start, the yardstick of the warm-start fallback
    double nRu_cold = INFINITY;
    const bool watch = use_warm && S.warm_fallback > 0;
    if (watch) {
        for (int i = tm.rank(); i < nm; i += tm.size()) W.u.v[i] = T(0);
        if (tm.leader()) *W.u.t = 1.0;
        tm.sync();
        cg_total += linsys(tm, P, W, W.u, W.ut, 0, S.cg_rtol, S.cg_max, hg, 0.0, S.refine != 0);
        OpResidual<T> op{W.u, W.ut, W.ub, W.Ru, T(0)};
        project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
        double red[1] = {(double)op.acc0};
        tm.reduce(red);
        nRu_cold = sqrt(red[0]);
    }
    // u0
    for (int i = tm.rank(); i < nm; i += tm.size()) W.u.v[i] = use_warm ? (T)W.warm[i] : T(0);
    if (tm.leader()) *W.u.t = use_warm ? W.warm[nm] : 1.0;
    tm.sync();
    cg_total += linsys(tm, P, W, W.u, W.ut, 0, S.cg_rtol, S.cg_max, hg, 0.0, S.refine != 0);
    double nRu;
    {
        OpResidual<T> op{W.u, W.ut, W.ub, W.Ru, T(0)};
        project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
        double red[1] = {(double)op.acc0};
        tm.reduce(red);
        nRu = sqrt(red[0]);
    }
    double eta0 = nRu, r_safe = nRu, eta = nRu, nz2 = 0.0;
    bool have_pair = false;
    DirState ds{0, 0};
    int nu_q = 0;  // outer iterations before this launch (the exponent of q^nu continues)
    if (S.resume && W.res->valid) {
        // continue the FP32 phase's iteration: its direction memory (Z, Xi and
        // the pending secant pair were widened by the hand-over), the Gram
        // matrix, and the K0/K1 references; u~, u_ and Ru were just evaluated
        // in this precision at the handed-over u
        const Resume* R = W.res;
        eta0 = R->eta0;
        eta = R->eta;
        r_safe = R->r_safe;
        nz2 = R->nz2;
        have_pair = R->have_pair != 0;
        ds.count = R->count;
        ds.inserted = R->inserted;
        nu_q = R->nu;
        if (S.direction == 0 || S.direction == 3)  // the Gram matrix, or R of the QR variant
            for (int i = threadIdx.x; i < AAMAX * AAMAX; i += blockDim.x) G[i] = R->G[i];
        __syncthreads();
    }
    int status = ST_MAX_ITERS;
    TermOut to;
    to.pr = to.dr = to.gap = to.ic = to.uc = INFINITY;
    to.pobj = to.dobj = NAN;
    to.bpsi = to.cchi = 0.0;
    double best_kkt = INFINITY;
    int best_it = 0;
    const int check_every = S.check_every > 0 ? S.check_every : 1;
    bool need_final_check = true;
    int nu;
    for (nu = 0; nu < S.max_iters - iter_base; ++nu) {
        if (tm.aborted()) break;
        if (watch && nu == S.warm_fallback && !(nRu < nRu_cold)) {
            iters_out = iter_base + nu;
            cg_out = cg_total;
            return 1;
        }
        if (!isfinite(nRu)) {
            if (watch) {
                iters_out = iter_base + nu;
                cg_out = cg_total;
                return 1;
            }
            status = ST_NUMERICAL;
            break;
        }
        unsigned long long tp = tm.leader() ? gtimer() : 0ull;  // start of this part
        auto part_end = [&](int k) {
            if (tm.leader()) {
                const unsigned long long t = gtimer();
                W.st->part_ns[k] += (double)(t - tp);
                tp = t;
            }
        };
        if (nu % check_every == 0) {
            const int st = termination(tm, P, W, S.eps, deadline, to);
            part_end(0);
            if (st != 0) {
                status = st;
                need_final_check = false;
                break;
            }
            if (to.time_up) {
                status = ST_TIME_LIMIT;
                need_final_check = false;
                break;
            }
            if (S.switch_kkt > 0.0 && fmax(to.pr, fmax(to.dr, to.gap)) <= S.switch_kkt) {
                status = ST_STALLED;  // hand over to the FP64 phase
                need_final_check = false;
                break;
            }
            if (S.stall_iters > 0) {
                // FP32 phase of SCS_MIXED: stop once ||Ru|| has not dropped 10% below
                // its best value for stall_iters iterations (the FP32 floor).  While
                // tau_ = 0 the residuals of Sec. 4.3 are undefined and the iterate is
                // still turning away from the tau axis, where ||Ru|| can plateau
                // without any floor being reached; a plateau with max(pr, dr, gap) still
                // above 100 times the hand-over level is not the FP32 floor either (the
                // FP32 phases measured here level off within a few times of it).  In
                // both cases the window is five times longer.
                const double kkt = fmax(to.pr, fmax(to.dr, to.gap));
                const bool far = !isfinite(to.pr) || (S.switch_kkt > 0.0 && kkt > 100.0 * S.switch_kkt);
                const int window = (S.stall_after_tau && far) ? 5 * S.stall_iters : S.stall_iters;
                if (nRu < 0.9 * best_kkt) {
                    best_kkt = nRu;
                    best_it = nu;
                } else if (nu - best_it >= window) {
                    status = ST_STALLED;
                    need_final_check = false;
                    break;
                }
            }
        }
        // direction d (Sec. 4.4)
        part_end(4);
        if (S.direction == 0)
            aa_direction(tm, P, W, S, have_pair, nz2, ds, G, sm_rhs, sm_L, sm_t);
        else if (S.direction == 3)
            aa_qr_direction(tm, P, W, S, have_pair, nz2, ds, G, sm_rhs, sm_L, sm_t);
        else if (S.direction == 1)
            rb_direction(tm, P, W, S, have_pair, nz2, ds);
        else {
            for (int i = tm.rank(); i < nm; i += tm.size()) W.d.v[i] = T(0);
            if (tm.leader()) *W.d.t = 0.0;
            tm.sync();
        }
        part_end(1);
        const double atol = S.cg_adapt > 0.0 ? S.cg_adapt * nRu : 0.0;
        cg_total += linsys(tm, P, W, W.d, W.dt, 1, S.cg_rtol, S.cg_max, hg, atol, S.refine != 0);
        double lin0 = 0.0;  // linear-solve time so far (a K2 step adds its own below)
        if (tm.leader()) {
            tp = gtimer();  // the linear solve timed itself
            lin0 = W.st->part_ns[2];
        }
        if (nRu <= S.c0 * eta) {
            // K0
            eta = nRu;
            OpK0<T> op{W.u, W.ut, W.ub, W.Ru, W.d, W.dt, W.zp, W.xip, T(0), T(0)};
            project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
            double red[2] = {(double)op.acc0, (double)op.acc1};
            tm.reduce(red);
            nRu = sqrt(red[0]);
            nz2 = red[1];
            ++k0;
        } else {
            double alpha = 1.0;
            for (int ls = 0; ls <= S.ls_max; ++ls) {
                if (ls == S.ls_max) alpha = 0.0;
                OpTrial<T> op{W.u, W.ut, W.d, W.dt, W.wb, W.Rw, alpha, T(0), T(0)};
                project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
                double red[2] = {(double)op.acc0, (double)op.acc1};
                tm.reduce(red);
                const double nRw = sqrt(red[0]);
                const double rho = red[1];
                if ((nRu <= r_safe && nRw <= S.c1 * nRu) || nRw == 0.0) {
                    // K1: u <- w, reuse w~, w_, Rw
                    r_safe = nRw + pow(S.q, (double)(nu + nu_q)) * eta0;
                    const T ta = (T)alpha;
                    T zz = 0;
                    for (int i = tm.rank(); i < nm; i += tm.size()) {
                        const T di = ta * W.d.v[i];
                        W.u.v[i] += di;
                        W.ut.v[i] += ta * W.dt.v[i];
                        W.ub.v[i] = W.wb.v[i];
                        W.zp.v[i] = di;
                        W.xip.v[i] = W.Rw.v[i] - W.Ru.v[i];
                        W.Ru.v[i] = W.Rw.v[i];
                        zz += di * di;
                    }
                    double red2[1] = {(double)zz};
                    if (tm.leader()) {
                        const double di = alpha * *W.d.t;
                        *W.u.t += di;
                        *W.ut.t += alpha * *W.dt.t;
                        *W.ub.t = *W.wb.t;
                        *W.zp.t = di;
                        *W.xip.t = *W.Rw.t - *W.Ru.t;
                        *W.Ru.t = *W.Rw.t;
                        red2[0] += di * di;
                    }
                    tm.reduce(red2);
                    nz2 = red2[0];
                    nRu = nRw;
                    ++k1;
                    break;
                } else if (rho >= S.sigma * nRu * nRw) {
                    // K2: u <- u - lambda rho / ||Rw||^2 Rw, then a fresh u~ solve
                    const double coef = S.lambda * rho / (nRw * nRw);
                    const T ta = (T)alpha, tc = (T)coef;
                    T zz = 0;
                    for (int i = tm.rank(); i < nm; i += tm.size()) {
                        const T di = ta * W.d.v[i];
                        W.zp.v[i] = di;
                        W.xip.v[i] = W.Rw.v[i] - W.Ru.v[i];
                        W.u.v[i] -= tc * W.Rw.v[i];
                        zz += di * di;
                    }
                    double red2[1] = {(double)zz};
                    if (tm.leader()) {
                        const double di = alpha * *W.d.t;
                        *W.zp.t = di;
                        *W.xip.t = *W.Rw.t - *W.Ru.t;
                        *W.u.t -= coef * *W.Rw.t;
                        red2[0] += di * di;
                    }
                    tm.reduce(red2);
                    nz2 = red2[0];
                    cg_total += linsys(tm, P, W, W.u, W.ut, 0, S.cg_rtol, S.cg_max, hg, atol, S.refine != 0);
                    OpResidual<T> opr{W.u, W.ut, W.ub, W.Ru, T(0)};
                    project_pass(tm, P, opr, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
                    double red3[1] = {(double)opr.acc0};
                    tm.reduce(red3);
                    nRu = sqrt(red3[0]);
                    ++k2;
                    break;
                }
                alpha *= 0.5;
                ++bt;
            }
        }
        have_pair = true;
        // the rest of the step (K0, line search, projections; K2's linear solve timed itself)
        if (tm.leader()) {
            const unsigned long long t = gtimer();
            W.st->part_ns[4] += (double)(t - tp) - (W.st->part_ns[2] - lin0);
        }
    }
    if (need_final_check && !tm.aborted()) {
        const int st = termination(tm, P, W, S.eps, 0.0, to);
        if (st != 0 && status != ST_NUMERICAL) status = st;
    }
    if (S.save_state) {
        // the loop state for a continuation in FP64 (the vectors stay in W)
        Resume* R = W.res;
        if (tm.leader()) {
            R->valid = 1;
            R->count = ds.count;
            R->inserted = ds.inserted;
            R->have_pair = have_pair ? 1 : 0;
            R->nu = nu + nu_q;
            R->eta = eta;
            R->eta0 = eta0;
            R->r_safe = r_safe;
            R->nz2 = nz2;
        }
        if (tm.block() == 0 && (S.direction == 0 || S.direction == 3))
            for (int i = threadIdx.x; i < AAMAX * AAMAX; i += blockDim.x) R->G[i] = G[i];
    }
    write_outputs(tm, P, W, status, to);
    iters_out = iter_base + nu;
    cg_out = cg_total;
    if (tm.leader()) {
        DevState* st = W.st;
        st->status = status;
        st->iters = iter_base + nu;
        st->k0 = k0;
        st->k1 = k1;
        st->k2 = k2;
        st->backtracks = bt;
        st->cg_iters = cg_total;
        st->pr = to.pr;
        st->dr = to.dr;
        st->gap = to.gap;
        st->ic = to.ic;
        st->uc = to.uc;
        st->nRu = nRu;
        if (status == ST_SOLVED || status == ST_MAX_ITERS || status == ST_TIME_LIMIT || status == ST_STALLED) {
            st->pobj = to.pobj;
            st->dobj = to.dobj;
        } else {
            st->pobj = NAN;
            st->dobj = NAN;
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// one entry for every mode
// ---------------------------------------------------------------------------
template <typename T, class Team>
__device__ void run_mode(Team& tm, const DevProb<T>& P, const DevWork<T>& W, const DevSettings& S, int mode, int slot,
                         double* G, double* sm_rhs, double* sm_L, double* sm_t, unsigned char* psd)
{
    const int n = P.n, m = P.m, nm = n + m;
    if (mode == MODE_FACTOR) {
        if constexpr (!Team::kGrid) {
            if (W.chol) chol_factor(tm, P, W);
        }
        return;
    }
    if (mode == MODE_SETUP) {
        // g = M^{-1}(c, b) from a zero start; ws[0] is zero on entry and left zero
        T* x = W.ws[0];
        double htp;
        const int it = minv(tm, P, W, P.c, P.b, x, S.cg_rtol, S.cg_max, htp);
        for (int i = tm.rank(); i < n; i += tm.size()) {
            W.g[i] = x[i];
            x[i] = T(0);
        }
        for (int i = tm.rank(); i < m; i += tm.size()) W.g[n + i] = W.py[i];
        if (tm.leader()) {
            W.st->hg = htp;
            W.st->setup_cg = it;
        }
        tm.sync();
        return;
    }
    if (mode == MODE_SOLVE) {
        int its = 0;
        long long cgs = 0;
        if (superscs(tm, P, W, S, G, sm_rhs, sm_L, sm_t, psd, S.use_warm != 0, 0, 0, its, cgs)) {
            // the warm start did not beat the cold start's residual: restart cold
            superscs(tm, P, W, S, G, sm_rhs, sm_L, sm_t, psd, false, its, cgs, its, cgs);
            if (tm.leader()) W.st->fallback = 1;
        }
        return;
    }
    if (mode == MODE_RESID) {
        // Sec. 4.3 residuals of a caller's candidate: x = io_in[0,n), y = io_in[n,n+m),
        // s = io_out2[0,m); io_out[0..2] = pr, dr, gap (FP64 data only)
        if constexpr (sizeof(T) == sizeof(double)) {
            const T* xv = W.io_in;
            const T* yv = W.io_in + n;
            const T* sv = W.io_out2;
            T* tmv = W.tm;
            T* tnv = W.tn;
            spmv(tm, P.A, xv, [&](int i, T v) { tmv[i] = v; });
            spmv(tm, P.AT, yv, [&](int j, T v) { tnv[j] = v; });
            tm.sync();
            double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            for (int i = tm.rank(); i < m; i += tm.size()) {
                const double bi = ro(P.b + i);
                const double e = tmv[i] + sv[i] - bi;
                a0 += e * e;
                a3 += bi * yv[i];
            }
            for (int j = tm.rank(); j < n; j += tm.size()) {
                const double cj = ro(P.c + j);
                const double g = tnv[j] + cj;
                a1 += g * g;
                a2 += cj * xv[j];
            }
            double red[4] = {a0, a1, a2, a3};
            tm.reduce(red);
            if (tm.leader()) {
                W.io_out[0] = sqrt(red[0]) / (1.0 + P.nb);
                W.io_out[1] = sqrt(red[1]) / (1.0 + P.nc);
                W.io_out[2] = fabs(red[2] + red[3]) / (1.0 + fabs(red[2]) + fabs(red[3]));
            }
            tm.sync();
        }
        return;
    }
    if (mode == MODE_SPMV) {
        // sparse products in precision T.  slot 0: io_out = A io_in[0,n);
        // slot 1: io_out = A^T io_in[0,m); slot 2: io_out = A^T io_in[0,m) and
        // io_out2 = A^T io_out2[0,m) in one fused pass.  x is staged at u's
        // start, y at u + n (the offset the solver's psi part has), the second
        // y in tm.
        T* xv = W.u.v;
        T* yv = W.u.v + n;
        T* y2 = W.tm;
        if (slot == 0) {
            for (int j = tm.rank(); j < n; j += tm.size()) xv[j] = (T)W.io_in[j];
        } else {
            for (int i = tm.rank(); i < m; i += tm.size()) {
                yv[i] = (T)W.io_in[i];
                if (slot == 2) y2[i] = (T)W.io_out2[i];
            }
        }
        tm.sync();
        if (slot == 0) {
            spmv(tm, P.A, xv, [&](int i, T v) { W.io_out[i] = (double)v; });
        } else if (slot == 1) {
            spmv(tm, P.AT, yv, [&](int j, T v) { W.io_out[j] = (double)v; });
        } else {
            spmv2(tm, P.AT, yv, y2, [&](int j, T v1, T v2) {
                W.io_out[j] = (double)v1;
                W.io_out2[j] = (double)v2;
            });
        }
        tm.sync();
        return;
    }
    if (mode == MODE_PROFILE) {
        // device-side timing of the solver's building blocks on this problem:
        // io_out[0..4] = ns per A pass, A^T pass, grid barrier, 1-value
        // reduction, and one CG iteration (A pass, barrier, A^T pass with
        // three dots, reduction, update pass, barrier)
        const int reps = slot > 0 ? slot : 10;
        T* xv = W.cp;
        T* yv = W.tm;
        T* zv = W.tn;
        for (int j = tm.rank(); j < n; j += tm.size()) {
            xv[j] = T(1) / T(1 + (j % 7));
            W.cr[j] = xv[j];
        }
        tm.sync();
        double t[6];
        t[0] = (double)gtimer();
        for (int r = 0; r < reps; ++r) {
            spmv(tm, P.A, xv, [&](int i, T s) { yv[i] = s; });
            tm.sync();
        }
        t[1] = (double)gtimer();
        for (int r = 0; r < reps; ++r) {
            spmv(tm, P.AT, yv, [&](int j, T s) { zv[j] = s; });
            tm.sync();
        }
        t[2] = (double)gtimer();
        for (int r = 0; r < reps; ++r) tm.sync();
        t[3] = (double)gtimer();
        for (int r = 0; r < reps; ++r) {
            double v1[1] = {1.0};
            tm.reduce(v1);
        }
        t[4] = (double)gtimer();
        T* q = W.cq;
        T* rr = W.cr;
        for (int r = 0; r < reps; ++r) {
            spmv(tm, P.A, xv, [&](int i, T s) { yv[i] = s; });
            tm.sync();
            T pq = 0, rq = 0, qq = 0;
            spmv(tm, P.AT, yv, [&](int j, T s) {
                const T qj = xv[j] + s;
                q[j] = qj;
                pq += xv[j] * qj;
                rq += rr[j] * qj;
                qq += qj * qj;
            });
            double red[4] = {(double)pq, (double)rq, (double)qq, 0.0};
            tm.reduce(red);
            const T ta = (T)(1e-30 * red[0]);
            for (int j = tm.rank(); j < n; j += tm.size()) {
                const T pj = xv[j];
                W.ws[1][j] += ta * pj;
                const T rj = rr[j] - ta * q[j];
                rr[j] = rj;
                xv[j] = rj + ta * pj;
            }
            tm.sync();
        }
        t[5] = (double)gtimer();
        if (tm.leader())
            for (int k = 0; k < 5; ++k) W.io_out[k] = (t[k + 1] - t[k]) / reps;
        tm.sync();
        return;
    }
    // single operators: io_in (FP64, N) -> u (T), results to io_out / io_out2
    for (int i = tm.rank(); i < nm; i += tm.size()) W.u.v[i] = (T)W.io_in[i];
    if (tm.leader()) {
        *W.u.t = W.io_in[nm];
        W.st->psd_resid = 0.0;
        W.st->psd_redo = 0;
    }
    tm.sync();
    if (mode == MODE_LINSYS) {
        // slot 0 / 1: the CG warm start of u~ / d~; + 2: by iterative refinement (FP64 data only)
        linsys(tm, P, W, W.u, W.ut, slot & 1, S.cg_rtol, S.cg_max, W.st->hg, 0.0, (slot & 2) != 0);
        for (int i = tm.rank(); i < nm; i += tm.size()) W.io_out[i] = (double)W.ut.v[i];
        if (tm.leader()) W.io_out[nm] = *W.ut.t;
    } else if (mode == MODE_PROJECT) {
        OpProject<T> op{W.u.v, W.u.t, W.ub.v, W.ub.t};
        project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
        tm.sync();
        for (int i = tm.rank(); i < nm; i += tm.size()) W.io_out[i] = (double)W.ub.v[i];
        if (tm.leader()) W.io_out[nm] = *W.ub.t;
    } else if (mode == MODE_APPLY_T) {
        linsys(tm, P, W, W.u, W.ut, 0, S.cg_rtol, S.cg_max, W.st->hg);
        OpResidual<T> op{W.u, W.ut, W.ub, W.Ru, T(0)};
        project_pass(tm, P, op, psd, PsdCheck{&W.st->psd_resid, &W.st->psd_redo, S.psd_tol, W.psd_v, P.v_off, W.psd_vok});
        tm.sync();
        for (int i = tm.rank(); i < nm; i += tm.size()) {
            W.io_out[i] = (double)W.u.v[i] - (double)W.Ru.v[i];
            W.io_out2[i] = (double)W.Ru.v[i];
        }
        if (tm.leader()) {
            W.io_out[nm] = *W.u.t - *W.Ru.t;
            W.io_out2[nm] = *W.Ru.t;
        }
    }
    tm.sync();
}

}  // namespace sscs
