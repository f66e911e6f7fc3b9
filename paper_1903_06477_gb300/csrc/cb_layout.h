// cb_layout.h -- host-side builder of the column-blocked sparse layout the
// grid team uses for large matrices (device side: Cblk, cb_spmv in
// solver.cuh).  Host code only; included by superscs.cu.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <thread>
#include <vector>

// One column-blocked copy of a matrix in one bulk precision (esize bytes per
// value); field meanings as in Cblk.
struct CbLayout {
    int ncb = 0, cw = 0, cols = 0, nw = 0, V = 1, acc_rows = 0, ms = 0, S = 0, stage_off = 0, stage_bytes = 0,
        off_x = 0, off_col = 0, off_val = 0, esize = 8;
    // two-dimensional tiles (tile = 1): R row blocks x ncb column blocks, tile
    // g = r * ncb + k on CTA g; its chunks are [cbeg[g], cbeg[g+1]) of meta
    int tile = 0, R = 0, rows = 0, nv = 1;
    std::vector<int> rbnd, meta, cbeg;
    std::vector<uint16_t> col;
    std::vector<double> val;
    size_t dyn() const { return ncb ? (size_t)stage_off + (size_t)S * stage_bytes : 0; }
    // partial sums of a tiled product: two buffers of nv vectors x ncb column blocks x rows
    size_t part_elems() const { return tile ? (size_t)2 * nv * ncb * rows : 0; }
};

// ---------------------------------------------------------------------------
// column-blocked layout (grid team)
// ---------------------------------------------------------------------------

// contiguous row ranges for G CTAs, balanced on (entries + 2) per row
static std::vector<int> cb_row_bounds(int rows, const std::vector<int>& rp, int G)
{
    std::vector<int> rb(G + 1, 0);
    const long long total = (long long)rp[rows] + 2LL * rows;
    int r = 0;
    for (int b = 1; b < G; ++b) {
        const long long target = total * b / G;
        while (r < rows && (long long)rp[r] + 2LL * r < target) ++r;
        rb[b] = r;
    }
    rb[G] = rows;
    return rb;
}

// The rows of CTA range [r0, r0 + R) bucketed by column block: cnt[k * R + lr]
// entries of local row lr in block k, their CSR indices in
// epos[start[k * R + lr] ...].
struct CbBuckets {
    std::vector<int> cnt, start, epos, fill;
    void build(int r0, int R, int ncb, int cw, const std::vector<int>& rp, const std::vector<int>& ci)
    {
        cnt.assign((size_t)ncb * R, 0);
        for (int lr = 0; lr < R; ++lr)
            for (int e = rp[r0 + lr]; e < rp[r0 + lr + 1]; ++e) cnt[(size_t)(ci[e] / cw) * R + lr]++;
        start.assign((size_t)ncb * R + 1, 0);
        for (size_t i = 0; i < (size_t)ncb * R; ++i) start[i + 1] = start[i] + cnt[i];
        epos.resize(start.back());
        fill.assign(start.begin(), start.end() - 1);
        for (int lr = 0; lr < R; ++lr)
            for (int e = rp[r0 + lr]; e < rp[r0 + lr + 1]; ++e) epos[fill[(size_t)(ci[e] / cw) * R + lr]++] = e;
    }
    // rows of block k with entries, by count descending (ties: row order)
    void sorted_rows(int k, int R, std::vector<int>& out) const
    {
        out.clear();
        for (int lr = 0; lr < R; ++lr)
            if (cnt[(size_t)k * R + lr] > 0) out.push_back(lr);
        std::stable_sort(out.begin(), out.end(),
                         [&](int a, int b) { return cnt[(size_t)k * R + a] > cnt[(size_t)k * R + b]; });
    }
};

// Deal slices (work = steps) to nw warps, largest first to the least-loaded
// warp.  Returns the warp of each slice; loads accumulate 2 * steps + 3.
static void cb_deal(const std::vector<int>& steps, int nw, std::vector<int>& warp, std::vector<long long>& load)
{
    load.assign(nw, 0);
    warp.resize(steps.size());
    for (size_t s = 0; s < steps.size(); ++s) {
        int best = 0;
        for (int w = 1; w < nw; ++w)
            if (load[w] < load[best]) best = w;
        warp[s] = best;
        load[best] += 2LL * steps[s] + 3;
    }
}

static void cb_slice_steps(const CbBuckets& bk, int k, int R, const std::vector<int>& rows, int V,
                           std::vector<int>& steps)
{
    const int H = 32 / V;
    const int ns = ((int)rows.size() + H - 1) / H;
    steps.resize(ns);
    for (int sl = 0; sl < ns; ++sl) steps[sl] = (bk.cnt[(size_t)k * R + rows[(size_t)sl * H]] + V - 1) / V;
}

// Lanes per row for the column-blocked layout: the V in {1, 2, 4, 8} with the
// least estimated time on a sample of CTAs -- per segment, the busiest
// warp's load plus eight times the mean load.  Segments are computed from
// shared memory while the matrix stream is the bound, so padding (the mean)
// weighs more than imbalance.
static int cb_pick_lanes(const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<int>& rb, int nw,
                         int ncb, int cw)
{
    const int G = (int)rb.size() - 1;
    const int stride = std::max(1, G / 16);
    long long cost[4] = {0, 0, 0, 0};
    CbBuckets bk;
    std::vector<int> rows, steps, warp;
    std::vector<long long> load;
    for (int b = 0; b < G; b += stride) {
        const int r0 = rb[b], R = rb[b + 1] - r0;
        bk.build(r0, R, ncb, cw, rp, ci);
        for (int k = 0; k < ncb; ++k) {
            bk.sorted_rows(k, R, rows);
            for (int vi = 0; vi < 4; ++vi) {
                cb_slice_steps(bk, k, R, rows, 1 << vi, steps);
                cb_deal(steps, nw, warp, load);
                long long mx = 0, sum = 0;
                for (long long l : load) {
                    mx = std::max(mx, l);
                    sum += l;
                }
                cost[vi] += mx + 8 * sum / nw;
            }
        }
    }
    int best = 0;
    for (int vi = 1; vi < 4; ++vi)
        if (cost[vi] < cost[best]) best = vi;
    return 1 << best;
}

// metadata words per segment for ns slices of H rows (layout of Cblk)
static int cb_meta_words(int nw, int ns, int H)
{
    return 5 + (nw + 1) + (ns + 1) + (ns * H + 1) / 2;
}

// Entry placement inside a slice.  Every lane of a step gathers one element
// of the vector slice from shared memory; lanes whose elements share a bank
// are served one after another.  The row of each lane is fixed, but which of
// its entries goes to which step is free, so each step takes, lane by lane,
// the row's remaining entry in the least-used bank (FP32: column mod 32 over
// the warp; FP64: column mod 16 within each half-warp, which is served
// separately).  Padding lanes point at a column in a free bank (value 0).  A
// staged slice starts at a shift that is the same for all its elements, so
// distinct banks stay distinct.  rem[rr] holds the CSR indices of the
// entries of the slice's row rr (consumed); the slice's nsteps x 32 entries
// are written at C.col / C.val [e0, ...) for column block k.
static void cb_place_slice(CbLayout& C, std::vector<std::vector<int>>& rem, size_t e0, int nsteps, int k, int cw,
                           int cols, int V, const std::vector<int>& ci, const std::vector<double>& vx)
{
    const int H = 32 / V;
    const int nbank = C.esize == 8 ? 16 : 32;
    const int len_k = std::min(cw, cols - k * cw);
    for (int t = 0; t < nsteps; ++t) {
        int cnt[2][32] = {};
        bool pad[32] = {};
        for (int q = 0; q < V; ++q)
            for (int rr = 0; rr < H; ++rr) {
                const int lane = q * H + rr, half = nbank == 16 ? lane >> 4 : 0;
                std::vector<int>& rl = rem[rr];
                if (rl.empty()) {
                    pad[lane] = true;
                    continue;
                }
                size_t best = 0;
                int bc = 1 << 30;
                for (size_t i = 0; i < rl.size(); ++i) {
                    const int c = cnt[half][(ci[rl[i]] - k * cw) % nbank];
                    if (c < bc) {
                        bc = c;
                        best = i;
                    }
                }
                const int e = rl[best];
                rl[best] = rl.back();
                rl.pop_back();
                const int lc = ci[e] - k * cw;
                cnt[half][lc % nbank]++;
                const size_t idx = e0 + (size_t)t * 32 + lane;
                C.col[idx] = (uint16_t)lc;
                C.val[idx] = vx[e];
            }
        for (int lane = 0; lane < 32; ++lane) {
            if (!pad[lane]) continue;
            const int half = nbank == 16 ? lane >> 4 : 0;
            int bb = 0;
            for (int b2 = 1; b2 < nbank && b2 < len_k; ++b2)
                if (cnt[half][b2] < cnt[half][bb]) bb = b2;
            cnt[half][bb]++;
            const size_t idx = e0 + (size_t)t * 32 + lane;
            C.col[idx] = (uint16_t)bb;
            C.val[idx] = 0.0;
        }
    }
}

// Build the column-blocked layout of a CSR matrix (rows x cols) for the row
// ranges rb, nw compute warps per CTA, blocks of cw columns and a ring of S
// stages.  The CTAs' segments are independent: a first pass sizes every
// segment, a prefix sum places them, and a second pass fills them; both
// passes split the CTAs over host threads, and the result is the same bit
// for bit whatever the thread count.
// Returns the largest segment (entries) or -1 if the layout is too large.
static long long build_cb(int rows, int cols, const std::vector<int>& rp, const std::vector<int>& ci,
                          const std::vector<double>& vx, const std::vector<int>& rb, int nw, int cw, int S,
                          CbLayout& C)
{
    (void)rows;
    const int G = (int)rb.size() - 1;
    const int ncb = (cols + cw - 1) / cw;
    const int V = cb_pick_lanes(rp, ci, rb, nw, ncb, cw);
    const int H = 32 / V;
    C.ncb = ncb;
    C.cw = cw;
    C.cols = cols;
    C.nw = nw;
    C.V = V;
    C.S = S;
    C.rbnd = rb;
    struct Seg {
        long long e0, e1;
        std::vector<int> words;  // [4] onwards of the segment's metadata
    };
    std::vector<Seg> segs((size_t)G * ncb);
    std::vector<long long> seg_len((size_t)G * ncb, 0);
    const int hw = (int)std::thread::hardware_concurrency();
    const int T = std::max(1, std::min(G, std::min(8, hw / 4)));
    auto parallel = [&](auto&& body) {  // body(b) for every CTA b, CTAs dealt round-robin to T threads
        std::vector<std::thread> th;
        for (int i = 1; i < T; ++i)
            th.emplace_back([&, i] {
                for (int b = i; b < G; b += T) body(b);
            });
        for (int b = 0; b < G; b += T) body(b);
        for (auto& t : th) t.join();
    };
    // pass 1: the entries of every segment
    parallel([&](int b) {
        thread_local CbBuckets bk;
        thread_local std::vector<int> rows_k, steps;
        const int r0 = rb[b], R = rb[b + 1] - r0;
        bk.build(r0, R, ncb, cw, rp, ci);
        for (int k = 0; k < ncb; ++k) {
            bk.sorted_rows(k, R, rows_k);
            cb_slice_steps(bk, k, R, rows_k, V, steps);
            long long e = 0;
            for (int st : steps) e += 32LL * st;
            seg_len[(size_t)b * ncb + k] = e;
        }
    });
    long long total = 0;
    for (size_t g = 0; g < segs.size(); ++g) {
        segs[g].e0 = total;
        total += seg_len[g];
        segs[g].e1 = total;
    }
    if (total >= (1LL << 31)) return -1;
    C.col.assign((size_t)total, 0);
    C.val.assign((size_t)total, 0.0);
    // pass 2: fill every segment at its place
    parallel([&](int b) {
        thread_local CbBuckets bk;
        thread_local std::vector<int> rows_k, steps, warp, order;
        thread_local std::vector<long long> load;
        thread_local std::vector<std::vector<int>> rem(32);
        const int r0 = rb[b], R = rb[b + 1] - r0;
        bk.build(r0, R, ncb, cw, rp, ci);
        for (int k = 0; k < ncb; ++k) {
            bk.sorted_rows(k, R, rows_k);
            cb_slice_steps(bk, k, R, rows_k, V, steps);
            cb_deal(steps, nw, warp, load);
            const int ns = (int)steps.size();
            order.resize(ns);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return warp[a] < warp[c]; });
            Seg& sg = segs[(size_t)b * ncb + k];
            std::vector<int> wstart(nw + 1, 0), sstart(ns + 1, 0);
            std::vector<uint16_t> srow((size_t)ns * H, 0xFFFF);
            int w = 0, t = 0;
            size_t e0 = (size_t)sg.e0;
            for (int oi = 0; oi < ns; ++oi) {
                const int sl = order[oi];
                while (w <= warp[sl]) wstart[w++] = oi;
                sstart[oi] = t;
                for (int rr = 0; rr < H; ++rr) {
                    const size_t pos = (size_t)sl * H + rr;
                    rem[rr].clear();
                    if (pos >= rows_k.size()) continue;
                    const int lr = rows_k[pos];
                    srow[(size_t)oi * H + rr] = (uint16_t)lr;
                    const size_t q0 = (size_t)bk.start[(size_t)k * R + lr];
                    const int len = bk.cnt[(size_t)k * R + lr];
                    for (int j = 0; j < len; ++j) rem[rr].push_back(bk.epos[q0 + j]);
                }
                cb_place_slice(C, rem, e0, steps[sl], k, cw, cols, V, ci, vx);
                e0 += (size_t)steps[sl] * 32;
                t += steps[sl];
            }
            sstart[ns] = t;
            while (w <= nw) wstart[w++] = ns;
            sg.words.clear();
            sg.words.push_back(ns);
            sg.words.insert(sg.words.end(), wstart.begin(), wstart.end());
            sg.words.insert(sg.words.end(), sstart.begin(), sstart.end());
            for (int i = 0; i < ns * H; i += 2) {
                const unsigned lo = srow[i], hi = i + 1 < ns * H ? srow[i + 1] : 0xFFFFu;
                sg.words.push_back((int)(lo | (hi << 16)));
            }
        }
    });
    int ms = 4;
    long long max_e = 0;
    for (const Seg& sg : segs) {
        ms = std::max(ms, 4 + (int)sg.words.size());
        max_e = std::max(max_e, sg.e1 - sg.e0);
    }
    ms = (ms + 3) & ~3;
    C.ms = ms;
    C.meta.assign((size_t)G * ncb * ms, 0);
    for (int b = 0; b < G; ++b)
        for (int k = 0; k < ncb; ++k) {
            const Seg& sg = segs[(size_t)b * ncb + k];
            int* m = C.meta.data() + ((size_t)b * ncb + k) * ms;
            m[0] = (int)sg.e0;
            m[1] = (int)sg.e1;
            const int k2 = (k + S) % ncb;  // visited S segments later (visits wrap around)
            m[2] = (int)segs[(size_t)b * ncb + k2].e0;
            m[3] = (int)segs[(size_t)b * ncb + k2].e1;
            std::copy(sg.words.begin(), sg.words.end(), m + 4);
        }
    return max_e;
}

// Plan (and build) the column-blocked copy of one matrix in one precision:
// nv vectors per product, dyn_max bytes of dynamic shared memory laid out as
// [2 nv partial-sum arrays | S stages of (metadata | vector slice | col | val)].
// The block width is sized so a stage holds one segment; a segment that
// turns out larger shrinks the width and the layout is rebuilt.  Leaves C
// empty (ncb = 0) where nothing fits or, unless forced, where the segments
// would be too short to pay for their per-segment cost.
static void plan_cb(int rows, int cols, const std::vector<int>& rp, const std::vector<int>& ci,
                    const std::vector<double>& vx, int G, int nw, int esize, int nv, size_t dyn_max, bool force,
                    CbLayout& C)
{
    // two stages of the largest size: measured against three and four, the
    // per-segment cost (metadata, waits, one flush per row and segment)
    // outweighs the deeper look-ahead
    constexpr int S = 2;
    C = CbLayout();
    C.esize = esize;
    const std::vector<int> rb = cb_row_bounds(rows, rp, G);
    int acc_rows = 0;
    long long nnz_cta = 0;
    for (int b = 0; b < G; ++b) {
        acc_rows = std::max(acc_rows, rb[b + 1] - rb[b]);
        nnz_cta = std::max<long long>(nnz_cta, rp[rb[b + 1]] - rp[rb[b]]);
    }
    if (acc_rows >= 0xFFFF || nw < 1) return;
    const int E = 16 / esize;
    // partial sums: two buffers (even / odd segments) per multiplied vector
    const size_t acc_bytes = ((size_t)2 * nv * std::max(acc_rows, 1) * esize + 15) & ~size_t(15);
    if (acc_bytes + 4096 > dyn_max) return;
    const long long stage_avail = (long long)((dyn_max - acc_bytes) / S) & ~15LL;
    // metadata bound: at most ceil(acc_rows / H) slices, H >= 4
    const int ms_cap = (cb_meta_words(nw, (acc_rows + 3) / 4, 4) + 16 + 3) & ~3;
    const double per_col = esize + 1.15 * (2 + esize) * (double)nnz_cta / std::max(cols, 1);
    long long budget = stage_avail - 4LL * ms_cap - 64 - 2LL * E * esize;
    int cw = (int)std::min<double>(65536.0, budget / per_col) & ~3;
    const long long nnz = rp[rows];
    for (int attempt = 0; attempt < 8 && cw >= 64; ++attempt) {
        const int ncb = (cols + cw - 1) / cw;
        const int cw2 = ((cols + ncb - 1) / ncb + 3) & ~3;
        if (!force && nnz < 1024LL * G * ncb) return;
        const long long max_e = build_cb(rows, cols, rp, ci, vx, rb, nw, cw2, S, C);
        if (max_e < 0) break;
        const long long off_x = 4LL * C.ms;
        const long long off_col = off_x + (((long long)(cw2 + 2 * E) * esize + 15) & ~15LL);
        const long long off_val = off_col + ((2 * max_e + 15) & ~15LL);
        const long long bytes = off_val + ((max_e * esize + 15) & ~15LL);
        if (bytes <= stage_avail) {
            C.esize = esize;
            C.acc_rows = acc_rows;
            C.stage_off = (int)acc_bytes;
            C.stage_bytes = (int)bytes;
            C.off_x = (int)off_x;
            C.off_col = (int)off_col;
            C.off_val = (int)off_val;
            return;
        }
        cw = (int)((double)cw2 * 0.95 * (double)stage_avail / (double)bytes) & ~3;
    }
    C = CbLayout();
}


// ---------------------------------------------------------------------------
// two-dimensional tiles (grid team)
// ---------------------------------------------------------------------------
// Tile (r, k) is row block r (rows rb[r] .. rb[r+1], balanced on entries)
// times column block k (cw columns) and runs on CTA r * ncb + k, which keeps
// only that column block of the multiplied vector in shared memory, copied
// once per product.  The tile's rows with entries in the block, by count
// descending, form slices of H = 32 / V rows (sliced ELL as above);
// consecutive slices are grouped into chunks that fit one stage of the copy
// ring (metadata, 16-bit column offsets, values), and inside a chunk the
// slices are dealt to the compute warps.  Every row of a tile lies in one
// slice, so its sum is complete when its slice is done: it goes to a
// per-tile row array in shared memory, which is written to the partial sums
// part[k][row] (global) once the tile is done; a second pass over the rows
// adds the ncb partials in block order.  Chunk metadata (ms words per chunk;
// the chunks of tile g are cbeg[g] .. cbeg[g+1]):
//   [0] E0  [1] E1  [2], [3] E0, E1 of the tile's chunk S later (0, 0: none)
//   [4] ns: slices  [5 .. 5+nw] first slice of each warp (nw+1 values)
//   [6+nw .. 6+nw+ns] slice start steps from E0 (ns+1 values)
//   then ns * H 16-bit row indices inside the row block (0xFFFF: none), two
//   per word, low half first.
// Chunks hold at most e_cap entries and ms_cap metadata words.  Returns false
// if one slice alone exceeds them.
static bool build_tile(int cols, const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<double>& vx,
                       const std::vector<int>& rb, int Cn, int cw, int nw, int S, int V, long long e_cap, int ms_cap,
                       CbLayout& L)
{
    const int R = (int)rb.size() - 1;
    const int H = 32 / V;
    L.tile = 1;
    L.R = R;
    L.ncb = Cn;
    L.cw = cw;
    L.cols = cols;
    L.nw = nw;
    L.V = V;
    L.S = S;
    L.rbnd = rb;
    L.col.clear();
    L.val.clear();
    L.cbeg.assign((size_t)R * Cn + 1, 0);
    struct Chunk {
        long long e0, e1;
        std::vector<int> words;  // [4] onwards
    };
    std::vector<Chunk> chunks;
    CbBuckets bk;
    std::vector<int> rows_k, steps, sub, warp, order;
    std::vector<long long> load;
    std::vector<std::vector<int>> rem(32);
    int ms = 4;
    for (int r = 0; r < R; ++r) {
        const int r0 = rb[r], Rr = rb[r + 1] - r0;
        bk.build(r0, Rr, Cn, cw, rp, ci);
        for (int k = 0; k < Cn; ++k) {
            L.cbeg[(size_t)r * Cn + k] = (int)chunks.size();
            bk.sorted_rows(k, Rr, rows_k);
            cb_slice_steps(bk, k, Rr, rows_k, V, steps);
            const int nst = (int)steps.size();
            for (int sl = 0; sl < nst;) {
                // the longest run of slices within both caps
                long long e = 0;
                int ns = 0;
                while (sl + ns < nst) {
                    const long long add = 32LL * steps[sl + ns];
                    if (e + add > e_cap || cb_meta_words(nw, ns + 1, H) > ms_cap) break;
                    e += add;
                    ++ns;
                }
                if (ns == 0) return false;
                sub.assign(steps.begin() + sl, steps.begin() + sl + ns);
                cb_deal(sub, nw, warp, load);
                order.resize(ns);
                std::iota(order.begin(), order.end(), 0);
                std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return warp[a] < warp[c]; });
                Chunk ch;
                ch.e0 = (long long)L.col.size();
                std::vector<int> wstart(nw + 1, 0), sstart(ns + 1, 0);
                std::vector<uint16_t> srow((size_t)ns * H, 0xFFFF);
                int w = 0, t = 0;
                for (int oi = 0; oi < ns; ++oi) {
                    const int ls = order[oi], gs = sl + ls;
                    while (w <= warp[ls]) wstart[w++] = oi;
                    sstart[oi] = t;
                    const size_t e0 = L.col.size();
                    const size_t size = (size_t)steps[gs] * 32;
                    L.col.resize(e0 + size, 0);
                    L.val.resize(e0 + size, 0.0);
                    for (int rr = 0; rr < H; ++rr) {
                        const size_t pos = (size_t)gs * H + rr;
                        rem[rr].clear();
                        if (pos >= rows_k.size()) continue;
                        const int lr = rows_k[pos];
                        srow[(size_t)oi * H + rr] = (uint16_t)lr;
                        const size_t q0 = (size_t)bk.start[(size_t)k * Rr + lr];
                        const int len = bk.cnt[(size_t)k * Rr + lr];
                        for (int j = 0; j < len; ++j) rem[rr].push_back(bk.epos[q0 + j]);
                    }
                    cb_place_slice(L, rem, e0, steps[gs], k, cw, cols, V, ci, vx);
                    t += steps[gs];
                }
                sstart[ns] = t;
                while (w <= nw) wstart[w++] = ns;
                ch.e1 = (long long)L.col.size();
                ch.words.push_back(ns);
                ch.words.insert(ch.words.end(), wstart.begin(), wstart.end());
                ch.words.insert(ch.words.end(), sstart.begin(), sstart.end());
                for (int i = 0; i < ns * H; i += 2) {
                    const unsigned lo = srow[i], hi = i + 1 < ns * H ? srow[i + 1] : 0xFFFFu;
                    ch.words.push_back((int)(lo | (hi << 16)));
                }
                ms = std::max(ms, 4 + (int)ch.words.size());
                chunks.push_back(std::move(ch));
                sl += ns;
            }
        }
    }
    L.cbeg[(size_t)R * Cn] = (int)chunks.size();
    if (L.col.size() >= (1ull << 31)) return false;
    ms = (ms + 3) & ~3;
    L.ms = ms;
    L.meta.assign(chunks.size() * (size_t)ms, 0);
    for (int g = 0; g < R * Cn; ++g)
        for (int j = L.cbeg[g]; j < L.cbeg[g + 1]; ++j) {
            const Chunk& ch = chunks[j];
            int* m = L.meta.data() + (size_t)j * ms;
            m[0] = (int)ch.e0;
            m[1] = (int)ch.e1;
            if (j + S < L.cbeg[g + 1]) {
                m[2] = (int)chunks[j + S].e0;
                m[3] = (int)chunks[j + S].e1;
            }
            std::copy(ch.words.begin(), ch.words.end(), m + 4);
        }
    return true;
}

// Plan (and build) the tiled copy of one matrix in one precision for G CTAs
// of nw compute warps and nv vectors per product, in dyn_max bytes of dynamic
// shared memory laid out as [row sums of one tile | vector slice | S stages
// of (metadata | col | val)].  The splits G = R x ncb that fit (rows per
// block below 0xFFFF, stages of at least 16 KB) are ranked by estimated time
// -- the partial sums written and read back, the vector slices copied, a
// fixed cost per chunk -- and the first one whose slices all fit a stage is
// built (a long row in a narrow split can need more than a stage; wider
// splits shorten it).  Leaves L empty (ncb = 0) where no split works or,
// unless forced, where the tiles would hold fewer than 4096 entries on
// average.
constexpr int TILE_STAGES = 2;  // stages of the tiles' copy ring

static void plan_tile(int rows, int cols, const std::vector<int>& rp, const std::vector<int>& ci,
                      const std::vector<double>& vx, int G, int nw, int esize, int nv, size_t dyn_max, bool force,
                      CbLayout& L)
{
    constexpr int S = TILE_STAGES;
    L = CbLayout();
    L.esize = esize;
    const long long nnz = rp[rows];
    if (nw < 1 || G < 1 || rows < 1 || cols < 1 || (!force && nnz < 4096LL * G)) return;
    const int E = 16 / esize;
    struct Split {
        int Cn, cw, acc_rows;
        long long acc_bytes, slice_bytes, stage;
        std::vector<int> rb;
    };
    auto split = [&](int Cn, Split& sp) {
        const int R = G / Cn;
        sp.Cn = Cn;
        sp.cw = (int)((((long long)cols + Cn - 1) / Cn + 3) & ~3LL);
        if (sp.cw > 65536 || (long long)(Cn - 1) * sp.cw >= cols || R > rows) return false;
        sp.rb = cb_row_bounds(rows, rp, R);
        sp.acc_rows = 0;
        for (int r = 0; r < R; ++r) sp.acc_rows = std::max(sp.acc_rows, sp.rb[r + 1] - sp.rb[r]);
        if (sp.acc_rows >= 0xFFFF) return false;
        sp.acc_bytes = ((long long)sp.acc_rows * esize + 15) & ~15LL;
        sp.slice_bytes = ((long long)(sp.cw + 2 * E) * esize + 15) & ~15LL;
        sp.stage = ((long long)dyn_max - sp.acc_bytes - sp.slice_bytes) / S & ~15LL;
        return sp.stage >= 16384;
    };
    std::vector<std::pair<double, int>> cand;
    for (int Cn = 1; Cn <= G; ++Cn) {
        Split sp;
        if (G % Cn || !split(Cn, sp)) continue;
        const double bytes = (double)nv * (2.0 * Cn * rows + (double)G * sp.cw) * esize;
        const double chunks = std::ceil(1.15 * (double)nnz * (2 + esize) / G / (0.85 * sp.stage)) * nv;
        cand.emplace_back(bytes / 6.8e12 + chunks * 0.3e-6, Cn);
    }
    std::sort(cand.begin(), cand.end());
    for (const auto& cd : cand) {
        Split sp;
        split(cd.second, sp);
        const int Cn = sp.Cn, R = G / Cn;
        const int V = cb_pick_lanes(rp, ci, sp.rb, nw, Cn, sp.cw);
        const int H = 32 / V;
        // metadata share of a stage from the mean slice (sampled row blocks):
        // 1 + H/2 words per slice against 32 x steps entries of 2 + esize bytes
        long long nslices = 0, nsteps = 0;
        {
            CbBuckets bk;
            std::vector<int> rows_k, steps;
            const int stride = std::max(1, R / 8);
            for (int r = 0; r < R; r += stride) {
                const int Rr = sp.rb[r + 1] - sp.rb[r];
                bk.build(sp.rb[r], Rr, Cn, sp.cw, rp, ci);
                for (int k = 0; k < Cn; ++k) {
                    bk.sorted_rows(k, Rr, rows_k);
                    cb_slice_steps(bk, k, Rr, rows_k, V, steps);
                    nslices += (long long)steps.size();
                    for (int st : steps) nsteps += st;
                }
            }
        }
        const double per_slice_meta = 4.0 * (1 + H / 2.0);
        const double per_slice_entries =
            32.0 * (2 + esize) * std::max(1.0, (double)nsteps / std::max<long long>(nslices, 1));
        const double frac = std::min(0.5, 1.3 * per_slice_meta / (per_slice_meta + per_slice_entries));
        const int ms_cap = std::max(cb_meta_words(nw, 1, H) + 4, (int)(frac * sp.stage / 4) & ~3);
        // entries: 2-byte offsets and esize-byte values, each region 16-byte aligned
        const long long e_cap = ((sp.stage - 4LL * ms_cap - 32) / (2 + esize)) & ~31LL;
        L = CbLayout();
        L.esize = esize;
        if (e_cap < 32 || !build_tile(cols, rp, ci, vx, sp.rb, Cn, sp.cw, nw, S, V, e_cap, ms_cap, L)) continue;
        long long max_e = 0;
        const size_t nch = L.meta.size() / (size_t)L.ms;
        for (size_t j = 0; j < nch; ++j) max_e = std::max<long long>(max_e, L.meta[j * L.ms + 1] - L.meta[j * L.ms]);
        L.rows = rows;
        L.nv = nv;
        L.acc_rows = sp.acc_rows;
        L.off_x = (int)sp.acc_bytes;
        L.stage_off = (int)(sp.acc_bytes + sp.slice_bytes);
        L.off_col = (4 * L.ms + 15) & ~15;
        L.off_val = L.off_col + (int)((2 * max_e + 15) & ~15LL);
        L.stage_bytes = L.off_val + (int)((max_e * esize + 15) & ~15LL);
        if ((long long)L.stage_bytes <= sp.stage) return;
    }
    L = CbLayout();
}
