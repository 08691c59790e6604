// Tile and K-step lists of the tensor-core products (the symbolic half of
// Algorithm 1's Gustavson merge, lifted to tiles of TBM x TBN blocks), shared
// by the tensor-core kernels.  A geometry G supplies TBM, TBN, kSlots =
// TBM + TBN, kColOff = 4 + TBM * TBN and kTileInts = kColOff + TBN.
#pragma once

#include <algorithm>

#include "tc_gemm.cuh"

namespace rdm {
namespace {

template <int TBM_, int TBN_>
struct PlanGeo {
    static constexpr int TBM = TBM_;                    // block rows per tile
    static constexpr int TBN = TBN_;                    // block columns per tile
    static constexpr int kSlots = TBM + TBN;            // operand blocks per K-step: A rows, then B rows
    static constexpr int kColOff = 4 + TBM * TBN;       // tile record: job, super-row, -, nsteps,
    static constexpr int kTileInts = kColOff + TBN;     //   mask slot[TBM x TBN], column j of each tile column
    static_assert(kSlots <= 32, "one producer lane per slot");
};

// ---------------------------------------------------------------------------
// tile lists
// ---------------------------------------------------------------------------
struct TileBuild {
    const int *rp;       // input set row_ptr (flat)
    const int *col;
    int NB, NBT;         // block rows, super-rows (ceil(NB / TBM))
    JobTable jt;
    const int *out_rp;   // mask row_ptr (flat, njob*NB+1)
    const int *mcol;     // mask columns
    const int *sys_of_row, *active, *sys_tier;
    JobMask job_mask;    // jobs computed on the tensor cores, per tier
    int u0, u1;          // super-row units (job * NBT + I) of this plan
    int *tile_cnt;       // [u1 - u0]
    const int *tile_off; // scanned
    int *tiles;          // [ntile * kTileInts]
    int *step_cnt;       // [ntile]
    const int64_t *step_off;
    int *steps;          // [nsteps * kSlots]
    int ntile;
    int max_words;       // bitmap window in 32-column words (<= 512); wider windows: serial merge
    const int *tpos;     // K-step entries point at tpos[e] (the planes' position), or at e if null
};

// upper mask range [cur, end) of block row TBM I + m of job p, empty for rows
// whose system is converged or whose job is not computed on the tensor cores
template <class G>
__device__ __forceinline__ void tile_row_range(const TileBuild &T, int p, int I, int m, int &cur, int &end) {
    const int i = G::TBM * I + m;
    cur = end = 0;
    if (i >= T.NB) return;
    int lo = T.out_rp[p * T.NB + i], hi = T.out_rp[p * T.NB + i + 1];
    end = hi;
    // first column >= i (upper triangle)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T.mcol[mid] < i) lo = mid + 1; else hi = mid;
    }
    cur = lo;
    // converged systems keep their blocks through the copy path of the
    // numeric phase, and jobs on the CUDA cores have their own launch:
    // neither produces tiles
    const int sys = T.sys_of_row[i];
    if (!T.active[sys] || !((T.job_mask.m[T.sys_tier[sys] & (kMaxTiers - 1)] >> p) & 1u)) cur = end;
}

// Tiles of one (job, super-row), warp-parallel: the upper mask columns of
// the TBM block rows are marked in a shared-memory bitmap over their column
// window; the rank of a column among the distinct ones (prefix popcounts)
// gives its tile (rank / TBN) and tile column (rank % TBN).  Windows wider
// than the bitmap fall back to a serial merge by lane 0 (count or fill).
constexpr int kTileRowWarps = 8, kTileRowWords = 512;   // 16,384 columns per window
template <class G>
__device__ void tile_rows_serial(const TileBuild &T, int t, int p, int I, const int *cur0, const int *end0,
                                 int fill);
template <class G>
__global__ void __launch_bounds__(32 * kTileRowWarps) k_tile_rows(TileBuild T, int fill) {
    __shared__ unsigned bits_s[kTileRowWarps][kTileRowWords];
    __shared__ int rank_s[kTileRowWarps][kTileRowWords];
    const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = T.u0 + blockIdx.x * kTileRowWarps + wq;
    if (t >= T.u1) return;
    const int p = t / T.NBT, I = t % T.NBT;
    unsigned *bm = bits_s[wq];
    int *wr = rank_s[wq];
    int c0 = 0, e0 = 0;
    if (lane < G::TBM) tile_row_range<G>(T, p, I, lane, c0, e0);
    int cur[G::TBM], end[G::TBM];
    int lo = 0x7fffffff, hi = -1;
#pragma unroll
    for (int m = 0; m < G::TBM; ++m) {
        cur[m] = __shfl_sync(0xffffffffu, c0, m);
        end[m] = __shfl_sync(0xffffffffu, e0, m);
        if (cur[m] < end[m]) {
            lo = min(lo, T.mcol[cur[m]]);
            hi = max(hi, T.mcol[end[m] - 1]);
        }
    }
    const int base = fill ? T.tile_off[t - T.u0] : 0;
    if (hi < lo) {                         // no tile
        if (!fill && lane == 0) T.tile_cnt[t - T.u0] = 0;
        return;
    }
    const int nw = ((hi - lo) >> 5) + 1;
    if (nw > T.max_words) {
        if (lane == 0) tile_rows_serial<G>(T, t, p, I, cur, end, fill);
        return;
    }
    for (int w = lane; w < nw; w += 32) bm[w] = 0u;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < G::TBM; ++m)
        for (int e = cur[m] + lane; e < end[m]; e += 32) {
            const int j = T.mcol[e] - lo;
            atomicOr(&bm[j >> 5], 1u << (j & 31));
        }
    __syncwarp();
    // exclusive prefix of the words' popcounts
    int carry = 0;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        const int c = w < nw ? __popc(bm[w]) : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (w < nw) wr[w] = carry + x - c;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    __syncwarp();
    const int ndist = carry, ntile = (ndist + G::TBN - 1) / G::TBN;
    if (!fill) {
        if (lane == 0) T.tile_cnt[t - T.u0] = ntile;
        return;
    }
    for (int q = lane; q < ntile; q += 32) {
        int *d = T.tiles + (size_t)(base + q) * G::kTileInts;
        d[0] = p; d[1] = I; d[2] = -1; d[3] = 0;
        for (int k = 4; k < G::kTileInts; ++k) d[k] = -1;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < G::TBM; ++m)
        for (int e = cur[m] + lane; e < end[m]; e += 32) {
            const int jc = T.mcol[e];
            const int j = jc - lo;
            const int r = wr[j >> 5] + __popc(bm[j >> 5] & ((1u << (j & 31)) - 1u));
            int *d = T.tiles + (size_t)(base + r / G::TBN) * G::kTileInts;
            d[4 + m * G::TBN + r % G::TBN] = e;
            d[G::kColOff + r % G::TBN] = jc;
        }
}

// the serial TBM-way merge (same tile order as the bitmap path)
template <class G>
__device__ void tile_rows_serial(const TileBuild &T, int t, int p, int I, const int *cur0, const int *end0,
                                 int fill) {
    int cur[G::TBM], end[G::TBM];
    for (int m = 0; m < G::TBM; ++m) { cur[m] = cur0[m]; end[m] = end0[m]; }
    // the distinct columns needed by the TBM rows, in increasing order, are
    // packed TBN at a time into tiles: every tile column is needed by at least
    // one row
    int ncol = 0, n = 0;
    const int base = fill ? T.tile_off[t - T.u0] : 0;
    int *d = nullptr;
    // list heads kept in registers: one load per advance
    int head[G::TBM];
#pragma unroll
    for (int m = 0; m < G::TBM; ++m) head[m] = cur[m] < end[m] ? T.mcol[cur[m]] : 0x7fffffff;
    while (true) {
        int jmin = 0x7fffffff;
#pragma unroll
        for (int m = 0; m < G::TBM; ++m) jmin = min(jmin, head[m]);
        if (jmin == 0x7fffffff) break;
        const int c = ncol % G::TBN;
        if (c == 0) {
            if (fill) {
                d = T.tiles + (size_t)(base + n) * G::kTileInts;
                d[0] = p; d[1] = I; d[2] = -1; d[3] = 0;
                for (int q = 4; q < G::kTileInts; ++q) d[q] = -1;
            }
            ++n;
        }
        if (fill) d[G::kColOff + c] = jmin;
#pragma unroll
        for (int m = 0; m < G::TBM; ++m)
            if (head[m] == jmin) {
                if (fill) d[4 + m * G::TBN + c] = cur[m];
                ++cur[m];
                head[m] = cur[m] < end[m] ? T.mcol[cur[m]] : 0x7fffffff;
            }
        ++ncol;
    }
    if (!fill) T.tile_cnt[t - T.u0] = n;
}

// one thread per tile: K-steps = union over the tile's A rows intersected with
// the union over its B rows, for each term (count or fill)
template <class G>
__device__ void tile_steps_serial(const TileBuild &T, int t, int fill) {
    const int *d = T.tiles + (size_t)t * G::kTileInts;
    const int p = d[0], I = d[1];
    const Job &job = T.jt.job[p];
    int64_t w = fill ? T.step_off[t] : 0;
    int n = 0;
    for (int term = 0; term < job.nterm; ++term) {
        const int am = job.a[term], bm = job.b[term];
        int cur[G::kSlots], end[G::kSlots];
        for (int q = 0; q < G::TBM; ++q) {
            const int i = G::TBM * I + q;
            cur[q] = end[q] = 0;
            if (i < T.NB) { cur[q] = T.rp[am * T.NB + i]; end[q] = T.rp[am * T.NB + i + 1]; }
        }
        for (int q = 0; q < G::TBN; ++q) {
            const int j = d[G::kColOff + q];
            cur[G::TBM + q] = end[G::TBM + q] = 0;
            if (j >= 0) { cur[G::TBM + q] = T.rp[bm * T.NB + j]; end[G::TBM + q] = T.rp[bm * T.NB + j + 1]; }
        }
        // list heads kept in registers: one load per advance
        int head[G::kSlots];
#pragma unroll
        for (int q = 0; q < G::kSlots; ++q) head[q] = cur[q] < end[q] ? T.col[cur[q]] : 0x7fffffff;
        while (true) {
            int kmin = 0x7fffffff;
#pragma unroll
            for (int q = 0; q < G::kSlots; ++q) kmin = min(kmin, head[q]);
            if (kmin == 0x7fffffff) break;
            bool anyA = false, anyB = false;
            int idx[G::kSlots];
#pragma unroll
            for (int q = 0; q < G::kSlots; ++q) {
                idx[q] = -1;
                if (head[q] == kmin) {
                    idx[q] = cur[q];
                    ++cur[q];
                    head[q] = cur[q] < end[q] ? T.col[cur[q]] : 0x7fffffff;
                    if (q < G::TBM) anyA = true; else anyB = true;
                }
            }
            if (anyA && anyB) {
                if (fill && w + n < T.step_off[t + 1]) {
                    int *s = T.steps + (size_t)(w + n) * G::kSlots;
                    for (int q = 0; q < G::kSlots; ++q) s[q] = idx[q] >= 0 && T.tpos ? T.tpos[idx[q]] : idx[q];
                }
                ++n;
            }
        }
    }
    if (!fill) T.step_cnt[t] = n;
    else if (n != (int)(T.step_off[t + 1] - T.step_off[t])) T.tiles[(size_t)t * G::kTileInts + 3] = -1;
}

// K-steps of one tile, warp-parallel: per term, the columns k of the tile's
// TBM A rows and of its TBN B rows are marked in two shared-memory bitmaps
// over the window where both can have columns; a K-step is a k marked in
// both, its index the rank of k among those (prefix popcounts).  Each list
// entry at such a k writes its block index into its slot of the step; the
// other slots stay -1 (zero block).  Same steps, same order as the serial
// merge, which lane 0 runs for windows wider than the bitmaps.
constexpr int kStepWarps = 4, kStepWords = 512;    // 16,384 columns per window
template <class G>
__global__ void __launch_bounds__(32 * kStepWarps) k_tile_steps(TileBuild T, int fill) {
    __shared__ unsigned ba_s[kStepWarps][kStepWords], bb_s[kStepWarps][kStepWords];
    __shared__ int rank_s[kStepWarps][kStepWords];
    const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kStepWarps + wq;
    if (t >= T.ntile) return;
    unsigned *ba = ba_s[wq], *bb = bb_s[wq];
    int *wr = rank_s[wq];
    const int *d = T.tiles + (size_t)t * G::kTileInts;
    const int p = d[0], I = d[1];
    const Job &job = T.jt.job[p];
    // the window of every term must fit the bitmaps, else the serial merge
    int lo_t[2], hi_t[2], cur[2][G::kSlots], end[2][G::kSlots];
    bool fits = true;
    for (int term = 0; term < job.nterm; ++term) {
        const int am = job.a[term], bm = job.b[term];
        int loA = 0x7fffffff, hiA = -1, loB = 0x7fffffff, hiB = -1;
        for (int q = 0; q < G::TBM; ++q) {
            const int i = G::TBM * I + q;
            cur[term][q] = end[term][q] = 0;
            if (i < T.NB) { cur[term][q] = T.rp[am * T.NB + i]; end[term][q] = T.rp[am * T.NB + i + 1]; }
            if (cur[term][q] < end[term][q]) {
                loA = min(loA, T.col[cur[term][q]]);
                hiA = max(hiA, T.col[end[term][q] - 1]);
            }
        }
        for (int q = 0; q < G::TBN; ++q) {
            const int j = d[G::kColOff + q];
            cur[term][G::TBM + q] = end[term][G::TBM + q] = 0;
            if (j >= 0) {
                cur[term][G::TBM + q] = T.rp[bm * T.NB + j];
                end[term][G::TBM + q] = T.rp[bm * T.NB + j + 1];
            }
            if (cur[term][G::TBM + q] < end[term][G::TBM + q]) {
                loB = min(loB, T.col[cur[term][G::TBM + q]]);
                hiB = max(hiB, T.col[end[term][G::TBM + q] - 1]);
            }
        }
        lo_t[term] = max(loA, loB);
        hi_t[term] = min(hiA, hiB);
        if (hi_t[term] >= lo_t[term] && ((hi_t[term] - lo_t[term]) >> 5) + 1 > T.max_words) fits = false;
    }
    if (!fits) {
        if (lane == 0) tile_steps_serial<G>(T, t, fill);
        return;
    }
    int64_t w = fill ? T.step_off[t] : 0;
    int n = 0;
    for (int term = 0; term < job.nterm; ++term) {
        const int lo = lo_t[term], hi = hi_t[term];
        if (hi < lo) continue;
        const int nw = ((hi - lo) >> 5) + 1;
        for (int x = lane; x < nw; x += 32) { ba[x] = 0u; bb[x] = 0u; }
        __syncwarp();
        for (int q = 0; q < G::kSlots; ++q) {
            unsigned *bmap = q < G::TBM ? ba : bb;
            for (int e = cur[term][q] + lane; e < end[term][q]; e += 32) {
                const int k = T.col[e];
                if (k < lo || k > hi) continue;
                atomicOr(&bmap[(k - lo) >> 5], 1u << ((k - lo) & 31));
            }
        }
        __syncwarp();
        int carry = 0;
        for (int x0 = 0; x0 < nw; x0 += 32) {
            const int x = x0 + lane;
            unsigned both = 0u;
            if (x < nw) {
                both = ba[x] & bb[x];
                ba[x] = both;
            }
            const int c = __popc(both);
            int y = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            if (x < nw) wr[x] = carry + y - c;
            carry += __shfl_sync(0xffffffffu, y, 31);
        }
        __syncwarp();
        if (fill) {
            const int64_t wend = T.step_off[t + 1];
            for (int64_t q = w + n + lane; q < min(w + n + carry, wend); q += 32) {
                int *st = T.steps + (size_t)q * G::kSlots;
                for (int k = 0; k < G::kSlots; ++k) st[k] = -1;
            }
            __syncwarp();
            for (int q = 0; q < G::kSlots; ++q)
                for (int e = cur[term][q] + lane; e < end[term][q]; e += 32) {
                    const int k = T.col[e];
                    if (k < lo || k > hi) continue;
                    const int kk = k - lo;
                    const unsigned word = ba[kk >> 5];
                    if (!((word >> (kk & 31)) & 1u)) continue;
                    const int r = wr[kk >> 5] + __popc(word & ((1u << (kk & 31)) - 1u));
                    if (w + n + r < wend) T.steps[(size_t)(w + n + r) * G::kSlots + q] = T.tpos ? T.tpos[e] : e;
                }
            __syncwarp();
        }
        n += carry;
    }
    if (lane == 0) {
        if (!fill) T.step_cnt[t] = n;
        else if (n != (int)(T.step_off[t + 1] - T.step_off[t])) T.tiles[(size_t)t * G::kTileInts + 3] = -1;
    }
}

template <class G>
__global__ void k_set_nsteps(int *tiles, const int *step_cnt, int ntile) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntile) tiles[(size_t)t * G::kTileInts + 3] = step_cnt[t];
}


template <class G>
TcPlan build_plan(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_rp, const int *mcol,
                  TcWork &w, JobMask job_mask, int unit0, int unit1, cudaStream_t st) {
    TcPlan plan{};
    const int NB = in.NB, NBT = (NB + G::TBM - 1) / G::TBM;
    const int nrowt = unit1 - unit0;
    if (nrowt <= 0) return plan;
    w.counters.ensure(8);
    RDM_CUDA_TRY(cudaMemsetAsync(w.counters.p, 0, 8 * sizeof(int), st));
    w.tile_cnt.ensure(nrowt + 1);
    w.tile_off.ensure(nrowt + 1);
    w.scan32.ensure(scan_tmp_elems(nrowt + 1));
    TileBuild T{};
    T.rp = in.row_ptr.p; T.col = in.col.p; T.NB = NB; T.NBT = NBT; T.jt = jt;
    T.out_rp = out_rp; T.mcol = mcol; T.sys_of_row = sd.sys_of_row.p; T.active = sd.active.p;
    T.job_mask = job_mask;
    T.u0 = unit0; T.u1 = unit1;
    T.sys_tier = sd.tier.p;
    T.tile_cnt = w.tile_cnt.p; T.tile_off = w.tile_off.p;
    T.tpos = w.tpos_valid ? w.tpos.p : nullptr;
    static_assert(kTileRowWords == kStepWords, "one window bound for both plan builders");
    T.max_words = w.knobs.window_words > 0 && w.knobs.window_words < kTileRowWords ? w.knobs.window_words
                                                                                    : kTileRowWords;
    k_tile_rows<G><<<(nrowt + kTileRowWarps - 1) / kTileRowWarps, 32 * kTileRowWarps, 0, st>>>(T, 0);
    RDM_LAUNCH_CHECK();
    scan_exclusive_i32(w.tile_cnt.p, w.tile_off.p, nrowt, w.scan32.p, st);
    int ntile = 0;
    RDM_CUDA_TRY(cudaMemcpyAsync(&ntile, w.tile_off.p + nrowt, sizeof(int), cudaMemcpyDeviceToHost, st));
    RDM_CUDA_TRY(cudaStreamSynchronize(st));
    plan.ntile = ntile;
    if (ntile == 0) return plan;
    w.tiles.ensure((size_t)ntile * G::kTileInts);
    T.tiles = w.tiles.p;
    k_tile_rows<G><<<(nrowt + kTileRowWarps - 1) / kTileRowWarps, 32 * kTileRowWarps, 0, st>>>(T, 1);
    RDM_LAUNCH_CHECK();
    w.step_cnt.ensure(ntile + 1);
    w.step_off.ensure(ntile + 1);
    w.scan64.ensure(scan_tmp_elems(ntile + 1));
    T.ntile = ntile;
    T.step_cnt = w.step_cnt.p;
    k_tile_steps<G><<<(ntile + kStepWarps - 1) / kStepWarps, 32 * kStepWarps, 0, st>>>(T, 0);
    RDM_LAUNCH_CHECK();
    scan_exclusive_i64(w.step_cnt.p, w.step_off.p, ntile, w.scan64.p, st);
    int64_t nsteps = 0;
    RDM_CUDA_TRY(cudaMemcpyAsync(&nsteps, w.step_off.p + ntile, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RDM_CUDA_TRY(cudaStreamSynchronize(st));
    plan.nsteps = nsteps;
    w.steps.ensure(std::max<int64_t>(nsteps, 1) * G::kSlots);
    T.step_off = w.step_off.p;
    T.steps = w.steps.p;
    k_set_nsteps<G><<<(ntile + 127) / 128, 128, 0, st>>>(w.tiles.p, w.step_cnt.p, ntile);
    RDM_LAUNCH_CHECK();
    k_tile_steps<G><<<(ntile + kStepWarps - 1) / kStepWarps, 32 * kStepWarps, 0, st>>>(T, 1);
    RDM_LAUNCH_CHECK();
    return plan;
}


}  // namespace
}  // namespace rdm
