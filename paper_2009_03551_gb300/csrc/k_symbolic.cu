// Symbolic phase of the block-sparse products: which output blocks to
// compute, and the list of block pairs feeding each of them.
//
// Mask.  For output row i of job p (C = c_lin X + c_sq sum_t A_t B_t) every
// column j reached by the Gustavson row expansion (Algorithm 1: for k in row
// i of A, for j in row k of B) accumulates the bound
//     beta_ij = |c_sq| sum_k ||A_ik|| ||B_kj||  +  |c_lin| ||X_ij||,
// which by the triangle inequality and Frobenius submultiplicativity is >=
// ||C_ij||.  Column j is kept iff beta_ij >= tau (any contribution when
// tau = 0), so every block that survives the truncation of Sec. 2.3 is in the
// mask and the numeric phase plus the truncation give exactly "full product,
// then drop blocks below tau".  Algorithm 1's dense label array becomes a
// per-row accumulator in shared memory over the system's block columns.
//
// Determinism and symmetry.  beta is accumulated in 64-bit fixed point (each
// term rounded UP to a unit of tau * 2^-24 and capped), so the sum does not
// depend on the order of the shared-memory atomics and beta_ij == beta_ji
// exactly: the mask of a symmetric product is exactly symmetric.
//
// Pairs.  For an upper-triangle output block (j >= i) the pairs are the k in
// row i of A_t whose block (j,k) exists in B_t (B symmetric: B_kj = B_jk^T),
// so C_ij = sum A_ik (B_jk)^T uses two row-major blocks; they are found by a
// warp-wide sorted intersection and stored in increasing k order.
#include "rdm_internal.cuh"

namespace rdm {
namespace {

constexpr int kSymThreads = 256;
constexpr float kFixOne = 16777216.0f;          // 2^24 units = the threshold
constexpr float kFixCap = 1099511627776.0f;     // 2^40 units per term

__device__ __forceinline__ int find_col(const int *col, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// lower_bound of key in col[lo,hi)
__device__ __forceinline__ int lower_bound(const int *col, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long fix_units(float prod, float inv_unit) {
    float u = __fmul_ru(prod, inv_unit);
    u = fminf(u, kFixCap);
    return (unsigned long long)__float2ull_ru(u);
}

template <class T>
__device__ T block_excl_scan(T v, T *sh, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < (kSymThreads / 32) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kSymThreads / 32)) sh[lane] = w;
    }
    __syncthreads();
    T ex = x - v + (wid > 0 ? sh[wid - 1] : T(0));
    *total = sh[kSymThreads / 32 - 1];
    __syncthreads();
    return ex;
}

struct SymParams {
    const int *rp;       // flat row_ptr of the input set (nmat*NB+1)
    const int *col;
    const float *nrm;
    int NB;
    JobTable jt;
    const int *sys_of_row, *row0, *nbs;
    const double *c_lin, *c_sq, *tau0, *tau1;
    const int *active;
    SymOut so;
};

// grid (NB, njob); dynamic shared memory: acc[ns] (u64) + cnt[ns] (u32)
__global__ void __launch_bounds__(kSymThreads) k_symbolic(SymParams P) {
    extern __shared__ unsigned long long sm_acc[];
    __shared__ int sh_scan[32];
    __shared__ int sh_off;
    const int i = blockIdx.x, p = blockIdx.y;
    const int NB = P.NB;
    const Job &job = P.jt.job[p];
    const int s = P.sys_of_row[i];
    const int c0 = P.row0[s], ns = P.nbs[s];
    unsigned int *cnt = reinterpret_cast<unsigned int *>(sm_acc + ns);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int out_r = p * NB + i;

    if (!P.active[s]) {
        // converged system: the output pattern is the current pattern of X
        const int xm = job.xmat;
        int lo = P.rp[xm * NB + i], hi = P.rp[xm * NB + i + 1];
        int n = hi - lo;
        if (tid == 0) {
            int off = atomicAdd(P.so.pool_top, n);
            if (off + n > P.so.pool_cap) { atomicExch(P.so.overflow, 1); off = -1; }
            sh_off = off;
            P.so.row_cnt[out_r] = n;
            P.so.row_off[out_r] = off;
        }
        __syncthreads();
        if (sh_off >= 0)
            for (int t = tid; t < n; t += blockDim.x) {
                P.so.pool_col[sh_off + t] = P.col[lo + t];
                P.so.pool_npair[sh_off + t] = 0;
            }
        return;
    }

    for (int t = tid; t < ns; t += blockDim.x) { sm_acc[t] = 0ull; cnt[t] = 0u; }
    __syncthreads();

    const double tau = job.tau_sel ? P.tau1[s] : P.tau0[s];
    const bool exact = !(tau > 0.0);
    // unit = tau (1 - 2^-10) 2^-24, rounded down so that 1/unit rounds up
    const float inv_unit = exact ? 0.f : __fdiv_ru(1.0f, __double2float_rd(tau * (1.0 - 1.0 / 1024.0))) * kFixOne;
    const float csq = (float)fabs(P.c_sq[s]);
    const double cl = P.c_lin[s];

    const int nw = blockDim.x >> 5;
    for (int t = 0; t < job.nterm; ++t) {
        const int am = job.a[t], bm = job.b[t];
        const int alo = P.rp[am * NB + i], ahi = P.rp[am * NB + i + 1];
        for (int pa = alo + wid; pa < ahi; pa += nw) {
            const int k = P.col[pa];
            const float na = __fmul_ru(P.nrm[pa], csq);
            const int blo = P.rp[bm * NB + k], bhi = P.rp[bm * NB + k + 1];
            for (int pb = blo + lane; pb < bhi; pb += 32) {
                const int j = P.col[pb] - c0;
                if (!exact) atomicAdd(&sm_acc[j], fix_units(__fmul_ru(na, P.nrm[pb]), inv_unit));
                atomicAdd(&cnt[j], 1u);
            }
        }
    }
    if (cl != 0.0 && job.xmat >= 0) {
        const float fcl = (float)fabs(cl);
        const int xlo = P.rp[job.xmat * NB + i], xhi = P.rp[job.xmat * NB + i + 1];
        for (int px = xlo + tid; px < xhi; px += blockDim.x) {
            const int j = P.col[px] - c0;
            if (!exact) atomicAdd(&sm_acc[j], fix_units(__fmul_ru(P.nrm[px], fcl), inv_unit));
            atomicOr(&cnt[j], 0x80000000u);   // linear term present
        }
    }
    __syncthreads();

    const unsigned long long thr = (unsigned long long)kFixOne;
    // pass 1: count kept columns
    int my = 0;
    for (int t = tid; t < ns; t += blockDim.x) {
        bool keep = exact ? (cnt[t] != 0u) : (sm_acc[t] >= thr);
        my += keep ? 1 : 0;
    }
    int total;
    block_excl_scan<int>(my, sh_scan, &total);
    if (tid == 0) {
        int off = atomicAdd(P.so.pool_top, total);
        if (off + total > P.so.pool_cap) { atomicExch(P.so.overflow, 1); off = -1; }
        sh_off = off;
        P.so.row_cnt[out_r] = total;
        P.so.row_off[out_r] = off;
    }
    __syncthreads();
    if (sh_off < 0) return;
    // pass 2: ordered write of the kept columns and their pair counts
    int base = 0;
    for (int seg = 0; seg < ns; seg += blockDim.x) {
        const int t = seg + tid;
        bool keep = false;
        if (t < ns) keep = exact ? (cnt[t] != 0u) : (sm_acc[t] >= thr);
        int segtot;
        int pos = block_excl_scan<int>(keep ? 1 : 0, sh_scan, &segtot);
        if (keep) {
            const int j = c0 + t;
            P.so.pool_col[sh_off + base + pos] = j;
            P.so.pool_npair[sh_off + base + pos] = (j >= i) ? (int)(cnt[t] & 0x7fffffffu) : 0;
        }
        base += segtot;
    }
}

// ---------------------------------------------------------------------------
// The same symbolic step for systems wider than the dense accumulator: the
// columns a row reaches (a few hundred, independent of the system size) go to
// an open-addressing hash table in shared memory; the kept columns are then
// sorted (bitonic) so that the row's list comes out in increasing order.  The
// fixed-point bound and the keep rule are those of k_symbolic.
// ---------------------------------------------------------------------------
constexpr int kHashSlots = 8192;                 // 128 KB: key + acc + cnt
constexpr int kHashMaxFill = kHashSlots * 3 / 4;

__device__ __forceinline__ int hash_slot(int j) { return (int)(((unsigned)j * 2654435761u) >> (32 - 13)); }

// returns the slot of key j (inserting it), or -1 when the table is full
__device__ __forceinline__ int hash_find(int *keys, int j, int *fill) {
    int h = hash_slot(j);
    for (int probe = 0; probe < kHashSlots; ++probe) {
        const int k = keys[h];
        if (k == j) return h;
        if (k < 0) {
            const int prev = atomicCAS(&keys[h], -1, j);
            if (prev == -1) {
                if (atomicAdd(fill, 1) >= kHashMaxFill) return -1;
                return h;
            }
            if (prev == j) return h;
        }
        h = (h + 1) & (kHashSlots - 1);
    }
    return -1;
}

__global__ void __launch_bounds__(kSymThreads) k_symbolic_hash(SymParams P) {
    extern __shared__ unsigned long long sm_acc[];                 // kHashSlots
    unsigned int *cnt = reinterpret_cast<unsigned int *>(sm_acc + kHashSlots);
    int *keys = reinterpret_cast<int *>(cnt + kHashSlots);
    __shared__ int sh_scan[32];
    __shared__ int sh_off, sh_fill, sh_bad;
    const int i = blockIdx.x, p = blockIdx.y;
    const int NB = P.NB;
    const Job &job = P.jt.job[p];
    const int s = P.sys_of_row[i];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int out_r = p * NB + i;

    if (!P.active[s]) {
        const int xm = job.xmat;
        int lo = P.rp[xm * NB + i], hi = P.rp[xm * NB + i + 1];
        int n = hi - lo;
        if (tid == 0) {
            int off = atomicAdd(P.so.pool_top, n);
            if (off + n > P.so.pool_cap) { atomicExch(P.so.overflow, 1); off = -1; }
            sh_off = off;
            P.so.row_cnt[out_r] = n;
            P.so.row_off[out_r] = off;
        }
        __syncthreads();
        if (sh_off >= 0)
            for (int t = tid; t < n; t += blockDim.x) {
                P.so.pool_col[sh_off + t] = P.col[lo + t];
                P.so.pool_npair[sh_off + t] = 0;
            }
        return;
    }
    for (int t = tid; t < kHashSlots; t += blockDim.x) { sm_acc[t] = 0ull; cnt[t] = 0u; keys[t] = -1; }
    if (tid == 0) { sh_fill = 0; sh_bad = 0; }
    __syncthreads();

    const double tau = job.tau_sel ? P.tau1[s] : P.tau0[s];
    const bool exact = !(tau > 0.0);
    const float inv_unit = exact ? 0.f : __fdiv_ru(1.0f, __double2float_rd(tau * (1.0 - 1.0 / 1024.0))) * kFixOne;
    const float csq = (float)fabs(P.c_sq[s]);
    const double cl = P.c_lin[s];
    const int nw = blockDim.x >> 5;
    for (int t = 0; t < job.nterm; ++t) {
        const int am = job.a[t], bm = job.b[t];
        const int alo = P.rp[am * NB + i], ahi = P.rp[am * NB + i + 1];
        for (int pa = alo + wid; pa < ahi; pa += nw) {
            const int k = P.col[pa];
            const float na = __fmul_ru(P.nrm[pa], csq);
            const int blo = P.rp[bm * NB + k], bhi = P.rp[bm * NB + k + 1];
            for (int pb = blo + lane; pb < bhi; pb += 32) {
                const int h = hash_find(keys, P.col[pb], &sh_fill);
                if (h < 0) { sh_bad = 1; continue; }
                if (!exact) atomicAdd(&sm_acc[h], fix_units(__fmul_ru(na, P.nrm[pb]), inv_unit));
                atomicAdd(&cnt[h], 1u);
            }
        }
    }
    if (cl != 0.0 && job.xmat >= 0) {
        const float fcl = (float)fabs(cl);
        const int xlo = P.rp[job.xmat * NB + i], xhi = P.rp[job.xmat * NB + i + 1];
        for (int px = xlo + tid; px < xhi; px += blockDim.x) {
            const int h = hash_find(keys, P.col[px], &sh_fill);
            if (h < 0) { sh_bad = 1; continue; }
            if (!exact) atomicAdd(&sm_acc[h], fix_units(__fmul_ru(P.nrm[px], fcl), inv_unit));
            atomicOr(&cnt[h], 0x80000000u);
        }
    }
    __syncthreads();
    if (sh_bad) {   // row reaches more columns than the table holds
        if (tid == 0) {
            atomicExch(P.so.overflow, 2);
            P.so.row_cnt[out_r] = 0;
            P.so.row_off[out_r] = -1;
        }
        return;
    }
    // keep decision, packed as (column << 32 | pair count); dropped slots sort last
    const unsigned long long thr = (unsigned long long)kFixOne;
    int my = 0;
    for (int t = tid; t < kHashSlots; t += blockDim.x) {
        unsigned long long packed = ~0ull;
        if (keys[t] >= 0) {
            const bool keep = exact ? (cnt[t] != 0u) : (sm_acc[t] >= thr);
            if (keep) {
                const int j = keys[t];
                const unsigned np = (j >= i) ? (cnt[t] & 0x7fffffffu) : 0u;
                packed = ((unsigned long long)(unsigned)j << 32) | np;
                ++my;
            }
        }
        sm_acc[t] = packed;
    }
    int total;
    block_excl_scan<int>(my, sh_scan, &total);
    // bitonic sort of the packed keys (ascending)
    for (int k = 2; k <= kHashSlots; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = tid; t < kHashSlots; t += blockDim.x) {
                const int partner = t ^ jj;
                if (partner > t) {
                    const unsigned long long a = sm_acc[t], b = sm_acc[partner];
                    const bool up = (t & k) == 0;
                    if ((a > b) == up) { sm_acc[t] = b; sm_acc[partner] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        int off = atomicAdd(P.so.pool_top, total);
        if (off + total > P.so.pool_cap) { atomicExch(P.so.overflow, 1); off = -1; }
        sh_off = off;
        P.so.row_cnt[out_r] = total;
        P.so.row_off[out_r] = off;
    }
    __syncthreads();
    if (sh_off < 0) return;
    for (int t = tid; t < total; t += blockDim.x) {
        const unsigned long long v = sm_acc[t];
        P.so.pool_col[sh_off + t] = (int)(v >> 32);
        P.so.pool_npair[sh_off + t] = (int)(v & 0xffffffffu);
    }
}

// one warp per (job,row): copy the pool lists into the output pattern
__global__ void k_gather(SymOut so, int nrows, const int *__restrict__ out_rp, int *out_col,
                         int *slot_row, int *slot_job, int *slot_npair, int NB) {
    int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    int n = so.row_cnt[r], off = so.row_off[r], dst = out_rp[r];
    int i = r % NB, p = r / NB;
    for (int t = lane; t < n; t += 32) {
        out_col[dst + t] = so.pool_col[off + t];
        slot_npair[dst + t] = so.pool_npair[off + t];
        slot_row[dst + t] = i;
        slot_job[dst + t] = p;
    }
}

struct PairParams {
    const int *rp, *col;      // input set
    int NB;
    JobTable jt;
    const int *out_rp, *out_col, *slot_row, *slot_job;
    const int64_t *pair_off;
    int64_t nslot;
    int *pair_a, *pair_b, *slot_x, *slot_t, *err;
    const int *sys_of_row, *active, *sys_tier;
    JobMask fill;    // jobs whose pair lists are filled, per tier (others: only slot_x / slot_t)
};

// one warp per output slot; only upper-triangle slots (j >= i) do work.
// slot_t pairs every off-diagonal upper slot with its lower mirror (both
// ways); a diagonal slot maps to itself
__global__ void k_pairs(PairParams P) {
    int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (s >= P.nslot) return;
    const int i = P.slot_row[s], j = P.out_col[s], p = P.slot_job[s];
    if (j < i) return;
    const int NB = P.NB;
    const Job &job = P.jt.job[p];
    if (lane == 0) {
        int t = s;
        if (j > i) {
            t = find_col(P.out_col, P.out_rp[p * NB + j], P.out_rp[p * NB + j + 1], i);
            if (t < 0) atomicOr(P.err, 1);
        }
        P.slot_t[s] = t;
        if (t >= 0 && t != s) P.slot_t[t] = (int)s;   // the lower partner points back
        int x = -1;
        if (job.xmat >= 0) x = find_col(P.col, P.rp[job.xmat * NB + i], P.rp[job.xmat * NB + i + 1], j);
        P.slot_x[s] = x;
    }
    // a converged system's blocks are copied: the symbolic phase gave them no pairs
    const int sys = P.sys_of_row[i];
    if (!P.active[sys] || !((P.fill.m[P.sys_tier[sys] & (kMaxTiers - 1)] >> p) & 1u)) return;
    int64_t w = P.pair_off[s];
    const int64_t wend = P.pair_off[s + 1];
    for (int t = 0; t < job.nterm; ++t) {
        const int am = job.a[t], bm = job.b[t];
        const int alo = P.rp[am * NB + i], ahi = P.rp[am * NB + i + 1];
        int blo = P.rp[bm * NB + j];
        const int bhi = P.rp[bm * NB + j + 1];
        for (int base = alo; base < ahi; base += 32) {
            const int pa = base + lane;
            int pb = -1;
            if (pa < ahi) {
                const int k = P.col[pa];
                int lb = lower_bound(P.col, blo, bhi, k);
                if (lb < bhi && P.col[lb] == k) pb = lb;
            }
            unsigned m = __ballot_sync(0xffffffffu, pb >= 0);
            if (pb >= 0) {
                int64_t dst = w + __popc(m & ((1u << lane) - 1u));
                if (dst < wend) { P.pair_a[dst] = pa; P.pair_b[dst] = pb; }
            }
            w += __popc(m);
            // rows are sorted: later A columns are >= the last one examined
            int last = P.col[min(base + 31, ahi - 1)];
            blo = lower_bound(P.col, blo, bhi, last);
        }
    }
    if (lane == 0 && w != wend) atomicOr(P.err, 2);
}

}  // namespace

void launch_symbolic(const MatSet &in, const JobTable &jt, const SysDev &sd, int S,
                     SymOut so, cudaStream_t st, int max_ns) {
    (void)S;
    if (in.NB == 0) return;
    SymParams P;
    P.rp = in.row_ptr.p; P.col = in.col.p; P.nrm = in.nrm.p; P.NB = in.NB; P.jt = jt;
    P.sys_of_row = sd.sys_of_row.p; P.row0 = sd.row0.p; P.nbs = sd.nbs.p;
    P.c_lin = sd.c_lin.p; P.c_sq = sd.c_sq.p; P.tau0 = sd.tau0.p; P.tau1 = sd.tau1.p;
    P.active = sd.active.p; P.so = so;
    func_smem_once((const void *)k_symbolic, kSymMaxNs * 12);
    func_smem_once((const void *)k_symbolic_hash, kHashSlots * 16);
    if (max_ns <= kSymMaxNs) {
        size_t smem = (size_t)max_ns * (sizeof(unsigned long long) + sizeof(unsigned int));
        k_symbolic<<<dim3(in.NB, jt.njob), kSymThreads, smem, st>>>(P);
    } else {
        k_symbolic_hash<<<dim3(in.NB, jt.njob), kSymThreads, kHashSlots * 16, st>>>(P);
    }
    RDM_LAUNCH_CHECK();
}

void launch_gather(const SymOut &so, int njob, int NB, const int *out_row_ptr, int *out_col,
                   int *slot_row, int *slot_job, int *slot_npair, cudaStream_t st) {
    int nrows = njob * NB;
    if (nrows == 0) return;
    int wpb = 8;
    k_gather<<<(nrows + wpb - 1) / wpb, wpb * 32, 0, st>>>(so, nrows, out_row_ptr, out_col,
                                                           slot_row, slot_job, slot_npair, NB);
    RDM_LAUNCH_CHECK();
}

void launch_pairs(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_row_ptr,
                  const int *out_col, const int *slot_row, const int *slot_job,
                  const int64_t *pair_off, int64_t nslot, int NB, int *pair_a, int *pair_b,
                  int *slot_x, int *slot_t, int *err, cudaStream_t st, JobMask fill) {
    if (nslot == 0) return;
    PairParams P;
    P.fill = fill;
    P.sys_tier = sd.tier.p;
    P.rp = in.row_ptr.p; P.col = in.col.p; P.NB = NB; P.jt = jt;
    P.out_rp = out_row_ptr; P.out_col = out_col; P.slot_row = slot_row; P.slot_job = slot_job;
    P.pair_off = pair_off; P.nslot = nslot; P.pair_a = pair_a; P.pair_b = pair_b;
    P.slot_x = slot_x; P.slot_t = slot_t; P.err = err;
    P.sys_of_row = sd.sys_of_row.p; P.active = sd.active.p;
    int wpb = 8;
    int64_t grid = (nslot + wpb - 1) / wpb;
    k_pairs<<<(unsigned)grid, wpb * 32, 0, st>>>(P);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
