// Stream compaction after truncation: per-row counts of the kept blocks, a
// scan (k_scan.cu) into the new row pointers, and an order-preserving copy of
// the kept blocks (columns, values, norm bounds); the products compute only
// the upper triangle and the copy writes each lower block as the transpose
// of its upper partner.  Also builds the work list of upper-triangle output
// blocks for the numeric phase.
#include "rdm_internal.cuh"

#include <algorithm>

namespace rdm {
namespace {

// work list: slots with col >= row, in slot order (one warp per 32 slots,
// ballot-ordered, block-level offsets through one atomic per warp; the order
// of the list does not affect results)
// keeps the upper slots of the active systems' jobs in job_mask and, with
// with_inactive, every upper slot of a converged system (those are copied)
__global__ void k_build_work(const int *__restrict__ slot_row, const int *__restrict__ out_col,
                             int64_t s0, int64_t s1, int *work, int *nwork, const int *__restrict__ sys_of_row,
                             const int *__restrict__ active, const int *__restrict__ slot_job,
                             const int *__restrict__ sys_tier, JobMask job_mask, int with_inactive) {
    int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool up = s < s1 && out_col[s] >= slot_row[s];
    if (up) {
        const int sys = sys_of_row[slot_row[s]];
        const bool act = active[sys] != 0;
        up = act ? ((job_mask.m[sys_tier[sys] & (kMaxTiers - 1)] >> slot_job[s]) & 1u) != 0 : with_inactive != 0;
    }
    unsigned m = __ballot_sync(0xffffffffu, up);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(nwork, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (up) work[base + __popc(m & ((1u << lane) - 1u))] = (int)s;
}

__global__ void k_class_pairs(const int *__restrict__ slot_row, const int *__restrict__ out_col,
                              const int *__restrict__ slot_npair, const int *__restrict__ slot_job, int64_t nslot,
                              const int *__restrict__ sys_of_row, const int *__restrict__ active,
                              const int *__restrict__ sys_tier, JobMask tc, JobMask m64, JobMask m32,
                              JobMask mff, JobMask moz, unsigned long long *out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c[5] = {0, 0, 0, 0, 0};
    if (s < nslot && out_col[s] >= slot_row[s]) {
        const int sys = sys_of_row[slot_row[s]];
        if (active[sys]) {
            const int t = sys_tier[sys] & (kMaxTiers - 1);
            const unsigned bit = 1u << slot_job[s];
            const unsigned long long np = (unsigned long long)slot_npair[s];
            if (tc.m[t] & bit) c[0] = np;
            else if (m64.m[t] & bit) c[1] = np;
            else if (m32.m[t] & bit) c[2] = np;
            else if (mff.m[t] & bit) c[3] = np;
            else if (moz.m[t] & bit) c[4] = np;
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        unsigned long long v = c[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&out[k], v);
    }
}

__global__ void k_upper_flags(const int *__restrict__ slot_row, const int *__restrict__ out_col,
                              int64_t nslot, int *__restrict__ uidx) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nslot) uidx[s] = out_col[s] >= slot_row[s] ? 1 : 0;
}

__global__ void k_gather_i32(const int *__restrict__ idx, const int *__restrict__ src, int n,
                             int *__restrict__ dst) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= n) dst[r] = src[idx[r]];
}

// one warp per row of the group: kept blocks (an upper slot on its own flag,
// a lower one on its upper partner's)
__global__ void k_compact_count(CompactArgs c, int *cnt) {
    const int rr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (rr >= c.nrows) return;
    const int r = c.r0 + rr;
    int n = 0;
    for (int p = c.out_rp[r] + lane; p < c.out_rp[r + 1]; p += 32) {
        const bool up = c.out_col[p] >= c.slot_row[p];
        n += c.keep[up ? p : c.slot_t[p]] ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[rr] = n;
}

// one warp per row: columns, norm bounds and destinations of the kept blocks
// (order-preserving); src[d - d0] receives the slot of output block d
__global__ void k_compact_index(CompactArgs c) {
    const int rr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (rr >= c.nrows) return;
    const int r = c.r0 + rr;
    const int rend = c.out_rp[r + 1];
    int dst = c.new_rp[r];
    for (int base = c.out_rp[r]; base < rend; base += 32) {
        const int p = base + lane;
        bool k = false, up = false;
        int src = p;
        if (p < rend) {
            up = c.out_col[p] >= c.slot_row[p];
            src = up ? p : c.slot_t[p];
            k = c.keep[src] != 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (k) {
            const int d = dst + __popc(m & ((1u << lane) - 1u));
            c.new_col[d] = c.out_col[p];
            c.new_nrm[d] = c.out_nrm[src];
            c.src[d - c.d0] = p;
            if (up) c.dest[p] = d;
        }
        dst += __popc(m);
    }
}

// one CTA per kept block (grid-stride): upper blocks are copied, lower ones
// transposed through shared memory (b x (b+1) doubles) from their upper
// partner, which is in this group's buffer or already compacted
__global__ void __launch_bounds__(128) k_compact_vals(CompactArgs c, int d1) {
    extern __shared__ double tile[];
    const int b = c.b, bb = b * b, ld = b + 1;
    for (int d = c.d0 + blockIdx.x; d < d1; d += gridDim.x) {
        const int p = c.src[d - c.d0];
        double *out = c.new_val + (size_t)d * bb;
        if (c.out_col[p] >= c.slot_row[p]) {
            const double *s = c.out_val + (size_t)(c.uidx[p] - c.u0) * bb;
            if ((bb & 1) == 0) {
                const double2 *s2 = reinterpret_cast<const double2 *>(s);
                double2 *o2 = reinterpret_cast<double2 *>(out);
                for (int e = threadIdx.x; e < bb / 2; e += blockDim.x) o2[e] = s2[e];
            } else {
                for (int e = threadIdx.x; e < bb; e += blockDim.x) out[e] = s[e];
            }
        } else {
            const int t = c.slot_t[p];
            const int ut = c.uidx[t];
            const double *s = ut >= c.u0 ? c.out_val + (size_t)(ut - c.u0) * bb
                                         : c.new_val + (size_t)c.dest[t] * bb;
            for (int e = threadIdx.x; e < bb; e += blockDim.x) tile[(e / b) * ld + (e % b)] = s[e];
            __syncthreads();
            for (int e = threadIdx.x; e < bb; e += blockDim.x) out[e] = tile[(e % b) * ld + (e / b)];
            __syncthreads();
        }
    }
}

}  // namespace

void launch_build_work(const int *slot_row, const int *out_col, int64_t s0, int64_t s1, int *work,
                       int *nwork, cudaStream_t st, const int *sys_of_row, const int *active,
                       const int *slot_job, const int *sys_tier, JobMask job_mask, int with_inactive) {
    if (s1 <= s0) return;
    int64_t grid = (s1 - s0 + 255) / 256;
    k_build_work<<<(unsigned)grid, 256, 0, st>>>(slot_row, out_col, s0, s1, work, nwork, sys_of_row,
                                                 active, slot_job, sys_tier, job_mask, with_inactive);
    RDM_LAUNCH_CHECK();
}

void launch_class_pairs(const int *slot_row, const int *out_col, const int *slot_npair, const int *slot_job,
                        int64_t nslot, const int *sys_of_row, const int *active, const int *sys_tier,
                        JobMask tc, JobMask m64, JobMask m32, JobMask mff, JobMask moz, unsigned long long *out,
                        cudaStream_t st) {
    if (nslot == 0) return;
    const int64_t grid = (nslot + 255) / 256;
    k_class_pairs<<<(unsigned)grid, 256, 0, st>>>(slot_row, out_col, slot_npair, slot_job, nslot, sys_of_row,
                                                  active, sys_tier, tc, m64, m32, mff, moz, out);
    RDM_LAUNCH_CHECK();
}

void launch_upper_flags(const int *slot_row, const int *out_col, int64_t nslot, int *uidx,
                        cudaStream_t st) {
    if (nslot == 0) return;
    k_upper_flags<<<(unsigned)((nslot + 255) / 256), 256, 0, st>>>(slot_row, out_col, nslot, uidx);
    RDM_LAUNCH_CHECK();
}

void launch_gather_i32(const int *idx, const int *src, int n, int *dst, cudaStream_t st) {
    k_gather_i32<<<(n + 256) / 256, 256, 0, st>>>(idx, src, n, dst);
    RDM_LAUNCH_CHECK();
}

void launch_compact_count(const CompactArgs &c, int *cnt, cudaStream_t st) {
    if (c.nrows == 0) return;
    const int wpb = 8;
    k_compact_count<<<(c.nrows + wpb - 1) / wpb, wpb * 32, 0, st>>>(c, cnt);
    RDM_LAUNCH_CHECK();
}

void launch_compact_copy(const CompactArgs &c, int d1, cudaStream_t st) {
    if (c.nrows == 0) return;
    const int wpb = 8;
    k_compact_index<<<(c.nrows + wpb - 1) / wpb, wpb * 32, 0, st>>>(c);
    RDM_LAUNCH_CHECK();
    if (d1 <= c.d0) return;
    const size_t smem = (size_t)c.b * (c.b + 1) * sizeof(double);
    func_smem_once((const void *)k_compact_vals, 64 * 65 * (int)sizeof(double));
    const int grid = (int)std::min<int64_t>((int64_t)d1 - c.d0, 152 * 16);
    k_compact_vals<<<grid, 128, smem, st>>>(c, d1);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
