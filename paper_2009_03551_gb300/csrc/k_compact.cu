// Stream compaction after truncation: per-row counts of the kept blocks, a
// scan (k_scan.cu) into the new row pointers, and an order-preserving copy of
// the kept blocks (columns, values, norm bounds).  Also builds the work list
// of upper-triangle output blocks for the numeric phase.
#include "rdm_internal.cuh"

namespace rdm {
namespace {

// work list: slots with col >= row, in slot order (one warp per 32 slots,
// ballot-ordered, block-level offsets through one atomic per warp; the order
// of the list does not affect results)
// keeps the upper slots of the active systems' jobs in job_mask and, with
// with_inactive, every upper slot of a converged system (those are copied)
__global__ void k_build_work(const int *__restrict__ slot_row, const int *__restrict__ out_col,
                             int64_t nslot, int *work, int *nwork, const int *__restrict__ sys_of_row,
                             const int *__restrict__ active, const int *__restrict__ slot_job,
                             const int *__restrict__ sys_tier, JobMask job_mask, int with_inactive) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool up = s < nslot && out_col[s] >= slot_row[s];
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
                              unsigned long long *out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c[3] = {0, 0, 0};
    if (s < nslot && out_col[s] >= slot_row[s]) {
        const int sys = sys_of_row[slot_row[s]];
        if (active[sys]) {
            const int t = sys_tier[sys] & (kMaxTiers - 1);
            const unsigned bit = 1u << slot_job[s];
            const unsigned long long np = (unsigned long long)slot_npair[s];
            if (tc.m[t] & bit) c[0] = np;
            else if (m64.m[t] & bit) c[1] = np;
            else if (m32.m[t] & bit) c[2] = np;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned long long v = c[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&out[k], v);
    }
}

__global__ void k_compact_count(const int *__restrict__ rp, const uint8_t *__restrict__ keep,
                                int nrows, int *cnt) {
    int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    int c = 0;
    for (int p = rp[r] + lane; p < rp[r + 1]; p += 32) c += keep[p] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[r] = c;
}

__global__ void k_compact_copy(const int *__restrict__ rp, const int *__restrict__ col,
                               const double *__restrict__ val, const float *__restrict__ nrm,
                               const uint8_t *__restrict__ keep, const int *__restrict__ nrp,
                               int nrows, int b, int *ncol, double *nval, float *nnrm) {
    int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int bb = b * b;
    int dst = nrp[r];
    for (int base = rp[r]; base < rp[r + 1]; base += 32) {
        int p = base + lane;
        bool k = p < rp[r + 1] && keep[p];
        unsigned m = __ballot_sync(0xffffffffu, k);
        if (k) {
            int d = dst + __popc(m & ((1u << lane) - 1u));
            ncol[d] = col[p];
            nnrm[d] = nrm[p];
        }
        // copy the kept blocks' values, one block at a time, lanes over elements
        unsigned mm = m;
        int d = dst;
        while (mm) {
            int l = __ffs(mm) - 1;
            mm &= mm - 1;
            const double *src = val + (size_t)(base + l) * bb;
            double *out = nval + (size_t)d * bb;
            for (int e = lane; e < bb; e += 32) out[e] = src[e];
            ++d;
        }
        dst += __popc(m);
    }
}

}  // namespace

void launch_build_work(const int *slot_row, const int *out_col, int64_t nslot, int *work,
                       int *nwork, cudaStream_t st, const int *sys_of_row, const int *active,
                       const int *slot_job, const int *sys_tier, JobMask job_mask, int with_inactive) {
    if (nslot == 0) return;
    int64_t grid = (nslot + 255) / 256;
    k_build_work<<<(unsigned)grid, 256, 0, st>>>(slot_row, out_col, nslot, work, nwork, sys_of_row,
                                                 active, slot_job, sys_tier, job_mask, with_inactive);
    RDM_LAUNCH_CHECK();
}

void launch_class_pairs(const int *slot_row, const int *out_col, const int *slot_npair, const int *slot_job,
                        int64_t nslot, const int *sys_of_row, const int *active, const int *sys_tier,
                        JobMask tc, JobMask m64, JobMask m32, unsigned long long *out, cudaStream_t st) {
    if (nslot == 0) return;
    const int64_t grid = (nslot + 255) / 256;
    k_class_pairs<<<(unsigned)grid, 256, 0, st>>>(slot_row, out_col, slot_npair, slot_job, nslot, sys_of_row,
                                                  active, sys_tier, tc, m64, m32, out);
    RDM_LAUNCH_CHECK();
}

void launch_compact_count(const int *out_row_ptr, const uint8_t *keep, int nrows_total, int *cnt,
                          cudaStream_t st) {
    if (nrows_total == 0) return;
    int wpb = 8;
    k_compact_count<<<(nrows_total + wpb - 1) / wpb, wpb * 32, 0, st>>>(out_row_ptr, keep,
                                                                        nrows_total, cnt);
    RDM_LAUNCH_CHECK();
}

void launch_compact_copy(const int *out_row_ptr, const int *out_col, const double *out_val,
                         const float *out_nrm, const uint8_t *keep, const int *new_row_ptr,
                         int nrows_total, int b, int *new_col, double *new_val, float *new_nrm,
                         cudaStream_t st) {
    if (nrows_total == 0) return;
    int wpb = 8;
    k_compact_copy<<<(nrows_total + wpb - 1) / wpb, wpb * 32, 0, st>>>(
        out_row_ptr, out_col, out_val, out_nrm, keep, new_row_ptr, nrows_total, b, new_col,
        new_val, new_nrm);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
