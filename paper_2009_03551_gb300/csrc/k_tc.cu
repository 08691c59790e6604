// Tensor-core numeric phase (tcgen05 + TMEM, sm_103a) for b x b blocks,
// b = 16, 32 or 64.
//
// Work decomposition.  Output blocks are grouped in 128 x 256 super-tiles:
// TBM = 128/b block rows times TBN = 256/b block columns taken, in increasing
// order, from the columns that these rows need (upper triangle of the mask),
// so that every tile column is needed by at least one tile row.  A super-tile
// is one MMA accumulator: D[128 x 256] = sum over K-steps of A[128 x b]
// B[256 x b]^T where a K-step is one block index k at which some row of the
// tile's A rows and some row of its B rows have a stored block (Gustavson's
// row merge, Algorithm 1, lifted to a TBM x TBN block tile).  Missing blocks
// are zero.  The X1 products (X0 X1 + X1 X0) simply concatenate the K-steps
// of both terms.  The tile is as wide as one MMA allows because operand bytes
// bound the kernel: a K-step brings (128 + 256) x b operand elements for
// 128 x 256 x b of MMA work whatever b is; at b = 32 on the masks of the
// 2,000-atom cluster the 4 x 8 tiles copied ~20% fewer bytes per product and
// ran the products 29% faster than 4 x 4 tiles.
//
// Split precision.  Every operand block is stored as a hi and a lo plane
// (bf16 or fp16, hi = rn(x), lo = rn(x - hi)); every K = 16 slice of a K-step
// issues the products hi*hi + hi*lo + lo*hi, all accumulated in FP32 in
// tensor memory.  The operand planes are laid out in global memory in the
// canonical K-major core-matrix order of the MMA (8 rows x 16 bytes per core
// matrix, core matrices adjacent along K 128 bytes apart), with the 8-row
// groups of a block's hi and lo planes alternating (16 b bytes each, 32 b
// bytes between the groups of one plane): one bulk copy of 4 b^2 bytes per
// block lands both planes ready for the MMA, and blocks stacked in a stage
// continue the same stride, so that a side of a K-step is one operand.  A
// streaming probe (one CTA per SM, no MMA) moves at most ~6.5 TB/s over the
// GPU in 4 KB bulk copies, from L2 as from DRAM, and ~7.4-8.9 TB/s in
// 16-32 KB copies: the rate of such copies into each SM bounds this kernel.
// So the planes of the operand block (i, k) are stored at the position of
// block (k, i) (the patterns are symmetric): the A blocks (i_0..i_3, k) of a
// K-step are then neighbours in block row k, and so are its B blocks
// (j_0..j_7, k) wherever row k holds them all, and the copy warp moves every
// run of slots whose blocks are neighbours in memory with one copy.
//
// Warp roles (320 threads, one CTA per SM, persistent over a static tile
// schedule, tiles round robin): warp 0 issues the bulk copies into a ring of stages, warp 1
// owns the tensor-memory allocation and one thread issues the MMAs, warps
// 2-9 (two per TMEM lane quarter, 128 accumulator columns each) run the
// epilogue.  Ten warps put three on some SM sub-partitions, which caps a
// thread at 168 registers: the epilogue keeps its 128 accumulators in
// registers and parks the tile metadata in shared memory.  At b = 64 an
// output block spans two lane quarters, so the two warps that share its
// columns combine their halves (norm, transpose of diagonal blocks) through
// shared memory, synchronised by a bounded mbarrier handshake.
//
// Accumulation in segments.  The tensor cores' FP32 accumulation truncates
// (it is not round-to-nearest), so a long accumulation chain drifts towards
// zero: measured on positive data, -2e-7 relative per 32-deep K-step, -2e-5
// after 96 of them.  The K-steps of a tile are therefore accumulated in
// segments of 128 K (kSegSteps K-steps) in fresh TMEM accumulators (2
// rotating buffers of 256 columns); the epilogue warps add every finished
// segment to registers with round-to-nearest FP32 adds and release the
// buffer.  The drift is then that of one segment (-7e-7 relative),
// independent of the tile's length.  After the last segment:
// C = c_lin X + c_sq D, diagonal blocks symmetrised, block Frobenius norm,
// truncation flag, FP64 store of the (upper-triangle) block; the old X
// blocks of the next tile's linear terms are prefetched into L2 two segments
// before this tile ends.  Every wait is bounded: on timeout the kernel raises
// an error flag, drains what it issued and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_plan.cuh"
#include "tc_ptx.cuh"

namespace rdm {
namespace {

// geometry of the tiles for block size B
template <int B>
struct Geo : PlanGeo<128 / B, 256 / B> {
    using P = PlanGeo<128 / B, 256 / B>;
    static constexpr int kPlaneElems = B * B;           // elements of one plane of a block
    static constexpr int kPairBytes = 4 * B * B;        // hi and lo planes of one block, interleaved
    static constexpr int kSideABytes = P::TBM * kPairBytes;     // A side of a stage: TBM blocks stacked
    static constexpr int kStageBytes = P::kSlots * kPairBytes;  // A side, then the TBN blocks of the B side
    static constexpr int kStages = B == 16 ? 7 : B == 32 ? 4 : 2;   // fit checked below
    static constexpr int kSegSteps = 128 / B;           // K-steps per accumulation segment (128 K)
    static constexpr int kSub = B / 16;                 // MMAs of K = 16 per K-step and product
    static constexpr uint32_t kSBO = 32 * B;            // bytes between the 8-row groups of one plane
    static constexpr uint32_t kLoOff = 16 * B;          // bytes from a group's hi part to its lo part
};

constexpr int kTileN = 256;                  // MMA N = accumulator columns in tensor memory
constexpr int kEpiWarps = 8;                 // epilogue warps: 2 per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kSegBufs = 512 / kTileN;       // segment accumulators: the 512 TMEM columns
// epilogue metadata per warp (8 words per output block): at b = 32 and 64
// (4 and 2 blocks per warp) it is parked in the padding column of the warp's
// 32 x 33 staging tile; at b = 16 (16 blocks per warp) in a region of its own
template <int B>
constexpr int meta_words() { return B == 16 ? 16 * 8 : 0; }
template <int B>
constexpr int meta_stride() { return B == 16 ? 1 : 33; }
// output blocks whose metadata an epilogue warp holds (one lane each)
template <int B>
constexpr int blocks_per_warp() { return B == 16 ? 16 : B == 32 ? 4 : 2; }
static_assert(kSegBufs >= 2 && (kSegBufs & (kSegBufs - 1)) == 0, "tile shape");

// Stays 0 for the life of the program: the test setting `hold` makes the
// producer wait for it, so that every wait of the kernel runs out.
__device__ int g_never_set = 0;

// Test setting `hold`: the MMA thread first waits (bounded) for g_never_set;
// the wait runs out and raises the abort flag before any MMA is issued, so
// the copy warp's wait for a free stage runs out too and it drains the copies
// it has in flight.  Kept out of line: inlined ahead of the loops it slowed
// the kernel down twofold.
__device__ __noinline__ void hold_until_timeout(volatile int *abort_flag, long long limit) {
    const long long t0 = clock64();
    while (*(volatile int *)&g_never_set == 0)
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return;
        }
}

// ---------------------------------------------------------------------------
// operand planes: hi/lo split in the K-major core-matrix layout
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ int pair_offset(int r, int c, int plane) {
    // element (r, c) of plane `plane` (0 hi, 1 lo) of a B x B block: the two
    // planes' 8-row groups alternate (8 B elements each), so that one copy
    // brings both and both are K-major core-matrix operands with a 32 B-byte
    // stride between 8-row groups; inside a group, core matrix (c/8) at 64
    // elements
    return (r >> 3) * (16 * B) + plane * (8 * B) + ((c >> 3) << 6) + ((r & 7) << 3) + (c & 7);
}

// Largest block norm of every matrix of the set: each CTA takes a contiguous
// chunk of blocks and folds the part of every matrix it overlaps into mx[m]
// (norms are non-negative, so their bit patterns order like the values).
__global__ void k_matrix_max(const float *__restrict__ nrm, const int *__restrict__ mat_first, int nmat,
                             unsigned *__restrict__ mx) {
    const int64_t total = mat_first[nmat];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * per, c1 = c0 + per < total ? c0 + per : total;
    __shared__ float sh[32];
    for (int m = 0; m < nmat; ++m) {
        const int64_t a = c0 > mat_first[m] ? c0 : mat_first[m];
        const int64_t b = c1 < mat_first[m + 1] ? c1 : mat_first[m + 1];
        if (a >= b) continue;                               // the same for the whole CTA
        float v = 0.f;
        for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) v = fmaxf(v, nrm[p]);
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = fmaxf(v, sh[k]);
            atomicMax(&mx[m], __float_as_uint(v));
        }
        __syncthreads();
    }
}

// per matrix m: scale[m] = 2^floor(log2(2^14 / max block norm)) for fp16 (the
// largest element then sits below 2^14, far from fp16 overflow, and values
// down to ~1e-9 of it stay normal); 1 for bf16, whose exponent range is FP32's
__global__ void k_matrix_scales(const unsigned *__restrict__ mxbits, int nmat, int fp16, float *__restrict__ scale) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmat) return;
    const float mx = __uint_as_float(mxbits[m]);
    float s = 1.f;
    if (fp16 && mx > 0.f) {
        int e = (int)floorf(log2f(16384.f / mx));
        e = max(-60, min(60, e));
        s = ldexpf(1.f, e);
    }
    scale[m] = s;
}

// one thread per 8 consecutive elements of a block row (one core-matrix row):
// 64 bytes of FP64 in, 16 bytes of hi and 16 bytes of lo out
template <bool BF16, int B>
__global__ void k_split_planes(const double *__restrict__ val, int64_t nblk, uint16_t *__restrict__ hi,
                               const float *__restrict__ scale,
                               const int *__restrict__ mat_first, int nmat, const int *__restrict__ tpos) {
    constexpr int kPE = B * B;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nblk * (kPE / 8)) return;
    const int64_t p = g / (kPE / 8);
    const int rc0 = (int)(g % (kPE / 8)) * 8;     // first element (row r, columns c0..c0+7)
    const int r = rc0 / B, c0 = rc0 % B;
    int m = 0;
    while (m + 1 < nmat && p >= mat_first[m + 1]) ++m;
    const float sc = scale[m];
    const double2 *v2 = reinterpret_cast<const double2 *>(val + p * kPE + rc0);
    uint16_t h[8], l[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 x2 = v2[k];
        const float xs[2] = {(float)x2.x * sc, (float)x2.y * sc};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float x = xs[u];
            if (BF16) {
                const __nv_bfloat16 bh = __float2bfloat16_rn(x);
                const __nv_bfloat16 bl = __float2bfloat16_rn(x - __bfloat162float(bh));
                h[2 * k + u] = __bfloat16_as_ushort(bh);
                l[2 * k + u] = __bfloat16_as_ushort(bl);
            } else {
                const __half hh = __float2half_rn(x);
                const __half hl = __float2half_rn(x - __half2float(hh));
                h[2 * k + u] = __half_as_ushort(hh);
                l[2 * k + u] = __half_as_ushort(hl);
            }
        }
    }
    uint4 hv, lv;
    hv.x = h[0] | ((uint32_t)h[1] << 16); hv.y = h[2] | ((uint32_t)h[3] << 16);
    hv.z = h[4] | ((uint32_t)h[5] << 16); hv.w = h[6] | ((uint32_t)h[7] << 16);
    lv.x = l[0] | ((uint32_t)l[1] << 16); lv.y = l[2] | ((uint32_t)l[3] << 16);
    lv.z = l[4] | ((uint32_t)l[5] << 16); lv.w = l[6] | ((uint32_t)l[7] << 16);
    // columns c0..c0+7 of row r are 8 consecutive elements of one core matrix;
    // the block's planes go to the position of its transpose (tpos), or to
    // its own position without one
    const int64_t at = tpos ? (int64_t)tpos[p] : p;
    if (at < 0) return;
    uint16_t *o = hi + at * (2 * kPE);
    *reinterpret_cast<uint4 *>(o + pair_offset<B>(r, c0, 0)) = hv;
    *reinterpret_cast<uint4 *>(o + pair_offset<B>(r, c0, 1)) = lv;
}

// Position of the transposed block: for block e = (i, k) of matrix m of the
// set, the global index of block (k, i) of the same matrix.  The patterns of
// the set are symmetric, so it exists; if not, -1 and error bit 8.
__global__ void k_transpose_pos(const int *__restrict__ rp, const int *__restrict__ col, int nrow_flat, int NB,
                                int64_t total, int *__restrict__ tpos, int *__restrict__ err) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    // flat row r of e: the last r with rp[r] <= e
    int lo = 0, hi = nrow_flat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int m = lo / NB, i = lo - m * NB, k = col[e];
    const int end = rp[m * NB + k + 1];
    int a = rp[m * NB + k], z = end;
    while (a < z) {
        const int mid = (a + z) >> 1;
        if (col[mid] < i) a = mid + 1; else z = mid;
    }
    if (a < end && col[a] == i) {
        tpos[e] = a;
    } else {
        tpos[e] = -1;
        atomicOr(err, 8);
    }
}

// ---------------------------------------------------------------------------
// the tensor-core product kernel
// ---------------------------------------------------------------------------
struct TcArgs {
    const uint16_t *planes;       // operand planes of the input set (hi and lo interleaved per block)
    const uint16_t *zero;         // zero blocks (kSlots per CTA)
    const int *tiles;
    const int64_t *step_off;
    const int *steps;
    int ntile;
    uint32_t idesc;
    const float *scale;           // per matrix operand scale
    int job_a[kMaxJobs], job_b[kMaxJobs];
    // epilogue
    const double *in_val;
    const int *slot_row, *slot_job, *slot_x, *slot_t;
    const int *sys_of_row;
    const double *c_lin, *c_sq, *tau0, *tau1;
    int job_tau_sel[kMaxJobs];
    double *out_val;        // upper slot s at index uidx[s] - u0
    float *out_nrm;
    uint8_t *keep;
    const int *uidx;
    int64_t u0;
    int *err;
    long long wait_cycles;        // bound of every mbarrier wait
    int hold;                     // test setting: the MMA thread waits for g_never_set first
    int runs;                     // 1: slots whose blocks are neighbours in memory share a copy
    const int *pre_err;           // error bits of the operand preparation, passed on to err
};

struct __align__(8) SmemCtl {
    uint64_t full[8], empty[8];
    uint64_t seg_full[kSegBufs], seg_empty[kSegBufs];
    uint64_t drain;
    uint64_t pair[4];             // b = 64: handshake of the two epilogue warps of a column range
    float pair_ss[kEpiWarps];     // b = 64: partial squared norms exchanged within a pair
    uint32_t tmem_base;
    int abort_flag;
};

// Epilogue metadata of one output block, gathered by one lane while the
// tile's MMAs run and parked in shared memory (8 words per block: slot, old
// slot, diagonal, output index, c_lin, c_sq, tau lo, tau hi).
template <int B>
__device__ __forceinline__ void gather_meta(const TcArgs &A, int s, float *q) {
    constexpr int W = meta_stride<B>();
    int m_sx = -1, m_diag = 0, m_keepidx = 0;
    float m_cl = 0.f, m_cq = 0.f;
    double m_tau = 0.0;
    if (s >= 0) {
        const int i = A.slot_row[s];
        const int sys = A.sys_of_row[i];
        const int job = A.slot_job[s];
        m_cl = (float)A.c_lin[sys];
        // undo the operand scaling: every term of a job has the same scale product
        m_cq = (float)A.c_sq[sys] / (A.scale[A.job_a[job]] * A.scale[A.job_b[job]]);
        m_tau = A.job_tau_sel[job] ? A.tau1[sys] : A.tau0[sys];
        m_sx = A.slot_x[s];
        m_diag = A.slot_t[s] == s;
        m_keepidx = A.uidx[s] - (int)A.u0;
    }
    q[0] = __int_as_float(s);
    q[W] = __int_as_float(m_sx);
    q[2 * W] = __int_as_float(m_diag);
    q[3 * W] = __int_as_float(m_keepidx);
    q[4 * W] = m_cl;
    q[5 * W] = m_cq;
    q[6 * W] = __int_as_float(__double2loint(m_tau));
    q[7 * W] = __int_as_float(__double2hiint(m_tau));
}

// The output block (slot) whose metadata lane `lane` of epilogue warp
// (eq, colhalf) gathers, from tile record d; -1 for lanes without one.
template <int B, class G>
__device__ __forceinline__ int lane_slot(const int *d, int eq, int colhalf, int lane) {
    if constexpr (B == 32) {
        // block row eq of the tile, block columns 4 colhalf .. 4 colhalf + 3
        return lane < 4 ? d[4 + eq * G::TBN + 4 * colhalf + lane] : -1;
    } else if constexpr (B == 16) {
        // block rows 2 eq (lanes 0-7) and 2 eq + 1 (lanes 8-15), block columns 8 colhalf .. + 7
        return lane < 16 ? d[4 + (2 * eq + (lane >> 3)) * G::TBN + 8 * colhalf + (lane & 7)] : -1;
    } else {
        // block row eq / 2 (row half eq & 1), block columns 2 colhalf, 2 colhalf + 1
        return lane < 2 ? d[4 + (eq >> 1) * G::TBN + 2 * colhalf + lane] : -1;
    }
}

// Prefetch into L2 the old X blocks of the linear terms of tile tn (the
// warp's next tile), two segments before they are read.
template <int B, class G>
__device__ __forceinline__ void prefetch_old_blocks(const TcArgs &A, int tn, int eq, int colhalf, int lane) {
    const int s = lane_slot<B, G>(A.tiles + (size_t)tn * G::kTileInts, eq, colhalf, lane);
    if (s < 0) return;
    const int sx = A.slot_x[s];
    if (sx < 0 || A.c_lin[A.sys_of_row[A.slot_row[s]]] == 0.0) return;
    const double *px = A.in_val + (size_t)sx * (B * B);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(px), "r"(8 * B * B) : "memory");
}

// b = 64: one step of the handshake of the two epilogue warps that share a
// block column range (their lane quarters hold the two row halves of the same
// blocks): both arrive on the pair's mbarrier (count 2) and wait, bounded like
// every wait of the kernel, for the phase to complete.
__device__ __forceinline__ bool pair_sync(SmemCtl *ctl, int pair, uint32_t &round, int lane,
                                          volatile int *abort_flag, long long limit) {
    __threadfence_block();     // this lane's shared-memory writes before the arrival
    __syncwarp();
    int ok = 1;
    if (lane == 0) {
        mbar_arrive(&ctl->pair[pair]);
        ok = mbar_wait(&ctl->pair[pair], round & 1, abort_flag, limit) ? 1 : 0;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __threadfence_block();     // the partner's writes before this lane's reads
    ++round;
    return ok != 0;
}

template <int B>
__global__ void __launch_bounds__(kThreads, 1) k_tc_bf16x3(TcArgs A) {
    using G = Geo<B>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *stages = smem_raw;                                                    // kStages stages
    float *stage_ep = reinterpret_cast<float *>(smem_raw + G::kStages * G::kStageBytes);   // kEpiWarps x 32 x 33
    float *meta_all = stage_ep + kEpiWarps * 32 * 33;                              // kEpiWarps x meta_words
    SmemCtl *ctl = reinterpret_cast<SmemCtl *>(meta_all + kEpiWarps * meta_words<B>());

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort_flag = &ctl->abort_flag;

    if (threadIdx.x == 0) {
        if (blockIdx.x == 0 && *A.pre_err) atomicOr(A.err, *A.pre_err);
        for (int s = 0; s < G::kStages; ++s) { mbar_init(&ctl->full[s], 1); mbar_init(&ctl->empty[s], 1); }
        for (int b = 0; b < kSegBufs; ++b) { mbar_init(&ctl->seg_full[b], 1); mbar_init(&ctl->seg_empty[b], kEpiWarps); }
        mbar_init(&ctl->drain, 1);
        for (int q = 0; q < 4; ++q) mbar_init(&ctl->pair[q], 2);
        ctl->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&ctl->tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        // ---------------- producer: bulk copies of the operand blocks ----------------
        // Lane m < kSlots owns slot m of every stage (slot m < TBM: A block row
        // m, else B block row m - TBM; slot m at m * kPairBytes): it loads the
        // block index of the next K-step while the current step's copies are
        // issued.  A slot whose block is missing needs zeros; a stage slot that
        // already holds zeros from its previous use is not copied again (zmask).
        uint32_t it = 0;
        bool ok = true;
        uint32_t zmask[G::kStages];
#pragma unroll
        for (int k = 0; k < G::kStages; ++k) zmask[k] = 0u;
        for (int t = blockIdx.x; t < A.ntile && ok; t += gridDim.x) {
            const int64_t s0 = A.step_off[t], s1 = A.step_off[t + 1];
            int nxt = (s0 < s1 && lane < G::kSlots) ? A.steps[s0 * G::kSlots + lane] : -1;
            for (int64_t q = s0; q < s1; ++q, ++it) {
                const int cur = nxt;
                if (q + 1 < s1 && lane < G::kSlots) nxt = A.steps[(q + 1) * G::kSlots + lane];
                const int st = it % G::kStages;
                const uint32_t ph = (it / G::kStages) & 1;
                const uint32_t zbits = __ballot_sync(0xffffffffu, lane < G::kSlots && cur < 0);
                uint32_t zprev = 0u;
#pragma unroll
                for (int k = 0; k < G::kStages; ++k)
                    if (k == st) zprev = zmask[k];
                const bool skip = lane >= G::kSlots || (cur < 0 && ((zprev >> lane) & 1u));
                const uint32_t need = __ballot_sync(0xffffffffu, !skip);
                int waited = 1;
                if (lane == 0) {
                    waited = mbar_wait(&ctl->empty[st], ph ^ 1, abort_flag, A.wait_cycles) ? 1 : 0;
                    if (waited) mbar_expect_tx(&ctl->full[st], (uint32_t)__popc(need) * G::kPairBytes);
                }
                waited = __shfl_sync(0xffffffffu, waited, 0);
                if (!waited) { ok = false; break; }
#pragma unroll
                for (int k = 0; k < G::kStages; ++k)
                    if (k == st) zmask[k] = zbits;
                // zero blocks: one per CTA and slot (so that the CTAs do not all
                // read the same few L2 sectors), adjacent like the slots
                const uint16_t *src = cur >= 0 ? A.planes + (size_t)cur * (2 * G::kPlaneElems)
                                               : A.zero + ((size_t)blockIdx.x * G::kSlots + lane) * (2 * G::kPlaneElems);
                // runs: a slot whose source follows its left neighbour's in
                // memory joins that neighbour's copy; the first slot of a run
                // copies the whole run
                const uint16_t *left = reinterpret_cast<const uint16_t *>(
                    __shfl_up_sync(0xffffffffu, reinterpret_cast<unsigned long long>(src), 1));
                const bool joins = A.runs && lane > 0 && !skip && ((need >> (lane - 1)) & 1u) &&
                                   src == left + 2 * G::kPlaneElems;
                const uint32_t jm = __ballot_sync(0xffffffffu, joins);
                if (!skip && !joins) {
                    const uint32_t above = lane < 31 ? jm >> (lane + 1) : 0u;
                    const uint32_t len = (uint32_t)__ffs(~above);      // this slot and the slots that join it
                    bulk_g2s(stages + st * G::kStageBytes + lane * G::kPairBytes, src, len * G::kPairBytes,
                             &ctl->full[st]);
                }
            }
        }
        if (!ok && lane == 0) {
            // after an abort, wait (bounded) until the copies of the stages
            // still in flight have landed before the CTA leaves: the last
            // min(it, kStages) issued stages, each at the phase of its last use
            const uint32_t n = it < (uint32_t)G::kStages ? it : (uint32_t)G::kStages;
            for (uint32_t q = it - n; q < it; ++q)
                mbar_wait_drain(&ctl->full[q % G::kStages], (q / G::kStages) & 1, A.wait_cycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            if (A.hold) hold_until_timeout(abort_flag, A.wait_cycles);
            uint32_t it = 0, seg = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < A.ntile && !*abort_flag; t += gridDim.x) {
                const int64_t s0 = A.step_off[t], s1 = A.step_off[t + 1];
                bool ok = true;
                for (int64_t q = s0; q < s1 && ok; ++seg) {
                    // one segment: up to kSegSteps K-steps into a fresh accumulator
                    const int buf = seg & (kSegBufs - 1);
                    const uint32_t use = seg / kSegBufs;
                    if (!mbar_wait(&ctl->seg_empty[buf], (use & 1) ^ 1, abort_flag, A.wait_cycles)) { ok = false; break; }
                    fence_after();
                    const uint32_t d_tmem = tmem + buf * kTileN;
                    const int64_t qe = q + G::kSegSteps < s1 ? q + G::kSegSteps : s1;
                    const int64_t qs = q;
                    for (; q < qe; ++q, ++it) {
                        const int st = it % G::kStages;
                        const uint32_t ph = (it / G::kStages) & 1;
                        if (!mbar_wait(&ctl->full[st], ph, abort_flag, A.wait_cycles)) { ok = false; break; }
                        fence_after();
                        const uint32_t base = smem_u32(stages + st * G::kStageBytes);
                        const uint32_t a_hi = base, a_lo = base + G::kLoOff;
                        const uint32_t b_hi = base + G::kSideABytes, b_lo = base + G::kSideABytes + G::kLoOff;
#pragma unroll
                        for (int kk = 0; kk < G::kSub; ++kk) {
                            const uint32_t ko = kk * 256;
                            const uint32_t first = (q == qs && kk == 0) ? 0u : 1u;
                            mma_f16(d_tmem, smem_desc(a_hi + ko, 128, G::kSBO), smem_desc(b_hi + ko, 128, G::kSBO), A.idesc, first);
                            mma_f16(d_tmem, smem_desc(a_hi + ko, 128, G::kSBO), smem_desc(b_lo + ko, 128, G::kSBO), A.idesc, 1u);
                            mma_f16(d_tmem, smem_desc(a_lo + ko, 128, G::kSBO), smem_desc(b_hi + ko, 128, G::kSBO), A.idesc, 1u);
                        }
                        issued = true;
                        mma_commit(&ctl->empty[st]);
                    }
                    if (ok) mma_commit(&ctl->seg_full[buf]);
                }
                if (!ok) break;
            }
            if (*abort_flag && issued) {
                // drain: wait (bounded) until every MMA this thread issued has completed
                mma_commit(&ctl->drain);
                long long t0 = clock64();
                while (!mbar_try_wait(&ctl->drain, 0) && clock64() - t0 < A.wait_cycles) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9 ----------------
        const int eq = warp & 3;                        // TMEM lanes 32*eq .. 32*eq+31
        const int colhalf = (warp - 2) >> 2;            // accumulator columns 128*colhalf .. +127
        float *S = stage_ep + (warp - 2) * 32 * 33;     // one 32 x 32 tile, transposed through shared memory
        // metadata of block n, word w at meta[(8 n + w) * MW]
        constexpr int MW = meta_stride<B>();
        float *meta = B == 16 ? meta_all + (warp - 2) * meta_words<B>() : S + 32;
        uint32_t seg = 0, pround = 0;
        for (int t = blockIdx.x; t < A.ntile && !*abort_flag; t += gridDim.x) {
            const int *d = A.tiles + (size_t)t * G::kTileInts;
            // metadata of this warp's output blocks, one lane each
            {
                const int s = lane_slot<B, G>(d, eq, colhalf, lane);
                // blocks per warp: 4 at b = 32, 16 at b = 16, 2 at b = 64 (each shared
                // with the partner warp that holds the other row half)
                if (lane < blocks_per_warp<B>()) gather_meta<B>(A, s, meta + lane * 8 * MW);
            }
            __syncwarp();
            const int nst = d[3];
            if (nst < 0 && lane == 0) atomicOr(A.err, 4);
            // the tile's accumulator: sum of its segments, added with
            // round-to-nearest in registers (row 32*eq + lane, this warp's 128 columns)
            float racc[128];
#pragma unroll
            for (int c = 0; c < 128; ++c) racc[c] = 0.f;
            const int nseg = nst > 0 ? (nst + G::kSegSteps - 1) / G::kSegSteps : 0;
            bool ok = true;
            for (int g = 0; g < nseg; ++g, ++seg) {
                const int buf = seg & (kSegBufs - 1);
                const uint32_t use = seg / kSegBufs;
                if (g == (nseg > 2 ? nseg - 2 : 0) && t + (int)gridDim.x < A.ntile)
                    prefetch_old_blocks<B, G>(A, t + gridDim.x, eq, colhalf, lane);
                if (!mbar_wait(&ctl->seg_full[buf], use & 1, abort_flag, A.wait_cycles)) { ok = false; break; }
                fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * eq) << 16) + buf * kTileN + 128 * colhalf;
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    float part[16];
                    tmem_ld16(ta + h * 16, part);
#pragma unroll
                    for (int c = 0; c < 16; ++c) racc[h * 16 + c] += part[c];
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->seg_empty[buf]);
            }
            if (!ok) break;

            if constexpr (B == 32) {
                // lane l holds row l of 4 blocks of 32 columns
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    const float *q = meta + n * 8 * MW;
                    const int s = __float_as_int(q[0]);
                    if (s < 0) continue;
                    float acc[32];
#pragma unroll
                    for (int c = 0; c < 32; ++c) acc[c] = racc[n * 32 + c];
                    const float cl = q[4 * MW];
                    const float cq = q[5 * MW];
                    const double tau = __hiloint2double(__float_as_int(q[7 * MW]), __float_as_int(q[6 * MW]));
                    const int sx = __float_as_int(q[1 * MW]);
                    const bool diag = __float_as_int(q[2 * MW]) != 0;
                    const int oidx = __float_as_int(q[3 * MW]);
                    __syncwarp();
                    // linear term: the old block is staged in S (coalesced row reads,
                    // rounded to FP32), then each lane takes its own row
                    if (sx >= 0 && cl != 0.f) {
                        const double *gx = A.in_val + (size_t)sx * G::kPlaneElems;
#pragma unroll 8
                        for (int r = 0; r < 32; ++r) S[r * 33 + lane] = (float)gx[r * 32 + lane];
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 32; ++c) acc[c] = fmaf(cl, S[lane * 33 + c], cq * acc[c]);
                        __syncwarp();
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) acc[c] = cq * acc[c];
                    }
                    // a diagonal block is symmetrised as (X + X^T) / 2
#pragma unroll
                    for (int c = 0; c < 32; ++c) S[lane * 33 + c] = acc[c];
                    __syncwarp();
                    if (diag) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) acc[c] = 0.5f * (S[lane * 33 + c] + S[c * 33 + lane]);
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 32; ++c) S[lane * 33 + c] = acc[c];
                        __syncwarp();
                    }
                    float ss = 0.f;
#pragma unroll
                    for (int c = 0; c < 32; ++c) ss = fmaf(acc[c], acc[c], ss);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    const float nrm = sqrtf(ss) * (1.0f + 1e-6f);
                    const bool kp = ((double)nrm >= tau) && (nrm > 0.f);
                    double *o = A.out_val + (size_t)oidx * G::kPlaneElems;
                    for (int r = 0; r < 32; ++r) o[r * 32 + lane] = (double)S[r * 33 + lane];
                    if (lane == 0) {
                        A.out_nrm[s] = nrm;
                        A.keep[s] = kp;
                    }
                    __syncwarp();
                }
            } else if constexpr (B == 16) {
                // half-warp h = lane / 16 holds rows of block row 2 eq + h: lane l
                // is row l & 15 of that block row, over 8 blocks of 16 columns
                const int h = lane >> 4, c16 = lane & 15;
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    const float *q = meta + (h * 8 + n) * 8 * MW;
                    const int s = __float_as_int(q[0]);
                    const float cl = q[4 * MW];
                    const float cq = q[5 * MW];
                    const double tau = __hiloint2double(__float_as_int(q[7 * MW]), __float_as_int(q[6 * MW]));
                    const int sx = __float_as_int(q[1 * MW]);
                    const bool diag = s >= 0 && __float_as_int(q[2 * MW]) != 0;
                    const int oidx = __float_as_int(q[3 * MW]);
                    const bool lin = s >= 0 && sx >= 0 && cl != 0.f;
                    float acc[16];
                    __syncwarp();
                    if (lin) {
                        const double *gx = A.in_val + (size_t)sx * G::kPlaneElems;
#pragma unroll
                        for (int r = 0; r < 16; ++r) S[(16 * h + r) * 33 + c16] = (float)gx[r * 16 + c16];
                    }
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        acc[c] = lin ? fmaf(cl, S[lane * 33 + c], cq * racc[n * 16 + c]) : cq * racc[n * 16 + c];
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < 16; ++c) S[lane * 33 + c] = acc[c];
                    __syncwarp();
                    // a diagonal block is symmetrised as (X + X^T) / 2
                    if (diag) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) acc[c] = 0.5f * (S[lane * 33 + c] + S[(16 * h + c) * 33 + c16]);
                    }
                    __syncwarp();
                    if (diag) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) S[lane * 33 + c] = acc[c];
                    }
                    __syncwarp();
                    float ss = 0.f;
#pragma unroll
                    for (int c = 0; c < 16; ++c) ss = fmaf(acc[c], acc[c], ss);
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    const float nrm = sqrtf(ss) * (1.0f + 1e-6f);
                    const bool kp = ((double)nrm >= tau) && (nrm > 0.f);
                    if (s >= 0) {
                        double *o = A.out_val + (size_t)oidx * G::kPlaneElems;
#pragma unroll
                        for (int r = 0; r < 16; ++r) o[r * 16 + c16] = (double)S[(16 * h + r) * 33 + c16];
                        if (c16 == 0) {
                            A.out_nrm[s] = nrm;
                            A.keep[s] = kp;
                        }
                    }
                    __syncwarp();
                }
            } else {
                // b = 64: lane l holds row 32 rh + l of 2 blocks of 64 columns; the
                // partner warp (warp ^ 1) holds the other 32 rows of the same blocks
                // (both see the same slots, so both take the same branches and
                // handshakes; after an abort both skip the rest)
                const int rh = eq & 1, pr = (warp - 2) >> 1;
                const float *Sp = stage_ep + ((warp ^ 1) - 2) * 32 * 33;   // the partner's staging tile
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    const float *q = meta + n * 8 * MW;
                    const int s = __float_as_int(q[0]);
                    if (s < 0 || !ok) continue;
                    const float cl = q[4 * MW];
                    const float cq = q[5 * MW];
                    const double tau = __hiloint2double(__float_as_int(q[7 * MW]), __float_as_int(q[6 * MW]));
                    const int sx = __float_as_int(q[1 * MW]);
                    const bool diag = __float_as_int(q[2 * MW]) != 0;
                    const int oidx = __float_as_int(q[3 * MW]);
                    // linear term, one 32-column half of the old rows at a time
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch) {
                        __syncwarp();
                        if (sx >= 0 && cl != 0.f) {
                            const double *gx = A.in_val + (size_t)sx * G::kPlaneElems + (size_t)(32 * rh) * 64 + 32 * ch;
#pragma unroll 8
                            for (int r = 0; r < 32; ++r) S[r * 33 + lane] = (float)gx[r * 64 + lane];
                            __syncwarp();
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                racc[n * 64 + 32 * ch + c] = fmaf(cl, S[lane * 33 + c], cq * racc[n * 64 + 32 * ch + c]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c) racc[n * 64 + 32 * ch + c] = cq * racc[n * 64 + 32 * ch + c];
                        }
                    }
                    if (diag) {
                        // (X + X^T) / 2: the off-diagonal quarter (rh, 1 - rh) pairs with
                        // the partner's quarter (1 - rh, rh), exchanged through S
                        __syncwarp();
                        if (rh == 0) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) S[lane * 33 + c] = racc[n * 64 + 32 + c];
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c) S[lane * 33 + c] = racc[n * 64 + c];
                        }
                        ok = pair_sync(ctl, pr, pround, lane, abort_flag, A.wait_cycles);
                        if (rh == 0) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) racc[n * 64 + 32 + c] = 0.5f * (racc[n * 64 + 32 + c] + Sp[c * 33 + lane]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c) racc[n * 64 + c] = 0.5f * (racc[n * 64 + c] + Sp[c * 33 + lane]);
                        }
                        ok = pair_sync(ctl, pr, pround, lane, abort_flag, A.wait_cycles) && ok;
                        // the diagonal quarter (rh, rh) with its own transpose
                        if (rh == 0) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) S[lane * 33 + c] = racc[n * 64 + c];
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c) S[lane * 33 + c] = racc[n * 64 + 32 + c];
                        }
                        __syncwarp();
                        if (rh == 0) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) racc[n * 64 + c] = 0.5f * (racc[n * 64 + c] + S[c * 33 + lane]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c) racc[n * 64 + 32 + c] = 0.5f * (racc[n * 64 + 32 + c] + S[c * 33 + lane]);
                        }
                    }
                    // Frobenius norm over both row halves
                    float ss = 0.f;
#pragma unroll
                    for (int c = 0; c < 64; ++c) ss = fmaf(racc[n * 64 + c], racc[n * 64 + c], ss);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    if (lane == 0) ctl->pair_ss[warp - 2] = ss;
                    ok = pair_sync(ctl, pr, pround, lane, abort_flag, A.wait_cycles) && ok;
                    const float other = *(volatile float *)&ctl->pair_ss[(warp ^ 1) - 2];
                    const float tot = rh == 0 ? ss + other : other + ss;
                    const float nrm = sqrtf(tot) * (1.0f + 1e-6f);
                    const bool kp = ((double)nrm >= tau) && (nrm > 0.f);
                    // store this warp's 32 rows, one 32-column half at a time
                    double *o = A.out_val + (size_t)oidx * G::kPlaneElems + (size_t)(32 * rh) * 64;
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch) {
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 32; ++c) S[lane * 33 + c] = racc[n * 64 + 32 * ch + c];
                        __syncwarp();
                        for (int r = 0; r < 32; ++r) o[r * 64 + 32 * ch + lane] = (double)S[r * 33 + lane];
                    }
                    if (lane == 0 && rh == 0) {
                        A.out_nrm[s] = nrm;
                        A.keep[s] = kp;
                    }
                    // the partner reuses pair_ss and its S only after this point
                    ok = pair_sync(ctl, pr, pround, lane, abort_flag, A.wait_cycles) && ok;
                }
                if (!ok) break;
            }
        }
    }

    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && ctl->abort_flag) atomicOr(A.err, 1);
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int B>
constexpr size_t smem_bytes() {
    return (size_t)Geo<B>::kStages * Geo<B>::kStageBytes + kEpiWarps * 32 * 33 * sizeof(float) +
           kEpiWarps * meta_words<B>() * sizeof(float) + sizeof(SmemCtl) + 1024;
}
static_assert(smem_bytes<16>() <= 227 * 1024 && smem_bytes<32>() <= 227 * 1024 && smem_bytes<64>() <= 227 * 1024,
              "shared memory of the tensor-core kernel exceeds 227 KB");
static_assert(Geo<16>::kStages <= 8 && Geo<32>::kStages <= 8 && Geo<64>::kStages <= 8, "mbarrier arrays");

template <int B>
void split_planes(MatSet &in, Arith ar, TcWork &w, cudaStream_t st) {
    const int64_t n = in.total * (int64_t)(B * B);
    const int64_t grid = (n / 8 + 255) / 256;
    const int *tpos = w.tpos_valid ? w.tpos.p : nullptr;
    if (ar == AR_BF16X3)
        k_split_planes<true, B><<<(unsigned)grid, 256, 0, st>>>(in.val.p, in.total, in.ophi.p, w.scale.p,
                                                                w.mat_first.p, in.nmat, tpos);
    else
        k_split_planes<false, B><<<(unsigned)grid, 256, 0, st>>>(in.val.p, in.total, in.ophi.p, w.scale.p,
                                                                 w.mat_first.p, in.nmat, tpos);
    RDM_LAUNCH_CHECK();
}

template <int B>
double launch_tc(const NumArgs &a, const MatSet &in, const JobTable &jt, Arith ar, TcWork &w,
                 const TcPlan &plan, cudaStream_t st) {
    using G = Geo<B>;
    int dev = 0, nsm = 0;
    RDM_CUDA_TRY(cudaGetDevice(&dev));
    RDM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t zero_elems = (size_t)nsm * G::kSlots * 2 * G::kPlaneElems;   // a zero block per CTA and slot
    if (!w.zero.p || w.zero.cap < zero_elems) {
        w.zero.ensure(zero_elems);
        RDM_CUDA_TRY(cudaMemsetAsync(w.zero.p, 0, w.zero.cap * sizeof(uint16_t), st));
    }
    TcArgs A{};
    A.planes = in.ophi.p; A.zero = w.zero.p;
    A.tiles = w.tiles.p; A.step_off = w.step_off.p; A.steps = w.steps.p; A.ntile = plan.ntile;
    // kind::f16: D = F32 (bit 4), A/B = BF16 (1) or F16 (0), K-major, N = kTileN, M = 128
    const uint32_t ab = ar == AR_BF16X3 ? 1u : 0u;
    A.idesc = (1u << 4) | (ab << 7) | (ab << 10) | (((uint32_t)kTileN >> 3) << 17) | ((128u >> 4) << 24);
    A.scale = w.scale.p;
    for (int p = 0; p < kMaxJobs; ++p) {
        A.job_a[p] = p < jt.njob ? jt.job[p].a[0] : 0;
        A.job_b[p] = p < jt.njob ? jt.job[p].b[0] : 0;
    }
    A.in_val = a.in_val; A.slot_row = a.slot_row; A.slot_job = a.slot_job; A.slot_x = a.slot_x;
    A.slot_t = a.slot_t; A.sys_of_row = a.sys_of_row; A.c_lin = a.c_lin; A.c_sq = a.c_sq;
    A.tau0 = a.tau0; A.tau1 = a.tau1;
    for (int p = 0; p < kMaxJobs; ++p) A.job_tau_sel[p] = a.job_tau_sel[p];
    A.out_val = a.out_val; A.out_nrm = a.out_nrm; A.keep = a.keep; A.uidx = a.uidx; A.u0 = a.u0;
    A.err = w.counters.p;
    A.wait_cycles = w.knobs.wait_cycles > 0 ? w.knobs.wait_cycles : kWaitCycles;
    A.hold = w.knobs.hold;
    A.runs = w.tpos_valid ? 1 : 0;
    A.pre_err = w.pre_err.p;
    func_smem_once((const void *)k_tc_bf16x3<B>, (int)smem_bytes<B>());
    const int grid = plan.ntile < nsm ? plan.ntile : nsm;
    k_tc_bf16x3<B><<<grid, kThreads, smem_bytes<B>(), st>>>(A);
    RDM_LAUNCH_CHECK();
    return (double)plan.nsteps * 3.0 * 2.0 * 128.0 * kTileN * B;
}

}  // namespace

bool tc_block_size_ok(int b) { return b == 16 || b == 32 || b == 64; }

int tc_tile_rows(int b) { return tc_block_size_ok(b) ? 128 / b : 4; }

void prepare_operands(MatSet &in, Arith ar, TcWork &w, cudaStream_t st) {
    if (!tc_block_size_ok(in.b)) throw Error{-1, "the tensor-core path handles 16 x 16, 32 x 32 and 64 x 64 blocks"};
    if (ar != AR_BF16X3 && ar != AR_FP16X3) throw Error{-1, "tensor-core arithmetic not available"};
    const int nmat = in.nmat;
    std::vector<int> first(nmat + 1, 0);
    for (int m = 0; m < nmat; ++m) first[m + 1] = first[m] + (int)in.nnzb[m];
    w.mat_first.ensure(nmat + 1);
    w.scale.ensure(std::max(nmat, 1));
    RDM_CUDA_TRY(cudaMemcpyAsync(w.mat_first.p, first.data(), (nmat + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    w.mx.ensure(std::max(nmat, 1));
    RDM_CUDA_TRY(cudaMemsetAsync(w.mx.p, 0, std::max(nmat, 1) * sizeof(unsigned), st));
    if (in.total > 0) {
        const int grid = (int)std::min<int64_t>(4 * 152, (in.total + 255) / 256);
        k_matrix_max<<<grid, 256, 0, st>>>(in.nrm.p, w.mat_first.p, nmat, w.mx.p);
        RDM_LAUNCH_CHECK();
    }
    k_matrix_scales<<<(nmat + 31) / 32, 32, 0, st>>>(w.mx.p, nmat, ar == AR_FP16X3 ? 1 : 0, w.scale.p);
    RDM_LAUNCH_CHECK();
    const int64_t n = in.total * (int64_t)in.b * in.b;
    in.ophi.ensure(std::max<int64_t>(2 * n, 1));   // hi and lo, interleaved per block
    w.pre_err.ensure(1);
    RDM_CUDA_TRY(cudaMemsetAsync(w.pre_err.p, 0, sizeof(int), st));
    w.tpos_valid = false;
    if (n == 0) return;
    // planes at the positions of the transposed blocks (the plan builder
    // points the K-step lists there), unless the test setting asks for one
    // copy per block
    if (!w.knobs.block_copies) {
        w.tpos.ensure(in.total);
        k_transpose_pos<<<(unsigned)((in.total + 255) / 256), 256, 0, st>>>(
            in.row_ptr.p, in.col.p, nmat * in.NB, in.NB, in.total, w.tpos.p, w.pre_err.p);
        RDM_LAUNCH_CHECK();
        w.tpos_valid = true;
    }
    switch (in.b) {
        case 16: split_planes<16>(in, ar, w, st); break;
        case 32: split_planes<32>(in, ar, w, st); break;
        default: split_planes<64>(in, ar, w, st); break;
    }
}

double launch_numeric_tc(const NumArgs &a, const MatSet &in, const JobTable &jt, Arith ar, TcWork &w,
                         int NB, const TcPlan &plan, cudaStream_t st) {
    (void)NB;
    if (!tc_block_size_ok(in.b)) throw Error{-1, "the tensor-core path handles 16 x 16, 32 x 32 and 64 x 64 blocks"};
    if (plan.ntile == 0) return 0.0;
    switch (in.b) {
        case 16: return launch_tc<16>(a, in, jt, ar, w, plan, st);
        case 32: return launch_tc<32>(a, in, jt, ar, w, plan, st);
        default: return launch_tc<64>(a, in, jt, ar, w, plan, st);
    }
}

TcPlan build_tc_plan(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_rp,
                     const int *mcol, TcWork &w, JobMask job_mask, int unit0, int unit1, cudaStream_t st) {
    switch (in.b) {
        case 16: return build_plan<Geo<16>>(in, jt, sd, out_rp, mcol, w, job_mask, unit0, unit1, st);
        case 32: return build_plan<Geo<32>>(in, jt, sd, out_rp, mcol, w, job_mask, unit0, unit1, st);
        case 64: return build_plan<Geo<64>>(in, jt, sd, out_rp, mcol, w, job_mask, unit0, unit1, st);
        default: throw Error{-1, "the tensor-core path handles 16 x 16, 32 x 32 and 64 x 64 blocks"};
    }
}

}  // namespace rdm
