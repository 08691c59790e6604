// FP64-class products on the tensor cores (tcgen05 + TMEM, sm_103a) for
// 32 x 32 blocks, by exact slice products: the splitting of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms 59, 2012), in which a matrix is cut into
// slices whose products a low-precision matrix multiply computes without
// rounding, and the slice products are summed in higher precision.  Used for
// X0^2 in the final tier of the precision ladder, where X0 must end
// idempotent to FP64 accuracy.
//
// Slices.  Row r of X (a matrix of the input set) is scaled by
// sigma_r = 2^e_r, e_r the smallest exponent with max_k |X_rk| < 2^e_r, and
// x = X_rk / sigma_r in (-1, 1) is cut into S = 7 integer slices:
//   a_1 = rint(128 x),  x_1 = 128 x - a_1,  a_i = rint(128 x_{i-1}), ...
// so that X_rk = sigma_r (sum_i a_i 2^(-7 i) + d) with |d| <= 2^(-50):
// |a_1| <= 128, |a_i| <= 64 for i > 1, every a_i exact in bf16.  X is
// symmetric, so the slices of row c serve as the B operand of output column c
// as well (B rows = output columns, K-major), with the column scale sigma_c.
//
// Exact groups.  C_rc = sum_k X_rk X_kc = sigma_r sigma_c
// sum_g 2^(-7 g) D_g[r, c],  D_g = sum_{i + j = g} sum_k a_i[r, k] a_j[c, k].
// Slice pairs with i + j <= S + 1 = 8 are kept (the first dropped pairs are
// ~2^-63 of the product).  Per k a group adds at most 9 * 2^12 < 2^15.2,
// so over a segment of 128 K the integer D_g stays below 2^22.2: each group
// accumulates in its own FP32 tensor-memory accumulator WITHOUT rounding (the
// tensor cores' truncating FP32 accumulation is exact on integers below
// 2^24).  Seven groups x 64 columns = 448 of the 512 TMEM columns, so a tile
// is 128 x 64 (4 block rows x 2 block columns) and there is one accumulator
// buffer.  28 slice pairs x 2 K-slices = 56 MMAs of 128 x 64 x 16 per K-step.
//
// Epilogue.  After every segment each epilogue warp (one 32 x 32 output block:
// lane quarter = block row, column half = block column) adds the seven exact
// group sums, scaled by 2^(-7 g) (exact), into a double-FP32 accumulator
// (hi, lo) with Knuth's error-free TwoSum (about 48 bits over the whole sum),
// and releases the buffer.  At the tile's end, in FP64:
// C = c_lin X + c_sq sigma_r sigma_c (hi + lo); Frobenius norm, truncation flag,
// FP64 store.  The result is exactly symmetric (D_g[r,c] = D_g[c,r] as
// integers and every later step is the same for (r,c) and (c,r)), so diagonal
// blocks need no symmetrisation.
//
// Operand bytes: a K-step brings 6 blocks of 7 bf16 slices (84 KB) for
// 128 x 64 x 32 FP64-class multiply-adds: the bulk-copy ingest per SM bounds
// this kernel as it bounds the split one.  Warp roles, bounded waits and the
// abort drain are those of the split kernel (k_tc.cu).
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_plan.cuh"
#include "tc_ptx.cuh"

namespace rdm {
namespace {

constexpr int kOzSlices = 7;                          // slices per element
constexpr int kOzGroups = kOzSlices;                  // groups g = i + j = 2 .. 8
constexpr int kOzPairs = kOzSlices * (kOzSlices + 1) / 2;   // slice pairs with i + j <= 8: 28
constexpr int kOzN = 64;                              // MMA N: 2 block columns
struct GeoOz : PlanGeo<4, 2> {
    static constexpr int kPlaneElems = 32 * 32;
    static constexpr int kSliceBytes = 2 * kPlaneElems;             // one bf16 slice of a block: 2 KB
    static constexpr int kBlockBytes = kOzSlices * kSliceBytes;     // 14 KB
    static constexpr int kSideABytes = TBM * kBlockBytes;
    static constexpr int kStageBytes = kSlots * kBlockBytes;        // 84 KB
    static constexpr int kStages = 2;
    static constexpr int kSegSteps = 4;                             // K-steps per segment: 128 K
    static constexpr uint32_t kSBO = kOzSlices * 512;               // bytes between 8-row groups of a slice
};
using G = GeoOz;
constexpr int kOzEpiWarps = 8;
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;

// element (r, c), slice i of a block: the 8-row groups of the 7 slices
// alternate (512 bytes each, 3.5 KB between the groups of one slice); inside
// a group, core matrix (c / 8) at 64 elements
__device__ __forceinline__ int oz_offset(int r, int c, int i) {
    return (r >> 3) * (kOzSlices * 256) + i * 256 + ((c >> 3) << 6) + ((r & 7) << 3) + (c & 7);
}

// e_r for every row of the first `nbrows` block rows (matrix 0 of the set):
// one block row per CTA, 8 threads per row
__global__ void __launch_bounds__(256) k_oz_row_exp(const int *__restrict__ row_ptr, const double *__restrict__ val,
                                                     int nbrows, int *__restrict__ e) {
    const int i = blockIdx.x;
    if (i >= nbrows) return;
    const int r = threadIdx.x >> 3, q = threadIdx.x & 7;   // row r of the block row, columns 4q .. 4q + 3
    double mx = 0.0;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const double2 *v = reinterpret_cast<const double2 *>(val + (size_t)p * 1024 + r * 32 + 4 * q);
        const double2 v0 = v[0], v1 = v[1];
        mx = fmax(mx, fmax(fmax(fabs(v0.x), fabs(v0.y)), fmax(fabs(v1.x), fabs(v1.y))));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (q == 0) e[(size_t)i * 32 + r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
}

// The kOzSlices base-128 digits of x0 = v 2^-er (|x0| < 1: 2^er bounds the
// row), each the round-half-even of the remainder times 128, as in the
// slicing of Ozaki, Ogita, Oishi and Rump: x0 = sum_i a_i 2^(-7(i+1)) + a
// remainder below 2^-49.  Integer arithmetic, exact (FP64 throughput is low
// on this part): X = x0 2^60 is held as its floor plus a sticky bit for the
// bits below; digit i has unit 2^(53 - 7i) in X.
__device__ __forceinline__ void oz_digits(double v, int er, int (&a)[kOzSlices]) {
    const uint64_t bits = (uint64_t)__double_as_longlong(v);
    const bool neg = (bits >> 63) != 0;
    const int E = (int)((bits >> 52) & 0x7FF);
    uint64_t M = bits & ((1ull << 52) - 1);
    int ex = 1 - 1075;                                   // subnormal
    if (E != 0) {
        M |= 1ull << 52;
        ex = E - 1075;
    }
    const int sh = ex - er + 60;                         // |x0| 2^60 = M 2^sh
    int64_t X = 0;
    bool sticky = false;
    if (M != 0) {
        if (sh >= 0) {
            X = (int64_t)(M << sh);                      // sh <= 7: M 2^sh < 2^60
        } else {
            const int rs = -sh;
            const uint64_t q = rs >= 64 ? 0ull : M >> rs;
            sticky = rs >= 64 ? true : (M & ((1ull << rs) - 1)) != 0;
            X = (int64_t)q;
        }
        if (neg) X = -X - (sticky ? 1 : 0);              // the floor of the negative value
    }
#pragma unroll
    for (int i = 0; i < kOzSlices; ++i) {
        const int s = 53 - 7 * i;
        int64_t q = X >> s;                              // floor
        const int64_t r = X - (q << s);                  // in [0, 2^s); true fraction (r + sticky) / 2^s
        const int64_t half = 1ll << (s - 1);
        if (r > half || (r == half && (sticky || (q & 1)))) q += 1;
        a[i] = (int)q;
        X -= q << s;
    }
}

// slices of matrix-0 blocks: one thread per 8 consecutive elements of a block row
__global__ void k_oz_slices(const double *__restrict__ val, const int *__restrict__ row_of_blk,
                            const int *__restrict__ e, int64_t nblk, __nv_bfloat16 *__restrict__ out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nblk * 128) return;
    const int64_t p = g >> 7;
    const int rc0 = (int)(g & 127) * 8;
    const int r = rc0 >> 5, c0 = rc0 & 31;
    const int er = e[(size_t)row_of_blk[p] * 32 + r];
    const double2 *v2 = reinterpret_cast<const double2 *>(val + p * 1024 + rc0);
    uint16_t s[kOzSlices][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 x2 = v2[k];
        const double xs[2] = {x2.x, x2.y};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            int a[kOzSlices];
            oz_digits(xs[u], er, a);
#pragma unroll
            for (int i = 0; i < kOzSlices; ++i) s[i][2 * k + u] = __bfloat16_as_ushort(__float2bfloat16_rn((float)a[i]));
        }
    }
    __nv_bfloat16 *o = out + p * (kOzSlices * 1024);
#pragma unroll
    for (int i = 0; i < kOzSlices; ++i) {
        uint4 w;
        w.x = s[i][0] | ((uint32_t)s[i][1] << 16); w.y = s[i][2] | ((uint32_t)s[i][3] << 16);
        w.z = s[i][4] | ((uint32_t)s[i][5] << 16); w.w = s[i][6] | ((uint32_t)s[i][7] << 16);
        *reinterpret_cast<uint4 *>(o + oz_offset(r, c0, i)) = w;
    }
}

__global__ void k_row_of_block(const int *__restrict__ row_ptr, int nbrows, int *__restrict__ row_of) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbrows) return;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) row_of[p] = i;
}

struct OzArgs {
    const __nv_bfloat16 *slices;  // slices of matrix 0 (14 KB per block)
    const __nv_bfloat16 *zero;    // zero blocks (kSlots per CTA)
    const int *e;                 // row exponents of matrix 0 (global rows)
    const int *tiles;
    const int64_t *step_off;
    const int *steps;
    int ntile;
    uint32_t idesc;
    // epilogue
    const double *in_val;
    const int *slot_row, *slot_job, *slot_x;
    const int *mcol;
    const int *sys_of_row;
    const double *c_lin, *c_sq, *tau0, *tau1;
    int job_tau_sel[kMaxJobs];
    double *out_val;
    float *out_nrm;
    uint8_t *keep;
    const int *uidx;
    int64_t u0;
    int *err;
    long long wait_cycles;
};

struct __align__(8) OzCtl {
    uint64_t full[G::kStages], empty[G::kStages];
    uint64_t seg_full, seg_empty;
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

// x added to (hi, lo) by Knuth's TwoSum (exact sum hi + x = s + t), the
// rounding error t carried in lo
__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, t);
}

__global__ void __launch_bounds__(kOzThreads, 1) k_tc_oz(OzArgs A) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *stages = smem_raw;
    OzCtl *ctl = reinterpret_cast<OzCtl *>(smem_raw + G::kStages * G::kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort_flag = &ctl->abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::kStages; ++s) { mbar_init(&ctl->full[s], 1); mbar_init(&ctl->empty[s], 1); }
        mbar_init(&ctl->seg_full, 1);
        mbar_init(&ctl->seg_empty, kOzEpiWarps);
        mbar_init(&ctl->drain, 1);
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
        // ---------------- producer: one bulk copy of 14 KB per operand block ----------------
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
                    if (waited) mbar_expect_tx(&ctl->full[st], (uint32_t)__popc(need) * G::kBlockBytes);
                }
                waited = __shfl_sync(0xffffffffu, waited, 0);
                if (!waited) { ok = false; break; }
#pragma unroll
                for (int k = 0; k < G::kStages; ++k)
                    if (k == st) zmask[k] = zbits;
                if (!skip) {
                    const __nv_bfloat16 *src = cur >= 0 ? A.slices + (size_t)cur * (kOzSlices * 1024)
                                                        : A.zero + ((size_t)blockIdx.x * G::kSlots + lane) * (kOzSlices * 1024);
                    bulk_g2s(stages + st * G::kStageBytes + lane * G::kBlockBytes, src, G::kBlockBytes, &ctl->full[st]);
                }
            }
        }
        if (!ok && lane == 0) {
            // after an abort, wait (bounded) for the copies still in flight
            const uint32_t n = it < (uint32_t)G::kStages ? it : (uint32_t)G::kStages;
            for (uint32_t q = it - n; q < it; ++q)
                mbar_wait_drain(&ctl->full[q % G::kStages], (q / G::kStages) & 1, A.wait_cycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer: 28 slice pairs x 2 K-slices per K-step ----------------
        if (lane == 0) {
            uint32_t it = 0, seg = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < A.ntile && !*abort_flag; t += gridDim.x) {
                const int64_t s0 = A.step_off[t], s1 = A.step_off[t + 1];
                bool ok = true;
                for (int64_t q = s0; q < s1 && ok; ++seg) {
                    if (!mbar_wait(&ctl->seg_empty, (seg & 1) ^ 1, abort_flag, A.wait_cycles)) { ok = false; break; }
                    fence_after();
                    const int64_t qe = q + G::kSegSteps < s1 ? q + G::kSegSteps : s1;
                    uint32_t fresh = (1u << kOzGroups) - 1u;   // groups not yet written in this segment
                    for (; q < qe; ++q, ++it) {
                        const int st = it % G::kStages;
                        const uint32_t ph = (it / G::kStages) & 1;
                        if (!mbar_wait(&ctl->full[st], ph, abort_flag, A.wait_cycles)) { ok = false; break; }
                        fence_after();
                        const uint32_t base = smem_u32(stages + st * G::kStageBytes);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t ko = kk * 256;
#pragma unroll
                            for (int i = 0; i < kOzSlices; ++i)
#pragma unroll
                                for (int j = 0; j + i < kOzSlices; ++j) {
                                    const int grp = i + j;           // group g = (i + 1) + (j + 1), minus 2
                                    const uint32_t acc = ((fresh >> grp) & 1u) ? 0u : 1u;
                                    fresh &= ~(1u << grp);
                                    mma_f16(tmem + grp * kOzN,
                                            smem_desc(base + i * 512 + ko, 128, G::kSBO),
                                            smem_desc(base + G::kSideABytes + j * 512 + ko, 128, G::kSBO), A.idesc, acc);
                                }
                        }
                        issued = true;
                        mma_commit(&ctl->empty[st]);
                    }
                    if (ok) mma_commit(&ctl->seg_full);
                }
                if (!ok) break;
            }
            if (*abort_flag && issued) {
                mma_commit(&ctl->drain);
                long long t0 = clock64();
                while (!mbar_try_wait(&ctl->drain, 0) && clock64() - t0 < A.wait_cycles) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9, one 32 x 32 output block each ----------------
        const int eq = warp & 3;                        // TMEM lanes 32 eq .. 32 eq + 31: block row eq
        const int bc = (warp - 2) >> 2;                 // block column of the tile (accumulator columns 32 bc ..)
        uint32_t seg = 0;
        for (int t = blockIdx.x; t < A.ntile && !*abort_flag; t += gridDim.x) {
            const int *d = A.tiles + (size_t)t * G::kTileInts;
            const int s = d[4 + eq * G::TBN + bc];
            const int nst = d[3];
            if (nst < 0 && lane == 0) atomicOr(A.err, 4);
            float hi[32], lo[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
            const int nseg = nst > 0 ? (nst + G::kSegSteps - 1) / G::kSegSteps : 0;
            bool ok = true;
            for (int g = 0; g < nseg; ++g, ++seg) {
                if (!mbar_wait(&ctl->seg_full, seg & 1, abort_flag, A.wait_cycles)) { ok = false; break; }
                fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * eq) << 16) + 32 * bc;
                // the exact group sums, largest first, scaled by 2^(-7 g); the
                // buffer is released once every group has been read
#pragma unroll
                for (int grp = 0; grp < kOzGroups; ++grp) {
                    const float sc = __int_as_float((127 - 7 * (grp + 2)) << 23);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float part[16];
                        tmem_ld16(ta + grp * kOzN + 16 * h, part);
#pragma unroll
                        for (int c = 0; c < 16; ++c) ff_add(hi[16 * h + c], lo[16 * h + c], part[c] * sc);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->seg_empty);
            }
            if (!ok) break;
            if (s < 0) continue;
            // C = c_lin X + c_sq sigma_r sigma_c (hi + lo), in FP64
            const int i = A.slot_row[s];
            const int j = A.mcol[s];
            const int sys = A.sys_of_row[i];
            const int job = A.slot_job[s];
            const double cl = A.c_lin[sys], cq = A.c_sq[sys];
            const double tau = A.job_tau_sel[job] ? A.tau1[sys] : A.tau0[sys];
            const int sx = A.slot_x[s];
            const int oidx = A.uidx[s] - (int)A.u0;
            const int er = A.e[(size_t)i * 32 + lane];
            const int ec_l = A.e[(size_t)j * 32 + lane];
            const double *gx = (sx >= 0 && cl != 0.0) ? A.in_val + (size_t)sx * 1024 + lane * 32 : nullptr;
            double *o = A.out_val + (size_t)oidx * 1024 + lane * 32;
            double ss = 0.0;
#pragma unroll
            for (int c2 = 0; c2 < 32; c2 += 2) {
                double2 xo = make_double2(0.0, 0.0);
                if (gx) xo = *reinterpret_cast<const double2 *>(gx + c2);
                const int e0 = __shfl_sync(0xffffffffu, ec_l, c2);
                const int e1 = __shfl_sync(0xffffffffu, ec_l, c2 + 1);
                const double p0 = ldexp((double)hi[c2] + (double)lo[c2], er + e0);
                const double p1 = ldexp((double)hi[c2 + 1] + (double)lo[c2 + 1], er + e1);
                double2 r;
                r.x = gx ? fma(cl, xo.x, cq * p0) : cq * p0;
                r.y = gx ? fma(cl, xo.y, cq * p1) : cq * p1;
                ss = fma(r.x, r.x, fma(r.y, r.y, ss));
                *reinterpret_cast<double2 *>(o + c2) = r;
            }
#pragma unroll
            for (int w = 16; w > 0; w >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, w);
            const float nrm = __double2float_ru(sqrt(ss)) * (1.0f + 1e-6f);
            if (lane == 0) {
                A.out_nrm[s] = nrm;
                A.keep[s] = ((double)nrm >= tau) && (nrm > 0.f);
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

constexpr size_t kOzSmem = (size_t)G::kStages * G::kStageBytes + sizeof(OzCtl) + 1024;
static_assert(kOzSmem <= 227 * 1024, "shared memory of the slice-product kernel exceeds 227 KB");
static_assert(kOzGroups * kOzN <= 512, "group accumulators exceed tensor memory");

}  // namespace

void prepare_oz_operands(const MatSet &in, OzWork &w, cudaStream_t st) {
    if (in.b != 32) throw Error{-1, "the slice-product (FP64-class tensor-core) path handles 32 x 32 blocks"};
    const int NB = in.NB;
    const int64_t nblk = in.nnzb.empty() ? 0 : in.nnzb[0];   // matrix 0 only
    w.e.ensure((size_t)NB * 32);
    w.row_of.ensure(std::max<int64_t>(nblk, 1));
    w.slices.ensure(std::max<int64_t>(nblk, 1) * kOzSlices * 1024);
    if (NB == 0) return;
    // matrix 0's row_ptr entries are global block indices starting at 0
    k_oz_row_exp<<<NB, 256, 0, st>>>(in.row_ptr.p, in.val.p, NB, w.e.p);
    RDM_LAUNCH_CHECK();
    if (nblk == 0) return;
    k_row_of_block<<<(NB + 127) / 128, 128, 0, st>>>(in.row_ptr.p, NB, w.row_of.p);
    RDM_LAUNCH_CHECK();
    const int64_t n = nblk * 128;
    k_oz_slices<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in.val.p, w.row_of.p, w.e.p, nblk,
                                                             reinterpret_cast<__nv_bfloat16 *>(w.slices.p));
    RDM_LAUNCH_CHECK();
}

TcPlan build_oz_plan(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_rp, const int *mcol,
                     TcWork &w, JobMask job_mask, int unit0, int unit1, cudaStream_t st) {
    if (in.b != 32) throw Error{-1, "the slice-product (FP64-class tensor-core) path handles 32 x 32 blocks"};
    return build_plan<GeoOz>(in, jt, sd, out_rp, mcol, w, job_mask, unit0, unit1, st);
}

double launch_numeric_oz(const NumArgs &a, const MatSet &in, const int *mcol, OzWork &ow, TcWork &w,
                         const TcPlan &plan, cudaStream_t st) {
    if (plan.ntile == 0) return 0.0;
    int dev = 0, nsm = 0;
    RDM_CUDA_TRY(cudaGetDevice(&dev));
    RDM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t zero_elems = (size_t)nsm * G::kSlots * kOzSlices * 1024;
    if (!ow.zero.p || ow.zero.cap < zero_elems) {
        ow.zero.ensure(zero_elems);
        RDM_CUDA_TRY(cudaMemsetAsync(ow.zero.p, 0, ow.zero.cap * sizeof(uint16_t), st));
    }
    OzArgs A{};
    A.slices = reinterpret_cast<const __nv_bfloat16 *>(ow.slices.p);
    A.zero = reinterpret_cast<const __nv_bfloat16 *>(ow.zero.p);
    A.e = ow.e.p;
    A.tiles = w.tiles.p; A.step_off = w.step_off.p; A.steps = w.steps.p; A.ntile = plan.ntile;
    // kind::f16: D = F32, A = B = BF16, K-major, N = 64, M = 128
    A.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (((uint32_t)kOzN >> 3) << 17) | ((128u >> 4) << 24);
    A.in_val = a.in_val; A.slot_row = a.slot_row; A.slot_job = a.slot_job; A.slot_x = a.slot_x; A.mcol = mcol;
    A.sys_of_row = a.sys_of_row; A.c_lin = a.c_lin; A.c_sq = a.c_sq; A.tau0 = a.tau0; A.tau1 = a.tau1;
    for (int p = 0; p < kMaxJobs; ++p) A.job_tau_sel[p] = a.job_tau_sel[p];
    A.out_val = a.out_val; A.out_nrm = a.out_nrm; A.keep = a.keep; A.uidx = a.uidx; A.u0 = a.u0;
    A.err = w.counters.p;
    A.wait_cycles = w.knobs.wait_cycles > 0 ? w.knobs.wait_cycles : kWaitCycles;
    func_smem_once((const void *)k_tc_oz, (int)kOzSmem);
    const int grid = plan.ntile < nsm ? plan.ntile : nsm;
    k_tc_oz<<<grid, kOzThreads, kOzSmem, st>>>(A);
    RDM_LAUNCH_CHECK();
    (void)in;
    return (double)plan.nsteps * kOzPairs * 2.0 * 2.0 * 128.0 * kOzN * 16.0;
}

}  // namespace rdm
