// Numeric phase on the CUDA cores (FP64 and FP32 operands), with the update
// and truncation of Eqs. TC2 / TC2-CPSCF fused into the epilogue:
//
//   C_ij = c_lin X_ij + c_sq sum_{(a,b) in pairs(i,j)} A_a (B_b)^T
//
// for every upper-triangle output block (j >= i); the lower block (j,i) is
// written as the transpose, so the result is exactly symmetric.  Diagonal
// blocks are symmetrised ((C + C^T)/2) because the accumulation order of
// C_mn and C_nm differs.  The block Frobenius norm is reduced in FP64 and the
// block is kept iff norm >= tau (the block-wise "filter" of Sec. 2.3).
//
// One CTA per output block (grid-stride over the work list); the two
// operand blocks of each pair are staged in shared memory, each thread owns
// ceil(b^2 / threads) outputs.  On GB300 the FP64 rate is the bound of this
// kernel; the FP32 variant converts the FP64 master values on load.
#include "rdm_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace rdm {
namespace {

template <int B>
struct Cfg {
    static constexpr int NT = (B * B >= 256) ? 256 : ((B * B < 32) ? 32 : B * B);
    static constexpr int PER = (B * B + NT - 1) / NT;
    static constexpr int LD = B + 1;
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;
}

template <int B, class T>
__global__ void __launch_bounds__(Cfg<B>::NT) k_numeric_simt(NumArgs a) {
    constexpr int NT = Cfg<B>::NT, PER = Cfg<B>::PER, LD = Cfg<B>::LD, BB = B * B;
    extern __shared__ double smem_d[];
    T *As = reinterpret_cast<T *>(smem_d);
    T *Bs = As + B * LD;
    double *Cs = smem_d;                    // reused for the epilogue (B*LD doubles)
    __shared__ double red[32];
    const int tid = threadIdx.x;

    __shared__ int s_w;
    for (;;) {
        // work items are handed out in list order by an atomic counter, so the
        // blocks in flight stay close in the list and share operands in L2
        if (threadIdx.x == 0) s_w = atomicAdd(a.work_next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= a.nwork) break;
        const int s = a.work[w];
        const int i = a.slot_row[s];
        const int sys = a.sys_of_row[i];
        const int job = a.slot_job[s];
        const double cl = a.c_lin[sys], cq = a.c_sq[sys];
        const double tau = a.job_tau_sel[job] ? a.tau1[sys] : a.tau0[sys];
        const int64_t p0 = a.pair_off[s], p1 = a.pair_off[s + 1];
        const int st = a.slot_t[s], sx = a.slot_x[s];

        T acc[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) acc[r] = T(0);

        for (int64_t q = p0; q < p1; ++q) {
            const double *ga = a.in_val + (size_t)a.pair_a[q] * BB;
            const double *gb = a.in_val + (size_t)a.pair_b[q] * BB;
            __syncthreads();
            for (int e = tid; e < BB; e += NT) {
                As[(e / B) * LD + (e % B)] = (T)ga[e];
                Bs[(e / B) * LD + (e % B)] = (T)gb[e];
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int e = tid + r * NT;
                if (e < BB) {
                    const int m = e / B, n = e % B;
                    const T *ar = As + m * LD;
                    const T *br = Bs + n * LD;
                    T sacc = acc[r];
#pragma unroll 8
                    for (int kk = 0; kk < B; ++kk) sacc = fma(ar[kk], br[kk], sacc);
                    acc[r] = sacc;
                }
            }
        }

        // epilogue: linear term, symmetrisation, norm, truncation (the lower
        // triangle is written by the compaction, as the transpose)
        double out[PER];
        const double *gx = sx >= 0 ? a.in_val + (size_t)sx * BB : nullptr;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * NT;
            if (e < BB) {
                double v = cq * (double)acc[r];
                if (gx) v = fma(cl, gx[e], v);
                out[r] = v;
                Cs[(e / B) * LD + (e % B)] = v;
            }
        }
        __syncthreads();
        const bool diag = (st == s);
        double ss = 0.0;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * NT;
            if (e < BB) {
                if (diag) {
                    const int m = e / B, n = e % B;
                    out[r] = 0.5 * (Cs[m * LD + n] + Cs[n * LD + m]);
                }
                ss += out[r] * out[r];
            }
        }
        const double nrm = sqrt(block_sum(ss, red));
        const bool keep = (nrm >= tau) && (nrm > 0.0);
        double *o = a.out_val + (size_t)(a.uidx[s] - a.u0) * BB;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * NT;
            if (e < BB) o[e] = out[r];
        }
        if (tid == 0) {
            a.out_nrm[s] = __double2float_ru(nrm);
            a.keep[s] = keep;
        }
    }
}

// ---------------------------------------------------------------------------
// Double-FP32 products of 32 x 32 blocks: 64 threads per output block, each a
// 4 x 4 register tile at rows r0 + 8i and columns c0 + 8j (r0 = t/8,
// c0 = t%8), so that the 16-byte shared-memory reads of a quarter warp hit 8
// different banks (B rows) or broadcast (A rows).  Operand blocks come from
// the FP32 (hi, lo) copies of the master values, double-buffered with
// cp.async.
// ---------------------------------------------------------------------------
constexpr int kF32Ld = 36;   // padded row stride in floats (144 B, 16-byte aligned)

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Double-FP32 ("float-float") products of the FP64 masters split as
// x = hi + lo (two FP32 planes): the
// hi*hi products are accumulated without rounding loss by the error-free
// transformations of Ogita, Rump and Oishi (2005) -- the exact product
// p + e = hi_a hi_b from one multiply and one fused multiply-add, the exact
// sum s + t = acc + p from six additions -- and the small cross terms hi*lo
// and lo*hi are added in plain FP32 into the low word.  The result carries
// about 46 bits, enough for FP64-class refinement of X0^2, on the FP32 pipe.
__global__ void __launch_bounds__(64) k_numeric_ff_b32(NumArgs a) {
    constexpr int NP = 2;                          // operand planes (hi, lo)
    __shared__ __align__(16) float sA[2][NP][32 * kF32Ld];
    __shared__ __align__(16) float sB[2][NP][32 * kF32Ld];
    __shared__ double sC[32 * 33];
    __shared__ float red[2];
    const int tid = threadIdx.x;
    const int r0 = tid >> 3, c0 = tid & 7;
    const float *planes[2] = {a.in_f32, a.in_f32lo};

    __shared__ int s_w;
    for (;;) {
        // work items are handed out in list order by an atomic counter, so the
        // blocks in flight stay close in the list and share operands in L2
        if (threadIdx.x == 0) s_w = atomicAdd(a.work_next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= a.nwork) break;
        const int s = a.work[w];
        const int i = a.slot_row[s];
        const int sys = a.sys_of_row[i];
        const int job = a.slot_job[s];
        const double tau = a.job_tau_sel[job] ? a.tau1[sys] : a.tau0[sys];
        const int64_t p0 = a.pair_off[s], p1 = a.pair_off[s + 1];
        const int st = a.slot_t[s], sx = a.slot_x[s];

        float acc[4][4], accl[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = accl[u][v] = 0.f;

        auto issue = [&](int64_t q, int buf) {
#pragma unroll
            for (int pl = 0; pl < NP; ++pl) {
                const float *ga = planes[pl] + (size_t)a.pair_a[q] * 1024;
                const float *gb = planes[pl] + (size_t)a.pair_b[q] * 1024;
#pragma unroll
                for (int c = tid; c < 256; c += 64) {
                    const int row = c >> 3, col4 = (c & 7) * 4;
                    cp_async16(&sA[buf][pl][row * kF32Ld + col4], ga + row * 32 + col4);
                    cp_async16(&sB[buf][pl][row * kF32Ld + col4], gb + row * 32 + col4);
                }
            }
            cp_async_commit();
        };
        __syncthreads();
        if (p0 < p1) issue(p0, 0);
        for (int64_t q = p0; q < p1; ++q) {
            const int buf = (int)((q - p0) & 1);
            if (q + 1 < p1) {
                issue(q + 1, buf ^ 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncthreads();
            const float *A_ = sA[buf][0];
            const float *B_ = sB[buf][0];
            // the double-FP32 body is large: not unrolled over kk, so that the
            // loop stays in the instruction cache
#pragma unroll 1
            for (int kk = 0; kk < 32; kk += 4) {
                float4 av[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) av[u] = *reinterpret_cast<const float4 *>(&A_[(r0 + 8 * u) * kF32Ld + kk]);
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = *reinterpret_cast<const float4 *>(&B_[(c0 + 8 * v) * kF32Ld + kk]);
                {
                    const float *Al = sA[buf][NP - 1];
                    const float *Bl = sB[buf][NP - 1];
                    float4 al[4], bl[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) al[u] = *reinterpret_cast<const float4 *>(&Al[(r0 + 8 * u) * kF32Ld + kk]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) bl[v] = *reinterpret_cast<const float4 *>(&Bl[(c0 + 8 * v) * kF32Ld + kk]);
                    // k outermost: the 16 accumulator chains of the thread are
                    // independent, so consecutive operations do not wait on each other
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float ah = k == 0 ? av[u].x : k == 1 ? av[u].y : k == 2 ? av[u].z : av[u].w;
                            const float alo = k == 0 ? al[u].x : k == 1 ? al[u].y : k == 2 ? al[u].z : al[u].w;
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                const float bh = k == 0 ? bv[v].x : k == 1 ? bv[v].y : k == 2 ? bv[v].z : bv[v].w;
                                const float blo = k == 0 ? bl[v].x : k == 1 ? bl[v].y : k == 2 ? bl[v].z : bl[v].w;
                                const float sh = acc[u][v];
                                const float p = __fmul_rn(ah, bh);
                                const float e = fmaf(ah, bh, -p);                // p + e = ah bh exactly
                                const float sn = __fadd_rn(sh, p);
                                const float z = __fsub_rn(sn, sh);
                                const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, z)), __fsub_rn(p, z));   // sn + t = sh + p
                                acc[u][v] = sn;
                                float sl = accl[u][v];
                                sl = fmaf(ah, blo, sl);
                                sl = fmaf(alo, bh, sl);
                                accl[u][v] = __fadd_rn(sl, __fadd_rn(t, e));
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }

        // epilogue: C = c_lin X + c_sq acc in FP64, symmetrised on the
        // diagonal, norm, truncation
        const double *gx = sx >= 0 ? a.in_val + (size_t)sx * 1024 : nullptr;
        const bool diag = (st == s);
        const double cl = a.c_lin[sys], cq = a.c_sq[sys];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = r0 + 8 * u, c = c0 + 8 * v;
                double x = cq * ((double)acc[u][v] + (double)accl[u][v]);
                if (gx) x = fma(cl, gx[r * 32 + c], x);
                sC[r * 33 + c] = x;
            }
        __syncthreads();
        float ss = 0.f;
        if (diag) {
            double sym[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = r0 + 8 * u, c = c0 + 8 * v;
                    sym[u][v] = 0.5 * (sC[r * 33 + c] + sC[c * 33 + r]);
                }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) sC[(r0 + 8 * u) * 33 + c0 + 8 * v] = sym[u][v];
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float x = (float)sC[(r0 + 8 * u) * 33 + c0 + 8 * v];
                ss = fmaf(x, x, ss);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if ((tid & 31) == 0) red[tid >> 5] = ss;
        __syncthreads();
        const float nrm = sqrtf(red[0] + red[1]) * (1.0f + 1e-6f);
        const bool keep = ((double)nrm >= tau) && (nrm > 0.f);
        double *o = a.out_val + (size_t)(a.uidx[s] - a.u0) * 1024;
        for (int e = tid; e < 1024; e += 64) o[e] = (double)sC[(e >> 5) * 33 + (e & 31)];
        if (tid == 0) {
            a.out_nrm[s] = nrm;
            a.keep[s] = keep;
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 products of 32 x 32 blocks with 8 x 4 register tiles.  A 4 x 4 tile
// (the layout of k_numeric_ff_b32) reads 2 bytes of shared memory per FMA, and a warp's 16-byte read takes four
// shared-memory cycles whatever it broadcasts, so the operand reads allow
// about half of the SM's FMA rate (ncu on the 4 x 4 version: FMA pipe 54%,
// short-scoreboard stalls first).  Here half-warp h of the CTA's four covers
// the k-half kh = h % 2 (k = 16 kh .. 16 kh + 15 of every pair) and the
// column half ch = h / 2, lane l of it rows r0 + 4u (u = 0..7) and columns
// 16 ch + c0 + 4v (v = 0..3), r0 = l / 4, c0 = l % 4: 12 reads of 16 bytes per
// 128 FMAs (1.5 bytes per FMA) within 128 registers, so that eight CTAs
// share an SM (44.5 against 41.6 TFLOP/s for the 4 x 4 version; an 8 x 8
// tile at 222 registers, four CTAs per SM, gained nothing).  A quarter warp reads two A rows (broadcast) and four B rows,
// in distinct banks.  The two k-halves are added in a fixed order at the end.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64, 8) k_numeric_f32_t84(NumArgs a) {
    __shared__ __align__(16) float sA[2][32 * kF32Ld];
    __shared__ __align__(16) float sB[2][32 * kF32Ld];
    __shared__ float sC[32 * 33];
    __shared__ float red[2];
    __shared__ int s_w;
    const int tid = threadIdx.x;
    const int hw = tid >> 4, l = tid & 15;
    const int kh = hw & 1, ch = hw >> 1;
    const int r0 = l >> 2, c0 = 16 * ch + (l & 3);
    const int k0 = 16 * kh;
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(a.work_next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= a.nwork) break;
        const int s = a.work[w];
        const int i = a.slot_row[s];
        const int sys = a.sys_of_row[i];
        const int job = a.slot_job[s];
        const double tau = a.job_tau_sel[job] ? a.tau1[sys] : a.tau0[sys];
        const int64_t p0 = a.pair_off[s], p1 = a.pair_off[s + 1];
        const int st = a.slot_t[s], sx = a.slot_x[s];

        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;

        auto issue = [&](int64_t q, int buf) {
            const float *ga = a.in_f32 + (size_t)a.pair_a[q] * 1024;
            const float *gb = a.in_f32 + (size_t)a.pair_b[q] * 1024;
#pragma unroll
            for (int c = tid; c < 256; c += 64) {
                const int row = c >> 3, col4 = (c & 7) * 4;
                cp_async16(&sA[buf][row * kF32Ld + col4], ga + row * 32 + col4);
                cp_async16(&sB[buf][row * kF32Ld + col4], gb + row * 32 + col4);
            }
            cp_async_commit();
        };
        __syncthreads();
        if (p0 < p1) issue(p0, 0);
        for (int64_t q = p0; q < p1; ++q) {
            const int buf = (int)((q - p0) & 1);
            if (q + 1 < p1) {
                issue(q + 1, buf ^ 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncthreads();
            const float *A_ = sA[buf];
            const float *B_ = sB[buf];
#pragma unroll
            for (int kk = 0; kk < 16; kk += 4) {
                float4 av[8], bv[4];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    av[u] = *reinterpret_cast<const float4 *>(&A_[(r0 + 4 * u) * kF32Ld + k0 + kk]);
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    bv[v] = *reinterpret_cast<const float4 *>(&B_[(c0 + 4 * v) * kF32Ld + k0 + kk]);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float t = acc[u][v];
                        t = fmaf(av[u].x, bv[v].x, t);
                        t = fmaf(av[u].y, bv[v].y, t);
                        t = fmaf(av[u].z, bv[v].z, t);
                        t = fmaf(av[u].w, bv[v].w, t);
                        acc[u][v] = t;
                    }
            }
            __syncthreads();
        }

        // the two k-halves' partial blocks into the free operand buffers, then
        // C = c_lin X + c_sq (P_0 + P_1)
        float *part = sA[kh];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) part[(r0 + 4 * u) * kF32Ld + c0 + 4 * v] = acc[u][v];
        __syncthreads();
        const double *gx = sx >= 0 ? a.in_val + (size_t)sx * 1024 : nullptr;
        const bool diag = (st == s);
        const float cl = (float)a.c_lin[sys], cq = (float)a.c_sq[sys];
        for (int e = tid; e < 1024; e += 64) {
            const int r = e >> 5, c = e & 31, o = r * kF32Ld + c;
            float x = cq * (sA[0][o] + sA[1][o]);
            if (gx) x = fmaf(cl, (float)gx[e], x);
            sC[r * 33 + c] = x;
        }
        __syncthreads();
        float sym[16];
        if (diag) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int e = tid + 64 * t, r = e >> 5, c = e & 31;
                sym[t] = 0.5f * (sC[r * 33 + c] + sC[c * 33 + r]);
            }
        }
        __syncthreads();
        float ss = 0.f;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 64 * t, r = e >> 5, c = e & 31;
            if (diag) sC[r * 33 + c] = sym[t];
            const float x = diag ? sym[t] : sC[r * 33 + c];
            ss = fmaf(x, x, ss);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if ((tid & 31) == 0) red[tid >> 5] = ss;
        __syncthreads();
        const float nrm = sqrtf(red[0] + red[1]) * (1.0f + 1e-6f);
        const bool keep = ((double)nrm >= tau) && (nrm > 0.f);
        double *o = a.out_val + (size_t)(a.uidx[s] - a.u0) * 1024;
        for (int e = tid; e < 1024; e += 64) o[e] = (double)sC[(e >> 5) * 33 + (e & 31)];
        if (tid == 0) {
            a.out_nrm[s] = nrm;
            a.keep[s] = keep;
        }
    }
}

// FP64 masters -> FP32 hi plane and (optionally) FP32 lo plane, x = hi + lo
__global__ void k_split_f32(const double *__restrict__ v, float *__restrict__ hi, float *__restrict__ lo, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double x = v[e];
    const float h = (float)x;
    hi[e] = h;
    if (lo) lo[e] = (float)(x - (double)h);
}


template <int B, class T>
void launch_b(const NumArgs &a, cudaStream_t st) {
    constexpr int NT = Cfg<B>::NT, LD = Cfg<B>::LD;
    size_t smem = (size_t)B * LD * sizeof(double);
    size_t ab = 2 * (size_t)B * LD * sizeof(T);
    if (ab > smem) smem = ab;
    func_smem_once((const void *)k_numeric_simt<B, T>, (int)smem);
    static int resident = 0;
    if (!resident) {
        int per_sm = 0, dev = 0, nsm = 0;
        RDM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_simt<B, T>, NT, smem));
        RDM_CUDA_TRY(cudaGetDevice(&dev));
        RDM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        resident = std::max(1, per_sm) * nsm;
    }
    const int grid = a.nwork < resident ? a.nwork : resident;
    if (grid <= 0) return;
    k_numeric_simt<B, T><<<grid, NT, smem, st>>>(a);
    RDM_LAUNCH_CHECK();
}

template <class T>
void dispatch(const NumArgs &a, cudaStream_t st) {
    switch (a.b) {
        case 1: launch_b<1, T>(a, st); break;
        case 2: launch_b<2, T>(a, st); break;
        case 4: launch_b<4, T>(a, st); break;
        case 8: launch_b<8, T>(a, st); break;
        case 16: launch_b<16, T>(a, st); break;
        case 32: launch_b<32, T>(a, st); break;
        case 64: launch_b<64, T>(a, st); break;
        default: throw Error{-1, "block size must be 1, 2, 4, 8, 16, 32 or 64"};
    }
}

// blocks of kernel k (threads per block nt, static shared memory) resident on the whole GPU
template <class K>
int resident_blocks(K k, int nt) {
    int per_sm = 0, dev = 0, nsm = 0;
    RDM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, 0));
    RDM_CUDA_TRY(cudaGetDevice(&dev));
    RDM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, per_sm) * nsm;
}

}  // namespace

void launch_numeric_simt(const NumArgs &a, Arith ar, cudaStream_t st) {
    if (a.nwork == 0) return;
    if (ar == AR_FF) {
        if (a.b != 32 || !a.in_f32 || !a.in_f32lo) throw Error{-1, "double-FP32 products need 32 x 32 blocks"};
        static const int res = resident_blocks(k_numeric_ff_b32, 64);
        k_numeric_ff_b32<<<std::min(a.nwork, res), 64, 0, st>>>(a);
        RDM_LAUNCH_CHECK();
    } else if (ar == AR_FP64) {
        dispatch<double>(a, st);
    } else if (a.b == 32 && a.in_f32) {
        static const int res = resident_blocks(k_numeric_f32_t84, 64);
        k_numeric_f32_t84<<<std::min(a.nwork, res), 64, 0, st>>>(a);
        RDM_LAUNCH_CHECK();
    } else {
        dispatch<float>(a, st);
    }
}

void launch_to_f32(const double *val, float *f32, int64_t n, cudaStream_t st, float *f32lo) {
    if (n == 0) return;
    k_split_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(val, f32, f32lo, n);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
