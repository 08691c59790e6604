// Reductions in FP64: the trace test of Eq. TC2, the idempotency error, the
// band energies of the stopping rule (Sec. 2.2: E0 = Tr(P0 H0),
// E1 = Tr(P1 H0)), and the polarizability trace (Eq. polar).
//
// Every reduction is two-stage and deterministic: one warp per block row
// writes per-row partial sums (warp-shuffle reduction inside the row), then
// one CTA per (system, quantity) adds the rows in a fixed order.  The branch
// decision therefore never depends on atomic ordering.
#include "rdm_internal.cuh"

namespace rdm {
namespace {

__device__ __forceinline__ int find_col(const int *col, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// row_part layout: [q][NB], q = 0 trace, 1 sumsq, 2 E0, 3+m-1 E1 of matrix m.
// One CTA per block row, warps over blocks, lanes over elements; the warp
// partials are added in a fixed order.  Tr X0 and ||X0||_F^2 run over the
// blocks of X0; the band energies Tr(X H0) only over the blocks of H0 (where
// H0 is zero they get no contribution), each looking up the matching block of
// X by binary search.
constexpr int kStatWarps = 8;
constexpr int kStatQ = 3 + 7;    // up to 7 first-order matrices

__global__ void __launch_bounds__(kStatWarps * 32) k_row_stats(
    const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val, int nmat, int NB, int b,
    const int *__restrict__ hrp, const int *__restrict__ hcol, const double *__restrict__ hval,
    double *__restrict__ row_part) {
    __shared__ double sh[kStatWarps][kStatQ];
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int bb = b * b;
    double q[kStatQ];
#pragma unroll
    for (int k = 0; k < kStatQ; ++k) q[k] = 0.0;
    // trace and squared norm of X0
    for (int p = rp[i] + wid; p < rp[i + 1]; p += kStatWarps) {
        const double *x = val + (size_t)p * bb;
        const bool dg = col[p] == i;
        for (int e = lane; e < bb; e += 32) {
            const double v = x[e];
            q[1] = fma(v, v, q[1]);
            if (dg && (e / b) == (e % b)) q[0] += v;
        }
    }
    // band energies over the pattern of H0
    for (int ph = hrp[i] + wid; ph < hrp[i + 1]; ph += kStatWarps) {
        const int j = hcol[ph];
        const double *h = hval + (size_t)ph * bb;
        for (int m = 0; m < nmat; ++m) {
            const int *rpm = rp + (size_t)m * NB;
            const int p = find_col(col, rpm[i], rpm[i + 1], j);
            if (p < 0) continue;
            const double *x = val + (size_t)p * bb;
            double eb = 0.0;
            for (int e = lane; e < bb; e += 32) eb = fma(x[e], h[e], eb);
            q[2 + m] += eb;
        }
    }
#pragma unroll
    for (int k = 0; k < kStatQ; ++k) {
        const double v = warp_sum(q[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 + nmat) {
        const int k = threadIdx.x;
        double t = 0.0;
        for (int w = 0; w < kStatWarps; ++w) t += sh[w][k];
        row_part[(size_t)k * NB + i] = t;
    }
}

// <P_d, H_g> summed over the blocks present in both, per row:
// row_part[(g*np + d)][NB]
__global__ void k_row_dots(const int *__restrict__ prp, const int *__restrict__ pcol,
                           const double *__restrict__ pval, int np,
                           const int *__restrict__ hrp, const int *__restrict__ hcol,
                           const double *__restrict__ hval, int nh, int NB, int b,
                           double *__restrict__ row_part) {
    int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (i >= NB) return;
    const int bb = b * b;
    for (int g = 0; g < nh; ++g) {
        const int *hr = hrp + (size_t)g * NB;
        for (int d = 0; d < np; ++d) {
            const int *pr = prp + (size_t)d * NB;
            double acc = 0.0;
            for (int q = hr[i]; q < hr[i + 1]; ++q) {
                int p = find_col(pcol, pr[i], pr[i + 1], hcol[q]);
                if (p < 0) continue;
                const double *x = pval + (size_t)p * bb;
                const double *h = hval + (size_t)q * bb;
                for (int e = lane; e < bb; e += 32) acc += x[e] * h[e];
            }
            acc = warp_sum(acc);
            if (lane == 0) row_part[(size_t)(g * np + d) * NB + i] = acc;
        }
    }
}

// out[s*nq + q] = sum_{i in system s} row_part[q][i], fixed order
__global__ void k_sys_sum(const double *__restrict__ row_part, int nq, int NB,
                          const int *__restrict__ row0, const int *__restrict__ nbs,
                          double *__restrict__ out) {
    __shared__ double sh[32];
    int s = blockIdx.x, q = blockIdx.y;
    const double *r = row_part + (size_t)q * NB + row0[s];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nbs[s]; i += blockDim.x) acc += r[i];
    acc = warp_sum(acc);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (w == 0) {
        double v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) out[(size_t)s * nq + q] = v;
    }
}

}  // namespace

void launch_row_stats(const int *row_ptr, const int *col, const double *val, int nmat, int NB,
                      int b, const int *h_row_ptr, const int *h_col, const double *h_val,
                      double *row_part, cudaStream_t st) {
    if (NB == 0) return;
    if (nmat > kStatQ - 2) throw Error{-1, "at most 7 first-order matrices"};
    k_row_stats<<<NB, kStatWarps * 32, 0, st>>>(row_ptr, col, val, nmat, NB, b, h_row_ptr, h_col, h_val,
                                                row_part);
    RDM_LAUNCH_CHECK();
}

void launch_row_dots(const int *p_row_ptr, const int *p_col, const double *p_val, int np,
                     const int *h_row_ptr, const int *h_col, const double *h_val, int nh,
                     int NB, int b, double *row_part, cudaStream_t st) {
    if (NB == 0 || np == 0 || nh == 0) return;
    int wpb = 8;
    k_row_dots<<<(NB + wpb - 1) / wpb, wpb * 32, 0, st>>>(p_row_ptr, p_col, p_val, np, h_row_ptr,
                                                          h_col, h_val, nh, NB, b, row_part);
    RDM_LAUNCH_CHECK();
}

void launch_sys_sum(const double *row_part, int nq, int NB, const int *row0, const int *nbs,
                    int S, double *out, cudaStream_t st) {
    if (S == 0 || nq == 0) return;
    k_sys_sum<<<dim3(S, nq), 256, 0, st>>>(row_part, nq, NB, row0, nbs, out);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
