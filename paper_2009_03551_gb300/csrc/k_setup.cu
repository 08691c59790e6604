// Set-up kernels: value validation, Gershgorin bounds, initial scaling.
//
// Gershgorin bounds (Sec. 2.2: the spectrum of H0 is bracketed with
// Gershgorin's circle theorem instead of an eigen-solve):
//   r_i = sum_{j != i} |H_ij|,  eps_min = min_i (H_ii - r_i),
//   eps_max = max_i (H_ii + r_i),   over the meaningful rows of each system.
// Initial matrices (Sec. 2.2):
//   X0_0 = (eps_max I - H0) / (eps_max - eps_min),
//   X1_0 = -H1 / (eps_max - eps_min)   (same bounds as X0_0).
// Padding orbitals (rows >= n of a system) get X0 = 0: a decoupled state at
// eps_max, which stays at 0 under both purification maps.
#include "rdm_internal.cuh"

namespace rdm {
namespace {

__device__ __forceinline__ int find_col(const int *col, int lo, int hi, int key) {
    // index of key in col[lo, hi) (sorted), or -1
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// one warp per block row; lane l handles orbital rows l, l+32 of the block row
__global__ void k_gershgorin(const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ val, int NB, int b,
                             const int *__restrict__ sys_of_row, const int *__restrict__ row0,
                             const int *__restrict__ n_orb, double *row_lo, double *row_hi) {
    int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (i >= NB) return;
    int s = sys_of_row[i];
    int r_base = (i - row0[s]) * b;
    double lo = 1e300, hi = -1e300;
    for (int rr = lane; rr < b; rr += 32) {
        if (r_base + rr >= n_orb[s]) continue;
        double rad = 0.0, d = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double *blk = val + (size_t)p * b * b + (size_t)rr * b;
            bool diag = col[p] == i;
            for (int c = 0; c < b; ++c) {
                double v = blk[c];
                if (diag && c == rr) d = v; else rad += fabs(v);
            }
        }
        lo = fmin(lo, d - rad);
        hi = fmax(hi, d + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { row_lo[i] = lo; row_hi[i] = hi; }
}

__global__ void k_sys_minmax(const double *row_lo, const double *row_hi, const int *row0,
                             const int *nbs, double *emin, double *emax) {
    __shared__ double slo[32], shi[32];
    int s = blockIdx.x;
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < nbs[s]; i += blockDim.x) {
        lo = fmin(lo, row_lo[row0[s] + i]);
        hi = fmax(hi, row_hi[row0[s] + i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { slo[w] = lo; shi[w] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { lo = fmin(lo, slo[k]); hi = fmax(hi, shi[k]); }
        lo = fmin(lo, slo[0]); hi = fmax(hi, shi[0]);
        emin[s] = lo;
        emax[s] = hi;
    }
}

// one CTA per block row, one warp per block
__global__ void k_init_scale(const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ hval, double *__restrict__ xval,
                             float *__restrict__ xnrm, int NB, int b,
                             const int *__restrict__ sys_of_row, const int *__restrict__ row0,
                             const int *__restrict__ n_orb, const double *__restrict__ emin,
                             const double *__restrict__ emax, int is_x0) {
    const int r = blockIdx.x;       // row of the (multi-matrix) set
    const int i = r % NB;           // block row inside its matrix
    int s = sys_of_row[i];
    double w = emax[s] - emin[s];
    double inv_w = 1.0 / w;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int r_base = (i - row0[s]) * b;
    int n = n_orb[s];
    for (int p = rp[r] + wid; p < rp[r + 1]; p += nw) {
        int j = col[p];
        int c_base = (j - row0[s]) * b;
        const double *h = hval + (size_t)p * b * b;
        double *x = xval + (size_t)p * b * b;
        double ss = 0.0;
        for (int e = lane; e < b * b; e += 32) {
            int rr = e / b, cc = e % b;
            double v;
            if (is_x0) {
                if (r_base + rr >= n || c_base + cc >= n) v = 0.0;   // padding
                else v = ((j == i && rr == cc) ? emax[s] : 0.0) - h[e];
                v *= inv_w;
            } else {
                v = -h[e] * inv_w;
            }
            x[e] = v;
            ss += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) xnrm[p] = __double2float_ru(sqrt(ss));
    }
}

// one warp per block: FP32 upper bound of the Frobenius norm
__global__ void k_block_norms(const double *__restrict__ val, float *__restrict__ nrm, int64_t nblk,
                              int b) {
    int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (p >= nblk) return;
    const double *x = val + (size_t)p * b * b;
    double ss = 0.0;
    for (int e = lane; e < b * b; e += 32) ss += x[e] * x[e];
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) nrm[p] = __double2float_ru(sqrt(ss));
}

__global__ void k_max_abs(const double *__restrict__ val, int64_t n, unsigned long long *out) {
    double m = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double v = fabs(val[e]);
        if (v == v && v > m) m = v;   // NaN handled by the finiteness check
        if (isinf(v)) m = 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// err bits: 1 non-finite, 2 asymmetric value, 4 non-zero padding, 8 missing mirror block
__global__ void k_check_values(const int *__restrict__ rp, const int *__restrict__ col,
                               const double *__restrict__ val, int NB, int b,
                               const int *__restrict__ sys_of_row, const int *__restrict__ row0,
                               const int *__restrict__ n_orb, const unsigned long long *maxabs,
                               double rel_tol, int *err) {
    int i = blockIdx.x;
    int s = sys_of_row[i];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double tol = rel_tol * __longlong_as_double((long long)*maxabs);
    int r_base = (i - row0[s]) * b, n = n_orb[s];
    for (int p = rp[i] + wid; p < rp[i + 1]; p += nw) {
        int j = col[p];
        int q = find_col(col, rp[j], rp[j + 1], i);
        if (q < 0) { if (lane == 0) atomicOr(err, 8); continue; }
        int c_base = (j - row0[s]) * b;
        const double *a = val + (size_t)p * b * b;
        const double *t = val + (size_t)q * b * b;
        int bits = 0;
        for (int e = lane; e < b * b; e += 32) {
            int rr = e / b, cc = e % b;
            double v = a[e];
            if (!isfinite(v)) bits |= 1;
            if (fabs(v - t[cc * b + rr]) > tol) bits |= 2;
            if ((r_base + rr >= n || c_base + cc >= n) && v != 0.0) bits |= 4;
        }
        for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        if (lane == 0 && bits) atomicOr(err, bits);
    }
}

}  // namespace

void launch_gershgorin(const int *row_ptr, const int *col, const double *val, int NB, int b,
                       const int *sys_of_row, const int *row0, const int *n_orb,
                       double *row_lo, double *row_hi, cudaStream_t st) {
    int wpb = 8;
    k_gershgorin<<<(NB + wpb - 1) / wpb, wpb * 32, 0, st>>>(row_ptr, col, val, NB, b, sys_of_row,
                                                            row0, n_orb, row_lo, row_hi);
    RDM_LAUNCH_CHECK();
}

void launch_sys_minmax(const double *row_lo, const double *row_hi, const int *row0, const int *nbs,
                       int S, double *emin, double *emax, cudaStream_t st) {
    k_sys_minmax<<<S, 256, 0, st>>>(row_lo, row_hi, row0, nbs, emin, emax);
    RDM_LAUNCH_CHECK();
}

void launch_init_scale(const int *row_ptr, const int *col, const double *hval, double *xval,
                       float *xnrm, int rows, int NB, int b, const int *sys_of_row,
                       const int *row0, const int *n_orb, const double *emin,
                       const double *emax, int is_x0, cudaStream_t st) {
    if (rows == 0) return;
    k_init_scale<<<rows, 128, 0, st>>>(row_ptr, col, hval, xval, xnrm, NB, b, sys_of_row, row0,
                                       n_orb, emin, emax, is_x0);
    RDM_LAUNCH_CHECK();
}

void launch_block_norms(const double *val, float *nrm, int64_t nblk, int b, cudaStream_t st) {
    if (nblk == 0) return;
    int64_t grid = (nblk + 7) / 8;
    k_block_norms<<<(unsigned)grid, 256, 0, st>>>(val, nrm, nblk, b);
    RDM_LAUNCH_CHECK();
}

void launch_check_values(const int *row_ptr, const int *col, const double *val, int64_t nval,
                         int NB, int b, const int *sys_of_row, const int *row0, const int *n_orb,
                         double rel_tol, int *err, cudaStream_t st) {
    // err[0]: error bits; err[2..3]: 64-bit max |H| accumulator (caller zeroes err[0..3])
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(err + 2);
    if (nval > 0) {
        k_max_abs<<<1024, 256, 0, st>>>(val, nval, mx);
        RDM_LAUNCH_CHECK();
    }
    if (NB > 0) {
        k_check_values<<<NB, 128, 0, st>>>(row_ptr, col, val, NB, b, sys_of_row, row0, n_orb, mx,
                                          rel_tol, err);
        RDM_LAUNCH_CHECK();
    }
}

}  // namespace rdm
