// Element-wise kernels of the non-orthogonal-basis transform (Sec. 2.2):
// per-system scaling of a block-sparse matrix (with the padding diagonal set
// to one, so that padding rows stay decoupled and invertible), and identity
// blocks.  The products of the transform run in the numeric kernels.
#include "rdm_internal.cuh"

namespace rdm {
namespace {

// out = fac[sys] * val over block row i (one CTA per block row); with
// pad_one, diagonal elements of padding rows (orbital index >= n_orb) are 1
__global__ void k_scale_sys(const int *__restrict__ row_ptr, const int *__restrict__ col,
                            const double *__restrict__ val, int NB, int b, const int *__restrict__ sys_of_row,
                            const int *__restrict__ row0, const int *__restrict__ n_orb,
                            const double *__restrict__ fac, int pad_one, double *__restrict__ out) {
    const int i = blockIdx.x;
    if (i >= NB) return;
    const int sys = sys_of_row[i];
    const double f = fac[sys];
    const int bb = b * b;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const bool diag = col[p] == i;
        for (int e = threadIdx.x; e < bb; e += blockDim.x) {
            const int r = e / b, c = e % b;
            double v = f * val[(size_t)p * bb + e];
            if (pad_one && diag && r == c && (i - row0[sys]) * b + r >= n_orb[sys]) v = 1.0;
            out[(size_t)p * bb + e] = v;
        }
    }
}

// identity blocks: every stored block of a diagonal-only pattern
__global__ void k_identity_blocks(double *__restrict__ val, int64_t nblk, int b) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t bb = (int64_t)b * b;
    if (e >= nblk * bb) return;
    const int rc = (int)(e % bb);
    val[e] = (rc / b == rc % b) ? 1.0 : 0.0;
}

}  // namespace

void launch_scale_sys(const int *row_ptr, const int *col, const double *val, int NB, int b, const int *sys_of_row,
                      const int *row0, const int *n_orb, const double *fac, int pad_one, double *out,
                      cudaStream_t st) {
    if (NB == 0) return;
    k_scale_sys<<<NB, 256, 0, st>>>(row_ptr, col, val, NB, b, sys_of_row, row0, n_orb, fac, pad_one, out);
    RDM_LAUNCH_CHECK();
}

void launch_identity_blocks(double *val, int64_t nblk, int b, cudaStream_t st) {
    const int64_t n = nblk * (int64_t)b * b;
    if (n == 0) return;
    k_identity_blocks<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(val, nblk, b);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
