// Change of block size of a block-sparse matrix: the same n x n matrix stored
// in b_out x b_out blocks instead of b_in x b_in ones (b_in, b_out powers of
// two).  The solve can then run its products at another block size than the
// caller's (16, 32 or 64 on the tensor cores, chosen by the autotuner), and
// the results go back to the caller's layout.
//
// Pattern (host): an output block exists where some stored input block
// overlaps it, so merging (b_out > b_in) keeps every stored element and
// splitting (b_out < b_in) keeps every sub-block of a stored block, zero or
// not.  Values (device): one thread per output element reads its element from
// the input block that holds it (binary search in the input row), or 0.
#include <algorithm>

#include "rdm_internal.cuh"

namespace rdm {
namespace {

__global__ void k_reblock_vals(const int *__restrict__ in_rp, const int *__restrict__ in_col,
                               const double *__restrict__ in_val, int nb_in, int b_in,
                               const int *__restrict__ out_row, const int *__restrict__ out_col,
                               double *__restrict__ out_val, int64_t nout, int b_out) {
    const int64_t bb = (int64_t)b_out * b_out;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nout * bb) return;
    const int64_t p = e / bb;
    const int rc = (int)(e - p * bb);
    const int64_t gi = (int64_t)out_row[p] * b_out + rc / b_out;
    const int64_t gj = (int64_t)out_col[p] * b_out + rc % b_out;
    const int i = (int)(gi / b_in), j = (int)(gj / b_in);
    double v = 0.0;
    if (i < nb_in && j < nb_in) {
        int lo = in_rp[i], hi = in_rp[i + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (in_col[mid] < j) lo = mid + 1; else hi = mid;
        }
        if (lo < in_rp[i + 1] && in_col[lo] == j)
            v = in_val[(int64_t)lo * b_in * b_in + (gi - (int64_t)i * b_in) * b_in + (gj - (int64_t)j * b_in)];
    }
    out_val[e] = v;
}

}  // namespace

void reblock_pattern(const std::vector<int> &rp, const std::vector<int> &col, int b_in, int n, int b_out,
                     std::vector<int> &rp_out, std::vector<int> &col_out) {
    const int nb_in = (int)rp.size() - 1;
    const int nb_out = (n + b_out - 1) / b_out;
    std::vector<std::vector<int>> rows(nb_out);
    for (int i = 0; i < nb_in; ++i) {
        const int64_t r0 = (int64_t)i * b_in / b_out;
        const int64_t r1 = std::min<int64_t>(((int64_t)(i + 1) * b_in - 1) / b_out, nb_out - 1);
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int j = col[p];
            const int64_t c0 = (int64_t)j * b_in / b_out;
            const int64_t c1 = std::min<int64_t>(((int64_t)(j + 1) * b_in - 1) / b_out, nb_out - 1);
            for (int64_t r = r0; r <= r1; ++r)
                for (int64_t c = c0; c <= c1; ++c) rows[r].push_back((int)c);
        }
    }
    rp_out.assign(nb_out + 1, 0);
    col_out.clear();
    for (int r = 0; r < nb_out; ++r) {
        auto &v = rows[r];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        col_out.insert(col_out.end(), v.begin(), v.end());
        rp_out[r + 1] = (int)col_out.size();
    }
}

void launch_reblock_vals(const int *in_rp, const int *in_col, const double *in_val, int nb_in, int b_in,
                         const int *out_row, const int *out_col, double *out_val, int64_t nout, int b_out,
                         cudaStream_t st) {
    const int64_t n = nout * (int64_t)b_out * b_out;
    if (n == 0) return;
    k_reblock_vals<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in_rp, in_col, in_val, nb_in, b_in, out_row,
                                                                 out_col, out_val, nout, b_out);
    RDM_LAUNCH_CHECK();
}

}  // namespace rdm
