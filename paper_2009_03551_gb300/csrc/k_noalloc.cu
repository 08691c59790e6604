// Allocation-free inner product of two block-sparse matrices.
//
// For callers that cannot call cudaMalloc — code whose device memory is owned
// by another allocator (a framework's caching pool that holds the free HBM),
// or latency-critical loops in which the implicit device synchronisation of
// cudaMalloc / cudaFree is not acceptable — this entry point computes
//     <A, B> = sum over blocks (i,j) stored in both of sum_mn A_ij[m][n] B_ij[m][n]
// (for symmetric matrices Tr(A B), the reduction behind the polarizability
// trace) with its scratch in a file-scope device array instead of allocated
// memory.  The caller passes the inputs and the output pointer.
//
// Scratch: one double per block row, at most kNoAllocMaxRows rows (2 MiB);
// every GPU that loads the library holds the array until process exit.
// Every call writes all the partial sums it reads, so nothing has to start at
// zero.  All calls share the one array: calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it and must be
// serialised by the caller.
//
// Set-up: the device address of the array is looked up (cudaGetSymbolAddress)
// once per device, with that device current, by the first call on that
// device; make that first call before any stream capture begins on the
// device.
#include <mutex>

#include "../../include/rdm.h"
#include "rdm_internal.cuh"

namespace rdm {
namespace {

constexpr int kNoAllocMaxRows = 1 << 18;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_rows[kNoAllocMaxRows];

std::mutex g_setup_mutex;
double *g_rows_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ int find_col_na(const int *col, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// one warp per block row: partial[i] = sum over the row's common blocks
__global__ void k_noalloc_rows(const int *__restrict__ arp, const int *__restrict__ acol,
                               const double *__restrict__ aval, const int *__restrict__ brp,
                               const int *__restrict__ bcol, const double *__restrict__ bval, int nb, int b,
                               double *__restrict__ partial) {
    int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (i >= nb) return;
    const int bb = b * b;
    double acc = 0.0;
    for (int q = arp[i]; q < arp[i + 1]; ++q) {
        int p = find_col_na(bcol, brp[i], brp[i + 1], acol[q]);
        if (p < 0) continue;
        const double *x = aval + (size_t)q * bb;
        const double *y = bval + (size_t)p * bb;
        for (int e = lane; e < bb; e += 32) acc += x[e] * y[e];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) partial[i] = acc;
}

// one CTA: out = sum of the nb partials, in a fixed order
__global__ void k_noalloc_sum(const double *__restrict__ partial, int nb, double *__restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

// device address of the scratch array for the current device (set-up on first use)
int scratch_for_current_device(double **ptr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RDM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_rows_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_rows);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RDM_ECUDA;
        }
        g_rows_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_rows_ptr[dev];
    return RDM_OK;
}

}  // namespace
}  // namespace rdm

extern "C" int rdm_bsr_dot_noalloc(const rdm_bsr *A, const rdm_bsr *B, double *out_device,
                                   void *cuda_stream) {
    using namespace rdm;
    if (!A || !B || !out_device) return RDM_EINVAL;
    if (!A->on_device || !B->on_device) return RDM_EINVAL;
    if (A->nb != B->nb || A->b != B->b || A->n != B->n || A->nb <= 0 || A->b <= 0 || A->b > 64)
        return RDM_EINVAL;
    if (A->nb > kNoAllocMaxRows) return RDM_EINVAL;   // beyond the scratch array
    if (!A->row_ptr || !B->row_ptr || (A->nnzb && (!A->col_idx || !A->vals)) ||
        (B->nnzb && (!B->col_idx || !B->vals)))
        return RDM_EINVAL;
    double *rows = nullptr;
    int st = scratch_for_current_device(&rows);
    if (st != RDM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int wpb = 8;
    k_noalloc_rows<<<(A->nb + wpb - 1) / wpb, wpb * 32, 0, s>>>(A->row_ptr, A->col_idx, A->vals, B->row_ptr,
                                                                 B->col_idx, B->vals, A->nb, A->b, rows);
    if (cudaGetLastError() != cudaSuccess) return RDM_ECUDA;
    k_noalloc_sum<<<1, 1024, 0, s>>>(rows, A->nb, out_device);
    if (cudaGetLastError() != cudaSuccess) return RDM_ECUDA;
    return RDM_OK;
}
