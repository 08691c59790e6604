// Internal declarations of the GB300 response-density-matrix library.
//
// Data model
// ----------
// A batch of independent systems is stored as ONE block-diagonal block-sparse
// matrix over NB = sum_s nb_s block rows; system s owns block rows (and block
// columns) [row0[s], row0[s] + nb[s]).  All systems share the block size b.
//
// A MatSet holds nmat such matrices over the same block-row space, in one set
// of arrays: blocks of matrix m occupy global block indices
// [row_ptr[m*NB], row_ptr[m*NB+NB]) (row_ptr has nmat*NB+1 entries, so row i
// of matrix m is [row_ptr[m*NB+i], row_ptr[m*NB+i+1])).  row_ptr entries are global
// block indices; col_idx holds global block columns (sorted inside a row);
// val holds b*b FP64 values per block (row-major); nrm holds an FP32 upper
// bound of every block's Frobenius norm.  In the solve, matrix 0 is X0 and
// matrices 1..nd are X1_gamma.  Patterns of every matrix are symmetric and
// values are symmetric (block (j,i) is the transpose of block (i,j)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <string>
#include <utility>
#include <vector>

namespace rdm {

// ---------------------------------------------------------------------------
// error handling inside the library (converted to status codes at the ABI)
// ---------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

#define RDM_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess)                                                    \
            throw ::rdm::Error{_e == cudaErrorMemoryAllocation ? -3 : -4,         \
                               std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

// every kernel launch of the library goes through RDM_LAUNCH_CHECK, which
// also counts it (the count is reported per solve in rdm_info)
extern thread_local long long g_kernel_launches;   // launches of this thread (a solve runs on one thread)
#define RDM_LAUNCH_CHECK()                      \
    do {                                        \
        ++::rdm::g_kernel_launches;             \
        RDM_CUDA_TRY(cudaGetLastError());       \
    } while (0)

// cudaFuncAttributeMaxDynamicSharedMemorySize of kernel `func`, set once per
// kernel and device (the attribute is per device; handles of one process may
// use several, and solves may run on worker threads)
void func_smem_once(const void *func, int bytes);

// device bytes held by all DevBufs of the process (current and high-water mark)
inline std::atomic<size_t> g_dev_bytes{0};
inline std::atomic<size_t> g_dev_bytes_peak{0};

inline void *dev_alloc(size_t bytes) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{-3, "cudaMalloc of " + std::to_string(bytes) + " bytes failed (" +
                            std::to_string(g_dev_bytes.load()) + " bytes held by the library)"};
    }
    const size_t now = g_dev_bytes += bytes;
    size_t pk = g_dev_bytes_peak.load();
    while (now > pk && !g_dev_bytes_peak.compare_exchange_weak(pk, now)) {
    }
    return p;
}

// grow-only device buffer (capacity is kept across iterations and solves)
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), cap(o.cap) { o.p = nullptr; o.cap = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; cap = o.cap; o.p = nullptr; o.cap = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void swap(DevBuf &o) noexcept { std::swap(p, o.p); std::swap(cap, o.cap); }
    // headroom for regrowth: a quarter, a sixteenth above 1 GiB
    static size_t with_headroom(size_t n) {
        if (n < 16) return 16;
        return n * sizeof(T) > (size_t(1) << 30) ? n + n / 16 : n + n / 4;
    }
    // contents are not kept
    T *ensure(size_t n) {
        if (n <= cap && p) return p;
        const size_t want = with_headroom(n);
        release();
        p = (T *)dev_alloc(want * sizeof(T));
        cap = want;
        return p;
    }
    // keeps the first `used` elements (copied on stream st); the old and the
    // new allocation coexist during the copy
    T *grow_keep(size_t n, size_t used, cudaStream_t st) {
        if (n <= cap && p) return p;
        const size_t want = with_headroom(n);
        T *q = (T *)dev_alloc(want * sizeof(T));
        if (p && used) {
            cudaError_t e = cudaMemcpyAsync(q, p, used * sizeof(T), cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                cudaFree(q);
                g_dev_bytes -= want * sizeof(T);
                throw Error{-4, std::string("buffer regrowth copy: ") + cudaGetErrorString(e)};
            }
        }
        release();
        p = q;
        cap = want;
        return p;
    }
    void release() {
        if (p) {
            cudaFree(p);
            g_dev_bytes -= cap * sizeof(T);
        }
        p = nullptr;
        cap = 0;
    }
};

// per-system scalars kept on the device (FP64 where the method needs it)
struct SysDev {
    DevBuf<int> row0, nbs, n_orb;      // [S]
    DevBuf<int> sys_of_row;            // [NB]
    DevBuf<double> emin, emax;         // [S]
    DevBuf<double> c_lin, c_sq;        // [S]   branch coefficients of the current step
    DevBuf<double> tau0, tau1;         // [S]   truncation thresholds of the current step
    DevBuf<int> active;                // [S]   1 = still iterating
    DevBuf<int> tier;                  // [S]
};

struct MatSet {
    int nmat = 0;
    int NB = 0;
    int b = 0;
    DevBuf<int> row_ptr;      // nmat*NB+1 (flat)
    DevBuf<int> col;          // total blocks
    DevBuf<double> val;       // total*b*b
    DevBuf<float> nrm;        // total
    DevBuf<uint16_t> ophi;    // tensor-core operand planes (hi and lo interleaved, 4 KB per block)
    DevBuf<float> opf32;      // FP32 operand copy for the CUDA-core FP32 products (hi word)
    DevBuf<float> opf32lo;    // lo word (x - hi) for the double-FP32 products
    std::vector<int64_t> nnzb;   // host copy, per matrix
    int64_t total = 0;
    void release() {
        row_ptr.release(); col.release(); val.release(); nrm.release();
        ophi.release(); opf32.release(); opf32lo.release();
        nnzb.clear(); total = 0;
    }
};

// One output matrix of a multiplication step:
//   C = c_lin * X + c_sq * sum_t (A_t B_t)
struct Job {
    int out;          // output matrix index
    int xmat;         // matrix of the linear term (-1: none)
    int nterm;        // 1 or 2
    int a[2], b[2];   // operand matrices of each term
    int tau_sel;      // 0: tau0[s], 1: tau1[s]
};

constexpr int kMaxJobs = 8;
struct JobTable {
    int njob;
    Job job[kMaxJobs];
};

// Operand arithmetic of a numeric launch
// (AR_FF: double-FP32 products on the FP32 pipe, about 46 bits; AR_OZ:
// exact bf16 slice products on the tensor cores, FP64-class)
enum Arith { AR_FP64 = 0, AR_FP32 = 1, AR_BF16X3 = 2, AR_FP16X3 = 3, AR_FF = 5, AR_OZ = 6 };

// Jobs selected per precision tier: bit p of m[t] selects job p for the rows
// of systems currently in tier t (systems of a batch move through the tiers
// independently)
constexpr int kMaxTiers = 4;
struct JobMask {
    unsigned m[kMaxTiers];
};

// ---------------------------------------------------------------------------
// kernel launchers (implemented in the k_*.cu files)
// ---------------------------------------------------------------------------

// k_scan.cu: exclusive scan (out may alias in); returns nothing, total at out[n]
void scan_exclusive_i32(const int *in, int *out, int n, int *tmp, cudaStream_t st, int init = 0);
void scan_exclusive_i64(const int *in, int64_t *out, int n, int64_t *tmp, cudaStream_t st);
size_t scan_tmp_elems(int n);

// k_setup.cu
void launch_gershgorin(const int *row_ptr, const int *col, const double *val, int NB, int b,
                       const int *sys_of_row, const int *row0, const int *n_orb,
                       double *row_lo, double *row_hi, cudaStream_t st);
void launch_sys_minmax(const double *row_lo, const double *row_hi, const int *row0, const int *nbs,
                       int S, double *emin, double *emax, cudaStream_t st);
// X := alpha * (diag_shift_sel ? emax[s] I : 0) + beta * H   (per system scaling), norms
// rows = number of block rows of the (possibly multi-matrix) set; NB = rows per matrix
void launch_init_scale(const int *row_ptr, const int *col, const double *hval, double *xval,
                       float *xnrm, int rows, int NB, int b, const int *sys_of_row,
                       const int *row0, const int *n_orb, const double *emin,
                       const double *emax, int is_x0, cudaStream_t st);
void launch_block_norms(const double *val, float *nrm, int64_t nblk, int b, cudaStream_t st);
void launch_check_values(const int *row_ptr, const int *col, const double *val, int64_t nval,
                         int NB, int b, const int *sys_of_row, const int *row0, const int *n_orb,
                         double rel_tol, int *err, cudaStream_t st);

// k_stats.cu: per-row partial sums then a deterministic per-system reduction.
// q-layout of the per-system output (double, [S][nq]):
//   0: Tr X0, 1: ||X0||_F^2, 2: Tr(X0 H0), 3+g: Tr(X1_g H0)
void launch_row_stats(const int *row_ptr, const int *col, const double *val, int nmat, int NB,
                      int b, const int *h_row_ptr, const int *h_col, const double *h_val,
                      double *row_part, cudaStream_t st);
void launch_sys_sum(const double *row_part, int nq, int NB, const int *row0, const int *nbs,
                    int S, double *out, cudaStream_t st);

// alpha: per-row partials of <P1_d, H1_g> over intersecting blocks
void launch_row_dots(const int *p_row_ptr, const int *p_col, const double *p_val, int np,
                     const int *h_row_ptr, const int *h_col, const double *h_val, int nh,
                     int NB, int b, double *row_part, cudaStream_t st);

// k_symbolic.cu
struct SymOut {
    int *row_cnt;        // [njob*NB] kept blocks per (job,row)
    int *row_off;        // [njob*NB] offset of the row's list in the pool
    int *pool_col;       // pool of kept columns
    int *pool_npair;     // pool of pair counts (per kept column)
    int *pool_top;       // [1] pool allocation counter
    int pool_cap;
    int *overflow;       // [1] set when the pool is too small
};
// largest system (in block rows) the shared-memory row accumulator handles
constexpr int kSymMaxNs = 8192;
void launch_symbolic(const MatSet &in, const JobTable &jt, const SysDev &sd, int S,
                     SymOut so, cudaStream_t st, int max_ns);
// gathers the pool into the output pattern; writes slot_row/slot_job and the
// per-slot pair counts (0 for lower-triangle slots)
void launch_gather(const SymOut &so, int njob, int NB, const int *out_row_ptr, int *out_col,
                   int *slot_row, int *slot_job, int *slot_npair, cudaStream_t st);
void launch_pairs(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_row_ptr,
                  const int *out_col, const int *slot_row, const int *slot_job,
                  const int64_t *pair_off, int64_t nslot, int NB, int *pair_a, int *pair_b,
                  int *slot_x, int *slot_t, int *err, cudaStream_t st, JobMask fill);

// k_numeric.cu: C(upper slot) = c_lin X + c_sq sum(pairs); lower slot = transpose
struct NumArgs {
    const double *in_val;
    const float *in_f32;       // FP32 copy of in_val (FP32 products), may be null
    const float *in_f32lo;     // in_val - in_f32 rounded to FP32 (double-FP32 products), may be null
    const float *in_nrm;
    const int *pair_a, *pair_b;
    const int64_t *pair_off;
    const int *slot_row, *slot_job, *slot_x, *slot_t;
    const int *work;        // upper slots to process
    int *work_next;         // zeroed counter: next work item to hand out
    int nwork;
    const int *sys_of_row;
    const double *c_lin, *c_sq, *tau0, *tau1;
    const int *active;
    int job_tau_sel[kMaxJobs];
    // outputs: only upper-triangle slots (col >= row) are computed; the
    // values of upper slot s go to out_val at index uidx[s] - u0 (uidx: rank
    // of s among the upper slots, u0: that of the group's first one);
    // norm bound and keep flag to out_nrm[s], keep[s]
    double *out_val;
    float *out_nrm;
    uint8_t *keep;
    const int *uidx;
    int64_t u0;
    int b;
};
void launch_numeric_simt(const NumArgs &a, Arith ar, cudaStream_t st);
// FP32 copy of the FP64 master values (for the FP32 products)
// FP32 copy (and, with f32lo, the FP32 remainder) of FP64 values
void launch_to_f32(const double *val, float *f32, int64_t n, cudaStream_t st, float *f32lo = nullptr);

// k_compact.cu
// block triples of the upper slots of active systems per kernel class:
// out[0] tensor cores (tc), out[1] FP64 (m64), out[2] FP32 (m32), out[3] double-FP32 (mff),
// out[4] tensor-core slice products (moz)
void launch_class_pairs(const int *slot_row, const int *out_col, const int *slot_npair, const int *slot_job,
                        int64_t nslot, const int *sys_of_row, const int *active, const int *sys_tier,
                        JobMask tc, JobMask m64, JobMask m32, JobMask mff, JobMask moz, unsigned long long *out,
                        cudaStream_t st);
// upper slots of the active systems' jobs selected by job_mask (per system
// tier), plus (with_inactive) all upper slots of converged systems
// (slots [s0, s1) only)
void launch_build_work(const int *slot_row, const int *out_col, int64_t s0, int64_t s1,
                       int *work, int *nwork, cudaStream_t st, const int *sys_of_row,
                       const int *active, const int *slot_job, const int *sys_tier, JobMask job_mask,
                       int with_inactive);
// uidx[s] = 1 for upper slots (col >= row), else 0 (scanned afterwards)
void launch_upper_flags(const int *slot_row, const int *out_col, int64_t nslot, int *uidx,
                        cudaStream_t st);
// urp[r] = uidx[out_row_ptr[r]] for r in [0, n]
void launch_gather_i32(const int *idx, const int *src, int n, int *dst, cudaStream_t st);

// Compaction of the rows [r0, r0 + nrows) of the mask.  An upper slot is kept
// on its own flag; a lower slot t on that of its upper partner slot_t[t],
// and receives that block's transpose, read from out_val when the partner
// belongs to the current group (uidx >= u0) and otherwise from the already
// compacted output (dest[partner]).  dest[s] receives the output position of
// every kept upper slot s.
struct CompactArgs {
    const int *out_rp, *out_col, *slot_row, *slot_t, *uidx;
    const double *out_val;
    const float *out_nrm;
    const uint8_t *keep;
    int64_t u0;
    int *dest;
    int *src;               // [kept blocks of the group]: slot of output block d0 + k
    const int *new_rp;
    int *new_col;
    double *new_val;
    float *new_nrm;
    int r0, nrows, b;
    int d0;                 // first output block of the group
};
void launch_compact_count(const CompactArgs &c, int *cnt, cudaStream_t st);
// output blocks [d0, d1) of the group
void launch_compact_copy(const CompactArgs &c, int d1, cudaStream_t st);

// k_lowdin.cu: out = fac[sys] * val for every block of the first NB block rows
// (pad_one: the diagonal of padding rows set to 1), and identity blocks.
void launch_scale_sys(const int *row_ptr, const int *col, const double *val, int NB, int b, const int *sys_of_row,
                      const int *row0, const int *n_orb, const double *fac, int pad_one, double *out,
                      cudaStream_t st);
void launch_identity_blocks(double *val, int64_t nblk, int b, cudaStream_t st);

// k_reblock.cu: the same matrix in b_out x b_out instead of b_in x b_in blocks.
// Host pattern (rp/col of one matrix, local block indices; n orbitals): an
// output block exists where a stored input block overlaps it.
void reblock_pattern(const std::vector<int> &rp, const std::vector<int> &col, int b_in, int n, int b_out,
                     std::vector<int> &rp_out, std::vector<int> &col_out);
// Values of the nout output blocks (out_row/out_col: block row and column of
// each, device) from the input matrix (device row_ptr/col/val, nb_in rows).
void launch_reblock_vals(const int *in_rp, const int *in_col, const double *in_val, int nb_in, int b_in,
                         const int *out_row, const int *out_col, double *out_val, int64_t nout, int b_out,
                         cudaStream_t st);

}  // namespace rdm
