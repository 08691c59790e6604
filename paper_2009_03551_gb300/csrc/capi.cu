// C ABI (include/rdm.h) and the host-side driver of the solve.
//
// The driver follows Sec. 2.2 of the paper: Gershgorin bounds, the initial
// matrices, then per iteration the trace test of Eq. TC2 choosing between
// X0 <- X0^2, X1 <- X1 X0 + X0 X1 and X0 <- 2X0 - X0^2,
// X1 <- 2X1 - X1 X0 - X0 X1 (Eq. TC2-CPSCF), each product followed by
// block-norm truncation (Sec. 2.3 "filter"), until the band energies
// Tr(X0 H0), Tr(X1 H0) stop changing (Sec. 2.3 "tolerance").  Finally the
// polarizability alpha_{gd} = -spin Tr(P1_d H1_g) (Eq. polar, field term
// -r.E).  Every arithmetic step runs in the kernels of k_*.cu; the host only
// makes the per-system scalar decisions and sizes the buffers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <mutex>
#include <numeric>
#include <set>
#include <thread>
#include <vector>

#include "../../include/rdm.h"
#include "rdm_internal.cuh"
#include "tc_gemm.cuh"

using namespace rdm;

thread_local long long rdm::g_kernel_launches = 0;

void rdm::func_smem_once(const void *func, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    RDM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({func, dev})) return;
    RDM_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.insert({func, dev});
}

namespace {

// one system's matrices at one block size: host patterns, device values
struct SysMats {
    int b = 0, nb = 0;
    std::vector<int> rp, col;          // H0
    DevBuf<double> val;
    std::vector<int> rp1[3], col1[3];  // H1_dir
    DevBuf<double> val1[3];
    std::vector<int> rps, cols;        // S (non-orthogonal basis)
    DevBuf<double> vals;
};

struct HostSys {
    bool has_h0 = false;
    int nb = 0, n = 0;
    int64_t n_elec = 0;
    std::vector<int> rp, col;          // host copies of the pattern
    DevBuf<double> val;                // device copy of the values
    bool has_h1[3] = {false, false, false};
    std::vector<int> rp1[3], col1[3];
    DevBuf<double> val1[3];
    bool has_s = false;                // overlap matrix uploaded (non-orthogonal basis, Sec. 2.2)
    std::vector<int> rps, cols;
    DevBuf<double> vals;
    SysMats rb;                        // the same matrices at the solve's block size (when it differs)
};

struct SysState {
    int iters = 0;
    int tier = 0;
    int tier_start = 0;
    int prev_branch = 0;
    bool active = true;
    bool converged = false;
    std::vector<double> e_hist;
    bool have_eb = false;
    double eb0 = 0, eb1[3] = {0, 0, 0};
    int tier_iters[4] = {0, 0, 0, 0};
};

}  // namespace

struct rdm_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    rdm_params prm;
    int S = 1;
    int b = 0;                 // block size of the uploaded matrices
    int bs = 0;                // block size of the current solve (b, or the re-blocked size)
    int tuned_b = 0;           // autotuner's choice (0: not tuned) ...
    std::vector<int64_t> tuned_key;   // ... for problems of this shape: systems, b, block rows, blocks of H0
    double autotune_ms = 0, probe_ms[3] = {0, 0, 0};
    std::thread worker;        // rdm_solve_async
    bool pending = false;
    int async_status = 0;
    std::vector<HostSys> hs;
    std::vector<uint8_t> forced;

    // assembled inputs
    int NB = 0;
    int nd = 0;
    int dirs[3] = {0, 0, 0};
    int dir_only = -1;          // >= 0: assemble only this field direction (split_directions)
    bool keep_assembled = false;  // run_solve starts from the current H0, H1 (the correction's response solves)
    std::vector<int> stop_at;     // non-empty: system s stops after stop_at[s] updates (the same)
    std::vector<int> row0, nbs, norb;
    MatSet H0, H1;
    MatSet Sm;                  // overlap matrices (non-orthogonal basis), when uploaded
    bool has_s = false;
    MatSet Zm, Lm;              // S^(-1/2) and S^(-1) of the last solve (Loewdin transform)
    int lowdin_iters = 0;
    SysDev sd;
    MatSet X[2];
    int cur = 0;

    // work buffers
    DevBuf<int> row_cnt, row_off, pool_col, pool_npair, counters, mask_col;
    DevBuf<int> out_rp, slot_row, slot_job, slot_npair, slot_x, slot_t, work, work2, work3;
    DevBuf<int64_t> pair_off, scan_tmp64;
    DevBuf<int> scan_tmp32, pair_a, pair_b, cnt_rows;
    DevBuf<int> uidx, scan_tmp_s, urp, dest, cpsrc;   // upper-slot ranks, compaction maps
    DevBuf<int> work_ctr;                             // work-item counters of the CUDA-core launches
    DevBuf<double> out_val, row_part, sys_q;
    DevBuf<float> out_nrm;
    DevBuf<uint8_t> keep;
    DevBuf<unsigned long long> class_pairs;
    DevBuf<double> row_lo, row_hi;
    TcWork tcw, tcw_oz;      // plans of the split and of the slice-product tensor-core launches
    OzWork ozw;
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void ensure_events() {
        for (auto &e : ev)
            if (!e) RDM_CUDA_TRY(cudaEventCreate(&e));
    }
    ~rdm_handle() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }

    // results
    bool solved = false;
    std::vector<rdm_info> info;
    std::vector<rdm_iter_log> log;
    std::vector<double> alpha;
    std::vector<int> final_rp;     // host copy of X row_ptr after the solve
    // results in the uploaded block size when the solve ran at another one:
    // pattern (row_ptr, col) per (system, matrix), made on first request
    std::vector<std::pair<std::vector<int>, std::vector<int>>> conv;
    int64_t pool_cap_hint = 0;
};

namespace {

int fail(rdm_handle *h, int code, const std::string &m) {
    if (h) h->err = m;
    return code;
}

template <class F>
int guarded(rdm_handle *h, F &&f) {
    try {
        return f();
    } catch (const Error &e) {
        return fail(h, e.code, e.msg);
    } catch (const std::bad_alloc &) {
        return fail(h, RDM_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(h, RDM_EINVAL, e.what());
    } catch (...) {
        return fail(h, RDM_EINVAL, "unknown error");
    }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) RDM_CUDA_TRY(cudaSetDevice(d));
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

void sync(rdm_handle *h) { RDM_CUDA_TRY(cudaStreamSynchronize(h->stream)); }

template <class T>
void h2d(T *dst, const T *src, size_t n, cudaStream_t st) {
    if (n) RDM_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
}
template <class T>
void d2h(T *dst, const T *src, size_t n, cudaStream_t st) {
    if (n) RDM_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
}

// ---------------------------------------------------------------------------
// upload and validation
// ---------------------------------------------------------------------------

void check_pattern(const rdm_bsr *A, const std::vector<int> &rp, const std::vector<int> &col,
                   bool need_diag) {
    const int nb = A->nb;
    if (rp[0] != 0 || rp[nb] != A->nnzb)
        throw Error{RDM_EBADBSR, "row_ptr[0] must be 0 and row_ptr[nb] must equal nnzb"};
    for (int i = 0; i < nb; ++i) {
        if (rp[i + 1] < rp[i]) throw Error{RDM_EBADBSR, "row_ptr is not non-decreasing"};
        bool diag = false;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= nb)
                throw Error{RDM_EBADBSR, "column index out of range in block row " + std::to_string(i)};
            if (p > rp[i] && col[p] <= col[p - 1])
                throw Error{RDM_EBADBSR, "columns not strictly increasing in block row " + std::to_string(i)};
            if (col[p] == i) diag = true;
        }
        if (need_diag && !diag)
            throw Error{RDM_EBADBSR, "diagonal block missing in block row " + std::to_string(i)};
    }
    // symmetric pattern: every (i,j) has (j,i)
    for (int i = 0; i < nb; ++i)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = col[p];
            if (!std::binary_search(col.begin() + rp[j], col.begin() + rp[j + 1], i))
                throw Error{RDM_EBADBSR, "block pattern is not symmetric"};
        }
}

void upload_matrix(rdm_handle *h, const rdm_bsr *A, std::vector<int> &rp, std::vector<int> &col,
                   DevBuf<double> &val, bool need_diag) {
    if (!A || !A->row_ptr || (A->nnzb > 0 && (!A->col_idx || !A->vals)))
        throw Error{RDM_EINVAL, "null matrix pointer"};
    if (A->nb <= 0 || A->b <= 0 || A->b > 64 || (A->b & (A->b - 1)))
        throw Error{RDM_EINVAL, "nb must be > 0 and b a power of two <= 64"};
    if (A->n <= (int64_t)(A->nb - 1) * A->b || A->n > (int64_t)A->nb * A->b)
        throw Error{RDM_EINVAL, "n must satisfy (nb-1)*b < n <= nb*b"};
    if (A->nnzb < 0 || A->nnzb > (int64_t)A->nb * A->nb)
        throw Error{RDM_EINVAL, "nnzb out of range"};
    if (h->b && h->b != A->b) throw Error{RDM_EINVAL, "all systems of a batch share the block size"};
    const int nb = A->nb;
    const size_t bb = (size_t)A->b * A->b;
    rp.resize(nb + 1);
    col.resize(A->nnzb);
    cudaMemcpyKind k = A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    RDM_CUDA_TRY(cudaMemcpy(rp.data(), A->row_ptr, (nb + 1) * sizeof(int), k));
    if (A->nnzb) RDM_CUDA_TRY(cudaMemcpy(col.data(), A->col_idx, A->nnzb * sizeof(int), k));
    check_pattern(A, rp, col, need_diag);
    val.ensure(A->nnzb * bb);
    if (A->nnzb)
        RDM_CUDA_TRY(cudaMemcpyAsync(val.p, A->vals, A->nnzb * bb * sizeof(double),
                                     A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     h->stream));
    // value checks on the device: finite, symmetric (1e-12 max|H|), zero padding
    DevBuf<int> drp, dcol, derr, dsys, dz;
    drp.ensure(nb + 1);
    dcol.ensure(std::max<int64_t>(1, A->nnzb));
    derr.ensure(4);
    dsys.ensure(nb);
    dz.ensure(2);
    h2d(drp.p, rp.data(), nb + 1, h->stream);
    h2d(dcol.p, col.data(), A->nnzb, h->stream);
    RDM_CUDA_TRY(cudaMemsetAsync(derr.p, 0, 4 * sizeof(int), h->stream));
    RDM_CUDA_TRY(cudaMemsetAsync(dsys.p, 0, nb * sizeof(int), h->stream));
    int zn[2] = {0, A->n};
    h2d(dz.p, zn, 2, h->stream);
    launch_check_values(drp.p, dcol.p, val.p, A->nnzb * (int64_t)bb, nb, A->b, dsys.p, dz.p,
                        dz.p + 1, 1e-12, derr.p, h->stream);
    int herr[4];
    d2h(herr, derr.p, 4, h->stream);
    sync(h);
    drp.release(); dcol.release(); derr.release(); dsys.release(); dz.release();
    if (herr[0] & 1) throw Error{RDM_EBADBSR, "matrix has non-finite values"};
    if (herr[0] & 8) throw Error{RDM_EBADBSR, "block pattern is not symmetric"};
    if (herr[0] & 2) throw Error{RDM_EBADBSR, "matrix values are not symmetric (tolerance 1e-12 max|H|)"};
    if (herr[0] & 4) throw Error{RDM_EBADBSR, "padding rows/columns (index >= n) must be zero"};
    h->b = A->b;
}

// ---------------------------------------------------------------------------
// assembly of the batch into global block-diagonal sets
// ---------------------------------------------------------------------------

// The matrices of system s at block size bs (the uploaded ones, or a
// re-blocked copy made once and kept until the next upload).
void ensure_reblocked(rdm_handle *h, int s, int bs) {
    HostSys &y = h->hs[s];
    if (bs == h->b || y.rb.b == bs) return;
    SysMats &r = y.rb;
    r.b = 0;
    auto one = [&](const std::vector<int> &rp, const std::vector<int> &col, const double *val,
                   std::vector<int> &orp, std::vector<int> &ocol, DevBuf<double> &oval) {
        reblock_pattern(rp, col, h->b, y.n, bs, orp, ocol);
        const int64_t nout = (int64_t)ocol.size();
        std::vector<int> orow(nout);
        for (int i = 0; i + 1 < (int)orp.size(); ++i)
            for (int p = orp[i]; p < orp[i + 1]; ++p) orow[p] = i;
        DevBuf<int> drp, dcol, dorow, docol;
        drp.ensure(rp.size());
        dcol.ensure(std::max<size_t>(col.size(), 1));
        dorow.ensure(std::max<int64_t>(nout, 1));
        docol.ensure(std::max<int64_t>(nout, 1));
        h2d(drp.p, rp.data(), rp.size(), h->stream);
        h2d(dcol.p, col.data(), col.size(), h->stream);
        h2d(dorow.p, orow.data(), (size_t)nout, h->stream);
        h2d(docol.p, ocol.data(), (size_t)nout, h->stream);
        oval.ensure(std::max<int64_t>(nout, 1) * bs * bs);
        launch_reblock_vals(drp.p, dcol.p, val, (int)rp.size() - 1, h->b, dorow.p, docol.p, oval.p, nout, bs,
                            h->stream);
        sync(h);
    };
    one(y.rp, y.col, y.val.p, r.rp, r.col, r.val);
    for (int d = 0; d < 3; ++d)
        if (y.has_h1[d]) one(y.rp1[d], y.col1[d], y.val1[d].p, r.rp1[d], r.col1[d], r.val1[d]);
    if (y.has_s) one(y.rps, y.cols, y.vals.p, r.rps, r.cols, r.vals);
    r.nb = (int)r.rp.size() - 1;
    r.b = bs;
}

void init_x(rdm_handle *h);
void init_sys_scalars(rdm_handle *h);

void assemble(rdm_handle *h) {
    const int S = h->S;
    h->row0.assign(S, 0);
    h->nbs.assign(S, 0);
    h->norb.assign(S, 0);
    int NB = 0;
    const bool rb = h->bs != h->b;
    for (int s = 0; s < S; ++s) {
        if (!h->hs[s].has_h0) throw Error{RDM_ESTATE, "H0 of system " + std::to_string(s) + " not uploaded"};
        if (rb) ensure_reblocked(h, s, h->bs);
        h->row0[s] = NB;
        h->nbs[s] = rb ? h->hs[s].rb.nb : h->hs[s].nb;
        h->norb[s] = h->hs[s].n;
        NB += h->nbs[s];
    }
    h->NB = NB;
    // directions: the set uploaded for system 0; every system must match
    int nd = 0;
    for (int d = 0; d < 3; ++d)
        if (h->hs[0].has_h1[d] && (h->dir_only < 0 || d == h->dir_only)) h->dirs[nd++] = d;
    for (int s = 1; s < S; ++s)
        for (int d = 0; d < 3; ++d)
            if (h->hs[s].has_h1[d] != h->hs[0].has_h1[d])
                throw Error{RDM_EINVAL, "every system of a batch needs the same H1 directions"};
    h->nd = nd;
    const int b = h->bs;
    const size_t bb = (size_t)b * b;

    auto build = [&](MatSet &M, int nmat, auto get_rp, auto get_col, auto get_val) {
        M.nmat = nmat;
        M.NB = NB;
        M.b = b;
        std::vector<int> rp((size_t)nmat * NB + 1);
        std::vector<int> col;
        M.nnzb.assign(nmat, 0);
        int64_t top = 0;
        for (int m = 0; m < nmat; ++m)
            for (int s = 0; s < S; ++s) {
                const std::vector<int> &r = get_rp(s, m);
                const std::vector<int> &c = get_col(s, m);
                for (int i = 0; i < h->nbs[s]; ++i) {
                    rp[(size_t)m * NB + h->row0[s] + i] = (int)(top + r[i]);
                }
                for (int p = 0; p < (int)c.size(); ++p) col.push_back(c[p] + h->row0[s]);
                top += r[h->nbs[s]];
                M.nnzb[m] += r[h->nbs[s]];
            }
        rp[(size_t)nmat * NB] = (int)top;
        if (top > INT32_MAX / 2) throw Error{RDM_EINVAL, "too many blocks"};
        M.total = top;
        M.row_ptr.ensure(rp.size());
        M.col.ensure(std::max<int64_t>(top, 1));
        M.val.ensure(std::max<int64_t>(top, 1) * bb);
        M.nrm.ensure(std::max<int64_t>(top, 1));
        h2d(M.row_ptr.p, rp.data(), rp.size(), h->stream);
        h2d(M.col.p, col.data(), col.size(), h->stream);
        int64_t off = 0;
        for (int m = 0; m < nmat; ++m)
            for (int s = 0; s < S; ++s) {
                int64_t n = get_rp(s, m)[h->nbs[s]];
                if (n)
                    RDM_CUDA_TRY(cudaMemcpyAsync(M.val.p + off * bb, get_val(s, m), n * bb * sizeof(double),
                                                 cudaMemcpyDeviceToDevice, h->stream));
                off += n;
            }
    };
    build(h->H0, 1, [&](int s, int) -> const std::vector<int> & { return rb ? h->hs[s].rb.rp : h->hs[s].rp; },
          [&](int s, int) -> const std::vector<int> & { return rb ? h->hs[s].rb.col : h->hs[s].col; },
          [&](int s, int) { return (const double *)(rb ? h->hs[s].rb.val.p : h->hs[s].val.p); });
    if (nd) {
        build(h->H1, nd,
              [&](int s, int m) -> const std::vector<int> & {
                  return rb ? h->hs[s].rb.rp1[h->dirs[m]] : h->hs[s].rp1[h->dirs[m]];
              },
              [&](int s, int m) -> const std::vector<int> & {
                  return rb ? h->hs[s].rb.col1[h->dirs[m]] : h->hs[s].col1[h->dirs[m]];
              },
              [&](int s, int m) {
                  return (const double *)(rb ? h->hs[s].rb.val1[h->dirs[m]].p : h->hs[s].val1[h->dirs[m]].p);
              });
    }
    h->has_s = false;
    int ns = 0;
    for (int s2 = 0; s2 < S; ++s2) ns += h->hs[s2].has_s ? 1 : 0;
    if (ns && ns != S) throw Error{RDM_EINVAL, "upload an overlap matrix for every system of the batch or for none"};
    if (ns) {
        h->has_s = true;
        build(h->Sm, 1, [&](int s2, int) -> const std::vector<int> & { return rb ? h->hs[s2].rb.rps : h->hs[s2].rps; },
              [&](int s2, int) -> const std::vector<int> & { return rb ? h->hs[s2].rb.cols : h->hs[s2].cols; },
              [&](int s2, int) { return (const double *)(rb ? h->hs[s2].rb.vals.p : h->hs[s2].vals.p); });
    }
    init_sys_scalars(h);
    init_x(h);
}

// X0 has the pattern of H0, X1_g that of H1_g
void init_x(rdm_handle *h) {
    const int NB = h->NB, nd = h->nd, b = h->bs;
    const size_t bb = (size_t)b * b;
    MatSet &X = h->X[0];
    h->cur = 0;
    X.nmat = 1 + nd;
    X.NB = NB;
    X.b = b;
    int64_t tot = h->H0.total + (nd ? h->H1.total : 0);
    X.total = tot;
    X.nnzb.assign(1 + nd, 0);
    X.nnzb[0] = h->H0.nnzb[0];
    for (int m = 0; m < nd; ++m) X.nnzb[1 + m] = h->H1.nnzb[m];
    X.row_ptr.ensure((size_t)(1 + nd) * NB + 1);
    X.col.ensure(std::max<int64_t>(tot, 1));
    X.val.ensure(std::max<int64_t>(tot, 1) * bb);
    X.nrm.ensure(std::max<int64_t>(tot, 1));
    {
        // row_ptr of X: H0 rows, then H1 rows shifted by nnzb(H0)
        std::vector<int> rp((size_t)(1 + nd) * NB + 1);
        std::vector<int> tmp((size_t)NB + 1);
        d2h(rp.data(), h->H0.row_ptr.p, (size_t)NB, h->stream);
        if (nd) {
            std::vector<int> r1((size_t)nd * NB + 1);
            d2h(r1.data(), h->H1.row_ptr.p, r1.size(), h->stream);
            sync(h);
            for (size_t t = 0; t < r1.size(); ++t) rp[NB + t] = r1[t] + (int)h->H0.total;
        } else {
            sync(h);
            rp[NB] = (int)h->H0.total;
        }
        h2d(X.row_ptr.p, rp.data(), rp.size(), h->stream);
    }
    RDM_CUDA_TRY(cudaMemcpyAsync(X.col.p, h->H0.col.p, h->H0.total * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    if (nd)
        RDM_CUDA_TRY(cudaMemcpyAsync(X.col.p + h->H0.total, h->H1.col.p, h->H1.total * sizeof(int),
                                     cudaMemcpyDeviceToDevice, h->stream));
}

// per-system device scalars
void init_sys_scalars(rdm_handle *h) {
    const int S = h->S, NB = h->NB;
    SysDev &sd = h->sd;
    sd.row0.ensure(S); sd.nbs.ensure(S); sd.n_orb.ensure(S);
    sd.emin.ensure(S); sd.emax.ensure(S); sd.c_lin.ensure(S); sd.c_sq.ensure(S);
    sd.tau0.ensure(S); sd.tau1.ensure(S); sd.active.ensure(S); sd.tier.ensure(S);
    sd.sys_of_row.ensure(NB);
    std::vector<int> sor(NB);
    for (int s = 0; s < S; ++s)
        for (int i = 0; i < h->nbs[s]; ++i) sor[h->row0[s] + i] = s;
    h2d(sd.row0.p, h->row0.data(), S, h->stream);
    h2d(sd.nbs.p, h->nbs.data(), S, h->stream);
    h2d(sd.n_orb.p, h->norb.data(), S, h->stream);
    h2d(sd.sys_of_row.p, sor.data(), NB, h->stream);
}

// ---------------------------------------------------------------------------
// one multiplication step: symbolic, pairs, numeric, truncation, compaction
// ---------------------------------------------------------------------------

struct StepStats {
    int64_t npairs = 0;
    int64_t nslot = 0;
    int64_t pairs_tc = 0, pairs_64 = 0, pairs_32 = 0, pairs_ff = 0, pairs_oz = 0;   // block triples per class
    double issued_tc = 0, issued_oz = 0;
    double bytes = 0;
    double ms[7] = {0, 0, 0, 0, 0, 0, 0};   // symbolic, tc, fp64, fp32, compaction, double-fp32, slice products
    int tc_launches = 0, oz_launches = 0, simt_launches = 0;
    int groups = 1;                         // job groups of the numeric phase
};

bool is_tc(Arith a) { return a == AR_BF16X3 || a == AR_FP16X3; }

// the mixed modes need a block size that the tensor-core kernel handles
bool tc_block_ok(int mode, int b) {
    return !(mode == RDM_MODE_MIXED_BF16 || mode == RDM_MODE_MIXED_FP16) || b == 0 || tc_block_size_ok(b);
}

// Arithmetic of every job (job 0 = X0^2, jobs 1.. = X1 products) for a tier.
// The fp16 ladder has two tiers: every product as a scaled fp16 split product
// on the tensor cores (22 bits), then the final tier, where X0^2 is refined
// (`refine_x0`; by default as exact bf16 slice products on the tensor cores,
// FP64-class) and the first-order products use `refine_x1` (by default they
// stay split: with the segmented accumulation of the tensor-core kernel they
// are as accurate as FP32 CUDA-core products).  The bf16 ladder: bf16 split
// products (16 bits), then the final tier (X0^2 as for fp16, the first-order
// products still bf16 split: alpha's error is the bulk tier's rotation of the
// occupied subspace, and FP64 first-order products in the final tier gave the
// same alpha at 11 times the solve time).  A three-tier bf16 ladder with an
// FP32 tier between (X1 in FP32 on the CUDA cores through both later tiers)
// was measured and left 2e-6 in alpha on a 90-atom cluster where this one
// leaves 1e-6.
int final_tier_of(int mode) { return mode == RDM_MODE_MIXED_BF16 || mode == RDM_MODE_MIXED_FP16 ? 1 : 0; }

void tier_arith(int mode, int tier, int njob, Arith *ar, int refine_x1 = 0, int refine_x0 = 0, int b = 32) {
    const bool bf16 = mode == RDM_MODE_MIXED_BF16;
    if (refine_x1 == RDM_REFINE_DEFAULT) refine_x1 = RDM_REFINE_SPLIT;
    if (refine_x0 == RDM_REFINE_DEFAULT) refine_x0 = b == 32 ? RDM_REFINE_SLICES : RDM_REFINE_FP64;
    const int final_tier = final_tier_of(mode);
    for (int p = 0; p < njob; ++p) {
        const Arith split = bf16 ? AR_BF16X3 : AR_FP16X3;
        switch (mode) {
            case RDM_MODE_FP64: ar[p] = AR_FP64; break;
            case RDM_MODE_FP32: ar[p] = AR_FP32; break;
            case RDM_MODE_MIXED_BF16:
            case RDM_MODE_MIXED_FP16:
                if (tier == 0 || tier < final_tier) ar[p] = split;
                else if (p == 0) ar[p] = refine_x0 == RDM_REFINE_FP32 ? AR_FP32
                                        : refine_x0 == RDM_REFINE_FP32X2 ? AR_FF
                                        : refine_x0 == RDM_REFINE_SLICES ? AR_OZ : AR_FP64;
                else if (refine_x1 == RDM_REFINE_FP64) ar[p] = AR_FP64;
                else if (refine_x1 == RDM_REFINE_FP32X2) ar[p] = AR_FF;
                else ar[p] = refine_x1 == RDM_REFINE_SPLIT ? split : AR_FP32;
                break;
            default: ar[p] = AR_FP64;
        }
    }
}

// tab[t][p]: arithmetic of job p for the systems in tier t; tiers_present:
// bit t set when some active system is in tier t (the per-system tiers are in
// h->sd.tier on the device)
StepStats multiply(rdm_handle *h, MatSet &in, MatSet &out, const JobTable &jt,
                   const Arith (*tab)[kMaxJobs], unsigned tiers_present) {
    cudaStream_t st = h->stream;
    const int NB = in.NB, b = in.b, njob = jt.njob;
    const size_t bb = (size_t)b * b;
    const int nrows = njob * NB;
    int max_ns = *std::max_element(h->nbs.begin(), h->nbs.end());
    StepStats ss;
    // CUDA-core classes, launched in this order: FP64, double-FP32, FP32
    constexpr int kSimt = 3;
    const Arith simt_ar[kSimt] = {AR_FP64, AR_FF, AR_FP32};
    JobMask tcm{}, cm[kSimt]{}, simt{}, ozm{};
    Arith tc_ar = AR_FP16X3;
    bool any_tc = false, any_oz = false, any_c[kSimt] = {false, false, false};
    for (int t = 0; t < kMaxTiers; ++t) {
        if (!((tiers_present >> t) & 1u)) continue;
        for (int p = 0; p < njob; ++p) {
            const Arith a = tab[t][p];
            if (a == AR_OZ) {
                ozm.m[t] |= 1u << p;
                any_oz = true;
                continue;
            }
            if (is_tc(a)) {
                tcm.m[t] |= 1u << p;
                tc_ar = a;
                any_tc = true;
                continue;
            }
            const int c = a == AR_FP64 ? 0 : a == AR_FF ? 1 : 2;
            cm[c].m[t] |= 1u << p;
            any_c[c] = true;
        }
        simt.m[t] = cm[0].m[t] | cm[1].m[t] | cm[2].m[t];
    }
    // the first class present also copies the blocks of converged systems (the
    // FP32 class when no CUDA-core product is left)
    int first_c = kSimt - 1;
    for (int c = kSimt - 1; c >= 0; --c)
        if (any_c[c]) first_c = c;
    const bool tc = any_tc;
    const bool f32_planes = any_c[1] || any_c[2];
    h->ensure_events();
    RDM_CUDA_TRY(cudaEventRecord(h->ev[0], st));
    // operand copies are made afresh from the input set at every step: one
    // set of buffers, moved to whichever set is the input, serves both
    auto take = [](auto &mine, auto &other) {
        if (other.cap > mine.cap) mine.swap(other);
        other.release();
    };
    take(in.ophi, out.ophi);
    take(in.opf32, out.opf32);
    take(in.opf32lo, out.opf32lo);
    // copies the step does not use are kept for the next solve, unless they
    // are large (above 4 GiB the solve's time dwarfs a re-allocation)
    const size_t big = size_t(4) << 30;
    if (!tc && in.ophi.cap * sizeof(uint16_t) > big) in.ophi.release();
    if (!f32_planes && in.opf32.cap * sizeof(float) > big) in.opf32.release();
    if (!any_c[1] && in.opf32lo.cap * sizeof(float) > big) in.opf32lo.release();
    if (tc) prepare_operands(in, tc_ar, h->tcw, st);
    if (any_oz) prepare_oz_operands(in, h->ozw, st);
    else if (h->ozw.slices.cap * sizeof(uint16_t) > big) h->ozw.slices.release();
    if (f32_planes) {
        in.opf32.ensure(std::max<int64_t>(in.total, 1) * bb);
        if (any_c[1]) in.opf32lo.ensure(std::max<int64_t>(in.total, 1) * bb);
        launch_to_f32(in.val.p, in.opf32.p, in.total * (int64_t)bb, st, any_c[1] ? in.opf32lo.p : nullptr);
    }

    h->row_cnt.ensure(nrows);
    h->row_off.ensure(nrows);
    h->counters.ensure(8);
    int64_t cap = std::max<int64_t>(h->pool_cap_hint, 4 * in.total + 1024);
    int top = 0;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (cap > INT32_MAX / 2) throw Error{RDM_ECAPACITY, "symbolic pool exceeds 2^30 blocks"};
        h->pool_col.ensure(cap);
        h->pool_npair.ensure(cap);
        RDM_CUDA_TRY(cudaMemsetAsync(h->counters.p, 0, 8 * sizeof(int), st));
        SymOut so{h->row_cnt.p, h->row_off.p, h->pool_col.p, h->pool_npair.p, h->counters.p,
                  (int)h->pool_col.cap, h->counters.p + 1};
        launch_symbolic(in, jt, h->sd, h->S, so, st, h->prm.symbolic_hash ? kSymMaxNs + 1 : max_ns);
        int hc[2];
        d2h(hc, h->counters.p, 2, st);
        sync(h);
        top = hc[0];
        if (!hc[1]) break;
        if (hc[1] == 2)
            throw Error{RDM_ECAPACITY, "a block row of a product reaches more than 6144 distinct block columns"};
        cap = (int64_t)top + top / 4 + 1024;
        if (attempt == 3) throw Error{RDM_ECAPACITY, "symbolic pool overflow after retries"};
    }
    h->pool_cap_hint = std::max<int64_t>(h->pool_cap_hint, top);

    // output pattern
    h->out_rp.ensure(nrows + 1);
    h->scan_tmp32.ensure(scan_tmp_elems(nrows + 1));
    scan_exclusive_i32(h->row_cnt.p, h->out_rp.p, nrows, h->scan_tmp32.p, st);
    const int64_t nslot = top;
    ss.nslot = nslot;
    out.nmat = njob;
    out.NB = NB;
    out.b = b;
    int *mcol = h->mask_col.ensure(std::max<int64_t>(nslot, 1));
    h->slot_row.ensure(std::max<int64_t>(nslot, 1));
    h->slot_job.ensure(std::max<int64_t>(nslot, 1));
    h->slot_npair.ensure(std::max<int64_t>(nslot, 1));
    SymOut so{h->row_cnt.p, h->row_off.p, h->pool_col.p, h->pool_npair.p, h->counters.p,
              (int)h->pool_col.cap, h->counters.p + 1};
    launch_gather(so, njob, NB, h->out_rp.p, mcol, h->slot_row.p, h->slot_job.p,
                  h->slot_npair.p, st);
    h->pair_off.ensure(nslot + 1);
    h->scan_tmp64.ensure(scan_tmp_elems((int)nslot + 1));
    scan_exclusive_i64(h->slot_npair.p, h->pair_off.p, (int)nslot, h->scan_tmp64.p, st);
    int64_t npairs = 0;
    d2h(&npairs, h->pair_off.p + nslot, 1, st);
    // block triples per kernel class (tensor cores, FP64, FP32, double-FP32) for the accounting
    h->class_pairs.ensure(5);
    RDM_CUDA_TRY(cudaMemsetAsync(h->class_pairs.p, 0, 5 * sizeof(unsigned long long), st));
    launch_class_pairs(h->slot_row.p, mcol, h->slot_npair.p, h->slot_job.p, nslot, h->sd.sys_of_row.p,
                       h->sd.active.p, h->sd.tier.p, tcm, cm[0], cm[2], cm[1], ozm, h->class_pairs.p, st);
    unsigned long long cls[5] = {0, 0, 0, 0, 0};
    d2h(cls, h->class_pairs.p, 5, st);
    sync(h);
    ss.npairs = npairs;
    ss.pairs_tc = (int64_t)cls[0];
    ss.pairs_64 = (int64_t)cls[1];
    ss.pairs_32 = (int64_t)cls[2];
    ss.pairs_ff = (int64_t)cls[3];
    ss.pairs_oz = (int64_t)cls[4];
    if (any_c[0] || any_c[1] || any_c[2]) {
        h->pair_a.ensure(std::max<int64_t>(npairs, 1));
        h->pair_b.ensure(std::max<int64_t>(npairs, 1));
    }
    h->slot_x.ensure(std::max<int64_t>(nslot, 1));
    h->slot_t.ensure(std::max<int64_t>(nslot, 1));
    // pair lists only for the jobs on the CUDA cores (the tensor-core kernel
    // builds its own K-steps); slot_x / slot_t for every job
    launch_pairs(in, jt, h->sd, h->out_rp.p, mcol, h->slot_row.p, h->slot_job.p, h->pair_off.p,
                 nslot, NB, h->pair_a.p, h->pair_b.p, h->slot_x.p, h->slot_t.p, h->counters.p + 2, st,
                 simt);
    DevBuf<int> *worklist[kSimt] = {&h->work, &h->work2, &h->work3};
    for (int c = 0; c < kSimt; ++c)
        if (any_c[c] || c == first_c) worklist[c]->ensure(std::max<int64_t>(nslot, 1));
    // rank of every upper slot among the upper slots (the products store
    // only those; compaction writes the lower blocks as transposes)
    h->uidx.ensure(nslot + 1);
    h->scan_tmp_s.ensure(scan_tmp_elems((int)nslot + 1));
    launch_upper_flags(h->slot_row.p, mcol, nslot, h->uidx.p, st);
    scan_exclusive_i32(h->uidx.p, h->uidx.p, (int)nslot, h->scan_tmp_s.p, st);
    int hq[2] = {0, 0};
    d2h(&hq[0], h->counters.p + 2, 1, st);
    d2h(&hq[1], h->uidx.p + nslot, 1, st);
    sync(h);
    if (hq[0]) throw Error{RDM_ECUDA, "internal error: pair lists inconsistent with the mask (code " + std::to_string(hq[0]) + ")"};
    const int64_t nupper = hq[1];

    // Numeric phase, fused truncation and compaction, one group of
    // consecutive super-rows (the block rows of a tensor-core tile, 128 / b of
    // them, of one job) at a time: the buffer of
    // untruncated blocks holds one group's upper slots.  A lower block's
    // upper partner lies in an earlier row, so it is in the same group or
    // already compacted; the result does not depend on the grouping.
    const size_t slot_bytes = bb * sizeof(double);
    int64_t budget = nupper;
    if (h->prm.chunk_mb > 0) {
        budget = std::max<int64_t>(1, (int64_t)(((size_t)h->prm.chunk_mb << 20) / slot_bytes));
    } else if ((size_t)nupper > h->out_val.cap / bb) {
        size_t fr = 0, totm = 0;
        RDM_CUDA_TRY(cudaMemGetInfo(&fr, &totm));
        // at most 1/16 of the device (at least 4 GiB) and what is free: the
        // current buffer is released before the new one is made; room is kept
        // for the output set (about the size of the input set) and a margin
        // for the plans, pair and work lists
        const size_t held = h->out_val.cap * sizeof(double);
        const size_t out_have = out.val.cap * sizeof(double);
        const size_t out_need = (size_t)in.total * bb * sizeof(double) * 9 / 8;
        const size_t reserve = (out_need > out_have ? out_need - out_have : 0) + (size_t(4) << 30);
        const size_t avail = fr + held > reserve ? fr + held - reserve : 0;
        const size_t cap = std::min(avail, std::max(totm / 16, size_t(4) << 30));
        budget = std::max<int64_t>(1, (int64_t)(cap / slot_bytes));
    }
    const int TR = tc_tile_rows(b), NBT = (NB + TR - 1) / TR, nunit = njob * NBT;
    auto unit_row = [&](int u) {   // first flat row of super-row unit u (u = nunit: nrows)
        if (u >= nunit) return nrows;
        return (u / NBT) * NB + TR * (u % NBT);
    };
    std::vector<int> gunit{0};          // first unit of every group
    std::vector<int> hrp, hurp;         // host out_rp and upper ranks at row starts (several groups)
    if (nupper <= budget) {
        gunit.push_back(nunit);
    } else {
        h->urp.ensure(nrows + 1);
        launch_gather_i32(h->out_rp.p, h->uidx.p, nrows, h->urp.p, st);
        hrp.resize(nrows + 1);
        hurp.resize(nrows + 1);
        d2h(hrp.data(), h->out_rp.p, nrows + 1, st);
        d2h(hurp.data(), h->urp.p, nrows + 1, st);
        sync(h);
        int u = 0;
        while (u < nunit) {
            int v = u + 1;
            while (v < nunit && hurp[unit_row(v + 1)] - hurp[unit_row(u)] <= budget) ++v;
            gunit.push_back(v);
            u = v;
        }
    }
    const int ngroup = (int)gunit.size() - 1;
    ss.groups = ngroup;
    auto gslot = [&](int u) -> int64_t { return ngroup == 1 ? (u == 0 ? 0 : nslot) : hrp[unit_row(u)]; };
    auto gupper = [&](int u) -> int64_t { return ngroup == 1 ? (u == 0 ? 0 : nupper) : hurp[unit_row(u)]; };
    int64_t gmax = 1;
    for (int g = 0; g < ngroup; ++g) gmax = std::max<int64_t>(gmax, gupper(gunit[g + 1]) - gupper(gunit[g]));
    h->out_val.ensure((size_t)gmax * bb);
    h->out_nrm.ensure(std::max<int64_t>(nslot, 1));
    h->keep.ensure(std::max<int64_t>(nslot, 1));
    h->dest.ensure(std::max<int64_t>(nslot, 1));
    h->cnt_rows.ensure(nrows + 1);
    out.row_ptr.ensure(nrows + 1);
    int kept = 0;
    float t_simt[kSimt] = {0, 0, 0}, t_tc = 0, t_cmp = 0, t_oz = 0;
    const int ev_simt[kSimt] = {5, 6, 4};   // events after each CUDA-core class
    for (int g = 0; g < ngroup; ++g) {
        const int ua = gunit[g], ub = gunit[g + 1];
        const int64_t s0 = gslot(ua), s1 = gslot(ub), u0 = gupper(ua);
        const int r0 = unit_row(ua), nr = unit_row(ub) - r0;
        RDM_CUDA_TRY(cudaMemsetAsync(h->counters.p + 3, 0, kSimt * sizeof(int), st));
        // CUDA-core work per class: the selected jobs, and in the first class
        // the copies of converged systems
        for (int c = 0; c < kSimt; ++c)
            if (any_c[c] || c == first_c)
                launch_build_work(h->slot_row.p, mcol, s0, s1, worklist[c]->p, h->counters.p + 3 + c, st,
                                  h->sd.sys_of_row.p, h->sd.active.p, h->slot_job.p, h->sd.tier.p, cm[c],
                                  c == first_c ? 1 : 0);
        TcPlan plan{}, oplan{};
        if (tc) plan = build_tc_plan(in, jt, h->sd, h->out_rp.p, mcol, h->tcw, tcm, ua, ub, st);
        if (any_oz) oplan = build_oz_plan(in, jt, h->sd, h->out_rp.p, mcol, h->tcw_oz, ozm, ua, ub, st);
        const bool tc_g = tc && plan.ntile > 0;
        const bool oz_g = any_oz && oplan.ntile > 0;
        int nwork[kSimt];
        d2h(nwork, h->counters.p + 3, kSimt, st);
        sync(h);

        NumArgs a{};
        a.in_val = in.val.p; a.in_nrm = in.nrm.p;
        a.in_f32 = f32_planes ? in.opf32.p : nullptr;
        a.in_f32lo = any_c[1] ? in.opf32lo.p : nullptr;
        a.pair_a = h->pair_a.p; a.pair_b = h->pair_b.p; a.pair_off = h->pair_off.p;
        a.slot_row = h->slot_row.p; a.slot_job = h->slot_job.p; a.slot_x = h->slot_x.p; a.slot_t = h->slot_t.p;
        a.sys_of_row = h->sd.sys_of_row.p;
        a.c_lin = h->sd.c_lin.p; a.c_sq = h->sd.c_sq.p; a.tau0 = h->sd.tau0.p; a.tau1 = h->sd.tau1.p;
        a.active = h->sd.active.p;
        for (int p = 0; p < njob; ++p) a.job_tau_sel[p] = jt.job[p].tau_sel;
        a.out_val = h->out_val.p; a.out_nrm = h->out_nrm.p; a.keep = h->keep.p;
        a.uidx = h->uidx.p; a.u0 = u0; a.b = b;
        h->work_ctr.ensure(kSimt);
        RDM_CUDA_TRY(cudaMemsetAsync(h->work_ctr.p, 0, kSimt * sizeof(int), st));
        RDM_CUDA_TRY(cudaEventRecord(h->ev[1], st));
        const long long lg = g_kernel_launches;
        for (int c = 0; c < kSimt; ++c) {
            if (nwork[c]) {
                NumArgs ac = a;
                ac.work = worklist[c]->p;
                ac.nwork = nwork[c];
                ac.work_next = h->work_ctr.p + c;
                launch_numeric_simt(ac, simt_ar[c], st);
            }
            RDM_CUDA_TRY(cudaEventRecord(h->ev[ev_simt[c]], st));
        }
        ss.simt_launches += (int)(g_kernel_launches - lg);
        if (tc_g) {
            const long long lt = g_kernel_launches;
            ss.issued_tc += launch_numeric_tc(a, in, jt, tc_ar, h->tcw, NB, plan, st);
            ss.tc_launches += (int)(g_kernel_launches - lt);
        }
        RDM_CUDA_TRY(cudaEventRecord(h->ev[2], st));
        if (oz_g) {
            const long long lt = g_kernel_launches;
            ss.issued_oz += launch_numeric_oz(a, in, mcol, h->ozw, h->tcw_oz, oplan, st);
            ss.oz_launches += (int)(g_kernel_launches - lt);
        }
        RDM_CUDA_TRY(cudaEventRecord(h->ev[7], st));

        // compaction of the group's rows, appended after the previous groups
        CompactArgs ca{};
        ca.out_rp = h->out_rp.p; ca.out_col = mcol; ca.slot_row = h->slot_row.p; ca.slot_t = h->slot_t.p;
        ca.uidx = h->uidx.p; ca.out_val = h->out_val.p; ca.out_nrm = h->out_nrm.p; ca.keep = h->keep.p;
        ca.u0 = u0; ca.dest = h->dest.p; ca.new_rp = out.row_ptr.p; ca.r0 = r0; ca.nrows = nr; ca.b = b;
        launch_compact_count(ca, h->cnt_rows.p, st);
        scan_exclusive_i32(h->cnt_rows.p, out.row_ptr.p + r0, nr, h->scan_tmp32.p, st, kept);
        int kept_end = 0;
        d2h(&kept_end, out.row_ptr.p + r0 + nr, 1, st);
        int tc_err = 0, oz_err = 0;
        if (tc_g) d2h(&tc_err, h->tcw.counters.p, 1, st);
        if (oz_g) d2h(&oz_err, h->tcw_oz.counters.p, 1, st);
        sync(h);
        tc_err |= oz_err;
        if (tc_err & 8) throw Error{RDM_EBADBSR, "an operand's block pattern is not symmetric"};
        if (tc_err)
            throw Error{tc_err & 1 ? RDM_ETIMEOUT : RDM_ECUDA,
                        "tensor-core product kernel failed (code " + std::to_string(tc_err) + ")"};
        if (g == 0) {
            // the output set's old contents are dead; reserve about the input's size
            const int64_t want = ngroup > 1 ? std::max<int64_t>(kept_end, in.total) : kept_end;
            out.col.ensure(std::max<int64_t>(want, 1));
            out.val.ensure((size_t)std::max<int64_t>(want, 1) * bb);
            out.nrm.ensure(std::max<int64_t>(want, 1));
        } else {
            out.col.grow_keep(std::max(kept_end, 1), kept, st);
            out.val.grow_keep((size_t)std::max(kept_end, 1) * bb, (size_t)kept * bb, st);
            out.nrm.grow_keep(std::max(kept_end, 1), kept, st);
        }
        ca.new_col = out.col.p; ca.new_val = out.val.p; ca.new_nrm = out.nrm.p;
        ca.src = h->cpsrc.ensure(std::max(kept_end - kept, 1));
        ca.d0 = kept;
        launch_compact_copy(ca, kept_end, st);
        kept = kept_end;
        RDM_CUDA_TRY(cudaEventRecord(h->ev[3], st));
        RDM_CUDA_TRY(cudaEventSynchronize(h->ev[3]));
        float mc[kSimt] = {0, 0, 0}, m42 = 0, m23 = 0, moz = 0;
        cudaEventElapsedTime(&mc[0], h->ev[1], h->ev[ev_simt[0]]);             // FP64 class
        cudaEventElapsedTime(&mc[1], h->ev[ev_simt[0]], h->ev[ev_simt[1]]);    // double-FP32 class
        cudaEventElapsedTime(&mc[2], h->ev[ev_simt[1]], h->ev[ev_simt[2]]);    // FP32 class (and copies)
        cudaEventElapsedTime(&m42, h->ev[ev_simt[2]], h->ev[2]);               // tensor-core launch
        cudaEventElapsedTime(&moz, h->ev[2], h->ev[7]);                        // slice-product launch
        cudaEventElapsedTime(&m23, h->ev[7], h->ev[3]);                        // compaction
        for (int c = 0; c < kSimt; ++c) t_simt[c] += mc[c];
        t_tc += m42; t_cmp += m23; t_oz += moz;
    }
    ss.bytes = ((double)in.total * (tc ? 4.0 : 8.0) + (any_oz ? (double)in.nnzb[0] * 14.0 : 0.0) +
                (double)nupper * 8.0) * (double)bb;
    out.total = kept;
    std::vector<int> rp(nrows + 1);
    d2h(rp.data(), out.row_ptr.p, nrows + 1, st);
    sync(h);
    float mall = 0;
    cudaEventElapsedTime(&mall, h->ev[0], h->ev[3]);
    ss.ms[1] = t_tc;          // tensor-core products
    ss.ms[2] = t_simt[0];     // FP64 products
    ss.ms[3] = t_simt[2];     // FP32 products (and copies of converged systems)
    ss.ms[4] = t_cmp;
    ss.ms[5] = t_simt[1];     // double-FP32 products
    ss.ms[6] = t_oz;          // tensor-core slice products
    ss.ms[0] = std::max(0.f, mall - (t_simt[0] + t_simt[1] + t_simt[2] + t_tc + t_cmp + t_oz));  // mask, lists, plans
    out.nnzb.assign(njob, 0);
    for (int p = 0; p < njob; ++p) out.nnzb[p] = rp[(size_t)(p + 1) * NB] - rp[(size_t)p * NB];
    return ss;
}

JobTable solve_jobs(int nd) {
    JobTable jt{};
    jt.njob = 1 + nd;
    jt.job[0] = Job{0, 0, 1, {0, 0}, {0, 0}, 0};
    for (int d = 0; d < nd; ++d) jt.job[1 + d] = Job{1 + d, 1 + d, 2, {0, 1 + d}, {1 + d, 0}, 1};
    return jt;
}

// per-system stats of the current X: [S][3+nd]
std::vector<double> stats(rdm_handle *h, MatSet &X) {
    const int nq = 3 + h->nd;
    h->row_part.ensure((size_t)nq * h->NB);
    h->sys_q.ensure((size_t)nq * h->S);
    launch_row_stats(X.row_ptr.p, X.col.p, X.val.p, X.nmat, h->NB, h->bs, h->H0.row_ptr.p,
                     h->H0.col.p, h->H0.val.p, h->row_part.p, h->stream);
    launch_sys_sum(h->row_part.p, nq, h->NB, h->sd.row0.p, h->sd.nbs.p, h->S, h->sys_q.p, h->stream);
    std::vector<double> q((size_t)nq * h->S);
    d2h(q.data(), h->sys_q.p, q.size(), h->stream);
    sync(h);
    return q;
}

// ---------------------------------------------------------------------------
// non-orthogonal basis: the Loewdin transform of Sec. 2.2 with the block
// products of the solve (FP64, truncated at tau)
// ---------------------------------------------------------------------------

// out = matrices [first, first + count) of each listed set, in that order
struct SetRange {
    const MatSet *m;
    int first, count;
};
void concat(rdm_handle *h, std::initializer_list<SetRange> parts, MatSet &out) {
    const int NB = h->NB, b = h->bs;
    const size_t bb = (size_t)b * b;
    int nmat = 0;
    int64_t total = 0;
    std::vector<std::vector<int>> rps;
    for (const auto &r : parts) {
        std::vector<int> rp((size_t)r.m->nmat * NB + 1);
        d2h(rp.data(), r.m->row_ptr.p, rp.size(), h->stream);
        rps.push_back(std::move(rp));
        nmat += r.count;
    }
    sync(h);
    std::vector<int> rp((size_t)nmat * NB + 1);
    out.nmat = nmat;
    out.NB = NB;
    out.b = b;
    out.nnzb.assign(nmat, 0);
    int m = 0;
    for (size_t k = 0; k < parts.size(); ++k) {
        const SetRange &r = *(parts.begin() + k);
        for (int q = r.first; q < r.first + r.count; ++q, ++m) {
            const int a0 = rps[k][(size_t)q * NB];
            for (int i = 0; i < NB; ++i) rp[(size_t)m * NB + i] = (int)(total + rps[k][(size_t)q * NB + i] - a0);
            out.nnzb[m] = rps[k][(size_t)(q + 1) * NB] - a0;
            total += out.nnzb[m];
        }
    }
    rp[(size_t)nmat * NB] = (int)total;
    out.total = total;
    out.row_ptr.ensure(rp.size());
    out.col.ensure(std::max<int64_t>(total, 1));
    out.val.ensure((size_t)std::max<int64_t>(total, 1) * bb);
    out.nrm.ensure(std::max<int64_t>(total, 1));
    h2d(out.row_ptr.p, rp.data(), rp.size(), h->stream);
    int64_t off = 0;
    for (size_t k = 0; k < parts.size(); ++k) {
        const SetRange &r = *(parts.begin() + k);
        const int64_t a0 = rps[k][(size_t)r.first * NB], a1 = rps[k][(size_t)(r.first + r.count) * NB];
        if (a1 > a0) {
            RDM_CUDA_TRY(cudaMemcpyAsync(out.col.p + off, r.m->col.p + a0, (a1 - a0) * sizeof(int),
                                         cudaMemcpyDeviceToDevice, h->stream));
            RDM_CUDA_TRY(cudaMemcpyAsync(out.val.p + off * bb, r.m->val.p + a0 * bb, (a1 - a0) * bb * sizeof(double),
                                         cudaMemcpyDeviceToDevice, h->stream));
        }
        off += a1 - a0;
    }
    launch_block_norms(out.val.p, out.nrm.p, total, b, h->stream);
}

// every job of jt, C = c_lin X + c_sq (A B [+ B A]) with per-system
// coefficients, in arithmetic `ar`, for every system
void set_products(rdm_handle *h, MatSet &in, const JobTable &jt, const std::vector<double> &cl,
                  const std::vector<double> &cq, double tau, Arith ar, MatSet &out) {
    const int S = h->S;
    std::vector<double> t(S, tau);
    std::vector<int> one(S, 1), zero(S, 0);
    h2d(h->sd.c_lin.p, cl.data(), S, h->stream);
    h2d(h->sd.c_sq.p, cq.data(), S, h->stream);
    h2d(h->sd.tau0.p, t.data(), S, h->stream);
    h2d(h->sd.tau1.p, t.data(), S, h->stream);
    h2d(h->sd.active.p, one.data(), S, h->stream);
    h2d(h->sd.tier.p, zero.data(), S, h->stream);
    Arith tab[kMaxTiers][kMaxJobs];
    for (int p = 0; p < kMaxJobs; ++p) tab[0][p] = ar;
    multiply(h, in, out, jt, tab, 1u);
}

// the same with one coefficient pair, in FP64
void fp64_products(rdm_handle *h, MatSet &in, const JobTable &jt, double c_lin, double c_sq, double tau,
                   MatSet &out) {
    set_products(h, in, jt, std::vector<double>(h->S, c_lin), std::vector<double>(h->S, c_sq), tau, AR_FP64, out);
}

// FP64-class products: double-FP32 at b = 32 (about 46 bits), FP64 otherwise
void fp64_class_products(rdm_handle *h, MatSet &in, const JobTable &jt, const std::vector<double> &cl,
                         const std::vector<double> &cq, double tau, MatSet &out) {
    set_products(h, in, jt, cl, cq, tau, h->bs == 32 ? AR_FF : AR_FP64, out);
}

// Job: out p = c_lin X_x + c_sq (A B + B A), or A A (a == b, one term)
Job sym_job(int out, int x, int a, int b) { return a == b ? Job{out, x, 1, {a, a}, {a, a}, 0} : Job{out, x, 2, {a, b}, {b, a}, 0}; }

// identity matrix of the batch layout: diagonal blocks only
void make_identity(rdm_handle *h, MatSet &I) {
    const int NB = h->NB, b = h->bs;
    std::vector<int> rp(NB + 1), col(NB);
    for (int i = 0; i <= NB; ++i) rp[i] = i;
    for (int i = 0; i < NB; ++i) col[i] = i;
    I.nmat = 1; I.NB = NB; I.b = b; I.total = NB; I.nnzb.assign(1, NB);
    I.row_ptr.ensure(NB + 1); I.col.ensure(std::max(NB, 1)); I.val.ensure((size_t)std::max(NB, 1) * b * b);
    I.nrm.ensure(std::max(NB, 1));
    h2d(I.row_ptr.p, rp.data(), rp.size(), h->stream);
    h2d(I.col.p, col.data(), col.size(), h->stream);
    launch_identity_blocks(I.val.p, NB, b, h->stream);
    launch_block_norms(I.val.p, I.nrm.p, NB, b, h->stream);
}

// M -> Z M Z for the k matrices of `ms` (Z = S^(-1/2), L = Z^2 = S^(-1)), with
// products of symmetric matrices only:  Z M Z = (Z K + K Z)/2 - (L M + M L)/2,
// K = Z M + M Z.
void lowdin_apply(rdm_handle *h, MatSet &ms, MatSet &out, double tau) {
    const int k = ms.nmat;
    MatSet in, K, M1;
    JobTable jt{};
    jt.njob = k;
    concat(h, {{&h->Zm, 0, 1}, {&ms, 0, k}}, in);
    for (int m = 0; m < k; ++m) jt.job[m] = sym_job(m, -1, 0, 1 + m);
    fp64_products(h, in, jt, 0.0, 1.0, tau, K);
    concat(h, {{&h->Zm, 0, 1}, {&K, 0, k}}, in);
    fp64_products(h, in, jt, 0.0, 1.0, tau, M1);
    K.release();
    concat(h, {{&M1, 0, k}, {&h->Lm, 0, 1}, {&ms, 0, k}}, in);
    for (int m = 0; m < k; ++m) jt.job[m] = sym_job(m, m, k, k + 1 + m);
    fp64_products(h, in, jt, 0.5, -0.5, tau, out);
}

// Z = S^(-1/2) by the coupled Newton-Schulz iteration (Higham): Y_0 = S / c,
// Z_0 = I with c a Gershgorin bound of every S; T = (3 I - Z Y) / 2,
// Y <- Y T, Z <- T Z until ||T - I||_F stops shrinking below 1e-6 sqrt(n) or
// drops below 1e-13 sqrt(n); then Z / sqrt(c).  Z and Y are polynomials in
// S, so every product is one of commuting symmetric matrices (taken as
// (A B + B A) / 2).  Then H0 and H1 are transformed in place.
void lowdin_forward(rdm_handle *h) {
    const int S = h->S, NB = h->NB, b = h->bs, nd = h->nd;
    const double tau = h->prm.tau;
    cudaStream_t st = h->stream;
    // c: Gershgorin upper bound of each system's S
    h->row_lo.ensure(NB);
    h->row_hi.ensure(NB);
    launch_gershgorin(h->Sm.row_ptr.p, h->Sm.col.p, h->Sm.val.p, NB, b, h->sd.sys_of_row.p, h->sd.row0.p,
                      h->sd.n_orb.p, h->row_lo.p, h->row_hi.p, st);
    launch_sys_minmax(h->row_lo.p, h->row_hi.p, h->sd.row0.p, h->sd.nbs.p, S, h->sd.emin.p, h->sd.emax.p, st);
    std::vector<double> lo(S), hi(S);
    d2h(lo.data(), h->sd.emin.p, S, st);
    d2h(hi.data(), h->sd.emax.p, S, st);
    sync(h);
    std::vector<double> inv_c(S), inv_sqrt_c(S);
    for (int s = 0; s < S; ++s) {
        if (!(hi[s] > 0)) throw Error{RDM_EBADBSR, "overlap matrix has no positive Gershgorin bound"};
        inv_c[s] = 1.0 / hi[s];
        inv_sqrt_c[s] = 1.0 / std::sqrt(hi[s]);
    }
    DevBuf<double> fac;
    fac.ensure(S);
    h2d(fac.p, inv_c.data(), S, st);
    MatSet Y, Z, I, T, in, YZ;
    concat(h, {{&h->Sm, 0, 1}}, Y);
    launch_scale_sys(Y.row_ptr.p, Y.col.p, Y.val.p, NB, b, h->sd.sys_of_row.p, h->sd.row0.p, h->sd.n_orb.p, fac.p, 1,
                     Y.val.p, st);
    launch_block_norms(Y.val.p, Y.nrm.p, Y.total, b, st);
    make_identity(h, I);
    concat(h, {{&I, 0, 1}}, Z);
    JobTable jt{};
    double prev = 1e300;
    int it = 0;
    const int nq = 3;     // Tr T, ||T||^2, Tr(T T) from the stats of a one-matrix set
    for (it = 0; it < 100; ++it) {
        concat(h, {{&Z, 0, 1}, {&Y, 0, 1}, {&I, 0, 1}}, in);
        jt.njob = 1;
        jt.job[0] = sym_job(0, 2, 0, 1);
        fp64_products(h, in, jt, 1.5, -0.25, tau, T);       // T = 3/2 I - (Z Y + Y Z)/4
        // ||T - I||_F^2 = ||T||^2 - 2 Tr T + n per system (padding rows included)
        h->row_part.ensure((size_t)nq * NB);
        h->sys_q.ensure((size_t)nq * S);
        launch_row_stats(T.row_ptr.p, T.col.p, T.val.p, 1, NB, b, T.row_ptr.p, T.col.p, T.val.p, h->row_part.p, st);
        launch_sys_sum(h->row_part.p, nq, NB, h->sd.row0.p, h->sd.nbs.p, S, h->sys_q.p, st);
        std::vector<double> q((size_t)nq * S);
        d2h(q.data(), h->sys_q.p, q.size(), st);
        sync(h);
        double dev = 0;
        for (int s = 0; s < S; ++s) {
            const double n = (double)h->nbs[s] * b;
            const double d2 = q[(size_t)s * nq + 1] - 2.0 * q[(size_t)s * nq] + n;
            dev = std::max(dev, std::sqrt(std::max(d2, 0.0)) / std::sqrt(n));
        }
        concat(h, {{&Y, 0, 1}, {&T, 0, 1}, {&Z, 0, 1}}, in);
        jt.njob = 2;
        jt.job[0] = sym_job(0, -1, 0, 1);                    // Y T
        jt.job[1] = sym_job(1, -1, 1, 2);                    // T Z
        fp64_products(h, in, jt, 0.0, 0.5, tau, YZ);
        concat(h, {{&YZ, 0, 1}}, Y);
        concat(h, {{&YZ, 1, 1}}, Z);
        if (dev < 1e-13 || (dev < 1e-6 && dev >= 0.5 * prev)) break;
        if (!std::isfinite(dev) || (it > 20 && dev > 1.0))
            throw Error{RDM_EBADBSR, "the Newton-Schulz iteration for S^(-1/2) does not converge (is S positive definite?)"};
        prev = dev;
    }
    h->lowdin_iters = it + 1;
    h2d(fac.p, inv_sqrt_c.data(), S, st);
    concat(h, {{&Z, 0, 1}}, h->Zm);
    launch_scale_sys(h->Zm.row_ptr.p, h->Zm.col.p, h->Zm.val.p, NB, b, h->sd.sys_of_row.p, h->sd.row0.p,
                     h->sd.n_orb.p, fac.p, 0, h->Zm.val.p, st);
    launch_block_norms(h->Zm.val.p, h->Zm.nrm.p, h->Zm.total, b, st);
    Y.release(); Z.release(); T.release(); YZ.release(); I.release();
    concat(h, {{&h->Zm, 0, 1}}, in);
    jt.njob = 1;
    jt.job[0] = sym_job(0, -1, 0, 0);
    fp64_products(h, in, jt, 0.0, 1.0, tau, h->Lm);       // L = Z Z = S^-1
    // H0 and every H1 in the orthogonal form
    MatSet hs, ho;
    if (nd) concat(h, {{&h->H0, 0, 1}, {&h->H1, 0, nd}}, hs);
    else concat(h, {{&h->H0, 0, 1}}, hs);
    lowdin_apply(h, hs, ho, tau);
    concat(h, {{&ho, 0, 1}}, h->H0);
    if (nd) concat(h, {{&ho, 1, nd}}, h->H1);
}

// P -> Z P Z for the solve's result set (P0 and every P1)
void lowdin_back(rdm_handle *h) {
    MatSet &X = h->X[h->cur];
    MatSet xs, out;
    concat(h, {{&X, 0, X.nmat}}, xs);
    lowdin_apply(h, xs, out, h->prm.tau);
    X.release();
    concat(h, {{&out, 0, out.nmat}}, X);
}

// alpha[g][d] = -spin <P1_d, H1_g> (Eq. polar) for every pair of the solved
// directions, from the result set (P0, P1_1..P1_nd) and the H1 set
void compute_alpha(rdm_handle *h) {
    const int S = h->S, NB = h->NB, nd = h->nd, b = h->bs;
    cudaStream_t st = h->stream;
    MatSet &Xf = h->X[h->cur];
    h->alpha.assign((size_t)S * 9, NAN);
    if (!nd) return;
    const int nq = nd * nd;
    h->row_part.ensure((size_t)nq * NB);
    h->sys_q.ensure((size_t)nq * S);
    launch_row_dots(Xf.row_ptr.p + NB, Xf.col.p, Xf.val.p, nd, h->H1.row_ptr.p, h->H1.col.p, h->H1.val.p, nd, NB, b,
                    h->row_part.p, st);
    launch_sys_sum(h->row_part.p, nq, NB, h->sd.row0.p, h->sd.nbs.p, S, h->sys_q.p, st);
    std::vector<double> dq((size_t)nq * S);
    d2h(dq.data(), h->sys_q.p, dq.size(), st);
    sync(h);
    for (int s = 0; s < S; ++s)
        for (int g = 0; g < nd; ++g)
            for (int d = 0; d < nd; ++d)
                h->alpha[(size_t)s * 9 + 3 * h->dirs[g] + h->dirs[d]] =
                    -h->prm.spin_factor * dq[(size_t)s * nq + g * nd + d];
}

int run_solve(rdm_handle *h, rdm_info *info_out) {
    DeviceGuard dg(h->device);
    if (h->hs.empty()) return fail(h, RDM_ESTATE, "no system uploaded");
    if (!tc_block_ok(h->prm.mode, h->bs))
        return fail(h, RDM_EINVAL, "the mixed modes run their products on the tensor cores, which take 16 x 16, 32 x 32 or 64 x 64 blocks");
    auto t_start = std::chrono::steady_clock::now();
    const long long launches0 = g_kernel_launches;
    if (h->keep_assembled) init_x(h);
    else assemble(h);
    if (h->has_s && !h->keep_assembled) {
        lowdin_forward(h);   // H0, H1 to the orthogonal form (Sec. 2.2)
        init_x(h);
    }
    const int S = h->S, NB = h->NB, nd = h->nd, b = h->bs;
    const rdm_params &P = h->prm;
    cudaStream_t st = h->stream;
    const bool mixed = P.mode == RDM_MODE_MIXED_BF16 || P.mode == RDM_MODE_MIXED_FP16;
    const bool lowprec = P.mode != RDM_MODE_FP64;
    const int final_tier = final_tier_of(P.mode);

    // Gershgorin bounds and the initial matrices
    h->row_lo.ensure(NB);
    h->row_hi.ensure(NB);
    launch_gershgorin(h->H0.row_ptr.p, h->H0.col.p, h->H0.val.p, NB, b, h->sd.sys_of_row.p,
                      h->sd.row0.p, h->sd.n_orb.p, h->row_lo.p, h->row_hi.p, st);
    launch_sys_minmax(h->row_lo.p, h->row_hi.p, h->sd.row0.p, h->sd.nbs.p, S, h->sd.emin.p,
                      h->sd.emax.p, st);
    MatSet &X = h->X[0];
    launch_init_scale(h->H0.row_ptr.p, h->H0.col.p, h->H0.val.p, X.val.p, X.nrm.p, NB, NB, b,
                      h->sd.sys_of_row.p, h->sd.row0.p, h->sd.n_orb.p, h->sd.emin.p, h->sd.emax.p, 1, st);
    if (nd) {
        const size_t bb = (size_t)b * b;
        // X1 blocks follow the X0 blocks; the H1 set's row_ptr indexes its own arrays
        launch_init_scale(h->H1.row_ptr.p, h->H1.col.p, h->H1.val.p, X.val.p + h->H0.total * bb,
                          X.nrm.p + h->H0.total, nd * NB, NB, b, h->sd.sys_of_row.p,
                          h->sd.row0.p, h->sd.n_orb.p, h->sd.emin.p, h->sd.emax.p, 0, st);
    }
    std::vector<double> emin(S), emax(S);
    d2h(emin.data(), h->sd.emin.p, S, st);
    d2h(emax.data(), h->sd.emax.p, S, st);
    sync(h);
    for (int s = 0; s < S; ++s)
        if (!(emax[s] > emin[s])) return fail(h, RDM_EBADBSR, "degenerate spectrum bounds (eps_max <= eps_min)");

    std::vector<SysState> ss(S);
    std::vector<double> nocc(S);
    for (int s = 0; s < S; ++s) nocc[s] = (double)(h->hs[s].n_elec / 2);
    const double tau0 = P.tau, tau1 = P.tau_x1 < 0 ? P.tau : P.tau_x1;
    const double tau_ref = P.tau_refine < 0 ? P.tau : P.tau_refine;
    const double tau1_ref = P.tau_x1 < 0 ? tau_ref : P.tau_x1;
    h->log.clear();
    JobTable jt = solve_jobs(nd);
    std::vector<double> c_lin(S), c_sq(S), t0(S), t1(S);
    std::vector<int> act(S);
    double useful = 0, issued = 0, nbytes = 0, flops_tc = 0, flops_64 = 0, flops_32 = 0, flops_ff = 0, flops_oz = 0;
    double kms[7] = {0, 0, 0, 0, 0, 0, 0};
    int tc_launches = 0, oz_launches = 0, simt_launches = 0, max_groups = 1;
    g_dev_bytes_peak = g_dev_bytes.load();
    cudaEvent_t ev0, ev1;
    RDM_CUDA_TRY(cudaEventCreate(&ev0));
    RDM_CUDA_TRY(cudaEventCreate(&ev1));
    int it = 0;
    bool any_active = true;
    std::vector<double> q;
    for (it = 0; it <= P.max_iter; ++it) {
        MatSet &Xc = h->X[h->cur];
        q = stats(h, Xc);
        const int nq = 3 + nd;
        any_active = false;
        for (int s = 0; s < S; ++s) {
            SysState &y = ss[s];
            act[s] = 0;
            c_lin[s] = 1.0;
            c_sq[s] = 0.0;
            t0[s] = tau0;
            t1[s] = tau1;
            if (!y.active) continue;
            const double tr = q[(size_t)s * nq + 0], sumsq = q[(size_t)s * nq + 1];
            const double e = tr - sumsq;
            const double eb0 = q[(size_t)s * nq + 2];
            // close the log record of the previous step with the new band energies
            for (auto r = h->log.rbegin(); r != h->log.rend(); ++r)
                if (r->sys == s) {
                    r->eb0 = eb0;
                    for (int d = 0; d < nd; ++d) r->eb1[d] = q[(size_t)s * nq + 3 + d];
                    break;
                }
            const int n = y.iters;   // number of updates done so far
            bool stop = false;
            if (!std::isfinite(tr) || !std::isfinite(sumsq)) {
                y.active = false;
                continue;
            }
            // band-energy stop (Sec. 2.3 tolerance), only in the final tier
            if (y.have_eb && P.tol > 0 && n >= std::max(2, P.min_iter) && y.tier == final_tier) {
                double d0 = fabs(eb0 - y.eb0), d1 = 0;
                for (int d = 0; d < nd; ++d) d1 = std::max(d1, fabs(q[(size_t)s * nq + 3 + d] - y.eb1[d]));
                if (d0 < P.tol && d1 < P.tol) stop = true;
            }
            // idempotency stall
            const double stall_tol = P.stall_tol;
            y.e_hist.push_back(e);
            const size_t E = y.e_hist.size();
            // stall window of the precision ladder (R10): |e_n| >= |e_{n-W}| / 2
            const int W = P.stall_window > 0 ? P.stall_window : 2;
            const bool stalled = (int)E >= W + 1 && fabs(e) >= 0.5 * fabs(y.e_hist[E - 1 - W]) &&
                                 fabs(e) < 1e-2 * nocc[s];
            if (!stop && n >= std::max(3, P.min_iter) && E >= 3) {
                // FP64: the oracle's stall stop (e not decreased over two iterations, below stall_tol)
                if (!lowprec && stall_tol > 0 && e >= y.e_hist[E - 3] && e < stall_tol) stop = true;
                if (lowprec && y.tier == final_tier && n - y.tier_start >= 2 && stalled) stop = true;
                // mixed modes: X0 refined in FP64 is idempotent to 1e-10 per
                // occupied state (four orders below the truncation error of any
                // useful tau; the FP64 rounding floor is ~1e-12 per state)
                if (mixed && y.tier == final_tier && n - y.tier_start >= 2 &&
                    fabs(e) <= 1e-10 * std::max(1.0, nocc[s]))
                    stop = true;
            }
            y.have_eb = true;
            y.eb0 = eb0;
            for (int d = 0; d < nd; ++d) y.eb1[d] = q[(size_t)s * nq + 3 + d];
            // a response solve of the correction repeats the solve's X0
            // recursion bit for bit (the same inputs, kernels and decisions):
            // it takes exactly as many updates
            if (!h->stop_at.empty()) stop = n >= h->stop_at[s];
            if (stop) {
                y.active = false;
                y.converged = true;
                continue;
            }
            if (n >= P.max_iter) {
                y.active = false;
                continue;
            }
            // tier switch on idempotency stall (mixed modes)
            // a stall moves a system to the next tier (after at least W
            // iterations in a tier above the first, so that the stall is its own)
            if (mixed && y.tier < final_tier && stalled && (y.tier == 0 || n - y.tier_start >= W)) {
                y.tier++;
                y.tier_start = n;
            }
            // branch: trace test of Eq. TC2 (tie -> square, the ">=" of Eq. TC2);
            // forced by the test hook.  Reading where the paper is silent (what TC2
            // does once rounding or the filter pushes eigenvalues out of [0, 1],
            // i.e. e = Tr X - ||X||^2 < 0): the branch alternates with the previous
            // one, so that both spectral edges contract instead of an eigenvalue
            // above 1 being squared again and again.
            //  - FP64 mode: only a clearly negative error, e < -1e-10 N_occ, the
            //    rule of the oracle; rounding at tau = 0 never reaches that level,
            //    the filter at large thresholds does (the trace test alone then
            //    diverges), so FP64 runs follow the oracle step for step.
            //  - reduced-precision modes: any e < 0, since their rounding alone
            //    leaves eigenvalues slightly outside [0, 1].  These trajectories
            //    have no oracle counterpart step for step; only their limits (P0,
            //    P1, alpha) are compared with the oracle.
            int branch = (tr >= nocc[s]) ? 1 : 2;
            if (n > 0 && (lowprec ? e < 0 : e < -1e-10 * std::max(1.0, nocc[s])))
                branch = y.prev_branch == 1 ? 2 : 1;
            if (n < (int)h->forced.size()) branch = h->forced[n];
            y.prev_branch = branch;
            c_lin[s] = branch == 1 ? 0.0 : 2.0;
            c_sq[s] = branch == 1 ? 1.0 : -1.0;
            if (y.tier == final_tier && mixed) {
                t0[s] = tau_ref;
                t1[s] = tau1_ref;
            }
            act[s] = 1;
            any_active = true;
            rdm_iter_log L{};
            L.iter = n;
            L.branch = branch;
            L.tier = y.tier;
            L.sys = s;
            L.trace = tr;
            L.idempotency = e;
            h->log.push_back(L);
        }
        if (!any_active) break;
        // every system computes in its own tier; the kernels select the rows of
        // each tier through per-tier job masks
        Arith tab[kMaxTiers][kMaxJobs];
        unsigned tiers_present = 0;
        std::vector<int> tier_of(S, 0);
        for (int t = 0; t <= final_tier; ++t) tier_arith(P.mode, t, jt.njob, tab[t], P.refine_x1, P.refine_x0, b);
        for (int s = 0; s < S; ++s) {
            tier_of[s] = ss[s].tier;
            if (act[s]) tiers_present |= 1u << ss[s].tier;
        }
        Arith ar[kMaxJobs];   // arithmetic of the lowest tier present (log only)
        for (int p = 0; p < jt.njob; ++p) ar[p] = tab[0][p];
        for (int t = 0; t <= final_tier; ++t)
            if ((tiers_present >> t) & 1u) {
                for (int p = 0; p < jt.njob; ++p) ar[p] = tab[t][p];
                break;
            }
        h2d(h->sd.tier.p, tier_of.data(), S, st);
        h2d(h->sd.c_lin.p, c_lin.data(), S, st);
        h2d(h->sd.c_sq.p, c_sq.data(), S, st);
        h2d(h->sd.tau0.p, t0.data(), S, st);
        h2d(h->sd.tau1.p, t1.data(), S, st);
        h2d(h->sd.active.p, act.data(), S, st);
        RDM_CUDA_TRY(cudaEventRecord(ev0, st));
        MatSet &Xn = h->X[1 - h->cur];
        StepStats sst = multiply(h, Xc, Xn, jt, tab, tiers_present);
        RDM_CUDA_TRY(cudaEventRecord(ev1, st));
        RDM_CUDA_TRY(cudaEventSynchronize(ev1));
        float ms = 0;
        cudaEventElapsedTime(&ms, ev0, ev1);
        const double fpb = 2.0 * b * b * b;
        useful += (double)sst.npairs * fpb;
        flops_tc += (double)sst.pairs_tc * fpb;
        flops_64 += (double)sst.pairs_64 * fpb;
        flops_32 += (double)sst.pairs_32 * fpb;
        flops_ff += (double)sst.pairs_ff * fpb;
        flops_oz += (double)sst.pairs_oz * fpb;
        issued += sst.issued_tc + sst.issued_oz + (double)(sst.pairs_64 + sst.pairs_32 + sst.pairs_ff) * fpb;
        nbytes += sst.bytes;
        tc_launches += sst.tc_launches;
        oz_launches += sst.oz_launches;
        simt_launches += sst.simt_launches;
        max_groups = std::max(max_groups, sst.groups);
        for (int k = 0; k < 7; ++k) kms[k] += sst.ms[k];
        h->cur = 1 - h->cur;
        for (int s = 0; s < S; ++s)
            if (act[s]) {
                ss[s].iters++;
                ss[s].tier_iters[ss[s].tier]++;
            }
        int nstep = 0;
        for (int s = 0; s < S; ++s) nstep += act[s];
        for (auto r = h->log.rbegin(); r != h->log.rend() && nstep > 0; ++r, --nstep) {
            r->ms = ms;
            r->nnzb0 = Xn.nnzb[0];
            for (int d = 0; d < nd; ++d) r->nnzb1[d] = Xn.nnzb[1 + d];
        }
        if (P.verbose) {
            fprintf(stderr,
                    "[rdm] step %d arith %d/%d pairs %lld slots %lld nnzb0 %lld %.3f ms (sym %.2f tc %.2f simt %.2f "
                    "cmp %.2f)\n",
                    it, (int)ar[0], (int)ar[jt.njob - 1], (long long)sst.npairs, (long long)sst.nslot,
                    (long long)Xn.nnzb[0], ms, sst.ms[0], sst.ms[1], sst.ms[2] + sst.ms[3], sst.ms[4]);
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);

    // polarizability: alpha[g][d] = -spin * <P1_d, H1_g>
    MatSet &Xf = h->X[h->cur];
    compute_alpha(h);
    // final pattern on the host for the getters, summary per system
    h->final_rp.resize((size_t)Xf.nmat * NB + 1);
    d2h(h->final_rp.data(), Xf.row_ptr.p, h->final_rp.size(), st);
    sync(h);
    auto t_end = std::chrono::steady_clock::now();
    double wall_ms = std::chrono::duration<double, std::milli>(t_end - t_start).count();
    h->info.assign(S, rdm_info{});
    const int nq = 3 + nd;
    bool all_conv = true;
    for (int s = 0; s < S; ++s) {
        rdm_info &I = h->info[s];
        I.iterations = ss[s].iters;
        I.converged = ss[s].converged ? 1 : 0;
        all_conv = all_conv && ss[s].converged;
        for (int t = 0; t < 4; ++t) I.tier_iters[t] = ss[s].tier_iters[t];
        I.eps_min = emin[s];
        I.eps_max = emax[s];
        I.trace_error = q[(size_t)s * nq] - nocc[s];
        I.idempotency = q[(size_t)s * nq] - q[(size_t)s * nq + 1];
        I.band_energy0 = 0;
        int r0 = h->row0[s], r1 = r0 + h->nbs[s];
        I.nnzb_p0 = h->final_rp[r1] - h->final_rp[r0];
        for (int d = 0; d < nd; ++d)
            I.nnzb_p1[h->dirs[d]] = h->final_rp[(size_t)(1 + d) * NB + r1] - h->final_rp[(size_t)(1 + d) * NB + r0];
        I.time_ms = wall_ms;
        I.useful_flops = useful;
        I.issued_flops = issued;
        for (int k = 0; k < 5; ++k) I.kernel_ms[k] = kms[k];
        I.kernel_ms[6] = kms[5];
        I.kernel_ms[7] = kms[6];
        I.kernel_ms[5] = std::max(0.0, wall_ms - kms[0] - kms[1] - kms[2] - kms[3] - kms[4] - kms[5] - kms[6]);
        I.kernel_flops[0] = flops_tc;
        I.kernel_flops[1] = flops_64;
        I.kernel_flops[2] = flops_32;
        I.kernel_flops[3] = flops_ff;
        I.kernel_flops[4] = flops_oz;
        I.kernel_launches = g_kernel_launches - launches0;
        I.tc_launches = tc_launches;
        I.oz_launches = oz_launches;
        I.simt_launches = simt_launches;
        I.numeric_bytes = nbytes;
        I.device_bytes_peak = (int64_t)g_dev_bytes_peak.load();
        I.product_groups = max_groups;
    }
    // band energy of the result: recompute the stats of the final X
    q = stats(h, Xf);
    for (int s = 0; s < S; ++s) {
        h->info[s].band_energy0 = q[(size_t)s * nq + 2];
        h->info[s].trace_error = q[(size_t)s * nq] - nocc[s];
        h->info[s].idempotency = q[(size_t)s * nq] - q[(size_t)s * nq + 1];
    }
    if (h->has_s && !h->keep_assembled) {
        // P0 and P1 back to the non-orthogonal basis; the summary above stays
        // that of the orthogonal form (Tr P0 = N_occ there)
        lowdin_back(h);
        MatSet &Xb = h->X[h->cur];
        h->final_rp.resize((size_t)Xb.nmat * NB + 1);
        d2h(h->final_rp.data(), Xb.row_ptr.p, h->final_rp.size(), st);
        sync(h);
        for (int s = 0; s < S; ++s) {
            const int r0 = h->row0[s], r1 = r0 + h->nbs[s];
            h->info[s].nnzb_p0 = h->final_rp[r1] - h->final_rp[r0];
            for (int d = 0; d < nd; ++d)
                h->info[s].nnzb_p1[h->dirs[d]] =
                    h->final_rp[(size_t)(1 + d) * NB + r1] - h->final_rp[(size_t)(1 + d) * NB + r0];
            h->info[s].lowdin_iterations = h->lowdin_iters;
        }
    }
    h->conv.assign((size_t)S * 4, {});
    for (int s = 0; s < S; ++s) h->info[s].block_size = b;
    h->solved = true;
    if (info_out) *info_out = h->info[0];
    return all_conv ? RDM_OK : RDM_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// accuracy correction (rdm_params.correct)
// ---------------------------------------------------------------------------

// per system, the largest block norm of the matrices [first, first + count) of
// m (the norms are computed afresh: the assembled H0 and H1 sets carry none)
std::vector<double> sys_max_norm(rdm_handle *h, const MatSet &m, int first, int count) {
    const int NB = h->NB;
    launch_block_norms(m.val.p, m.nrm.p, m.total, h->bs, h->stream);
    std::vector<int> rp((size_t)m.nmat * NB + 1);
    std::vector<float> nrm((size_t)std::max<int64_t>(m.total, 1));
    d2h(rp.data(), m.row_ptr.p, rp.size(), h->stream);
    if (m.total) d2h(nrm.data(), m.nrm.p, (size_t)m.total, h->stream);
    sync(h);
    std::vector<double> mx(h->S, 0.0);
    for (int k = first; k < first + count; ++k)
        for (int s = 0; s < h->S; ++s)
            for (int i = h->row0[s]; i < h->row0[s] + h->nbs[s]; ++i)
                for (int p = rp[(size_t)k * NB + i]; p < rp[(size_t)k * NB + i + 1]; ++p)
                    mx[s] = std::max(mx[s], (double)nrm[p]);
    return mx;
}

// Scale every matrix of m, per system s, by lam_s: the power of two that
// brings the largest block norm of s's matrices nearest to ref_s (1 where
// either is 0).  Returns lam.
std::vector<double> scale_to(rdm_handle *h, MatSet &m, const std::vector<double> &ref) {
    const int S = h->S, NB = h->NB, b = h->bs;
    const std::vector<double> mx = sys_max_norm(h, m, 0, m.nmat);
    std::vector<double> lam(S, 1.0);
    for (int s = 0; s < S; ++s)
        if (mx[s] > 0 && ref[s] > 0) lam[s] = std::ldexp(1.0, (int)std::lround(std::log2(ref[s] / mx[s])));
    DevBuf<double> fac;
    fac.ensure(S);
    h2d(fac.p, lam.data(), S, h->stream);
    for (int k = 0; k < m.nmat; ++k)
        launch_scale_sys(m.row_ptr.p + (size_t)k * NB, m.col.p, m.val.p, NB, b, h->sd.sys_of_row.p, h->sd.row0.p,
                         h->sd.n_orb.p, fac.p, 0, m.val.p, h->stream);
    launch_block_norms(m.val.p, m.nrm.p, m.total, b, h->stream);
    sync(h);
    return lam;
}

// Accuracy correction of P0 and P1.  P0 is fixed by [H0, P0] = 0 with
// P0^2 = P0, P1 by [H0, P1] + [H1, P0] = 0 with P1 = P0 P1 + P1 P0
// (Sec. 2.1).  The reduced-precision tiers leave a small rotation of the
// occupied subspace in P0 (purification drives eigenvalues to 0 and 1 but
// never refers to H0 again, so it does not undo a rotation of the
// eigenvectors) and with it an error in P1.  Both errors are first-order
// responses to symmetric perturbations made of the residuals
// ({A, B} = A B + B A; every product one of symmetric matrices):
//  - P0: dP0 = dP/dH[H'0] with H'0 = [[H0, P0], P0] = 2 G0 - {P0, G0},
//        G0 = {P0, H0} (P0 idempotent);
//  - P1, with the corrected P0: dP1 = dP/dH[H'1] with H'1 = [R1, P0],
//        R1 = [H0, P1] + [H1, P0]:  H'1 = 2 G - {P0, G} + {D, P1},
//        G = {P0, H1}, D = H0 - {P0, H0}; P1 + dP1 is then projected on
//        its occupied-virtual part 2 {P0, X} - {P0, {P0, X}}.
// Each response is one more solve of the same mode with the H' in place of
// H1, scaled per system by a power of two to H1's size so that the solve's
// filter treats it as it treats H1 (a response is linear in its
// perturbation).  The residual products are FP64-class with a filter well
// below tau (rdm_params.correct_tau, by default tau / 100): the residuals are
// small differences of O(1) terms.
int run_solve_corr(rdm_handle *h, rdm_info *info_out) {
    if (!h->prm.correct) return run_solve(h, info_out);
    for (const auto &y : h->hs)
        if (y.has_s) return fail(h, RDM_EINVAL, "correct does not take an overlap matrix");
    int status = run_solve(h, nullptr);
    if (status < 0) return status;
    const auto t0 = std::chrono::steady_clock::now();
    auto tprev = t0;
    auto phase = [&](const char *what) {   // verbose: wall time of each phase
        if (!h->prm.verbose) return;
        sync(h);
        const auto t = std::chrono::steady_clock::now();
        fprintf(stderr, "[rdm] correction: %s %.1f ms\n", what,
                std::chrono::duration<double, std::milli>(t - tprev).count());
        tprev = t;
    };
    const int S = h->S, NB = h->NB, nd = h->nd;
    const int dirs0[3] = {h->dirs[0], h->dirs[1], h->dirs[2]};
    const double tc = h->prm.correct_tau > 0 ? h->prm.correct_tau : h->prm.tau * 1e-2;
    const std::vector<rdm_info> info0 = h->info;
    const std::vector<rdm_iter_log> log0 = h->log;
    h->solved = false;
    struct Reset {
        rdm_handle *h;
        ~Reset() {
            h->keep_assembled = false;
            h->stop_at.clear();
        }
    } reset{h};
    const std::vector<double> c0(S, 0.0), c1(S, 1.0), c2(S, 2.0), cm1(S, -1.0), ch(S, 0.5);
    std::vector<double> cq(S);
    MatSet Pt, H1s, I, A, G0, H0p, P0c, P1c;
    concat(h, {{&h->X[h->cur], 0, 1 + nd}}, Pt);      // P0~, P1~_1..nd
    if (nd) H1s = std::move(h->H1);
    make_identity(h, I);
    // the size each H' is scaled to: H1's largest block norm (H0's without H1)
    const std::vector<double> ref = nd ? sys_max_norm(h, H1s, 0, nd) : sys_max_norm(h, h->H0, 0, 1);
    JobTable jt{};

    // P0: H'0 = 2 G0 - {P0~, G0}, G0 = {P0~, H0}; P0 = P0~ + {I, E0} / (2 lam)
    concat(h, {{&h->H0, 0, 1}, {&Pt, 0, 1}}, A);
    jt.njob = 1;
    jt.job[0] = sym_job(0, -1, 0, 1);
    fp64_class_products(h, A, jt, c0, c1, tc, G0);
    concat(h, {{&Pt, 0, 1}, {&G0, 0, 1}}, A);
    jt.job[0] = sym_job(0, 1, 0, 1);
    fp64_class_products(h, A, jt, c2, cm1, tc, H0p);
    G0.release();
    std::vector<double> lam = scale_to(h, H0p, ref);
    phase("perturbation of P0 (2 products)");
    h->H1 = std::move(H0p);
    h->nd = 1;
    h->dirs[0] = 0;
    h->keep_assembled = true;
    h->stop_at.assign(S, 0);
    for (int s = 0; s < S; ++s) h->stop_at[s] = info0[s].iterations;
    int st = run_solve(h, nullptr);
    if (st < 0) return st;
    if (st == RDM_NOT_CONVERGED) status = st;
    if (h->prm.verbose) {
        const std::vector<double> e = sys_max_norm(h, h->X[h->cur], 1, 1);
        for (int s = 0; s < S; ++s)
            fprintf(stderr, "[rdm] correction of P0, system %d: scale 2^%d, largest block of the response %.3e\n", s,
                    (int)std::lround(std::log2(lam[s])), e[s] / lam[s]);
    }
    phase("response solve for P0");
    concat(h, {{&I, 0, 1}, {&Pt, 0, 1}, {&h->X[h->cur], 1, 1}}, A);
    for (int s = 0; s < S; ++s) cq[s] = 0.5 / lam[s];
    jt.job[0] = sym_job(0, 1, 0, 2);
    fp64_class_products(h, A, jt, c1, cq, tc, P0c);
    phase("corrected P0");

    if (nd) {
        // P1: H'1_d = U_d + {I, V_d} / 2, U_d = 2 G_d - {P0, G_d}, G_d = {P0, H1_d},
        // V_d = {D, P1~_d}, D = H0 - {P0, H0}
        MatSet G, D, U, V, H1p, P1s, W;
        concat(h, {{&P0c, 0, 1}, {&h->H0, 0, 1}, {&H1s, 0, nd}}, A);
        jt.njob = nd;
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, -1, 0, 2 + d);
        fp64_class_products(h, A, jt, c0, c1, tc, G);
        jt.njob = 1;
        jt.job[0] = sym_job(0, 1, 0, 1);
        fp64_class_products(h, A, jt, c1, cm1, tc, D);
        concat(h, {{&P0c, 0, 1}, {&G, 0, nd}}, A);
        jt.njob = nd;
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, 1 + d, 0, 1 + d);
        fp64_class_products(h, A, jt, c2, cm1, tc, U);
        G.release();
        concat(h, {{&D, 0, 1}, {&Pt, 1, nd}}, A);
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, -1, 0, 1 + d);
        fp64_class_products(h, A, jt, c0, c1, tc, V);
        D.release();
        concat(h, {{&I, 0, 1}, {&U, 0, nd}, {&V, 0, nd}}, A);
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, 1 + d, 0, 1 + nd + d);
        fp64_class_products(h, A, jt, c1, ch, tc, H1p);
        U.release();
        V.release();
        lam = scale_to(h, H1p, ref);
        phase("perturbations of P1 (1 + 4 nd products)");
        h->H1 = std::move(H1p);
        h->nd = nd;
        for (int d = 0; d < 3; ++d) h->dirs[d] = dirs0[d];
        st = run_solve(h, nullptr);
        if (st < 0) return st;
        if (st == RDM_NOT_CONVERGED) status = st;
        if (h->prm.verbose) {
            const std::vector<double> e = sys_max_norm(h, h->X[h->cur], 1, nd);
            for (int s = 0; s < S; ++s)
                fprintf(stderr, "[rdm] correction of P1, system %d: scale 2^%d, largest block of the response %.3e\n",
                        s, (int)std::lround(std::log2(lam[s])), e[s] / lam[s]);
        }
        phase("response solve for P1");
        // P1 = projection of P1~ + {I, E} / (2 lam)
        concat(h, {{&I, 0, 1}, {&Pt, 1, nd}, {&h->X[h->cur], 1, nd}}, A);
        for (int s = 0; s < S; ++s) cq[s] = 0.5 / lam[s];
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, 1 + d, 0, 1 + nd + d);
        fp64_class_products(h, A, jt, c1, cq, tc, P1s);
        concat(h, {{&P0c, 0, 1}, {&P1s, 0, nd}}, A);
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, -1, 0, 1 + d);
        fp64_class_products(h, A, jt, c0, c1, tc, W);
        concat(h, {{&P0c, 0, 1}, {&W, 0, nd}}, A);
        for (int d = 0; d < nd; ++d) jt.job[d] = sym_job(d, 1 + d, 0, 1 + d);
        fp64_class_products(h, A, jt, c2, cm1, tc, P1c);
        phase("corrected P1 (nd + 2 nd products)");
    }
    A.release();
    Pt.release();
    I.release();

    // the result set (P0, P1_1..nd) with the uploaded H1 back in place
    h->keep_assembled = false;
    h->stop_at.clear();
    if (nd) h->H1 = std::move(H1s);
    else h->H1.release();
    h->nd = nd;
    for (int d = 0; d < 3; ++d) h->dirs[d] = dirs0[d];
    h->X[1 - h->cur].release();
    MatSet &Xf = h->X[h->cur];
    if (nd) concat(h, {{&P0c, 0, 1}, {&P1c, 0, nd}}, Xf);
    else concat(h, {{&P0c, 0, 1}}, Xf);
    P0c.release();
    P1c.release();
    compute_alpha(h);
    h->final_rp.resize((size_t)Xf.nmat * NB + 1);
    d2h(h->final_rp.data(), Xf.row_ptr.p, h->final_rp.size(), h->stream);
    sync(h);
    const std::vector<double> q = stats(h, Xf);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int nq = 3 + nd;
    h->info = info0;
    for (int s = 0; s < S; ++s) {
        rdm_info &R = h->info[s];
        const double nocc = (double)(h->hs[s].n_elec / 2);
        R.correction_ms = ms;
        R.time_ms += ms;
        R.trace_error = q[(size_t)s * nq] - nocc;
        R.idempotency = q[(size_t)s * nq] - q[(size_t)s * nq + 1];
        R.band_energy0 = q[(size_t)s * nq + 2];
        const int r0 = h->row0[s], r1 = r0 + h->nbs[s];
        R.nnzb_p0 = h->final_rp[r1] - h->final_rp[r0];
        for (int d = 0; d < nd; ++d)
            R.nnzb_p1[h->dirs[d]] = h->final_rp[(size_t)(1 + d) * NB + r1] - h->final_rp[(size_t)(1 + d) * NB + r0];
    }
    h->log = log0;
    h->conv.assign((size_t)S * 4, {});
    h->solved = true;
    if (info_out) *info_out = h->info[0];
    return status;
}

// split_directions: the field directions one after another, each a solve
// with that H1 alone from freed work buffers (the X sets then hold P0 and one
// P1; the X0 recursion is repeated),
// then the result set P0, P1_x, P1_y, P1_z and every alpha component
// (cross terms <P1_d, H1_g> included).  The summary adds up the passes'
// times and work; iterations and convergence are the worst pass's.
int run_solve(rdm_handle *h, rdm_info *info_out);
void release_work(rdm_handle *h);
int run_solve_dirs(rdm_handle *h, rdm_info *info_out) {
    int all[3], na = 0;
    if (!h->hs.empty())
        for (int d = 0; d < 3; ++d)
            if (h->hs[0].has_h1[d]) all[na++] = d;
    if (!h->prm.split_directions || na <= 1) return run_solve_corr(h, info_out);
    const int S = h->S;
    for (int s = 0; s < S; ++s)
        if (h->hs[s].has_s) return fail(h, RDM_EINVAL, "split_directions does not take an overlap matrix");
    MatSet p0, p1[3], h1[3];
    std::vector<rdm_info> acc;
    std::vector<rdm_iter_log> log0;
    int status = RDM_OK;
    for (int k = 0; k < na; ++k) {
        // the passes share nothing but the saved results: each starts from
        // freed work buffers and matrix sets
        if (k > 0) release_work(h);
        h->dir_only = all[k];
        int st;
        try {
            st = run_solve(h, nullptr);
        } catch (...) {
            h->dir_only = -1;
            throw;
        }
        h->dir_only = -1;
        if (st < 0) return st;
        if (st == RDM_NOT_CONVERGED) status = st;
        MatSet &X = h->X[h->cur];
        if (k == 0) {
            concat(h, {{&X, 0, 1}}, p0);
            acc = h->info;
            log0 = h->log;
        } else {
            for (int s = 0; s < S; ++s) {
                rdm_info &A = acc[s];
                const rdm_info &I = h->info[s];
                A.iterations = std::max(A.iterations, I.iterations);
                A.converged = A.converged && I.converged;
                A.time_ms += I.time_ms;
                A.useful_flops += I.useful_flops;
                A.issued_flops += I.issued_flops;
                for (int q = 0; q < 8; ++q) A.kernel_ms[q] += I.kernel_ms[q];
                for (int q = 0; q < 5; ++q) A.kernel_flops[q] += I.kernel_flops[q];
                A.kernel_launches += I.kernel_launches;
                A.tc_launches += I.tc_launches;
                A.oz_launches += I.oz_launches;
                A.simt_launches += I.simt_launches;
                A.numeric_bytes += I.numeric_bytes;
                A.device_bytes_peak = std::max(A.device_bytes_peak, I.device_bytes_peak);
                A.product_groups = std::max(A.product_groups, I.product_groups);
            }
        }
        for (int s = 0; s < S; ++s) acc[s].nnzb_p1[all[k]] = h->info[s].nnzb_p1[all[k]];
        concat(h, {{&X, 1, 1}}, p1[k]);
        concat(h, {{&h->H1, 0, 1}}, h1[k]);
    }
    // the result set and the H1 set of every direction
    release_work(h);
    h->nd = na;
    for (int k = 0; k < na; ++k) h->dirs[k] = all[k];
    MatSet &X = h->X[h->cur];
    if (na == 2) {
        concat(h, {{&p0, 0, 1}, {&p1[0], 0, 1}, {&p1[1], 0, 1}}, X);
        concat(h, {{&h1[0], 0, 1}, {&h1[1], 0, 1}}, h->H1);
    } else {
        concat(h, {{&p0, 0, 1}, {&p1[0], 0, 1}, {&p1[1], 0, 1}, {&p1[2], 0, 1}}, X);
        concat(h, {{&h1[0], 0, 1}, {&h1[1], 0, 1}, {&h1[2], 0, 1}}, h->H1);
    }
    p0.release();
    for (int k = 0; k < 3; ++k) { p1[k].release(); h1[k].release(); }
    compute_alpha(h);
    h->final_rp.resize((size_t)X.nmat * h->NB + 1);
    d2h(h->final_rp.data(), X.row_ptr.p, h->final_rp.size(), h->stream);
    sync(h);
    h->info = acc;
    h->log = log0;
    h->conv.assign((size_t)S * 4, {});
    h->solved = true;
    if (info_out) *info_out = h->info[0];
    return status;
}

// Free the solve's work buffers and matrix sets (the uploaded matrices stay):
// between autotuning probes at different block sizes, whose grow-only buffers
// would otherwise add up.
void release_work(rdm_handle *h) {
    for (auto *b : {&h->row_cnt, &h->row_off, &h->pool_col, &h->pool_npair, &h->mask_col, &h->out_rp, &h->slot_row,
                    &h->slot_job, &h->slot_npair, &h->slot_x, &h->slot_t, &h->work, &h->work2, &h->work3,
                    &h->scan_tmp32, &h->pair_a, &h->pair_b, &h->cnt_rows, &h->uidx, &h->scan_tmp_s, &h->urp,
                    &h->dest, &h->cpsrc})
        b->release();
    h->pair_off.release();
    h->scan_tmp64.release();
    h->out_val.release();
    h->out_nrm.release();
    h->keep.release();
    h->X[0].release();
    h->X[1].release();
    h->H0.release();
    h->H1.release();
    h->tcw.tiles.release();
    h->tcw.steps.release();
    h->tcw.step_cnt.release();
    h->tcw.step_off.release();
    h->tcw.tile_cnt.release();
    h->tcw.tile_off.release();
    h->tcw.zero.release();
    h->pool_cap_hint = 0;
    h->solved = false;
}

// The solve at the chosen block size: the uploaded b, rdm_params.block_size,
// or (autotune) the fastest of one probe solve at each of 16, 32 and 64,
// remembered until the next upload or parameter change.  A probe that runs
// out of memory or pool capacity is skipped; any other error ends the call.
int solve_entry(rdm_handle *h, rdm_info *info_out) {
    DeviceGuard dg(h->device);
    const rdm_params &P = h->prm;
    if (h->hs.empty() || !h->b) return fail(h, RDM_ESTATE, "no system uploaded");
    bool have_result = false;
    int status = RDM_OK;
    // the autotuner's choice is kept for later uploads of the same shape
    // (a size class: number of systems, block size, block rows, H0 blocks)
    std::vector<int64_t> key{h->S, h->b};
    for (const auto &y : h->hs) {
        key.push_back(y.nb);
        key.push_back((int64_t)y.col.size());
    }
    if (key != h->tuned_key) h->tuned_b = 0;
    if (P.autotune && !h->tuned_b) {
        const int cand[3] = {16, 32, 64};
        const auto t0 = std::chrono::steady_clock::now();
        double best = 0;
        int best_b = 0, last_b = 0;
        for (int k = 0; k < 3; ++k) {
            h->probe_ms[k] = 0;
            if (k > 0) release_work(h);
            h->bs = cand[k];
            int st;
            try {
                for (int sy = 0; sy < h->S; ++sy)
                    if (h->hs[sy].has_h0) ensure_reblocked(h, sy, cand[k]);   // outside the timed solve
                st = run_solve_dirs(h, nullptr);
            } catch (const Error &e) {
                st = e.code;
                h->err = e.msg;
            }
            last_b = 0;
            if (st == RDM_ENOMEM || st == RDM_ECAPACITY) continue;
            if (st < 0) return st;
            h->probe_ms[k] = h->info[0].time_ms;
            last_b = cand[k];
            status = st;
            if (!best_b || h->probe_ms[k] < best) {
                best = h->probe_ms[k];
                best_b = cand[k];
            }
        }
        h->autotune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (!best_b) return fail(h, RDM_ENOMEM, "autotune: no block size in {16, 32, 64} fits the device");
        h->tuned_b = best_b;
        h->tuned_key = key;
        have_result = last_b == best_b;   // the last probe already is the solve at the chosen size
    } else if (!P.autotune) {
        h->autotune_ms = 0;
        for (double &x : h->probe_ms) x = 0;
    }
    if (!have_result) {
        const int want = P.autotune ? h->tuned_b : P.block_size > 0 ? P.block_size : h->b;
        if (P.autotune && h->bs != want) release_work(h);
        h->bs = want;
        status = run_solve_dirs(h, nullptr);
        if (status < 0) return status;
    }
    for (auto &I : h->info) {
        I.autotune_ms = h->autotune_ms;
        for (int k = 0; k < 3; ++k) I.probe_ms[k] = h->probe_ms[k];
    }
    if (info_out) *info_out = h->info[0];
    return status;
}

// Wait for a solve started by rdm_solve_async (every call but rdm_sync,
// rdm_last_error and the parameter-free queries does this first).
void join_pending(rdm_handle *h) {
    if (h && h->pending) {
        if (h->worker.joinable()) h->worker.join();
        h->pending = false;
    }
}

// Pattern of matrix `mat` of system `sys` in the uploaded block size when the
// solve ran at another one (cached until the next solve): host copies of the
// solve's pattern, re-blocked.
const std::pair<std::vector<int>, std::vector<int>> &uploaded_pattern(rdm_handle *h, int sys, int mat) {
    auto &slot = h->conv[(size_t)sys * 4 + mat];
    if (slot.first.empty()) {
        const int NB = h->NB, r0 = h->row0[sys], nbs = h->nbs[sys];
        const int *rp = h->final_rp.data() + (size_t)mat * NB;
        const int64_t first = rp[r0], n = rp[r0 + nbs] - first;
        std::vector<int> lrp(nbs + 1), lcol(n);
        for (int i = 0; i <= nbs; ++i) lrp[i] = (int)(rp[r0 + i] - first);
        d2h(lcol.data(), h->X[h->cur].col.p + first, (size_t)n, h->stream);
        sync(h);
        for (auto &c : lcol) c -= r0;
        reblock_pattern(lrp, lcol, h->bs, h->norb[sys], h->b, slot.first, slot.second);
    }
    return slot;
}

int64_t result_nnzb(rdm_handle *h, int sys, int mat) {
    if (h->bs == h->b) {
        const int *rp = h->final_rp.data() + (size_t)mat * h->NB;
        return rp[h->row0[sys] + h->nbs[sys]] - rp[h->row0[sys]];
    }
    return (int64_t)uploaded_pattern(h, sys, mat).second.size();
}

int get_matrix(rdm_handle *h, int sys, int mat, rdm_bsr_out *out) {
    if (!h->solved) return fail(h, RDM_ESTATE, "no solve result");
    if (sys < 0 || sys >= h->S) return fail(h, RDM_EINVAL, "system index out of range");
    if (!out) return fail(h, RDM_EINVAL, "null output");
    DeviceGuard dg(h->device);
    MatSet &X = h->X[h->cur];
    const int NB = h->NB, r0 = h->row0[sys], nbs = h->nbs[sys], bs = h->bs;
    const size_t bbs = (size_t)bs * bs;
    const int *rp = h->final_rp.data() + (size_t)mat * NB;
    const int64_t first = rp[r0], last = rp[r0 + nbs];
    const bool conv = bs != h->b;
    const int64_t n = conv ? result_nnzb(h, sys, mat) : last - first;
    out->nb = conv ? h->hs[sys].nb : nbs;
    out->b = h->b;
    out->n = h->norb[sys];
    if (!out->row_ptr) {   // size query
        out->nnzb = n;
        return RDM_OK;
    }
    if (out->nnzb < n || (n && (!out->col_idx || !out->vals))) {
        out->nnzb = n;
        return fail(h, RDM_EINVAL, "output capacity too small (need " + std::to_string(n) + " blocks)");
    }
    if (!conv) {
        for (int i = 0; i <= nbs; ++i) out->row_ptr[i] = (int)(rp[r0 + i] - first);
        d2h(out->col_idx, X.col.p + first, (size_t)n, h->stream);
        d2h(out->vals, X.val.p + first * bbs, (size_t)n * bbs, h->stream);
        sync(h);
        for (int64_t p = 0; p < n; ++p) out->col_idx[p] -= r0;
        out->nnzb = n;
        return RDM_OK;
    }
    // the solve ran at block size bs: the matrix goes back to the uploaded b
    const auto &pat = uploaded_pattern(h, sys, mat);
    const int b = h->b, nbu = (int)pat.first.size() - 1;
    std::vector<int> lrp(nbs + 1), orow(n);
    for (int i = 0; i <= nbs; ++i) lrp[i] = (int)(rp[r0 + i] - first);
    for (int i = 0; i < nbu; ++i)
        for (int p = pat.first[i]; p < pat.first[i + 1]; ++p) orow[p] = i;
    DevBuf<int> drp, dcol, dorow, docol;
    DevBuf<double> dval;
    drp.ensure(nbs + 1);
    dcol.ensure(std::max<int64_t>(last - first, 1));
    dorow.ensure(std::max<int64_t>(n, 1));
    docol.ensure(std::max<int64_t>(n, 1));
    dval.ensure(std::max<int64_t>(n, 1) * b * b);
    h2d(drp.p, lrp.data(), lrp.size(), h->stream);
    // the solve's columns are global (row0 offset): local copies for the kernel
    std::vector<int> lcol(last - first);
    d2h(lcol.data(), X.col.p + first, lcol.size(), h->stream);
    sync(h);
    for (auto &c : lcol) c -= r0;
    h2d(dcol.p, lcol.data(), lcol.size(), h->stream);
    h2d(dorow.p, orow.data(), (size_t)n, h->stream);
    h2d(docol.p, pat.second.data(), (size_t)n, h->stream);
    launch_reblock_vals(drp.p, dcol.p, X.val.p + first * bbs, nbs, bs, dorow.p, docol.p, dval.p, n, b, h->stream);
    d2h(out->vals, dval.p, (size_t)n * b * b, h->stream);
    sync(h);
    for (int i = 0; i <= nbu; ++i) out->row_ptr[i] = pat.first[i];
    std::copy(pat.second.begin(), pat.second.end(), out->col_idx);
    out->nnzb = n;
    return RDM_OK;
}

}  // namespace

// ===========================================================================
// exported C ABI
// ===========================================================================
extern "C" {

const char *rdm_version(void) { return "rdm-gb300 0.1 (sm_103a)"; }

int rdm_default_params(rdm_params *p) {
    if (!p) return RDM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->tau = 1e-6;
    p->tau_x1 = -1;
    p->tau_refine = -1;
    p->tol = 1e-9;
    p->stall_tol = 0;
    p->spin_factor = 2.0;
    p->max_iter = 100;
    p->mode = RDM_MODE_FP64;
    p->min_iter = 1;
    p->use_graphs = 0;
    p->verbose = 0;
    p->stall_window = 2;
    return RDM_OK;
}

static thread_local std::string g_create_err;

int rdm_create(rdm_handle **out, int device, void *cuda_stream) {
    if (!out) return RDM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return RDM_ECUDA;
    }
    if (device < 0 || device >= ndev) {
        g_create_err = "device index out of range";
        return RDM_EINVAL;
    }
    rdm_handle *h = new (std::nothrow) rdm_handle();
    if (!h) return RDM_ENOMEM;
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    rdm_default_params(&h->prm);
    h->S = 1;
    h->hs.resize(1);
    *out = h;
    return RDM_OK;
}

int rdm_destroy(rdm_handle *h) {
    if (!h) return RDM_OK;
    join_pending(h);
    {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(h->device);
        cudaStreamSynchronize(h->stream);
        delete h;   // DevBuf members are released below through their owners
        if (prev >= 0) cudaSetDevice(prev);
    }
    return RDM_OK;
}

const char *rdm_last_error(const rdm_handle *h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

int rdm_set_params(rdm_handle *h, const rdm_params *p) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!p) return fail(h, RDM_EINVAL, "null params");
    if (!(p->tau >= 0) || !(p->tol >= 0) || p->max_iter < 1 || p->mode < 0 || p->mode > 3 ||
        !(p->spin_factor > 0) || p->min_iter < 0 || p->refine_x1 < 0 || p->refine_x1 > 4 ||
        p->refine_x0 < 0 || p->refine_x0 > 5 || p->refine_x0 == RDM_REFINE_SPLIT || p->chunk_mb < 0 ||
        p->use_graphs != 0 || p->stall_window < 0 || p->block_size < 0 || p->block_size > 64 ||
        (p->block_size & (p->block_size - 1)) || p->autotune < 0 || p->autotune > 1 || p->split_directions < 0 ||
        p->split_directions > 1 || p->correct < 0 || p->correct > 1 || (p->correct && p->split_directions) ||
        !(p->correct_tau <= 0 || p->correct_tau >= 0))
        return fail(h, RDM_EINVAL, "invalid parameters (tau >= 0, tol >= 0, max_iter >= 1, mode 0..3, "
                                   "refine_x1 0..4, refine_x0 0, 1, 3, 4 or 5, chunk_mb >= 0, use_graphs 0, "
                                   "stall_window >= 0, block_size 0 or a power of two <= 64, autotune, "
                                   "split_directions and correct 0 or 1, not both of the last two)");
    if (!tc_block_ok(p->mode, p->autotune ? 32 : p->block_size > 0 ? p->block_size : h->b))
        return fail(h, RDM_EINVAL, "the mixed modes run their products on the tensor cores, which take 16 x 16, "
                                   "32 x 32 or 64 x 64 blocks (the uploaded matrices have b = " + std::to_string(h->b) +
                                   "; rdm_params.block_size or autotune can re-block them)");
    h->prm = *p;
    h->tuned_b = 0;
    return RDM_OK;
}

int rdm_batch_create(rdm_handle *h, int n_systems) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (n_systems < 1 || n_systems > 65536) return fail(h, RDM_EINVAL, "n_systems out of range");
    return guarded(h, [&] {
        DeviceGuard dg(h->device);
        h->hs.clear();
        h->hs.resize(n_systems);
        h->S = n_systems;
        h->b = 0;
        h->solved = false;
        return RDM_OK;
    });
}

int rdm_upload_h0(rdm_handle *h, int sys, const rdm_bsr *H0, int64_t n_electrons) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (sys < 0 || sys >= h->S) return fail(h, RDM_EINVAL, "system index out of range");
    return guarded(h, [&] {
        DeviceGuard dg(h->device);
        if (!H0) return fail(h, RDM_EINVAL, "null matrix");
        if (n_electrons <= 0 || (n_electrons & 1) || n_electrons / 2 >= H0->n)
            return fail(h, RDM_EINVAL, "electron count must be even with 0 < N_e/2 < n");
        if (!h->prm.autotune && !h->prm.block_size && !tc_block_ok(h->prm.mode, H0->b))
            return fail(h, RDM_EINVAL, "the mixed modes run their products on the tensor cores, which take 16 x 16, "
                                       "32 x 32 or 64 x 64 blocks; set another mode first to upload b = " + std::to_string(H0->b));
        HostSys &y = h->hs[sys];
        int saved_b = h->b;
        if (h->S == 1) h->b = 0;
        try {
            upload_matrix(h, H0, y.rp, y.col, y.val, true);
        } catch (...) {
            h->b = saved_b;
            throw;
        }
        y.has_h0 = true;
        y.rb = SysMats{};
        y.nb = H0->nb;
        y.n = H0->n;
        y.n_elec = n_electrons;
        if (h->S == 1) {
            for (int d = 0; d < 3; ++d)
                if (y.has_h1[d] && (int)y.rp1[d].size() != y.nb + 1) y.has_h1[d] = false;
            if (y.has_s && (int)y.rps.size() != y.nb + 1) y.has_s = false;
        }
        h->solved = false;
        return RDM_OK;
    });
}

int rdm_upload_h1(rdm_handle *h, int sys, int dir, const rdm_bsr *H1) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (sys < 0 || sys >= h->S) return fail(h, RDM_EINVAL, "system index out of range");
    if (dir < 0 || dir > 2) return fail(h, RDM_EINVAL, "direction must be 0, 1 or 2");
    return guarded(h, [&] {
        DeviceGuard dg(h->device);
        HostSys &y = h->hs[sys];
        if (!y.has_h0) return fail(h, RDM_ESTATE, "upload H0 of the system before H1");
        if (!H1) return fail(h, RDM_EINVAL, "null matrix");
        if (H1->nb != y.nb || H1->n != y.n || H1->b != h->b)
            return fail(h, RDM_EINVAL, "H1 must have the same nb, b and n as H0");
        upload_matrix(h, H1, y.rp1[dir], y.col1[dir], y.val1[dir], false);
        y.has_h1[dir] = true;
        y.rb = SysMats{};
        h->solved = false;
        return RDM_OK;
    });
}

int rdm_upload_s(rdm_handle *h, int sys, const rdm_bsr *S) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (sys < 0 || sys >= h->S) return fail(h, RDM_EINVAL, "system index out of range");
    return guarded(h, [&] {
        DeviceGuard dg(h->device);
        HostSys &y = h->hs[sys];
        if (!y.has_h0) return fail(h, RDM_ESTATE, "upload H0 of the system before S");
        if (!S) return fail(h, RDM_EINVAL, "null matrix");
        if (S->nb != y.nb || S->n != y.n || S->b != h->b)
            return fail(h, RDM_EINVAL, "S must have the same nb, b and n as H0");
        upload_matrix(h, S, y.rps, y.cols, y.vals, true);
        y.has_s = true;
        y.rb = SysMats{};
        h->solved = false;
        return RDM_OK;
    });
}

int rdm_force_branches(rdm_handle *h, const uint8_t *seq, int len) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (len < 0 || (len > 0 && !seq)) return fail(h, RDM_EINVAL, "bad branch sequence");
    for (int i = 0; i < len; ++i)
        if (seq[i] != 1 && seq[i] != 2) return fail(h, RDM_EINVAL, "branches must be 1 or 2");
    h->forced.assign(seq, seq + len);
    return RDM_OK;
}

int rdm_solve(rdm_handle *h, rdm_info *info) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    return guarded(h, [&] { return solve_entry(h, info); });
}

int rdm_solve_async(rdm_handle *h) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (h->hs.empty() || !h->b) return fail(h, RDM_ESTATE, "no system uploaded");
    h->async_status = RDM_OK;
    try {
        h->worker = std::thread([h] { h->async_status = guarded(h, [&] { return solve_entry(h, nullptr); }); });
    } catch (const std::exception &e) {
        return fail(h, RDM_EINVAL, std::string("cannot start the solve thread: ") + e.what());
    }
    h->pending = true;
    return RDM_OK;
}

int rdm_sync(rdm_handle *h, rdm_info *info) {
    if (!h) return RDM_EINVAL;
    if (!h->pending) return fail(h, RDM_ESTATE, "no solve in flight");
    join_pending(h);
    if (info && h->solved && h->async_status >= 0) *info = h->info[0];
    return h->async_status;
}

int rdm_set_test_knobs(rdm_handle *h, const rdm_test_knobs *k) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    rdm_test_knobs z{};
    if (!k) k = &z;
    if (k->tc_wait_cycles < 0 || k->tc_hold < 0 || k->tc_hold > 1 || k->tc_window_cols < 0 ||
        k->tc_window_cols > 16384 || (k->tc_window_cols & 31) || k->tc_block_copies < 0 ||
        k->tc_block_copies > 1 || k->pad0 != 0)
        return fail(h, RDM_EINVAL, "invalid test settings");
    h->tcw.knobs.wait_cycles = k->tc_wait_cycles;
    h->tcw.knobs.hold = k->tc_hold;
    h->tcw.knobs.window_words = k->tc_window_cols / 32;
    h->tcw.knobs.block_copies = k->tc_block_copies;
    return RDM_OK;
}

int rdm_get_info(rdm_handle *h, int sys, rdm_info *info) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!h->solved) return fail(h, RDM_ESTATE, "no solve result");
    if (sys < 0 || sys >= h->S || !info) return fail(h, RDM_EINVAL, "bad system index or null output");
    *info = h->info[sys];
    return RDM_OK;
}

int rdm_get_p0_nnzb(rdm_handle *h, int sys, int64_t *nnzb) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!h->solved) return fail(h, RDM_ESTATE, "no solve result");
    if (sys < 0 || sys >= h->S || !nnzb) return fail(h, RDM_EINVAL, "bad system index or null output");
    return guarded(h, [&] {
        DeviceGuard dg(h->device);
        *nnzb = result_nnzb(h, sys, 0);
        return RDM_OK;
    });
}

int rdm_get_p1_nnzb(rdm_handle *h, int sys, int dir, int64_t *nnzb) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!h->solved) return fail(h, RDM_ESTATE, "no solve result");
    if (sys < 0 || sys >= h->S || !nnzb || dir < 0 || dir > 2) return fail(h, RDM_EINVAL, "bad index or null output");
    for (int d = 0; d < h->nd; ++d)
        if (h->dirs[d] == dir)
            return guarded(h, [&] {
                DeviceGuard dg(h->device);
                *nnzb = result_nnzb(h, sys, 1 + d);
                return RDM_OK;
            });
    return fail(h, RDM_EINVAL, "direction was not uploaded");
}

int rdm_get_p0(rdm_handle *h, int sys, rdm_bsr_out *out) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    return guarded(h, [&] { return get_matrix(h, sys, 0, out); });
}

int rdm_get_p1(rdm_handle *h, int sys, int dir, rdm_bsr_out *out) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    return guarded(h, [&] {
        for (int d = 0; d < h->nd; ++d)
            if (h->dirs[d] == dir) return get_matrix(h, sys, 1 + d, out);
        return fail(h, RDM_EINVAL, "direction was not uploaded");
    });
}

int rdm_get_alpha(rdm_handle *h, int sys, double alpha[9]) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!h->solved) return fail(h, RDM_ESTATE, "no solve result");
    if (sys < 0 || sys >= h->S || !alpha) return fail(h, RDM_EINVAL, "bad system index or null output");
    for (int k = 0; k < 9; ++k) alpha[k] = h->alpha[(size_t)sys * 9 + k];
    return RDM_OK;
}

int rdm_get_log(rdm_handle *h, rdm_iter_log *out, int cap, int *n) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    if (!n || (cap > 0 && !out)) return fail(h, RDM_EINVAL, "null output");
    int m = std::min<int>(cap, (int)h->log.size());
    for (int k = 0; k < m; ++k) out[k] = h->log[k];
    *n = (int)h->log.size();
    return RDM_OK;
}

int rdm_block_product(rdm_handle *h, const rdm_bsr *A, const rdm_bsr *B, const rdm_bsr *X,
                      double c_lin, double c_sq, int terms, double tau, int mode,
                      rdm_bsr_out *out, int64_t *needed) {
    if (!h) return RDM_EINVAL;
    join_pending(h);
    return guarded(h, [&]() -> int {
        DeviceGuard dg(h->device);
        if (!A || (terms == 2 && !B)) return fail(h, RDM_EINVAL, "null operand");
        if (terms != 1 && terms != 2) return fail(h, RDM_EINVAL, "terms must be 1 or 2");
        const bool slices = mode == RDM_PRODUCT_SLICES;
        if (!(tau >= 0) || ((mode < 0 || mode > 3) && !slices)) return fail(h, RDM_EINVAL, "bad tau or mode");
        if (slices && (terms != 1 || A->b != 32))
            return fail(h, RDM_EINVAL, "the slice product takes terms = 1 (A A) and 32 x 32 blocks");
        // a private single-system context so that the solve state is untouched
        rdm_handle t;
        t.device = h->device;
        t.stream = h->stream;
        t.S = 1;
        t.hs.resize(1);
        const rdm_bsr *mats[3] = {A, terms == 2 ? B : nullptr, X};
        std::vector<int> rps[3], cols[3];
        DevBuf<double> vals[3];
        int nm = 0;
        int idx[3] = {-1, -1, -1};
        for (int k = 0; k < 3; ++k) {
            if (!mats[k]) continue;
            if (mats[k]->nb != A->nb || mats[k]->b != A->b || mats[k]->n != A->n)
                return fail(h, RDM_EINVAL, "operands must share nb, b and n");
            upload_matrix(&t, mats[k], rps[k], cols[k], vals[k], false);
            idx[k] = nm++;
        }
        const int NB = A->nb, b = A->b;
        const size_t bb = (size_t)b * b;
        MatSet in;
        in.nmat = nm;
        in.NB = NB;
        in.b = b;
        std::vector<int> rp((size_t)nm * NB + 1);
        std::vector<int> col;
        int64_t top = 0;
        in.nnzb.assign(nm, 0);
        for (int k = 0; k < 3; ++k) {
            if (idx[k] < 0) continue;
            for (int i = 0; i < NB; ++i) rp[(size_t)idx[k] * NB + i] = (int)(top + rps[k][i]);
            col.insert(col.end(), cols[k].begin(), cols[k].end());
            in.nnzb[idx[k]] = rps[k][NB];
            top += rps[k][NB];
        }
        rp[(size_t)nm * NB] = (int)top;
        in.total = top;
        in.row_ptr.ensure(rp.size());
        in.col.ensure(std::max<int64_t>(top, 1));
        in.val.ensure(std::max<int64_t>(top, 1) * bb);
        in.nrm.ensure(std::max<int64_t>(top, 1));
        h2d(in.row_ptr.p, rp.data(), rp.size(), t.stream);
        h2d(in.col.p, col.data(), col.size(), t.stream);
        int64_t off = 0;
        for (int k = 0; k < 3; ++k) {
            if (idx[k] < 0) continue;
            int64_t n = rps[k][NB];
            if (n) RDM_CUDA_TRY(cudaMemcpyAsync(in.val.p + off * bb, vals[k].p, n * bb * sizeof(double),
                                                cudaMemcpyDeviceToDevice, t.stream));
            off += n;
        }
        launch_block_norms(in.val.p, in.nrm.p, top, b, t.stream);
        t.NB = NB;
        t.b = b;
        t.nbs = {NB};
        t.row0 = {0};
        t.norb = {A->n};
        SysDev &sd = t.sd;
        sd.row0.ensure(1); sd.nbs.ensure(1); sd.n_orb.ensure(1); sd.sys_of_row.ensure(NB);
        sd.c_lin.ensure(1); sd.c_sq.ensure(1); sd.tau0.ensure(1); sd.tau1.ensure(1); sd.active.ensure(1);
        sd.tier.ensure(1);
        RDM_CUDA_TRY(cudaMemsetAsync(sd.tier.p, 0, sizeof(int), t.stream));
        RDM_CUDA_TRY(cudaMemsetAsync(sd.row0.p, 0, sizeof(int), t.stream));
        RDM_CUDA_TRY(cudaMemsetAsync(sd.sys_of_row.p, 0, NB * sizeof(int), t.stream));
        int one = 1;
        h2d(sd.nbs.p, &NB, 1, t.stream);
        h2d(sd.n_orb.p, &A->n, 1, t.stream);
        h2d(sd.active.p, &one, 1, t.stream);
        h2d(sd.c_lin.p, &c_lin, 1, t.stream);
        h2d(sd.c_sq.p, &c_sq, 1, t.stream);
        h2d(sd.tau0.p, &tau, 1, t.stream);
        h2d(sd.tau1.p, &tau, 1, t.stream);
        JobTable jt{};
        jt.njob = 1;
        int ia = idx[0], ib = terms == 2 ? idx[1] : idx[0];
        int ix = X ? idx[2] : -1;
        if (terms == 1) jt.job[0] = Job{0, ix, 1, {ia, ia}, {ia, ia}, 0};
        else jt.job[0] = Job{0, ix, 2, {ia, ib}, {ib, ia}, 0};
        Arith tab[kMaxTiers][kMaxJobs];
        if (slices) tab[0][0] = AR_OZ;
        else tier_arith(mode, 0, jt.njob, tab[0]);
        MatSet res;
        multiply(&t, in, res, jt, tab, 1u);
        int64_t n = res.nnzb[0];
        if (needed) *needed = n;
        if (!out || !out->row_ptr || out->nnzb < n || (n && (!out->col_idx || !out->vals))) {
            if (out) out->nnzb = n;
            res.release();
            in.release();
            return out && out->row_ptr ? fail(h, RDM_EINVAL, "output capacity too small") : RDM_OK;
        }
        std::vector<int> rrp((size_t)NB + 1);
        d2h(rrp.data(), res.row_ptr.p, NB + 1, t.stream);
        d2h(out->col_idx, res.col.p, (size_t)n, t.stream);
        d2h(out->vals, res.val.p, (size_t)n * bb, t.stream);
        RDM_CUDA_TRY(cudaStreamSynchronize(t.stream));
        for (int i = 0; i <= NB; ++i) out->row_ptr[i] = rrp[i];
        out->nb = NB;
        out->b = b;
        out->n = A->n;
        out->nnzb = n;
        res.release();
        in.release();
        return RDM_OK;
    });
}

}  // extern "C"
