/*
 * rdm.h - C ABI of the GB300 response-density-matrix library.
 *
 * The library computes, for a gapped Hamiltonian H0 and first-order
 * perturbations H1_gamma given in an orthogonal basis (the orthogonal form of
 * Sec. 2.2 of Shang, Liang, Zhang, Yang, "Efficient Parallel Linear Scaling
 * Method to get the Response Density Matrix in All-Electron Real-Space DFPT"):
 *
 *   P0       = lim X0_n     (TC2 purification, Eq. TC2)
 *   P1_gamma = lim X1_n     (first-order recursion, Eq. TC2-CPSCF)
 *   alpha    = polarizability tensor (Eq. polar, field term -r.E)
 *
 * starting from X0_0 = (eps_max I - H0)/(eps_max - eps_min) and
 * X1_0 = -H1/(eps_max - eps_min) with Gershgorin bounds eps_min, eps_max
 * (Sec. 2.2).  Every product is a block-sparse (BSR) product followed by
 * block-norm truncation (the "filter" of Sec. 2.3); the loop stops on the
 * band-energy change (the "tolerance" of Sec. 2.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an int status: RDM_OK (0) on success, a positive
 *   warning (results readable), or a negative error.  No C++ exception and no
 *   abort crosses this boundary.  rdm_last_error() gives a message for the
 *   last failing call on that handle.
 * - Units: Hartree and bohr; alpha in bohr^3.  Matrices are real symmetric.
 * - BSR layout (struct rdm_bsr): nb block rows of b x b blocks; row_ptr has
 *   nb+1 int32 entries (row_ptr[0] = 0); col_idx has nnzb int32 entries,
 *   strictly increasing inside each block row; vals holds nnzb blocks of
 *   b*b doubles, each block row-major.  n <= nb*b is the number of
 *   meaningful orbitals; rows and columns n..nb*b-1 are padding and must be
 *   zero.  The block pattern must be symmetric and every diagonal block of
 *   H0 must be present.
 * - Ownership: the caller owns every buffer it passes.  Uploads copy the
 *   data (in the order of the handle's stream); caller buffers may be reused
 *   once the call has returned (host buffers) or once the handle's stream has
 *   been synchronised (device buffers).  Getters write into caller-allocated
 *   host buffers and return after the copy has completed.
 * - A handle is bound to one CUDA device and one stream, and must not be
 *   used from two threads at once.
 */
#ifndef RDM_H_
#define RDM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define RDM_OK               0
#define RDM_NOT_CONVERGED    1   /* warning: max_iter reached; results readable */
#define RDM_EINVAL          -1   /* bad argument (null pointer, range, call order) */
#define RDM_EBADBSR         -2   /* malformed matrix: pattern, symmetry, non-finite values */
#define RDM_ENOMEM          -3   /* device allocation failed */
#define RDM_ECUDA           -4   /* CUDA runtime error */
#define RDM_ECAPACITY       -5   /* a work pool overflowed and could not be grown */
#define RDM_ETIMEOUT        -6   /* a bounded device wait expired */
#define RDM_ESTATE          -7   /* call made in the wrong state (e.g. getter before solve) */

/* ---- precision modes (rdm_params.mode) ------------------------------- */
#define RDM_MODE_FP64        0   /* every product in FP64 (CUDA cores) */
#define RDM_MODE_FP32        1   /* every product in FP32 (CUDA cores), FP64 scalars */
#define RDM_MODE_MIXED_BF16  2   /* bf16 hi+lo split products on the tensor cores
                                    (tcgen05, FP32 accumulate) until the idempotency
                                    error stalls, then a final tier: X0^2 FP64-class
                                    (RDM_REFINE_SLICES for 32 x 32 blocks, else FP64),
                                    the first-order products still split (refine_x0 /
                                    refine_x1 choose otherwise) */
#define RDM_MODE_MIXED_FP16  3   /* the same with fp16 hi+lo operands, each matrix scaled
                                    by a power of two into fp16's normal range
                                    (22-bit products instead of 16-bit); final tier:
                                    X0^2 as exact bf16 slice products on the tensor
                                    cores (FP64-class, RDM_REFINE_SLICES; FP64 on the
                                    CUDA cores for blocks other than 32 x 32),
                                    first-order products still split */

/* ---- final-tier arithmetic of the first-order products (rdm_params.refine_x1) */
#define RDM_REFINE_DEFAULT   0   /* refine_x1: the split product (both mixed modes);
                                    refine_x0: see rdm_params */
#define RDM_REFINE_FP64      1
#define RDM_REFINE_SPLIT     2   /* keep the tensor-core split product */
#define RDM_REFINE_FP32      3   /* FP32 on the CUDA cores (round-to-nearest accumulation) */
#define RDM_REFINE_FP32X2    4   /* double-FP32 on the CUDA cores: each FP64 value as the sum of
                                    two FP32 words, the products accumulated with error-free
                                    transformations (about 46 bits; 32 x 32 blocks) */
#define RDM_REFINE_SLICES    5   /* refine_x0 only: X0^2 on the tensor cores from exact products of
                                    7 bf16 slices per element (row-scaled integer slices summed in
                                    exact groups, then in double-FP32; about 48 bits; the splitting of
                                    Ozaki, Ogita, Oishi and Rump 2012; 32 x 32 blocks) */

typedef struct rdm_handle rdm_handle;

/* Input matrix (H0 or one H1_gamma).  on_device = 1: the three arrays are
 * device pointers on the handle's device; 0: host pointers. */
typedef struct {
    int32_t nb;             /* block rows (= block columns) */
    int32_t b;              /* block size, 1..64 */
    int32_t n;              /* meaningful orbitals, (nb-1)*b < n <= nb*b */
    int32_t on_device;
    int64_t nnzb;           /* stored blocks */
    const int32_t *row_ptr; /* nb+1 */
    const int32_t *col_idx; /* nnzb */
    const double  *vals;    /* nnzb*b*b, row-major blocks */
} rdm_bsr;

/* Output matrix: caller-allocated HOST arrays of the sizes returned by the
 * matching *_nnzb getter. */
typedef struct {
    int32_t nb, b, n;
    int64_t nnzb;           /* in: capacity in blocks; out: blocks written */
    int32_t *row_ptr;       /* nb+1 */
    int32_t *col_idx;       /* nnzb */
    double  *vals;          /* nnzb*b*b */
} rdm_bsr_out;

typedef struct {
    double  tau;            /* block-norm truncation threshold for X0 (filter), >= 0 */
    double  tau_x1;         /* the same for X1; < 0 means "use tau" */
    double  tau_refine;     /* threshold in the final (FP64) tier of the mixed modes; < 0: tau */
    double  tol;            /* band-energy change stop (Hartree); 0 disables it */
    double  stall_tol;      /* idempotency-stall stop level (0 disables; mixed modes set their own) */
    double  spin_factor;    /* 2.0 for closed shells; enters alpha only */
    int32_t max_iter;       /* iteration cap; reaching it returns RDM_NOT_CONVERGED */
    int32_t mode;           /* RDM_MODE_* */
    int32_t min_iter;       /* never stop before this many iterations */
    int32_t use_graphs;     /* reserved, must be 0 (else RDM_EINVAL): the iteration is not captured in
                               CUDA graphs, since it takes host decisions (sizes, branch, tier) every step */
    int32_t verbose;        /* 1: per-iteration log to stderr */
    int32_t refine_x1;      /* mixed modes, final tier, arithmetic of the first-order products
                               (RDM_REFINE_*) */
    int32_t symbolic_hash;  /* 1: use the hash-table symbolic phase (otherwise chosen only for
                               systems above 8,192 block rows); results are identical */
    int32_t chunk_mb;       /* cap in MiB on the buffer of untruncated product blocks (8 b^2 + 5
                               bytes per upper-triangle block); the products of a step (X0^2,
                               each X1 product) are then computed in groups of consecutive
                               super-rows (4 block rows of one product) that fit it (at least
                               one super-row per group).  0: automatic, from the free device
                               memory.  Results do not depend on the grouping. */
    int32_t refine_x0;      /* mixed modes, final tier, arithmetic of X0^2: RDM_REFINE_DEFAULT
                               (RDM_REFINE_SLICES with 32 x 32 blocks, otherwise
                               RDM_REFINE_FP64), RDM_REFINE_FP64, RDM_REFINE_FP32X2
                               (32 x 32 blocks only), or RDM_REFINE_FP32 (the final tier then ends
                               on the FP32 idempotency stall) */
    int32_t stall_window;   /* mixed modes: the idempotency error e "stalls" when |e_n| >= |e_{n-w}| / 2
                               with w = stall_window iterations (0: 2); a stall moves a system to the
                               final tier, and in the final tier ends its iteration */
    int32_t block_size;     /* block size of the solve's products: 0 = the uploaded b; 16, 32 or 64
                               re-blocks every system (the same matrices in b' x b' blocks; the
                               filter then acts on b' x b' blocks) and the getters return P0 and P1
                               in the uploaded layout.  Ignored while autotune is on. */
    int32_t autotune;       /* 1: the first solve of a problem shape (number of systems, b, block rows
                               and H0 blocks of every system) times one probe solve at each block
                               size in {16, 32, 64} and keeps the fastest for this and later solves
                               of that shape, whatever values are uploaded (rdm_info.block_size,
                               probe_ms); setting parameters forgets the choice; 0: off */
    int32_t split_directions; /* 1: the field directions are solved one after another (each solve holds
                               P0 and one P1 instead of P0 and every P1: about half the device memory
                               at three directions, for a repeated X0 recursion); the results, alpha
                               with its cross terms included, are those of the joint solve up to the
                               stopping tolerance.  Not with an overlap matrix (RDM_EINVAL at the
                               solve).  0: off */
    int32_t correct;        /* 1: after the solve, correct P0 and P1 for the residuals of their
                               defining conditions (Sec. 2.1: [H0, P0] = 0 and, with P1 occupied-
                               virtual, [H0, P1] + [H1, P0] = 0) by two more solves of the same
                               mode: the error of P0 is the response to H'0 = [[H0, P0], P0], that
                               of P1, with the corrected P0, the response to H'1 = [R1, P0], R1 the
                               residual; the H' are formed by FP64-class block products (double-
                               FP32 at b = 32, else FP64) with the filter correct_tau.  Removes the
                               rounding error of the reduced-precision tiers (the rotation of the
                               occupied subspace they leave); costs the two response solves and
                               about 3 + 5 nd FP64-class products.  Not with an overlap matrix or
                               split_directions (RDM_EINVAL).  0: off */
    double  correct_tau;    /* filter of the correction's block products (the residuals are small
                               differences of O(1) terms, so it must lie well below tau); <= 0:
                               tau / 100 */
} rdm_params;

/* Per-solve summary (per system s of a batch: rdm_get_info). */
typedef struct {
    int32_t iterations;
    int32_t converged;
    int32_t tier_iters[4];  /* iterations spent per precision tier (mixed modes) */
    double  eps_min, eps_max;
    double  trace_error;    /* Tr P0 - N_occ */
    double  idempotency;    /* Tr P0 - ||P0||_F^2 */
    double  band_energy0;   /* Tr(P0 H0) */
    int64_t nnzb_p0;
    int64_t nnzb_p1[3];
    double  time_ms;        /* wall time of the solve on the handle's stream */
    double  useful_flops;   /* 2 b^3 per (i,k,j) block triple, summed over the solve */
    double  issued_flops;   /* flops the kernels executed (split products count 3x, padding counted) */
    double  kernel_ms[8];   /* device time per kernel class (CUDA events on the handle's stream):
                               0 symbolic mask + pair / tile lists, 1 tensor-core split products,
                               2 FP64 CUDA-core products, 3 FP32 CUDA-core products (and copies
                               of converged systems), 4 truncation compaction, 5 reductions,
                               set-up and host decisions (the remainder of the solve),
                               6 double-FP32 CUDA-core products, 7 tensor-core slice products */
    double  kernel_flops[5];   /* useful flops (2 b^3 per block triple) of the tensor-core split (0),
                                  FP64 (1), FP32 (2), double-FP32 (3) and slice-product (4) launches */
    int64_t kernel_launches;   /* kernels launched by the solve */
    int32_t tc_launches;       /* launches of the tensor-core split-product kernel */
    int32_t simt_launches;     /* launches of the CUDA-core product kernel */
    double  numeric_bytes;  /* algorithmic bytes of the product launches: operand blocks read
                               once (8 bytes/element FP64, 4 bytes hi+lo planes) + output
                               blocks written (8 bytes/element) */
    int64_t device_bytes_peak; /* largest device memory held by the library's buffers during
                                  the solve (all handles of the process) */
    int32_t product_groups;    /* most super-row groups a step of the solve was split into (chunk_mb) */
    int32_t block_size;        /* block size the products ran at (rdm_params.block_size / autotune) */
    double  autotune_ms;       /* wall time of the autotuner's probe solves (0 when it did not run) */
    double  probe_ms[3];       /* device time of the probe solve at b = 16, 32, 64 (0: not probed) */
    int32_t lowdin_iterations; /* Newton-Schulz iterations for S^(-1/2) (0: orthogonal basis) */
    int32_t oz_launches;       /* launches of the tensor-core slice-product kernel */
    double  correction_ms;     /* wall time of the correction (rdm_params.correct; included in
                                  time_ms; 0: off); the other fields describe the solve before it,
                                  except the summary of P0 and P1 (trace, idempotency, band energy,
                                  nnzb), which is that of the corrected matrices */
} rdm_info;

/* One record per iteration (rdm_get_log). */
typedef struct {
    int32_t iter, branch, tier, sys;
    double  trace;          /* Tr X0_n */
    double  idempotency;    /* Tr X0_n - ||X0_n||_F^2 */
    double  eb0;            /* Tr(X0_{n+1} H0) */
    double  eb1[3];         /* Tr(X1_{n+1,gamma} H0) */
    int64_t nnzb0, nnzb1[3];
    double  ms;             /* device time of the iteration */
} rdm_iter_log;

/* ---- lifetime ---------------------------------------------------------- */

/* Create a handle on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle (NULL on failure). */
int rdm_create(rdm_handle **out, int device, void *cuda_stream);

/* Free every device buffer of the handle (after synchronising its stream). */
int rdm_destroy(rdm_handle *h);

/* Message of the last failing call on h (never NULL; valid until the next
 * call on h).  h may be NULL for creation errors. */
const char *rdm_last_error(const rdm_handle *h);

/* Fill *p with the defaults: tau 1e-6, tau_x1/tau_refine -1, tol 1e-9,
 * stall_tol 0, spin 2, max_iter 100, mode FP64, min_iter 1, graphs 0, the
 * rest 0. */
int rdm_default_params(rdm_params *p);

/* Set the solve parameters.  Validated: tau >= 0, tol >= 0, max_iter >= 1, a
 * known mode, refine_x1 in 0..4, refine_x0 in {0, 1, 3, 4, 5}, chunk_mb >= 0,
 * use_graphs == 0, stall_window >= 0, block_size 0 or a power of two up to 64,
 * autotune, split_directions and correct 0 or 1, not both of the last two;
 * anything else returns RDM_EINVAL and keeps the old set. */
int rdm_set_params(rdm_handle *h, const rdm_params *p);

/* ---- problem definition ------------------------------------------------ */

/* Declare a batch of n_systems independent systems (default 1).  Clears any
 * uploaded matrices.  All systems of a batch share the block size b. */
int rdm_batch_create(rdm_handle *h, int n_systems);

/* Upload H0 of system `sys` with its electron count (even, 0 < N_e/2 < n).
 * Validates the pattern (sorted, unique, in range, symmetric, diagonal
 * present) and the values (finite, symmetric to 1e-12 max|H|, padding zero)
 * and returns RDM_EBADBSR with a message if any check fails. */
int rdm_upload_h0(rdm_handle *h, int sys, const rdm_bsr *H0, int64_t n_electrons);

/* Upload H1 for direction dir (0 = x, 1 = y, 2 = z) of system sys: the
 * matrix dH/dlambda of the first-order perturbation (Sec. 2.1, the H^(1) of
 * Eq. CPSCF-U; for a homogeneous field this is the dipole matrix D_dir, the
 * field term -r.E of Sec. 2 entering through the sign convention of alpha).
 * Same checks as H0 (the diagonal need not be present); same nb, b, n as H0. */
int rdm_upload_h1(rdm_handle *h, int sys, int dir, const rdm_bsr *H1);

/* Upload the overlap matrix S of system sys for a NON-ORTHOGONAL basis
 * (Sec. 2.2: H C = S C E).  The solve then forms S^(-1/2) by the coupled
 * Newton-Schulz iteration (with the same block products and filter as the
 * purification), transforms H0 and every H1 to the orthogonal form
 * S^(-1/2) H S^(-1/2), runs the solve there and transforms P0 and P1 back
 * (P = S^(-1/2) P_orth S^(-1/2)); alpha is basis independent.  rdm_get_p0 /
 * rdm_get_p1 return the non-orthogonal-basis matrices (Tr(P0 S) = N_occ);
 * rdm_info's trace and idempotency are those of the orthogonal form.  S must
 * be symmetric positive definite with the pattern rules of H0 (diagonal blocks
 * present, padding zero) and the same nb, b, n; upload it for every system of
 * a batch or for none (RDM_EINVAL at the solve otherwise).  A perturbation
 * that changes S (atomic displacements) is out of scope: H1 is a field term. */
int rdm_upload_s(rdm_handle *h, int sys, const rdm_bsr *S);

/* ---- solve -------------------------------------------------------------- */

/* Run the coupled TC2 / first-order recursion for every uploaded system and
 * direction (Sec. 2.2: X0_0, X1_0 from the Gershgorin bounds; Eq. TC2 for X0
 * and Eq. TC2-CPSCF for every X1 in the branch the trace test of Eq. TC2
 * picks; the filter of Sec. 2.3 after every product; stop on the band-energy
 * change, the "tolerance" of Sec. 2.3), then the polarizability (Eq. polar).
 * Blocks until done.  *info (may be NULL) receives the summary of system 0.
 * Returns RDM_OK, the warning RDM_NOT_CONVERGED, or an error (RDM_ECAPACITY,
 * RDM_ECUDA, RDM_ENOMEM, RDM_ETIMEOUT). */
int rdm_solve(rdm_handle *h, rdm_info *info);

/* The same solve, asynchronous: it runs on a host thread of the library that
 * drives the handle's stream, and the call returns at once (RDM_OK, or
 * RDM_ESTATE when nothing is uploaded).  rdm_sync waits for it and returns its
 * status (as rdm_solve would) with *info (may be NULL) for system 0;
 * RDM_ESTATE if no solve is in flight.  Every other call on the handle waits
 * for a solve in flight first, so results are never read half-written. */
int rdm_solve_async(rdm_handle *h);
int rdm_sync(rdm_handle *h, rdm_info *info);

/* Test hook: force the branch of Eq. TC2 at iteration n to seq[n] (1 = X^2,
 * 2 = 2X - X^2) for n < len; len = 0 clears it.  Applies to every system. */
int rdm_force_branches(rdm_handle *h, const uint8_t *seq, int len);

/* ---- results ------------------------------------------------------------ */

/* Summary of system sys of the last solve (iterations, branch tiers, the
 * Gershgorin bounds of Sec. 2.2, Tr P0 - N_occ and the idempotency error of
 * Eq. TC2's fixed point, the band energy Tr(P0 H0) of the Sec. 2.3 stopping
 * rule, block counts, timings).  RDM_ESTATE before a solve. */
int rdm_get_info(rdm_handle *h, int sys, rdm_info *info);

/* Number of stored blocks of P0 = lim X0_n (Eq. TC2) (resp. P1_dir = lim X1_n,
 * Eq. TC2-CPSCF) of system sys, in the uploaded block layout. */
int rdm_get_p0_nnzb(rdm_handle *h, int sys, int64_t *nnzb);
int rdm_get_p1_nnzb(rdm_handle *h, int sys, int dir, int64_t *nnzb);

/* Copy P0 (resp. P1_dir) into caller host buffers (out->nnzb = capacity on
 * entry).  With out->row_ptr == NULL the call is a size query: it fills
 * out->nb, b, n, nnzb and returns RDM_OK.  Block order and indices are the
 * caller's: the library does not permute.  Padding rows/columns come back as
 * zeros. */
int rdm_get_p0(rdm_handle *h, int sys, rdm_bsr_out *out);
int rdm_get_p1(rdm_handle *h, int sys, int dir, rdm_bsr_out *out);

/* alpha[3*g + d] = -spin * Tr(P1_d H1_g) (Eq. polar with field term -r.E);
 * entries of directions that were not uploaded are NaN. */
int rdm_get_alpha(rdm_handle *h, int sys, double alpha[9]);

/* Copy up to cap per-iteration records of the last solve (branch of Eq. TC2,
 * tier, Tr X0_n, idempotency error, the band energies of the Sec. 2.3
 * stopping rule, block counts); *n gets the count. */
int rdm_get_log(rdm_handle *h, rdm_iter_log *out, int cap, int *n);

/* ---- single-product primitive (kernel-level testing and benchmarking) ---- */

/* One truncated block-sparse product on the handle's device:
 *   C = c_lin * X + c_sq * (A B)          (terms = 1)
 *   C = c_lin * X + c_sq * (A B + B A)    (terms = 2; requires symmetric A, B)
 * followed by dropping every block whose Frobenius norm is below tau — the
 * update step of Eqs. TC2 / TC2-CPSCF for one matrix.  A, B, X are symmetric
 * host BSR matrices with the same nb, b, n (X may be NULL: no linear term).
 * `mode` selects the product arithmetic (RDM_MODE_*; the mixed modes use the
 * hi+lo split tensor-core product; RDM_PRODUCT_SLICES the exact bf16 slice
 * product of RDM_REFINE_SLICES, for terms = 1 and 32 x 32 blocks; both take symmetric block
 * patterns, else RDM_EBADBSR).  The result goes to *out as for
 * rdm_get_p0; call with out->nnzb = 0 / NULL arrays to query the size only
 * (*needed receives the block count). */
#define RDM_PRODUCT_SLICES   8   /* rdm_block_product only: the tensor-core slice product */
int rdm_block_product(rdm_handle *h, const rdm_bsr *A, const rdm_bsr *B, const rdm_bsr *X,
                      double c_lin, double c_sq, int terms, double tau, int mode,
                      rdm_bsr_out *out, int64_t *needed);

/* ---- allocation-free inner product (no counterpart in the paper) ---------- */

/* <A, B> = sum over the blocks (i,j) stored in both A and B of the
 * elementwise products (Tr(A B) for symmetric A, B: the reduction behind the
 * polarizability trace), written as one double to out_device, in the order
 * of the CUDA stream `cuda_stream` (NULL = legacy default stream), on the
 * current device.  For callers that must not allocate device memory: a
 * framework whose caching pool owns the free HBM, or a latency-critical loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
 * The call allocates nothing: its scratch (one double per block row) is a
 * file-scope device array of at most 262,144 block rows, held by every GPU
 * that loads the library until exit.
 *  - A and B: device BSR (on_device = 1) with the same nb, b and n; nb above
 *    262,144 returns RDM_EINVAL, as do null pointers and host matrices.
 *  - The call cannot inspect device data, so it trusts the layout: each
 *    row_ptr must have nb+1 non-decreasing entries from 0 to that matrix's
 *    nnzb, and the column indices of every block row must be strictly
 *    increasing and in [0, nb) (B's columns are binary-searched).  A
 *    malformed matrix gives a wrong result or out-of-range reads.
 *  - The first call on a device looks up the array's device address (once,
 *    with that device current); make it before any stream capture.
 *  - All calls share the array: calls whose kernels overlap on the GPU race
 *    and must be serialised by the caller.  Nothing in the array has to start
 *    at zero (every call writes each partial it reads).
 * Returns RDM_OK, RDM_EINVAL or RDM_ECUDA (launch failure). */
int rdm_bsr_dot_noalloc(const rdm_bsr *A, const rdm_bsr *B, double *out_device, void *cuda_stream);

/* ---- test settings (kernel-level tests; no counterpart in the paper) ------ */

/* Settings that tests use to reach paths a production solve rarely takes.
 * All zeros (the state of a new handle) is production behaviour. */
typedef struct {
    int64_t tc_wait_cycles;  /* bound of every wait inside the tensor-core product kernel, in SM clock
                                cycles; 0 = the default (~2 s).  A wait that runs out makes the kernel
                                raise its abort flag, let its copies and MMAs in flight finish, free
                                its tensor memory and return; the solve then fails with RDM_ETIMEOUT
                                and the handle stays usable. */
    int32_t tc_hold;         /* 1: the tensor-core kernel's MMA thread first waits for a device flag that
                                nothing sets, so that its wait runs out (with tc_wait_cycles), the copy
                                warp's wait for a free stage runs out after it and drains its copies,
                                and the solve returns RDM_ETIMEOUT without a fault */
    int32_t tc_window_cols;  /* column window (a multiple of 32, at most 16,384) of the warp-parallel
                                builders of the tensor-core tile and K-step lists; rows whose columns
                                span more take the serial merges.  0 = 16,384.  Results do not depend
                                on it. */
    int32_t tc_block_copies; /* 1: the split-precision kernel's operand planes sit at their blocks' own
                                positions and every block is one bulk copy (0: at the positions of the
                                transposed blocks, so that neighbouring slots of a K-step share a copy).
                                Results do not depend on it. */
    int32_t pad0;            /* zero */
} rdm_test_knobs;

/* Set the test settings of h (NULL restores all zeros).  RDM_EINVAL for a
 * negative value, a window that is not a multiple of 32 up to 16,384, or a
 * flag other than 0 or 1. */
int rdm_set_test_knobs(rdm_handle *h, const rdm_test_knobs *k);

/* Library version string. */
const char *rdm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RDM_H_ */
