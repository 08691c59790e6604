"""Tensor-core (tcgen05) products and the mixed-precision solve against the
CPU oracle.

The split products hi*hi + hi*lo + lo*hi with 8-bit (bf16) or 11-bit (fp16)
significands and FP32 accumulation have a relative error of order 2^-16
(bf16: |x - hi - lo| <= 2^-16 |x|, the dropped lo*lo term is of the same
order) plus the FP32 accumulation error; the product test allows 3e-5
relative Frobenius error.  The mixed solve (split products until the
idempotency error stalls, then FP64) must reproduce the FP64 oracle's alpha
to 1e-6 relative and P0/P1 to 1e-5.
"""

import numpy as np
import pytest

from oracle import polarizability, tc2_response
from oracle.dense import rel_frobenius
from blockcheck import max_rel_err
from oracle.tc2 import block_norms, block_truncate
from synth import Bsr, make_chain, make_cluster

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def _sym_bsr(rng, n, b, density, scale=1.0, decay=None):
    nb = -(-n // b)
    mask = rng.random((nb, nb)) < density
    mask = mask | mask.T
    np.fill_diagonal(mask, True)
    a = rng.standard_normal((n, n)) * scale
    if decay is not None:
        idx = np.arange(n)
        a *= np.exp(-np.abs(idx[:, None] - idx[None, :]) / decay)
    a = a + a.T
    full = np.repeat(np.repeat(mask, b, 0), b, 1)[:n, :n]
    a = np.where(full, a, 0.0)
    return a, Bsr.from_dense(a, b, drop_zero_blocks=False, keep_diagonal=True)


@pytest.mark.parametrize("b", [16, 32, 64])
@pytest.mark.parametrize("mode", ["mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("terms", [1, 2])
@pytest.mark.parametrize("nblk", [3, 9, 13])
def test_tc_block_product(rdm, b, mode, terms, nblk):
    """Split products on the tensor cores for every block size they take
    (16 x 16 blocks: 8 x 16-block tiles; 32: 4 x 8; 64: 2 x 4, each output
    block spread over two TMEM lane quarters), ragged last block, with and
    without the linear term and truncation."""
    rng = np.random.default_rng(7 * nblk + terms + b)
    n = nblk * b - 5                                  # ragged last block
    a, A = _sym_bsr(rng, n, b, 0.35)
    bd, B = _sym_bsr(rng, n, b, 0.35, 0.5)
    x, X = _sym_bsr(rng, n, b, 0.5, 0.25)
    h = rdm.rdm_create(0)
    try:
        # the solver's coefficients, and a ratio c_lin / c_sq that is not a power of two
        for c_lin, c_sq, tau in ((0.0, 1.0, 0.0), (2.0, -1.0, 2.0), (0.5, 3.0, 0.0)):
            prod = a @ a if terms == 1 else a @ bd + bd @ a
            exact = c_lin * x + c_sq * prod
            ref = block_truncate(exact, b, tau)
            res = rdm.rdm_block_product(h, A, B if terms == 2 else None, X, c_lin, c_sq, terms, tau,
                                        rdm.MODES[mode])
            got = res.to_dense()
            assert rel_frobenius(got, ref) <= 3e-5, mode
            assert max_rel_err(got, ref) <= 3e-5, mode
            # blocks clearly above / below the threshold are kept / dropped
            nrm = block_norms(exact, b)
            nb = nrm.shape[0]
            kept = np.zeros((nb, nb), bool)
            rows = np.repeat(np.arange(nb), np.diff(res.row_ptr))
            kept[rows, res.col_idx] = True
            assert np.all(kept[(nrm >= tau * 1.001) & (nrm > 0)])
            if tau > 0:
                assert not np.any(kept[nrm < tau * 0.999])
            assert np.allclose(got, got.T, rtol=0, atol=0)     # exactly symmetric
    finally:
        rdm.rdm_destroy(h)


def test_tc_product_with_c_sq_zero_is_the_linear_term(rdm):
    """c_sq = 0 leaves C = c_lin X: on the tensor-core paths X enters the
    epilogue rounded to FP32, so C matches c_lin X to FP32 rounding."""
    rng = np.random.default_rng(5)
    a, A = _sym_bsr(rng, 3 * 32, 32, 0.5)
    h = rdm.rdm_create(0)
    try:
        for mode in (rdm.MODE_MIXED_BF16, rdm.MODE_MIXED_FP16):
            r = rdm.rdm_block_product(h, A, None, A, 1.5, 0.0, 1, 0.0, mode).to_dense()
            assert max_rel_err(r, 1.5 * a) <= 1e-7
        r = rdm.rdm_block_product(h, A, None, A, 1.5, 0.0, 1, 0.0, rdm.MODE_FP64).to_dense()
        assert np.array_equal(r, 1.5 * a)
    finally:
        rdm.rdm_destroy(h)


def test_tc_product_matches_fp64_kernel_closely(rdm):
    """The same product through the FP64 CUDA-core kernel and the split
    tensor-core kernel: differences of order 2^-16 relative, not more."""
    rng = np.random.default_rng(3)
    n = 10 * 32
    a, A = _sym_bsr(rng, n, 32, 0.5, decay=40.0)
    h = rdm.rdm_create(0)
    try:
        r64 = rdm.rdm_block_product(h, A, None, None, 0.0, 1.0, 1, 0.0, rdm.MODE_FP64).to_dense()
        rbf = rdm.rdm_block_product(h, A, None, None, 0.0, 1.0, 1, 0.0, rdm.MODE_MIXED_BF16).to_dense()
        assert rel_frobenius(r64, a @ a) <= 1e-13
        assert max_rel_err(r64, a @ a) <= 1e-13
        assert 1e-9 < rel_frobenius(rbf, r64) <= 3e-5
    finally:
        rdm.rdm_destroy(h)


def test_tc_accumulation_does_not_drift_with_k(rdm):
    """The tensor cores' FP32 accumulation truncates; on positive data one
    accumulator over 96 K-steps loses 2e-5 of the result.  The kernel
    accumulates segments of 4 K-steps and adds them with round-to-nearest,
    so the bias stays at the level of one segment for any K."""
    h = rdm.rdm_create(0)
    try:
        for nblk in (8, 96):
            rng = np.random.default_rng(nblk)
            n = nblk * 32
            a = rng.random((n, n))
            a = a + a.T
            A = Bsr.from_dense(a, 32, drop_zero_blocks=False)
            got = rdm.rdm_block_product(h, A, None, None, 0.0, 1.0, 1, 0.0, rdm.MODES["mixed_fp16"]).to_dense()
            bias = float(np.mean((got - a @ a) / (a @ a)))
            assert -1.5e-6 < bias < 1.5e-6, (nblk, bias)
    finally:
        rdm.rdm_destroy(h)


@pytest.fixture(scope="module")
def cluster150():
    return make_cluster(150, opa=8, b=32, cutoff=10.0, seed=11, dirs=("x", "y", "z"))


@pytest.fixture(scope="module")
def oracle150(cluster150):
    s = cluster150
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    return tc2_response(h0, h1s, s.n_occ, s.b, tau=1e-6, tol=1e-9), h1s


@pytest.mark.parametrize("mode", ["mixed_bf16", "mixed_fp16"])
def test_mixed_solve_vs_oracle(rdm, cluster150, oracle150, mode):
    s = cluster150
    ob, h1s = oracle150
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode=mode, max_iter=100)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK and info.converged
    assert info.tier_iters[0] > 0 and info.tier_iters[1] > 0      # both tiers used
    a = sol.alpha()
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(a - ao)) / np.max(np.abs(ao)) <= 1e-6
    assert rel_frobenius(sol.p0().to_dense(), ob.p0) <= 1e-5
    assert max_rel_err(sol.p0().to_dense(), ob.p0) <= 1e-5
    for d in range(3):
        assert rel_frobenius(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-4
        assert max_rel_err(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-4
    assert abs(info.idempotency) < 1e-8 and abs(info.trace_error) < 1e-8


@pytest.mark.parametrize("refine,tol", [(1, 1e-6), (3, 1e-6), (2, 1e-6)])
def test_final_tier_first_order_arithmetic(rdm, cluster150, oracle150, refine, tol):
    """Final tier of the fp16 ladder (X0^2 refined as tensor-core slice products, the default): X1 products in FP64 (1),
    FP32 on the CUDA cores (3), or kept on the tensor cores (2, the default;
    with segmented accumulation as accurate as FP32)."""
    s = cluster150
    ob, h1s = oracle150
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100, refine_x1=refine)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK and info.converged
    a = sol.alpha()
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(a - ao)) / np.max(np.abs(ao)) <= tol
    assert abs(info.idempotency) < 1e-8


def test_final_tier_double_fp32_purification(rdm, cluster150):
    """refine_x0 = double-FP32 (error-free transformations on the FP32 pipe):
    the refined X0 is FP64-class, so P0, P1 and alpha agree with the FP64
    refinement far below the split tier's own error, and P0 is idempotent to
    the same floor."""
    s = cluster150
    out = {}
    for r0 in (1, 4):
        sol = rdm.Solver(0)
        sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100, refine_x0=r0)
        sol.load(s)
        code, info = sol.solve()
        assert code == rdm.RDM_OK and info.converged
        out[r0] = (sol.alpha(), sol.p0().to_dense(), info)
    (a64, p64, i64), (aff, pff, iff) = out[1], out[4]
    assert iff.kernel_flops[3] > 0 and iff.kernel_flops[1] == 0.0
    assert iff.iterations == i64.iterations
    assert rel_frobenius(pff, p64) <= 1e-9
    assert max_rel_err(pff, p64) <= 1e-9
    assert np.max(np.abs(aff - a64)) / np.max(np.abs(a64)) <= 1e-9
    assert abs(iff.idempotency) < 1e-8


@pytest.mark.parametrize("nblk", [3, 9, 13])
def test_slice_product_is_fp64_class(rdm, nblk):
    """X^2 from exact bf16 slice products on the tensor cores (row-scaled
    integer slices, 7 per element, slice pairs summed exactly per group in
    FP32 tensor memory, groups in double-FP32): FP64-class, i.e. within a few
    2^-48 of the product's scale, where the split product is at 2^-22 and the
    FP64 kernel at 2^-53.  Entries of very different sizes (exponential decay
    away from the diagonal) exercise the row scaling."""
    rng = np.random.default_rng(100 + nblk)
    b = 32
    n = nblk * b - 5
    a, A = _sym_bsr(rng, n, b, 0.6, decay=12.0)
    h = rdm.rdm_create(0)
    try:
        ref = a @ a
        got = rdm.rdm_block_product(h, A, None, None, 0.0, 1.0, 1, 0.0, rdm.PRODUCT_SLICES).to_dense()
        split = rdm.rdm_block_product(h, A, None, None, 0.0, 1.0, 1, 0.0, rdm.MODES["mixed_fp16"]).to_dense()
        scale = np.max(np.abs(ref))
        err = np.max(np.abs(got - ref)) / scale
        assert err <= 2e-13, err
        assert np.max(np.abs(split - ref)) / scale > 100 * err
        assert np.array_equal(got, got.T)                 # exactly symmetric without symmetrisation
        # the linear term and truncation in FP64: C = 2 X - X^2, blocks below tau dropped
        x, X = _sym_bsr(rng, n, b, 0.6, decay=12.0)
        got2 = rdm.rdm_block_product(h, A, None, X, 2.0, -1.0, 1, 1e-3, rdm.PRODUCT_SLICES).to_dense()
        ref2 = block_truncate(2.0 * x - ref, b, 1e-3)
        assert np.max(np.abs(got2 - ref2)) / np.max(np.abs(ref2)) <= 2e-13
    finally:
        rdm.rdm_destroy(h)


def test_final_tier_slice_products(rdm, cluster150, oracle150):
    """refine_x0 = slices: the final tier's X0^2 on the tensor cores as exact
    slice products.  P0 agrees with the FP64 refinement far below the split
    tier's own error and ends idempotent to the FP64 floor; alpha meets the
    oracle."""
    s = cluster150
    ob, h1s = oracle150
    out = {}
    for r0 in (1, rdm.REFINE_SLICES):
        sol = rdm.Solver(0)
        sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100, refine_x0=r0)
        sol.load(s)
        code, info = sol.solve()
        assert code == rdm.RDM_OK and info.converged
        out[r0] = (sol.alpha(), sol.p0().to_dense(), info)
    (a64, p64, i64), (aoz, poz, ioz) = out[1], out[rdm.REFINE_SLICES]
    assert ioz.kernel_flops[4] > 0 and ioz.kernel_flops[1] == 0.0 and ioz.kernel_ms[7] > 0
    assert rel_frobenius(poz, p64) <= 1e-9
    assert max_rel_err(poz, p64) <= 1e-9
    assert np.max(np.abs(aoz - a64)) / np.max(np.abs(a64)) <= 1e-9
    assert abs(ioz.idempotency) < 1e-8
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(aoz - ao)) / np.max(np.abs(ao)) <= 1e-6


def test_final_tier_fp32_purification(rdm, cluster150, oracle150):
    """refine_x0 = FP32: the whole final tier on the FP32 CUDA cores.  It ends
    on the idempotency stall (FP32 floor) instead of the FP64 one; alpha stays
    within 1e-6 of the oracle."""
    s = cluster150
    ob, h1s = oracle150
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100, refine_x0=3)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK and info.converged
    assert info.kernel_flops[1] == 0.0          # no FP64 products
    a = sol.alpha()
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(a - ao)) / np.max(np.abs(ao)) <= 1e-6
    assert abs(info.idempotency) < 1e-3


def test_mixed_batch_with_converged_copies(rdm):
    systems = [make_chain(40, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=21, dirs=("x", "y", "z")),
               make_cluster(90, opa=8, b=32, cutoff=10.0, seed=22, dirs=("x", "y", "z"))]
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_bf16", max_iter=100)
    sol.load(systems)
    code, info = sol.solve()
    assert code == rdm.RDM_OK
    # the chain's alpha carries the dipole range (|x| up to 55 bohr) as an error
    # amplifier: the 16-bit bf16 split reaches ~2e-6 there (the CPU emulation
    # of the same split gives 2.9e-6), the cluster 8e-7
    tol = [5e-6, 1e-6]
    for k, s in enumerate(systems):
        one = rdm.Solver(0)
        one.set_params(tau=1e-6, tol=1e-9, mode="fp64", max_iter=100)
        one.load(s)
        one.solve()
        a1, a0 = sol.alpha(k), one.alpha()
        assert np.max(np.abs(a1 - a0)) / np.max(np.abs(a0)) <= tol[k]
        assert np.allclose(sol.p0(k).to_dense(), one.p0().to_dense(), atol=1e-5)
    # the scaled fp16 split with the FP32 refinement of X1 meets 1e-6 on both
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100)
    code, info = sol.solve()
    assert code == rdm.RDM_OK
    for k, s in enumerate(systems):
        one = rdm.Solver(0)
        one.set_params(tau=1e-6, tol=1e-9, mode="fp64", max_iter=100)
        one.load(s)
        one.solve()
        a1, a0 = sol.alpha(k), one.alpha()
        assert np.max(np.abs(a1 - a0)) / np.max(np.abs(a0)) <= 1e-6


def test_bf16_final_tier_keeps_the_first_order_products_split(rdm, cluster150, oracle150):
    """The bf16 ladder's final tier refines X0^2 (slice products) and keeps the
    first-order products as bf16 split products by default: no FP64 products
    at all, alpha within 1e-6 of the oracle and within 5e-7 of the same ladder
    with FP64 first-order products in the final tier (the bulk tier's error
    dominates both)."""
    s = cluster150
    ob, h1s = oracle150
    ao = polarizability(ob.p1s, h1s)
    out = {}
    for r1 in (0, 1):
        sol = rdm.Solver(0)
        sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_bf16", max_iter=100, refine_x1=r1)
        sol.load(s)
        code, info = sol.solve()
        assert code == rdm.RDM_OK and info.converged
        assert info.tier_iters[0] > 0 and info.tier_iters[1] > 0
        out[r1] = (sol.alpha().copy(), info)
    (a_split, i_split), (a_64, i_64) = out[0], out[1]
    assert i_split.kernel_flops[1] == 0.0 and i_64.kernel_flops[1] > 0
    assert np.max(np.abs(a_split - ao)) / np.max(np.abs(ao)) <= 1e-6
    assert np.max(np.abs(a_split - a_64)) / np.max(np.abs(a_64)) <= 5e-7


@pytest.mark.parametrize("b", [16, 64])
@pytest.mark.parametrize("mode", ["mixed_bf16", "mixed_fp16"])
def test_mixed_solve_other_block_sizes_vs_oracle(rdm, b, mode):
    """The whole mixed ladder with 16 x 16 and 64 x 64 blocks (ragged last
    block at 64) against oracle B at the same block partition."""
    s = make_cluster(150, opa=8, b=b, cutoff=10.0, seed=11, dirs=("x", "y", "z"))
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    ob = tc2_response(h0, h1s, s.n_occ, s.b, tau=1e-6, tol=1e-9)
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode=mode, max_iter=100, refine_x0=3, refine_x1=2)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK and info.converged
    assert info.tc_launches > 0 and info.kernel_flops[1] == 0.0
    a = sol.alpha()
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(a - ao)) / np.max(np.abs(ao)) <= 1e-6
    assert rel_frobenius(sol.p0().to_dense(), ob.p0) <= 1e-5
    assert max_rel_err(sol.p0().to_dense(), ob.p0) <= 1e-5
    for d in range(3):
        assert rel_frobenius(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-4
        assert max_rel_err(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-4


def test_expired_wait_returns_etimeout_and_the_handle_stays_usable(rdm, cluster150):
    """The tensor-core kernel bounds every wait.  With a short bound and its
    copy warp waiting for a flag that nothing sets, the wait runs out: the
    kernel raises its abort flag, drains, frees its tensor memory and returns;
    the solve reports RDM_ETIMEOUT, and the same handle then solves to the
    same bits as before."""
    s = cluster150
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100)
    sol.load(s)
    code, _ = sol.solve()
    assert code == rdm.RDM_OK
    a_ref, p0_ref = sol.alpha().copy(), sol.p0().vals.copy()
    rdm.rdm_set_test_knobs(sol.h, tc_wait_cycles=2_000_000, tc_hold=1)     # ~1 ms
    with pytest.raises(rdm.RdmError) as e:
        sol.solve()
    assert e.value.code == rdm.RDM_ETIMEOUT
    rdm.rdm_set_test_knobs(sol.h)
    code, _ = sol.solve()
    assert code == rdm.RDM_OK
    assert np.array_equal(sol.alpha(), a_ref) and np.array_equal(sol.p0().vals, p0_ref)


def test_serial_plan_builders_give_the_same_tiles(rdm, cluster150):
    """Tile rows and K-steps whose columns span more than the bitmap window
    are built by serial merges; with a 32-column window most of them take
    that path here.  The tiles, their K-steps and so every bit of the result
    are the same as with the warp-parallel builders."""
    s = cluster150
    res = []
    for window in (0, 32):
        sol = rdm.Solver(0)
        rdm.rdm_set_test_knobs(sol.h, tc_window_cols=window)
        sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100)
        sol.load(s)
        code, _ = sol.solve()
        assert code == rdm.RDM_OK
        res.append((sol.alpha().copy(), sol.p0().vals.copy(), [sol.p1(0, d).vals.copy() for d in range(3)]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    for d in range(3):
        assert np.array_equal(res[0][2][d], res[1][2][d])


@pytest.mark.parametrize("b,mode", [(16, "mixed_fp16"), (32, "mixed_fp16"), (32, "mixed_bf16"), (64, "mixed_fp16")])
def test_run_copies_give_the_same_bits_as_block_copies(rdm, b, mode):
    """The operand planes sit at the positions of the transposed blocks so
    that neighbouring slots of a K-step come in one bulk copy; with the test
    setting the planes sit at their own positions and every block is a copy
    of its own.  The MMAs see the same operands either way: every bit of the
    result is the same."""
    s = make_cluster(150, opa=8, b=b, cutoff=10.0, seed=11, dirs=("x", "y", "z"))
    res = []
    for block_copies in (0, 1):
        sol = rdm.Solver(0)
        rdm.rdm_set_test_knobs(sol.h, tc_block_copies=block_copies)
        sol.set_params(tau=1e-6, tol=1e-9, mode=mode, max_iter=100, block_size=b, autotune=0)
        sol.load(s)
        code, info = sol.solve()
        assert code == rdm.RDM_OK and info.tc_launches > 0
        res.append((sol.alpha().copy(), sol.p0().vals.copy(), [sol.p1(0, d).vals.copy() for d in range(3)]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    for d in range(3):
        assert np.array_equal(res[0][2][d], res[1][2][d])


def test_test_knobs_are_validated(rdm):
    h = rdm.rdm_create(0)
    try:
        for bad in (dict(tc_window_cols=33), dict(tc_window_cols=16416), dict(tc_wait_cycles=-1), dict(tc_hold=2),
                    dict(tc_block_copies=2), dict(tc_block_copies=-1)):
            with pytest.raises(rdm.RdmError):
                rdm.rdm_set_test_knobs(h, **bad)
    finally:
        rdm.rdm_destroy(h)


def test_mixed_modes_reject_unsupported_block_sizes_up_front(rdm):
    s = make_chain(8, opa=4, b=4, spacing=2.8, cutoff=8.0, seed=0, dirs=("x",))   # b = 4: below 16
    sol = rdm.Solver(0)
    sol.set_params(mode="mixed_fp16")
    with pytest.raises(rdm.RdmError) as e:
        sol.load(s)
    assert e.value.code == rdm.RDM_EINVAL
    sol.set_params(mode="fp64")
    sol.load(s)
    with pytest.raises(rdm.RdmError) as e:
        sol.set_params(mode="mixed_bf16")
    assert e.value.code == rdm.RDM_EINVAL
