"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative Frobenius error <= 1e-10 for the FP64 path (P0, P1 and
alpha), <= 1e-5 for the FP32 path; integer results (block patterns, branch
sequences) exactly.
"""

import numpy as np
import pytest

from oracle import exact_response, polarizability, tc2_response
from oracle.dense import rel_frobenius
from blockcheck import max_rel_err
from oracle.tc2 import block_truncate
from synth import Bsr, make_batch_config, make_chain, make_cluster, make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def gpu_solve(rdm, systems, **params):
    s = rdm.Solver(0)
    s.set_params(**params)
    s.load(systems)
    code, info = s.solve()
    return s, code, info


def dense_list(sys_):
    return sys_.h0.to_dense(), [m.to_dense() for m in sys_.h1]


# ---------------------------------------------------------------------------
# workload 1: FP64 at zero threshold vs the exact definition
# ---------------------------------------------------------------------------

def test_cfg1_fp64_tau0_vs_exact(rdm):
    s = make_config(1)
    h0, h1s = dense_list(s)
    p0, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    ob = tc2_response(h0, h1s, s.n_occ, s.b, tau=0.0, tol=1e-12)
    sol, code, info = gpu_solve(rdm, s, tau=0.0, tol=1e-12, mode="fp64", max_iter=100)
    assert code == rdm.RDM_OK and info.converged
    assert rel_frobenius(sol.p0().to_dense(), p0) <= 1e-10
    assert max_rel_err(sol.p0().to_dense(), p0) <= 1e-10
    assert rel_frobenius(sol.p1(0, 0).to_dense(), p1s[0]) <= 1e-10
    assert max_rel_err(sol.p1(0, 0).to_dense(), p1s[0]) <= 1e-10
    a = sol.alpha()[0, 0]
    assert a == pytest.approx(polarizability(p1s, h1s)[0, 0], rel=1e-10)
    # same iteration count and branch sequence as the step-by-step oracle
    log = sol.log()
    assert [r["branch"] for r in log] == ob.branches
    assert info.iterations == ob.iterations
    for r, o in zip(log, ob.log):
        assert r["trace"] == pytest.approx(o["trace"], rel=1e-12, abs=1e-12)
    assert abs(info.trace_error) < 1e-10 and abs(info.idempotency) < 1e-9


# ---------------------------------------------------------------------------
# cluster with a ragged last block, tau > 0: per-step replay of the oracle
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cluster150():
    return make_cluster(150, opa=8, b=32, cutoff=10.0, seed=11, dirs=("x", "y", "z"))


@pytest.fixture(scope="module")
def oracle150(cluster150):
    s = cluster150
    h0, h1s = dense_list(s)
    return tc2_response(h0, h1s, s.n_occ, s.b, tau=1e-6, tol=1e-9)


def test_cluster_fp64_tau_vs_stepwise_oracle(rdm, cluster150, oracle150):
    s = cluster150
    assert s.n % s.b != 0          # ragged tail
    ob = oracle150
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=0.0, mode="fp64", max_iter=ob.iterations)
    sol.load(s)
    rdm.rdm_force_branches(sol.h, ob.branches)
    code, info = sol.solve()
    assert info.iterations == ob.iterations
    p0 = sol.p0().to_dense()
    assert rel_frobenius(p0, ob.p0) <= 1e-10
    assert max_rel_err(p0, ob.p0) <= 1e-10
    for d in range(3):
        assert rel_frobenius(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-10
        assert max_rel_err(sol.p1(0, d).to_dense(), ob.p1s[d]) <= 1e-10
    a = sol.alpha()
    h0, h1s = dense_list(s)
    ao = polarizability(ob.p1s, h1s)
    assert np.max(np.abs(a - ao)) <= 1e-10 * np.max(np.abs(ao))
    # block counts per step (integer results): identical except blocks whose
    # norm sits within rounding of tau
    log = sol.log()
    for r, o in zip(log, ob.log):
        assert abs(r["nnzb0"] - o["nnzb0"]) <= 2
        assert r["trace"] == pytest.approx(o["trace"], rel=1e-11)


def test_cluster_fp64_free_run_matches_oracle_limit(rdm, cluster150, oracle150):
    s = cluster150
    sol, code, info = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode="fp64")
    assert code == rdm.RDM_OK
    assert rel_frobenius(sol.p0().to_dense(), oracle150.p0) <= 1e-9
    assert max_rel_err(sol.p0().to_dense(), oracle150.p0) <= 1e-9
    for d in range(3):
        assert rel_frobenius(sol.p1(0, d).to_dense(), oracle150.p1s[d]) <= 1e-8
        assert max_rel_err(sol.p1(0, d).to_dense(), oracle150.p1s[d]) <= 1e-8


def test_fp64_large_threshold_stays_bounded(rdm, cluster150):
    """tau = 1e-4: the filter pushes eigenvalues out of [0, 1]; the FP64 path
    alternates the branch like the oracle (e < -1e-10 N_occ) and stays bounded
    with alpha at the accuracy the threshold allows (the trace test alone
    diverges here)."""
    s = cluster150
    h0, h1s = dense_list(s)
    _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    ae = polarizability(p1s, h1s)
    sol, code, info = gpu_solve(rdm, s, tau=1e-4, tol=0.0, mode="fp64", max_iter=40)
    a = sol.alpha()
    assert np.isfinite(a).all()
    assert np.max(np.abs(a - ae)) / np.max(np.abs(ae)) < 1e-5
    assert abs(info.trace_error) < 1e-3


def test_hash_symbolic_phase_is_identical(rdm, cluster150):
    """The hash-table symbolic phase (used above 8,192 block rows) gives the same
    masks, pair counts and therefore bit-identical results as the dense one."""
    s = cluster150
    ref, _, _ = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode="fp64")
    hsh, code, info = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode="fp64", symbolic_hash=1)
    assert code == rdm.RDM_OK
    assert np.array_equal(hsh.p0().col_idx, ref.p0().col_idx)
    assert np.array_equal(hsh.p0().vals, ref.p0().vals)
    for d in range(3):
        assert np.array_equal(hsh.p1(0, d).vals, ref.p1(0, d).vals)


@pytest.mark.parametrize("mode", ["fp64", "mixed_fp16"])
def test_job_groups_are_identical(rdm, cluster150, mode):
    """A cap on the untruncated-product buffer (1 MiB: 128 blocks) splits every
    step into many groups of super-rows, so most lower blocks take their
    transpose from an earlier group's compacted output; masks, values and
    alpha stay bit-identical to the single-group run."""
    s = cluster150
    ref, _, rinfo = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode=mode)
    grp, code, info = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode=mode, chunk_mb=1)
    assert code == rdm.RDM_OK
    assert rinfo.product_groups == 1 and info.product_groups >= 8
    assert info.iterations == rinfo.iterations
    assert info.device_bytes_peak > 0
    assert np.array_equal(grp.p0().col_idx, ref.p0().col_idx)
    assert np.array_equal(grp.p0().vals, ref.p0().vals)
    for d in range(3):
        assert np.array_equal(grp.p1(0, d).col_idx, ref.p1(0, d).col_idx)
        assert np.array_equal(grp.p1(0, d).vals, ref.p1(0, d).vals)
    assert np.array_equal(grp.alpha(), ref.alpha())


def test_job_groups_batch_identical(rdm):
    """Job groups over a batch of uneven systems (chains and clusters)."""
    systems = make_batch_config(n_systems=4, lo=40, hi=160)
    ref, _, _ = gpu_solve(rdm, systems, tau=1e-6, tol=1e-9, mode="mixed_fp16")
    grp, code, info = gpu_solve(rdm, systems, tau=1e-6, tol=1e-9, mode="mixed_fp16", chunk_mb=1)
    assert code == rdm.RDM_OK and info.product_groups > 1
    for k in range(len(systems)):
        assert np.array_equal(grp.p0(k).vals, ref.p0(k).vals)
        for d in range(3):
            assert np.array_equal(grp.p1(k, d).vals, ref.p1(k, d).vals)
        assert np.array_equal(grp.alpha(k), ref.alpha(k))


def test_cluster_fp32_vs_oracle(rdm, cluster150, oracle150):
    s = cluster150
    sol, code, info = gpu_solve(rdm, s, tau=1e-6, tol=1e-9, mode="fp32")
    assert code in (rdm.RDM_OK, rdm.RDM_NOT_CONVERGED)
    assert rel_frobenius(sol.p0().to_dense(), oracle150.p0) <= 1e-5
    assert max_rel_err(sol.p0().to_dense(), oracle150.p0) <= 1e-5
    for d in range(3):
        assert rel_frobenius(sol.p1(0, d).to_dense(), oracle150.p1s[d]) <= 1e-5
        assert max_rel_err(sol.p1(0, d).to_dense(), oracle150.p1s[d]) <= 1e-5


# ---------------------------------------------------------------------------
# the single-product primitive for every block size
# ---------------------------------------------------------------------------

def _sym_bsr(rng, n, b, density, scale=1.0):
    nb = -(-n // b)
    mask = rng.random((nb, nb)) < density
    mask = mask | mask.T
    np.fill_diagonal(mask, True)
    a = rng.standard_normal((n, n)) * scale
    a = a + a.T
    full = np.repeat(np.repeat(mask, b, 0), b, 1)[:n, :n]
    a = np.where(full, a, 0.0)
    return a, Bsr.from_dense(a, b, drop_zero_blocks=False, keep_diagonal=True)


@pytest.mark.parametrize("b", [4, 16, 32, 64])
@pytest.mark.parametrize("terms", [1, 2])
def test_block_product_fp32(rdm, b, terms):
    """FP32 CUDA-core products (the tuned 32 x 32 kernel for b = 32) against
    the dense FP64 product: FP32 rounding only (<= 2e-6 relative)."""
    rng = np.random.default_rng(300 + b + terms)
    n = 6 * b + b // 2
    a, A = _sym_bsr(rng, n, b, 0.4)
    bd, B = _sym_bsr(rng, n, b, 0.4, 0.5)
    x, X = _sym_bsr(rng, n, b, 0.5, 0.25)
    h = rdm.rdm_create(0)
    try:
        for c_lin, c_sq in ((0.0, 1.0), (2.0, -1.0)):
            prod = a @ a if terms == 1 else a @ bd + bd @ a
            ref = c_lin * x + c_sq * prod
            res = rdm.rdm_block_product(h, A, B if terms == 2 else None, X, c_lin, c_sq, terms, 0.0,
                                        rdm.MODES["fp32"])
            got = res.to_dense()
            assert rel_frobenius(got, ref) <= 2e-6
            assert max_rel_err(got, ref) <= 2e-6
            assert np.array_equal(got, got.T)
    finally:
        rdm.rdm_destroy(h)


@pytest.mark.parametrize("b", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("terms", [1, 2])
def test_block_product_fp64(rdm, b, terms):
    rng = np.random.default_rng(100 + b + terms)
    n = 5 * b + max(1, b // 2) if b > 1 else 13     # ragged
    a, A = _sym_bsr(rng, n, b, 0.3)
    bd, B = _sym_bsr(rng, n, b, 0.3, 0.5)
    x, X = _sym_bsr(rng, n, b, 0.5, 0.25)
    h = rdm.rdm_create(0)
    try:
        for c_lin, c_sq, tau in ((0.0, 1.0, 0.0), (2.0, -1.0, 0.5)):
            prod = a @ a if terms == 1 else a @ bd + bd @ a
            ref = block_truncate(c_lin * x + c_sq * prod, b, tau)
            res = rdm.rdm_block_product(h, A, B if terms == 2 else None, X, c_lin, c_sq, terms, tau,
                                        rdm.MODE_FP64)
            got = res.to_dense()
            assert rel_frobenius(got, ref) <= 1e-13
            assert max_rel_err(got, ref) <= 1e-13
            # kept blocks: exactly the blocks of ref with norm >= tau
            nb = -(-n // b)
            pad = np.zeros((nb * b, nb * b))
            pad[:n, :n] = ref
            ref_blocks = np.linalg.norm(pad.reshape(nb, b, nb, b), axis=(1, 3)) > 0
            got_blocks = np.zeros((nb, nb), bool)
            rows = np.repeat(np.arange(nb), np.diff(res.row_ptr))
            got_blocks[rows, res.col_idx] = True
            assert np.array_equal(got_blocks, ref_blocks)
    finally:
        rdm.rdm_destroy(h)


# ---------------------------------------------------------------------------
# batching, errors, edge cases
# ---------------------------------------------------------------------------

def test_batch_matches_individual_solves(rdm):
    systems = [make_chain(30, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=5, dirs=("x", "y", "z")),
               make_cluster(60, opa=8, b=32, cutoff=10.0, seed=6, dirs=("x", "y", "z")),
               make_cluster(23, opa=8, b=32, cutoff=10.0, seed=7, dirs=("x", "y", "z"))]
    sol, code, info = gpu_solve(rdm, systems, tau=1e-7, tol=1e-9, mode="fp64")
    assert code == rdm.RDM_OK
    for k, s in enumerate(systems):
        one, _, _ = gpu_solve(rdm, s, tau=1e-7, tol=1e-9, mode="fp64")
        assert np.array_equal(sol.p0(k).vals, one.p0().vals)
        assert np.allclose(sol.alpha(k), one.alpha(), rtol=1e-13)
        h0, h1s = dense_list(s)
        _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
        ae = polarizability(p1s, h1s)
        assert np.max(np.abs(sol.alpha(k) - ae)) <= 1e-6 * np.max(np.abs(ae))


def test_partitioned_batch_matches_the_whole_batch(rdm):
    """The multi-GPU path partitions a batch over ranks (bench.partition) and
    each rank solves its share as a batch of its own.  On one GPU: the two
    shares of a 2-rank partition, solved one after the other, give every
    system's P0 bit for bit, and alpha to rounding (the per-system sum of the
    row partials may group differently), as the whole batch does (FP64)."""
    import bench
    systems = [make_chain(30, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=5, dirs=("x", "y", "z")),
               make_cluster(60, opa=8, b=32, cutoff=10.0, seed=6, dirs=("x", "y", "z")),
               make_cluster(23, opa=8, b=32, cutoff=10.0, seed=7, dirs=("x", "y", "z")),
               make_chain(44, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=8, dirs=("x", "y", "z"))]
    whole, code, _ = gpu_solve(rdm, systems, tau=1e-7, tol=1e-9, mode="fp64")
    assert code == rdm.RDM_OK
    shares = bench.partition([bench.work_estimate(s) for s in systems], 2)
    assert sorted(shares[0] + shares[1]) == [0, 1, 2, 3] and shares[0] and shares[1]
    for share in shares:
        part, code, _ = gpu_solve(rdm, [systems[k] for k in share], tau=1e-7, tol=1e-9, mode="fp64")
        assert code == rdm.RDM_OK
        for q, k in enumerate(share):
            assert np.array_equal(part.p0(q).vals, whole.p0(k).vals)
            assert np.allclose(part.alpha(q), whole.alpha(k), rtol=1e-13, atol=0)


def test_bad_inputs_are_rejected(rdm):
    s = make_config(1, n_atoms=8)
    h = rdm.rdm_create(0)
    try:
        bad = Bsr(s.h0.nb, s.h0.b, s.h0.n, s.h0.row_ptr.copy(), s.h0.col_idx.copy(), s.h0.vals.copy())
        bad.vals[0, 0, 1] += 1.0                      # breaks value symmetry of a diagonal block
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_upload_h0(h, 0, bad, s.n_electrons)
        assert e.value.code == rdm.RDM_EBADBSR
        nan = Bsr(s.h0.nb, s.h0.b, s.h0.n, s.h0.row_ptr.copy(), s.h0.col_idx.copy(), s.h0.vals.copy())
        nan.vals[1, 0, 0] = np.nan
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_upload_h0(h, 0, nan, s.n_electrons)
        assert e.value.code == rdm.RDM_EBADBSR
        unsorted = Bsr(s.h0.nb, s.h0.b, s.h0.n, s.h0.row_ptr.copy(), s.h0.col_idx.copy(), s.h0.vals.copy())
        r0, r1 = unsorted.row_ptr[1], unsorted.row_ptr[2]
        unsorted.col_idx[r0:r1] = unsorted.col_idx[r0:r1][::-1]
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_upload_h0(h, 0, unsorted, s.n_electrons)
        assert e.value.code == rdm.RDM_EBADBSR
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_upload_h0(h, 0, s.h0, 7)          # odd electron count
        assert e.value.code == rdm.RDM_EINVAL
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_get_alpha(h, 0)                   # no solve yet
        assert e.value.code == rdm.RDM_ESTATE
        p = rdm.rdm_default_params()
        p.use_graphs = 1                              # reserved: graph capture is not implemented
        with pytest.raises(rdm.RdmError) as e:
            rdm.rdm_set_params(h, p)
        assert e.value.code == rdm.RDM_EINVAL
    finally:
        rdm.rdm_destroy(h)


def test_not_converged_is_a_warning_with_readable_results(rdm):
    s = make_config(1)
    sol, code, info = gpu_solve(rdm, s, tau=0.0, tol=1e-12, mode="fp64", max_iter=3)
    assert code == rdm.RDM_NOT_CONVERGED and info.iterations == 3 and not info.converged
    assert sol.p0().nnzb > 0


def test_no_perturbation_and_single_block(rdm):
    s = make_chain(4, opa=4, b=16, spacing=2.8, cutoff=8.0, seed=2, dirs=("x",))
    s.h1 = []
    s.dirs = ()
    sol, code, info = gpu_solve(rdm, s, tau=0.0, tol=1e-12, mode="fp64")
    assert code == rdm.RDM_OK and s.h0.nb == 1
    p0, _, _, _ = exact_response(s.h0.to_dense(), [], s.n_occ)
    assert rel_frobenius(sol.p0().to_dense(), p0) <= 1e-10
    assert max_rel_err(sol.p0().to_dense(), p0) <= 1e-10
    assert np.all(np.isnan(sol.alpha()))
