"""Block size of the solve (re-blocking, autotuning), the asynchronous solve
and the stall window of the precision ladder, through the C ABI.

Re-blocking stores the same matrices in other blocks; the filter then acts
on the new blocks, so a solve of matrices uploaded with 32 x 32 blocks and
run at block size b' equals, bit for bit in FP64, the solve of the same
matrices uploaded with b' x b' blocks (the extra blocks the split keeps are
zero and drop out at the first truncation)."""

import numpy as np
import pytest

from oracle import exact_response, polarizability
from synth import make_cluster
from blockcheck import max_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def cluster(b):
    return make_cluster(150, opa=8, b=b, cutoff=10.0, seed=11, dirs=("x", "y", "z"))


@pytest.fixture(scope="module")
def exact_alpha():
    s = cluster(32)
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    return polarizability(p1s, h1s)


def solve(rdm, s, **params):
    sol = rdm.Solver(0)
    sol.set_params(**params)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK
    return sol, info


@pytest.mark.parametrize("bs", [16, 64])
def test_fp64_solve_at_another_block_size_equals_native_upload(rdm, bs):
    native, _ = solve(rdm, cluster(bs), tau=1e-6, tol=1e-9, mode="fp64")
    reblocked, info = solve(rdm, cluster(32), tau=1e-6, tol=1e-9, mode="fp64", block_size=bs)
    assert info.block_size == bs
    p = reblocked.p0()
    assert p.b == 32 and p.nb == 38                       # back in the uploaded layout
    assert np.array_equal(p.to_dense(), native.p0().to_dense())
    for d in range(3):
        assert np.array_equal(reblocked.p1(0, d).to_dense(), native.p1(0, d).to_dense())
    assert np.array_equal(reblocked.alpha(), native.alpha())
    # the size queries agree with what the getters return
    assert rdm.rdm_get_p0_nnzb(reblocked.h, 0) == p.nnzb


@pytest.mark.parametrize("mode", ["mixed_fp16", "mixed_bf16"])
def test_autotune_probes_every_block_size_and_keeps_the_fastest(rdm, exact_alpha, mode):
    s = cluster(32)
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode=mode, autotune=1)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK
    probes = list(info.probe_ms)
    assert all(p > 0 for p in probes) and info.autotune_ms >= sum(probes) * 0.99
    assert info.block_size == [16, 32, 64][int(np.argmin(probes))]
    a = sol.alpha()
    assert np.max(np.abs(a - exact_alpha)) / np.max(np.abs(exact_alpha)) <= 1e-6
    assert sol.p0().b == 32
    # later solves keep the choice without probing again, also after a new
    # upload of a problem of the same shape
    code, info2 = sol.solve()
    assert info2.block_size == info.block_size and list(info2.probe_ms) == probes
    sol.load(s)
    code, info3 = sol.solve()
    assert info3.block_size == info.block_size and list(info3.probe_ms) == probes
    assert info3.time_ms < 0.8 * info.autotune_ms
    assert np.max(np.abs(sol.alpha() - exact_alpha)) / np.max(np.abs(exact_alpha)) <= 1e-6


def test_async_solve_matches_the_blocking_one(rdm):
    s = cluster(32)
    ref, _ = solve(rdm, s, tau=1e-6, tol=1e-9, mode="mixed_fp16")
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16")
    sol.load(s)
    with pytest.raises(rdm.RdmError) as e:
        sol.sync()                                        # nothing in flight
    assert e.value.code == rdm.RDM_ESTATE
    sol.solve_async()
    code, info = sol.sync()
    assert code == rdm.RDM_OK and info.converged
    assert np.array_equal(sol.alpha(), ref.alpha())
    # a getter called while the solve runs waits for it
    sol.solve_async()
    assert np.array_equal(sol.p0().vals, ref.p0().vals)


def test_stall_window_sets_when_the_ladder_moves_on(rdm, exact_alpha):
    s = cluster(32)
    tiers = {}
    for w in (2, 4):
        sol, info = solve(rdm, s, tau=1e-6, tol=1e-9, mode="mixed_fp16", stall_window=w)
        tiers[w] = info.tier_iters[0]
        assert np.max(np.abs(sol.alpha() - exact_alpha)) / np.max(np.abs(exact_alpha)) <= 1e-6
    assert tiers[4] >= tiers[2]


@pytest.mark.parametrize("mode", ["fp64", "mixed_fp16"])
def test_split_directions_match_the_joint_solve(rdm, mode):
    """split_directions: each field direction solved on its own (P0 and one P1
    in the X set), then P0, every P1 and every alpha component, cross terms
    included.  Against the joint solve of the same batch (two systems, two
    directions and three directions)."""
    from synth import make_chain
    for dirs in (("x", "z"), ("x", "y", "z")):
        systems = [make_cluster(60, opa=8, b=32, cutoff=10.0, seed=41, dirs=dirs),
                   make_chain(30, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=42, dirs=dirs)]
        res = []
        for split in (0, 1):
            sol = rdm.Solver(0)
            sol.set_params(tau=1e-6, tol=1e-9, mode=mode, max_iter=100, split_directions=split)
            sol.load(systems)
            code, info = sol.solve()
            assert code == rdm.RDM_OK and info.converged
            res.append(([sol.alpha(k) for k in range(2)], [sol.p0(k).to_dense() for k in range(2)],
                        [[sol.p1(k, "xyz".index(d)).to_dense() for d in dirs] for k in range(2)],
                        sol.info(1)))
        tol = 1e-8 if mode == "fp64" else 1e-6
        for k in range(2):
            a0, a1 = res[0][0][k], res[1][0][k]
            m = ~np.isnan(a0)
            assert np.array_equal(m, ~np.isnan(a1)) and m.sum() == len(dirs) ** 2
            assert np.max(np.abs(a1[m] - a0[m])) / np.max(np.abs(a0[m])) <= tol
            assert max_rel_err(res[1][1][k], res[0][1][k]) <= tol
            for q in range(len(dirs)):
                assert max_rel_err(res[1][2][k][q], res[0][2][k][q]) <= 100 * tol
        # the summary adds up the passes
        assert res[1][3].time_ms > 0 and res[1][3].tc_launches >= res[0][3].tc_launches


def test_split_directions_refuse_an_overlap(rdm):
    from synth import make_overlap
    s = make_cluster(40, opa=8, b=32, cutoff=10.0, seed=12, dirs=("x", "y"))
    s.s = make_overlap(s)
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="fp64", split_directions=1)
    sol.load(s)
    with pytest.raises(rdm.RdmError) as e:
        sol.solve()
    assert e.value.code == rdm.RDM_EINVAL


def test_split_directions_parameter_is_validated(rdm):
    sol = rdm.Solver(0)
    for bad in (2, -1):
        with pytest.raises(rdm.RdmError) as e:
            sol.set_params(tau=1e-6, mode="fp64", split_directions=bad)
        assert e.value.code == rdm.RDM_EINVAL
    sol.set_params(tau=1e-6, mode="fp64", split_directions=1)
    sol.close()
