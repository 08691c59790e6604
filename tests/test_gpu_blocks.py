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
