"""Non-orthogonal basis (Sec. 2.2) through the C ABI: the overlap S is
uploaded beside H0 and H1, the library forms S^(-1/2) by Newton-Schulz
iterations with its block products, solves in the orthogonal form and
transforms P0 and P1 back.  Checked against the Loewdin oracle (itself pinned
to the generalized eigenproblem solved directly, tests/test_oracle_pins.py)."""

import numpy as np
import pytest

from blockcheck import max_rel_err
from oracle import lowdin_response, polarizability
from oracle.dense import rel_frobenius
from synth import Bsr, make_chain, make_cluster, make_overlap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def with_overlap(s):
    s.s = make_overlap(s)
    return s


@pytest.fixture(scope="module")
def case():
    s = with_overlap(make_cluster(60, opa=8, b=32, cutoff=10.0, seed=6, dirs=("x", "y", "z")))
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    p0, p1s, z = lowdin_response(h0, h1s, s.s.to_dense(), s.n_occ)
    return s, h1s, p0, p1s


def solve(rdm, s, **params):
    sol = rdm.Solver(0)
    sol.set_params(**params)
    sol.load(s)
    code, info = sol.solve()
    assert code == rdm.RDM_OK
    return sol, info


def test_fp64_zero_threshold_matches_the_loewdin_oracle(rdm, case):
    s, h1s, p0, p1s = case
    sol, info = solve(rdm, s, tau=0.0, tol=1e-12, mode="fp64")
    assert info.lowdin_iterations > 0
    g0 = sol.p0().to_dense()
    assert rel_frobenius(g0, p0) <= 1e-10 and max_rel_err(g0, p0) <= 1e-10
    for d in range(3):
        g1 = sol.p1(0, d).to_dense()
        assert rel_frobenius(g1, p1s[d]) <= 1e-9 and max_rel_err(g1, p1s[d]) <= 1e-9
    a = polarizability(p1s, h1s)
    assert np.max(np.abs(sol.alpha() - a)) <= 1e-10 * np.max(np.abs(a))
    # the orthogonal-form summary: Tr P0 = N_occ there; in the uploaded basis Tr(P0 S) = N_occ
    assert abs(info.trace_error) < 1e-9
    assert abs(np.trace(g0 @ s.s.to_dense()) - s.n_occ) < 1e-8


def test_identity_overlap_changes_nothing(rdm):
    s = make_chain(30, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=5, dirs=("x",))
    plain, _ = solve(rdm, s, tau=1e-7, tol=1e-10, mode="fp64")
    s.s = Bsr.from_dense(np.eye(s.n), 32)
    ident, info = solve(rdm, s, tau=1e-7, tol=1e-10, mode="fp64")
    assert info.lowdin_iterations >= 1
    assert max_rel_err(ident.p0().to_dense(), plain.p0().to_dense()) <= 1e-12
    assert np.allclose(ident.alpha()[:1, :1], plain.alpha()[:1, :1], rtol=1e-12, atol=0)   # one direction: alpha_xx


@pytest.mark.parametrize("mode", ["fp64", "mixed_fp16"])
def test_thresholded_solve_in_a_non_orthogonal_basis(rdm, case, mode):
    s, h1s, p0, p1s = case
    sol, info = solve(rdm, s, tau=1e-6, tol=1e-9, mode=mode)
    a = polarizability(p1s, h1s)
    assert np.max(np.abs(sol.alpha() - a)) / np.max(np.abs(a)) <= 1e-6
    assert rel_frobenius(sol.p0().to_dense(), p0) <= 1e-5


def test_overlap_for_some_systems_of_a_batch_is_rejected(rdm):
    a = with_overlap(make_chain(20, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=1, dirs=("x",)))
    b = make_chain(24, opa=8, b=32, spacing=2.8, cutoff=8.0, seed=2, dirs=("x",))
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-6, tol=1e-9, mode="fp64")
    sol.load([a, b])
    with pytest.raises(rdm.RdmError) as e:
        sol.solve()
    assert e.value.code == rdm.RDM_EINVAL
