"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here uses a route independent of the code it pins: the matrix
sign function by Newton's iteration (no eigen-decomposition) for P0, central
finite differences for P1 and alpha, closed forms for 2x2 and hopping-free
systems, and the scalar maps of TC2 in the eigenbasis for the iteration
sequence.  ``test_planted_*`` show that a plausible mistake in the oracle
fails these pins.
"""

import json
import os

import numpy as np
import pytest

from oracle import block_truncate, exact_response, gershgorin_bounds, polarizability, tc2_response
from oracle.dense import polarizability_sos, projector_invariants, rel_frobenius, response_invariants
from oracle.tc2 import block_norms
from synth import make_chain, make_config, make_cluster

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# independent reference routes
# ---------------------------------------------------------------------------

def sign_projector(h: np.ndarray, mu: float, iters: int = 60) -> np.ndarray:
    """Projector onto the eigenvalues of h below mu, from the matrix sign
    function sign(mu I - h) by Newton's iteration X <- (X + X^-1)/2 (Higham);
    no eigen-decomposition involved."""
    x = mu * np.eye(h.shape[0]) - h
    for _ in range(iters):
        xn = 0.5 * (x + np.linalg.inv(x))
        if np.linalg.norm(xn - x) <= 1e-15 * np.linalg.norm(xn):
            x = xn
            break
        x = xn
    return 0.5 * (np.eye(h.shape[0]) + x)


def chain_sys(n_atoms=24, seed=0):
    return make_chain(n_atoms, opa=4, b=4, spacing=2.8, cutoff=8.0, seed=seed, dirs=("x", "y", "z"))


MU_GAP = -0.15   # inside the model gap: occupied onsite <= -0.5, virtual >= 0.2, hopping << 0.3


# ---------------------------------------------------------------------------
# Gershgorin bounds (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_gershgorin_contains_spectrum():
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 40):
        a = rng.standard_normal((n, n))
        a = a + a.T
        lo, hi = gershgorin_bounds(a)
        w = np.linalg.eigvalsh(a)
        assert lo <= w[0] + 1e-12 and w[-1] <= hi + 1e-12


def test_gershgorin_special_cases():
    d = np.diag([3.0, -1.0, 0.5])
    assert gershgorin_bounds(d) == (-1.0, 3.0)
    a, h, dd = 0.3, -0.2, -0.9
    lo, hi = gershgorin_bounds(np.array([[a, h], [h, dd]]))
    assert lo == pytest.approx(min(a - abs(h), dd - abs(h)))
    assert hi == pytest.approx(max(a + abs(h), dd + abs(h)))


# ---------------------------------------------------------------------------
# Oracle A: exact P0, P1, alpha (Sec. 2.1, Eq. polar)
# ---------------------------------------------------------------------------

def test_p0_matches_sign_function_and_invariants():
    s = chain_sys()
    h0 = s.h0.to_dense()
    p0, _, _, _ = exact_response(h0, [], s.n_occ)
    ps = sign_projector(h0, MU_GAP)
    assert np.trace(ps) == pytest.approx(s.n_occ, abs=1e-9)
    assert rel_frobenius(p0, ps) < 1e-12
    inv = projector_invariants(p0, h0, s.n_occ)
    assert inv["idempotency"] < 1e-12 and abs(inv["trace"]) < 1e-10 and inv["commutator"] < 1e-12


def test_p1_matches_finite_difference_of_p0():
    s = chain_sys()
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    for h1, p1 in zip(h1s, p1s):
        eps = 1e-4 / np.linalg.norm(h1, 2)
        fd = (sign_projector(h0 + eps * h1, MU_GAP) - sign_projector(h0 - eps * h1, MU_GAP)) / (2 * eps)
        assert rel_frobenius(p1, fd) < 1e-6


def test_p1_invariants():
    s = make_config(2, n_atoms=60)
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    p0, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    for h1, p1 in zip(h1s, p1s):
        r = response_invariants(p0, p1, h0, h1)
        scale = np.linalg.norm(p1)
        assert r["idempotency1"] < 1e-11 * scale
        assert r["occ_occ"] < 1e-11 * scale
        assert abs(r["trace1"]) < 1e-10 * scale
        assert r["commutator1"] < 1e-10 * max(scale, 1.0) * np.linalg.norm(h1)


def test_alpha_two_routes_symmetric_positive():
    s = chain_sys()
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    a = polarizability(p1s, h1s)
    b = polarizability_sos(h0, h1s, s.n_occ)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-12)
    assert np.allclose(a, a.T, rtol=1e-10, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(0.5 * (a + a.T)) > 0)


def test_alpha_is_dipole_derivative():
    """Eq. polar: alpha_gd = d mu_g / d e_d with mu_g = 2 Tr(P0 D_g) and the
    field term -r.E, i.e. H(e) = H0 - e D_d.  P0 from the sign function."""
    s = chain_sys(16)
    h0 = s.h0.to_dense()
    ds = [m.to_dense() for m in s.h1]
    _, p1s, _, _ = exact_response(h0, ds, s.n_occ)
    a = polarizability(p1s, ds)
    e = 1e-4
    for d in range(3):
        pp = sign_projector(h0 - e * ds[d], MU_GAP)
        pm = sign_projector(h0 + e * ds[d], MU_GAP)
        for g in range(3):
            mu_p = 2.0 * np.sum(pp * ds[g])
            mu_m = 2.0 * np.sum(pm * ds[g])
            fd = (mu_p - mu_m) / (2 * e)
            assert fd == pytest.approx(a[g, d], rel=1e-6, abs=1e-8)


def test_alpha_origin_shift_invariant():
    s = chain_sys()
    h0 = s.h0.to_dense()
    d = s.h1[0].to_dense()
    _, p1, _, _ = exact_response(h0, [d, d + 7.5 * np.eye(d.shape[0])], s.n_occ)
    a0 = polarizability([p1[0]], [d])[0, 0]
    a1 = polarizability([p1[1]], [d + 7.5 * np.eye(d.shape[0])])[0, 0]
    assert a1 == pytest.approx(a0, rel=1e-10)


def test_special_cases_zero_response():
    s = chain_sys()
    h0 = s.h0.to_dense()
    n = h0.shape[0]
    _, p1s, _, _ = exact_response(h0, [np.eye(n), h0], s.n_occ)
    assert np.linalg.norm(p1s[0]) < 1e-12
    assert np.linalg.norm(p1s[1]) < 1e-10


def test_hopping_free_closed_form():
    """No hopping: eigenvectors are unit vectors, P0 = diag(occupied) and
    P1_ia = H1_ia / (eps_i - eps_a) inside each atom (Eq. cpscf-LCAO)."""
    s = make_chain(6, opa=4, b=4, spacing=50.0, cutoff=8.0, seed=3, dirs=("x", "z"))
    h0 = s.h0.to_dense()
    assert np.count_nonzero(h0 - np.diag(np.diag(h0))) == 0
    h1s = [m.to_dense() for m in s.h1]
    p0, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    eps = np.diag(h0)
    occ = np.zeros(h0.shape[0], bool)
    for atom in range(6):
        occ[atom * 4: atom * 4 + 2] = True
    assert np.allclose(p0, np.diag(occ.astype(float)), atol=1e-14)
    for h1, p1 in zip(h1s, p1s):
        ref = np.zeros_like(h1)
        for i in np.nonzero(occ)[0]:
            for a in np.nonzero(~occ)[0]:
                ref[i, a] = ref[a, i] = h1[i, a] / (eps[i] - eps[a])
        assert np.allclose(p1, ref, atol=1e-13)
    # alpha = 4 sum |S_ai|^2 / (eps_a - eps_i)
    a = polarizability(p1s, h1s)
    for g in range(2):
        ref = 4.0 * sum(h1s[g][i, a] ** 2 / (eps[a] - eps[i])
                        for i in np.nonzero(occ)[0] for a in np.nonzero(~occ)[0])
        assert a[g, g] == pytest.approx(ref, rel=1e-12)


def test_two_by_two_closed_form():
    """P0 = I/2 - (H0 - m I)/(2r) for the lower state of a 2x2 matrix and its
    derivative along H1."""
    a, h, d = -0.7, 0.15, 0.4
    p, q, t = 0.3, -0.2, 1.1
    h0 = np.array([[a, h], [h, d]])
    h1 = np.array([[p, q], [q, t]])
    m = 0.5 * (a + d)
    r = np.sqrt((0.5 * (a - d)) ** 2 + h * h)
    p0_ref = 0.5 * np.eye(2) - (h0 - m * np.eye(2)) / (2 * r)
    dr = (0.25 * (a - d) * (p - t) + h * q) / r
    p1_ref = -(h1 - 0.5 * (p + t) * np.eye(2)) / (2 * r) + (h0 - m * np.eye(2)) * dr / (2 * r * r)
    p0, (p1,), _, _ = exact_response(h0, [h1], 1)
    assert np.allclose(p0, p0_ref, atol=1e-14)
    assert np.allclose(p1, p1_ref, atol=1e-13)


# ---------------------------------------------------------------------------
# Oracle B: TC2 + first-order recursion (Eqs. TC2, TC2-CPSCF)
# ---------------------------------------------------------------------------

def test_block_truncate_semantics():
    rng = np.random.default_rng(1)
    n, b = 11, 4                      # ragged last block (3 rows)
    x = rng.standard_normal((n, n)) * 1e-3
    x[:4, :4] = 1.0
    nrm = block_norms(x, b)
    tau = float(np.median(nrm))
    y = block_truncate(x, b, tau)
    for bi in range(3):
        for bj in range(3):
            blk_x = x[bi * b:(bi + 1) * b, bj * b:(bj + 1) * b]
            blk_y = y[bi * b:(bi + 1) * b, bj * b:(bj + 1) * b]
            if np.linalg.norm(blk_x) < tau:
                assert not blk_y.any()
            else:
                assert np.array_equal(blk_x, blk_y)
    assert np.array_equal(block_truncate(x, b, 0.0), x)


def test_tc2_converges_to_exact_at_zero_threshold():
    s = make_config(1)
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    p0, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    r = tc2_response(h0, h1s, s.n_occ, s.b, tau=0.0, tol=1e-12)
    assert r.converged
    assert rel_frobenius(r.p0, p0) < 1e-10
    assert rel_frobenius(r.p1s[0], p1s[0]) < 1e-10
    # the paper reports about 25 recursion cycles (Sec. 2.2, Fig. band_energy)
    assert 10 <= r.iterations <= 40


def test_tc2_matches_scalar_maps_in_eigenbasis():
    """At tau = 0 every eigenvalue x of X0 follows x -> x^2 or 2x - x^2 and
    the element (p,q) of X1 in the H0 eigenbasis is multiplied by
    x_p + x_q or 2 - x_p - x_q (the branch chosen by the trace)."""
    s = chain_sys(20)
    h0 = s.h0.to_dense()
    h1 = s.h1[0].to_dense()
    eps, c = np.linalg.eigh(h0)
    lo, hi = gershgorin_bounds(h0)
    w = hi - lo
    x = (hi - eps) / w
    u = c.T @ (-h1 / w) @ c
    for k in range(1, 9):
        r = tc2_response(h0, [h1], s.n_occ, s.b, tau=0.0, tol=0.0, max_iter=k)
        # predicted iterate after k steps
        xs, us = x.copy(), u.copy()
        branches = []
        for _ in range(k):
            if xs.sum() >= s.n_occ:
                branches.append(1)
                us = (xs[:, None] + xs[None, :]) * us
                xs = xs * xs
            else:
                branches.append(2)
                us = (2.0 - xs[:, None] - xs[None, :]) * us
                xs = 2.0 * xs - xs * xs
        assert r.branches == branches
        assert np.allclose(c.T @ r.p0 @ c, np.diag(xs), atol=1e-11)
        assert np.allclose(c.T @ r.p1s[0] @ c, us, atol=1e-10 * max(1.0, np.abs(us).max()))


def test_tc2_truncation_error_shrinks_with_threshold():
    s = make_config(2, n_atoms=40)
    h0 = s.h0.to_dense()
    h1s = [s.h1[0].to_dense()]
    _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    errs = []
    for tau in (1e-3, 1e-5, 1e-7):
        # tolerance one decade above the filter, the paper's pairing (Sec. 3.1: filter 1e-6, tol 1e-5)
        r = tc2_response(h0, h1s, s.n_occ, 8, tau=tau, tol=10 * tau)
        assert r.converged
        errs.append(rel_frobenius(r.p1s[0], p1s[0]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_tc2_large_threshold_stays_bounded():
    """At tau = 1e-4 the filter pushes eigenvalues of X0 out of [0, 1]; with the
    trace test alone TC2 then diverges on this cluster (X0 overflows).  With
    the branch alternating while Tr X - ||X||^2 < -1e-10 N_occ, X0 stays
    bounded, P0 stays a projector to the filter's accuracy and alpha keeps the
    accuracy the threshold allows."""
    s = make_cluster(150, opa=8, b=32, cutoff=10.0, seed=11, dirs=("x", "y", "z"))
    h0 = s.h0.to_dense()
    h1s = [m.to_dense() for m in s.h1]
    p0, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
    r = tc2_response(h0, h1s, s.n_occ, s.b, tau=1e-4, tol=0.0, max_iter=40)
    assert np.isfinite(r.p0).all()
    assert abs(np.trace(r.p0) - s.n_occ) < 1e-3
    assert rel_frobenius(r.p0, p0) < 1e-3
    ae = polarizability(p1s, h1s)
    a = polarizability(r.p1s, h1s)
    assert np.max(np.abs(a - ae)) / np.max(np.abs(ae)) < 1e-5
    # the safeguard acted: some step took the other branch than the trace test
    assert any(rec["idempotency"] < -1e-10 * s.n_occ for rec in r.log)


def test_tc2_idempotency_stall_stop_iteration():
    """The idempotency-stall stop (stall_tol > 0) fires when e = Tr X0 -
    ||X0||_F^2 has not decreased over two iterations while below stall_tol.
    Predicted by hand for H0 = diag(-1, 0, 1), N_occ = 1: the Gershgorin
    bounds are -1 and 1, so X0_0 = diag(1, 1/2, 0); the trace never drops
    below N_occ, every step squares, and the middle eigenvalue runs through
    2^-1, 2^-2, 2^-4, ..., 2^-64.  Every value and every sum is exact in FP64
    until Tr X0 = 1 + 2^-64 rounds to 1 at X0_6; so e_n = 1/4, 3/16, 15/256,
    2^-8 - 2^-16, 2^-16 - 2^-32, 2^-32 (1 + 2^-64 rounds to 1 in ||X0||^2),
    then 0, 0, 0.  The first n with e_{n+1} >= e_{n-1} is n = 7 (0 >= 0): the
    loop stops after 8 updates.  With the stop disabled it runs to max_iter."""
    h0 = np.diag([-1.0, 0.0, 1.0])
    h1s = [np.diag([0.3, -0.2, 0.1])]
    r = tc2_response(h0, h1s, 1, 1, tau=0.0, tol=0.0, max_iter=50, stall_tol=1e-3)
    assert r.converged and r.iterations == 8
    assert r.branches == [1] * 8
    e = [rec["idempotency"] for rec in r.log]
    assert e[:6] == [0.25, 0.1875, 0.05859375, 2.0 ** -8 - 2.0 ** -16, 2.0 ** -16 - 2.0 ** -32, 2.0 ** -32]
    assert e[6:] == [0.0, 0.0]
    # the level matters only as an upper bound; 0 disables the stop
    assert tc2_response(h0, h1s, 1, 1, tau=0.0, tol=0.0, max_iter=50, stall_tol=1e-300).iterations == 8
    off = tc2_response(h0, h1s, 1, 1, tau=0.0, tol=0.0, max_iter=50, stall_tol=0.0)
    assert off.iterations == 50 and not off.converged


def test_tc2_forced_branches_replay():
    s = chain_sys(12)
    h0 = s.h0.to_dense()
    h1s = [s.h1[0].to_dense()]
    r = tc2_response(h0, h1s, s.n_occ, 4, tau=1e-6, tol=1e-10)
    r2 = tc2_response(h0, h1s, s.n_occ, 4, tau=1e-6, tol=0.0, max_iter=r.iterations,
                      force_branches=r.branches)
    assert r2.branches == r.branches
    assert np.array_equal(r.p0, r2.p0) and np.array_equal(r.p1s[0], r2.p1s[0])


# ---------------------------------------------------------------------------
# planted mistakes: the pins above catch them
# ---------------------------------------------------------------------------

def _broken_dmpt(h0, h1s, n_occ, b, drop_term=False, wrong_sign=False, n_iter=40):
    lo, hi = gershgorin_bounds(h0)
    w = hi - lo
    x0 = (hi * np.eye(h0.shape[0]) - h0) / w
    x1s = [(h1 if wrong_sign else -h1) / w for h1 in h1s]
    for _ in range(n_iter):
        sq = x0 @ x0
        if np.trace(x0) >= n_occ:
            x1s = [x1 @ x0 + (0 if drop_term else x0 @ x1) for x1 in x1s]
            x0 = sq
        else:
            x1s = [2 * x1 - x1 @ x0 - (0 if drop_term else x0 @ x1) for x1 in x1s]
            x0 = 2 * x0 - sq
    return x0, x1s


@pytest.mark.parametrize("mistake", ["drop_term", "wrong_sign"])
def test_planted_mistake_is_caught(mistake):
    s = chain_sys(12)
    h0 = s.h0.to_dense()
    h1 = s.h1[0].to_dense()
    _, (p1b,) = _broken_dmpt(h0, [h1], s.n_occ, 4, **{mistake: True})
    eps = 1e-4 / np.linalg.norm(h1, 2)
    fd = (sign_projector(h0 + eps * h1, MU_GAP) - sign_projector(h0 - eps * h1, MU_GAP)) / (2 * eps)
    assert not rel_frobenius(p1b, fd) < 1e-6


# ---------------------------------------------------------------------------
# stored values written by tests/golden/make_golden.py (oracle only)
# ---------------------------------------------------------------------------

def test_golden_values_reproduce():
    with open(os.path.join(GOLDEN, "alpha_small.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        if case["kind"] != "chain":
            continue
        s = make_chain(case["n_atoms"], opa=case["opa"], b=case["b"], spacing=case["spacing"],
                       cutoff=case["cutoff"], seed=case["seed"], dirs=tuple(case["dirs"]))
        h0 = s.h0.to_dense()
        h1s = [m.to_dense() for m in s.h1]
        _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
        a = polarizability(p1s, h1s)
        assert np.allclose(a, np.array(case["alpha"]), rtol=1e-12)


# ---------------------------------------------------------------------------
# non-orthogonal basis (Sec. 2.2): the Loewdin oracle against the generalized
# eigenproblem solved directly, finite differences and S-metric invariants
# ---------------------------------------------------------------------------

def _nonorth_case():
    from synth import make_overlap
    s_ = make_cluster(40, opa=8, b=32, cutoff=10.0, seed=12, dirs=("x", "y"))
    return s_, s_.h0.to_dense(), [m.to_dense() for m in s_.h1], make_overlap(s_).to_dense()


def _generalized(h0, s, n_occ):
    import scipy.linalg
    eps, c = scipy.linalg.eigh(h0, s)          # C^T S C = I
    return eps, c, c[:, :n_occ] @ c[:, :n_occ].T


def test_lowdin_reduces_to_the_orthogonal_oracle_for_identity_overlap():
    from oracle import lowdin_response
    s_ = chain_sys(10)
    h0, h1s = s_.h0.to_dense(), [m.to_dense() for m in s_.h1]
    p0, p1s, z = lowdin_response(h0, h1s, np.eye(h0.shape[0]), s_.n_occ)
    q0, q1s, _, _ = exact_response(h0, h1s, s_.n_occ)
    assert np.allclose(z, np.eye(h0.shape[0]), atol=1e-14)
    assert rel_frobenius(p0, q0) < 1e-13
    assert max(rel_frobenius(a, b) for a, b in zip(p1s, q1s)) < 1e-12


def test_lowdin_p0_equals_the_generalized_eigenproblem_projector():
    from oracle import lowdin_response
    s_, h0, h1s, s = _nonorth_case()
    p0, p1s, z = lowdin_response(h0, h1s, s, s_.n_occ)
    eps, c, pg = _generalized(h0, s, s_.n_occ)
    assert rel_frobenius(p0, pg) < 1e-11
    # S-metric projector: P S P = P, Tr(P S) = N_occ
    assert rel_frobenius(p0 @ s @ p0, p0) < 1e-11
    assert abs(np.trace(p0 @ s) - s_.n_occ) < 1e-9
    # Z really is S^(-1/2)
    assert rel_frobenius(z @ s @ z, np.eye(s.shape[0])) < 1e-13


def test_lowdin_p1_and_alpha_match_generalized_sum_over_states_and_finite_differences():
    from oracle import lowdin_response, polarizability
    s_, h0, h1s, s = _nonorth_case()
    p0, p1s, _ = lowdin_response(h0, h1s, s, s_.n_occ)
    eps, c, _ = _generalized(h0, s, s_.n_occ)
    n_occ = s_.n_occ
    co, cv = c[:, :n_occ], c[:, n_occ:]
    for h1, p1 in zip(h1s, p1s):
        v = cv.T @ h1 @ co                                   # V_ai in the S-orthonormal eigenbasis
        u = v / (eps[:n_occ][None, :] - eps[n_occ:][:, None])
        t = cv @ u @ co.T
        assert rel_frobenius(p1, t + t.T) < 1e-10
        # central finite difference of the generalized projector (S fixed)
        e = 1e-4 / np.max(np.abs(h1))
        fd = (_generalized(h0 + e * h1, s, n_occ)[2] - _generalized(h0 - e * h1, s, n_occ)[2]) / (2 * e)
        assert rel_frobenius(p1, fd) < 1e-6
        # S-metric response invariant: P1 = P0 S P1 + P1 S P0, and Tr(P1 S) = 0
        assert rel_frobenius(p0 @ s @ p1 + p1 @ s @ p0, p1) < 1e-9
        assert abs(np.trace(p1 @ s)) < 1e-9 * np.max(np.abs(p1)) * s.shape[0]
    # alpha: Tr(P1 H1) is the same in both bases, and equals 4 sum V^2 / (e_a - e_i)
    a = polarizability(p1s, h1s)
    vs = [cv.T @ h1 @ co for h1 in h1s]
    d = eps[n_occ:][:, None] - eps[:n_occ][None, :]
    a2 = np.array([[4.0 * np.sum(vg * vd / d) for vd in vs] for vg in vs])
    assert np.allclose(a, a2, rtol=1e-10, atol=0)
