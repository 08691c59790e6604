"""CPU checks of the algebra behind the accuracy correction (rdm_params.correct).

The library forms the residual perturbations with products of symmetric
matrices only ({A, B} = A B + B A).  These tests check, in dense FP64 with
numpy, that each anticommutator form equals the commutator it stands for
(Sec. 2.1 fixes P0 by [H0, P0] = 0 with P0 idempotent, and P1 by
[H0, P1] + [H1, P0] = 0 with P1 occupied-virtual).  They also check that one
correction step, with exact responses from oracle A, restores P0 and P1 from
perturbed copies.  The GPU path is compared with oracle A in
tests/test_gpu_correct.py.
"""

import numpy as np

from oracle import exact_response, polarizability


def sym(a, b):
    return a @ b + b @ a


def comm(a, b):
    return a @ b - b @ a


def small_system(n=24, nocc=9, seed=3):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    h0 = (a + a.T) / 2 + np.diag(np.linspace(-3, 3, n))
    d = rng.standard_normal((n, n))
    h1 = (d + d.T) / 2
    return h0, h1, nocc


def rotated_projector(p0, theta, seed=5):
    """P0 rotated by exp(theta K), K antisymmetric: idempotent, trace kept."""
    n = p0.shape[0]
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((n, n))
    k = (k - k.T) / 2
    w, v = np.linalg.eigh(1j * k)           # i K is Hermitian
    u = (v @ np.diag(np.exp(-1j * theta * w)) @ v.conj().T).real
    return u @ p0 @ u.T


def test_p0_perturbation_is_the_double_commutator():
    """H'0 = [[H0, P0], P0] = 2 G0 - {P0, G0}, G0 = {P0, H0}, for any
    idempotent P0 (here a rotated one, so that [H0, P0] != 0)."""
    h0, _, nocc = small_system()
    p0, _, _, _ = exact_response(h0, [h0], nocc)
    p = rotated_projector(p0, 1e-3)
    assert np.abs(p @ p - p).max() < 1e-12
    g0 = sym(p, h0)
    form = 2 * g0 - sym(p, g0)
    direct = comm(comm(h0, p), p)
    assert np.abs(direct).max() > 1e-4
    assert np.abs(form - direct).max() <= 1e-12 * np.abs(h0).max()


def test_p1_perturbation_is_the_residual_commutator():
    """H'1 = [R1, P0], R1 = [H0, P1] + [H1, P0], equals 2 G - {P0, G} + {D, P1}
    with G = {P0, H1}, D = H0 - {P0, H0}, for idempotent P0 and P1
    occupied-virtual with respect to it."""
    h0, h1, nocc = small_system()
    p0, (p1,), _, _ = exact_response(h0, [h1], nocc)
    p = rotated_projector(p0, 1e-3)
    q = np.eye(len(p)) - p
    rng = np.random.default_rng(7)
    e = rng.standard_normal(p1.shape) * 1e-3
    x = p1 + (e + e.T) / 2
    x = p @ x @ q + q @ x @ p                # occupied-virtual with respect to p
    g = sym(p, h1)
    d = h0 - sym(p, h0)
    form = 2 * g - sym(p, g) + sym(d, x)
    r1 = comm(h0, x) + comm(h1, p)
    direct = comm(r1, p)
    assert np.abs(form - direct).max() <= 1e-11 * np.abs(direct).max()


def test_occupied_virtual_projection():
    """2 {P0, X} - {P0, {P0, X}} = P0 X Q + Q X P0 (Q = I - P0) for idempotent P0."""
    h0, h1, nocc = small_system()
    p0, _, _, _ = exact_response(h0, [h1], nocc)
    q = np.eye(len(p0)) - p0
    x = np.random.default_rng(2).standard_normal(p0.shape)
    x = (x + x.T) / 2
    form = 2 * sym(p0, x) - sym(p0, sym(p0, x))
    assert np.abs(form - (p0 @ x @ q + q @ x @ p0)).max() <= 1e-12 * np.abs(x).max()


def correction_step(h0, h1, nocc, pt, p1t):
    """The two corrections with exact responses (oracle A): P0 from H'0, then
    P1 from H'1 with the corrected P0, then the occupied-virtual projection."""
    g0 = sym(pt, h0)
    pc = pt + exact_response(h0, [2 * g0 - sym(pt, g0)], nocc)[1][0]
    g = sym(pc, h1)
    d = h0 - sym(pc, h0)
    x = p1t + exact_response(h0, [2 * g - sym(pc, g) + sym(d, p1t)], nocc)[1][0]
    return pc, 2 * sym(pc, x) - sym(pc, sym(pc, x))


def test_one_correction_step_is_second_order():
    """A P0 rotated by theta and a P1 carrying the matching error plus noise
    of size theta / 10: one correction step leaves errors of order theta^2
    in P0, P1 and alpha (a tenfold smaller theta leaves a hundredfold smaller
    error), so a rotation of 1e-6 comes back to ~1e-11."""
    h0, h1, nocc = small_system()
    p0, (p1,), _, _ = exact_response(h0, [h1], nocc)
    ax = polarizability([p1], [h1])
    after = []
    for theta in (1e-5, 1e-6):
        pt = rotated_projector(p0, theta)
        rng = np.random.default_rng(11)
        noise = rng.standard_normal(p1.shape) * 0.1 * theta * np.abs(p1).max()
        p1t = p1 + (noise + noise.T) / 2 + comm(comm(pt - p0, p0), p1)
        pc, p1c = correction_step(h0, h1, nocc, pt, p1t)
        a_before = np.abs(polarizability([p1t], [h1]) - ax).max() / np.abs(ax).max()
        a_after = np.abs(polarizability([p1c], [h1]) - ax).max() / np.abs(ax).max()
        e = (np.abs(pc - p0).max(), np.abs(p1c - p1).max(), a_after)
        assert e[0] < 1e-3 * np.abs(pt - p0).max()
        assert e[1] < 1e-3 * np.abs(p1t - p1).max()
        assert a_after < 1e-3 * a_before
        after.append(e)
    for big, small in zip(*after):
        assert 50 < big / small < 200
    assert after[1][2] < 1e-10
