"""Oracle A: the exact zero- and first-order density matrices.

Test infrastructure only (see the package docstring).  Plain dense FP64
NumPy/LAPACK; no blocking, fusion or reordering.

For an orthogonal basis (S = I, the orthogonal form of Sec. 2.2) the
generalized eigenproblem of Eq. KS-matrix becomes H0 C = C E.  Then

* P0 = sum over the N_occ lowest states of c_i c_i^T            (Sec. 2.2)
* V  = C^T H1 C                      (the matrix of Eqs. CPSCF-U/epsilon1)
* U_pq = -V_pq / (eps_p - eps_q), U_pp = 0                 (Eq. cpscf-LCAO)
* C1 = C U, P1 = sum_i f_i (C1_i C_i^T + C_i C1_i^T)              (Eq. DM1)

with f_i = 1 for occupied states (P is normalised as sum_occ c c^T, so
Tr P0 = N_occ; the spin factor 2 enters only the polarizability).  In DM1 the
occupied-occupied terms of U cancel pairwise because U is antisymmetric, so
only occupied-virtual pairs remain:

  P1 = sum_{i occ, a virt} V_ai / (eps_i - eps_a) (c_a c_i^T + c_i c_a^T).

The polarizability follows Eq. polar with the field term h_E = -r.E of
Sec. 2: the first-order Hamiltonian for field component delta is -D_delta,
so with P1[D] the response to H1 = D,

  alpha_{gamma delta} = 2 * Tr(dP/de_delta D_gamma) = -2 Tr(P1[D_delta] D_gamma)
                      = 4 sum_{i,a} V^gamma_ai V^delta_ai / (eps_a - eps_i).
"""

from __future__ import annotations

from typing import List, Sequence

import numpy as np


def exact_response(h0: np.ndarray, h1s: Sequence[np.ndarray], n_occ: int):
    """Return (P0, [P1_gamma], eps, C) for dense symmetric H0 and H1_gamma.

    Follows Sec. 2.1 (Eqs. DM1, CPSCF-U, epsilon1, cpscf-LCAO) in the
    orthogonal basis.  Raises if the HOMO-LUMO gap is not positive.
    """
    h0 = np.asarray(h0, dtype=np.float64)
    n = h0.shape[0]
    if not (0 < n_occ < n):
        raise ValueError("need 0 < n_occ < n")
    eps, c = np.linalg.eigh(h0)
    gap = eps[n_occ] - eps[n_occ - 1]
    if not gap > 0:
        raise ValueError("no HOMO-LUMO gap: the projector is not defined")
    c_occ = c[:, :n_occ]
    c_vir = c[:, n_occ:]
    p0 = c_occ @ c_occ.T
    p1s = []
    denom = eps[:n_occ][None, :] - eps[n_occ:][:, None]       # (n_vir, n_occ): eps_i - eps_a
    for h1 in h1s:
        v_ai = c_vir.T @ np.asarray(h1, dtype=np.float64) @ c_occ   # V_ai
        u_ai = v_ai / denom
        t = c_vir @ u_ai @ c_occ.T                             # sum u_ai c_a c_i^T
        p1s.append(t + t.T)
    return p0, p1s, eps, c


def polarizability(p1s: Sequence[np.ndarray], h1s: Sequence[np.ndarray], spin: float = 2.0) -> np.ndarray:
    """alpha_{gamma delta} = -spin * Tr(P1_delta D_gamma)  (Eq. polar, field
    term -r.E).  Entry [g, d] uses the response to direction d."""
    m = len(h1s)
    a = np.zeros((m, m))
    for g in range(m):
        for d in range(m):
            a[g, d] = -spin * float(np.sum(p1s[d] * h1s[g]))   # Tr(P D) for symmetric P, D
    return a


def polarizability_sos(h0: np.ndarray, h1s: Sequence[np.ndarray], n_occ: int) -> np.ndarray:
    """The same tensor from the spectral sum 4 sum V^g_ai V^d_ai/(eps_a-eps_i)
    (a second route used to pin ``polarizability``)."""
    eps, c = np.linalg.eigh(np.asarray(h0, dtype=np.float64))
    c_occ, c_vir = c[:, :n_occ], c[:, n_occ:]
    vs = [c_vir.T @ h1 @ c_occ for h1 in h1s]
    de = eps[n_occ:][:, None] - eps[:n_occ][None, :]
    m = len(h1s)
    a = np.zeros((m, m))
    for g in range(m):
        for d in range(m):
            a[g, d] = 4.0 * float(np.sum(vs[g] * vs[d] / de))
    return a


def projector_invariants(p0: np.ndarray, h0: np.ndarray, n_occ: int) -> dict:
    """Residuals that vanish for the exact P0: idempotency, trace, and
    commutation with H0 (Sec. 2.2: P_orth P_orth = P_orth)."""
    return {
        "idempotency": float(np.linalg.norm(p0 @ p0 - p0)),
        "trace": float(np.trace(p0) - n_occ),
        "commutator": float(np.linalg.norm(h0 @ p0 - p0 @ h0)),
    }


def response_invariants(p0: np.ndarray, p1: np.ndarray, h0: np.ndarray, h1: np.ndarray) -> dict:
    """Residuals that vanish for the exact P1 = dP0/dlambda: the derivative of
    P^2 = P, of Tr P = N_occ and of [H, P] = 0."""
    return {
        "idempotency1": float(np.linalg.norm(p0 @ p1 + p1 @ p0 - p1)),
        "occ_occ": float(np.linalg.norm(p0 @ p1 @ p0)),
        "trace1": float(np.trace(p1)),
        "commutator1": float(np.linalg.norm(h0 @ p1 - p1 @ h0 + h1 @ p0 - p0 @ h1)),
    }


def rel_frobenius(a: np.ndarray, ref: np.ndarray) -> float:
    den = float(np.linalg.norm(ref))
    return float(np.linalg.norm(a - ref)) / (den if den > 0 else 1.0)


__all__: List[str] = [
    "exact_response", "polarizability", "polarizability_sos",
    "projector_invariants", "response_invariants", "rel_frobenius",
]
