"""Oracle B: TC2 purification coupled to the first-order recursion, step by
step in dense FP64, with the block-norm truncation the GPU path applies.

Test infrastructure only (see the package docstring).  Dense NumPy; every
product is computed literally (X1 X0 and X0 X1 separately), in the paper's
order:

1. Gershgorin bounds eps_min, eps_max of H0 (Sec. 2.2, "estimated with
   Gershgorin's Circle Theorem").
2. X0_0 = (eps_max I - H0) / (eps_max - eps_min)                  (Sec. 2.2)
   X1_0 = -H1 / (eps_max - eps_min), with the same bounds          (Sec. 2.2)
   The initial matrices are not truncated.
3. For n = 0, 1, ...:
     Tr X0_n >= N_occ:  X0' = X0^2,        X1' = X1 X0 + X0 X1     (Eq. TC2,
     Tr X0_n <  N_occ:  X0' = 2X0 - X0^2,  X1' = 2X1 - X1 X0 - X0 X1  Eq. TC2-CPSCF)
   then every b x b block of X0' whose Frobenius norm is below tau, and every
   block of X1' below tau_x1, is set to zero (the "filter" of Sec. 2.3 read
   block-wise; a block is dropped only if all its elements are below tau).
4. Stop when the band energies E0 = Tr(X0 H0) and E1 = Tr(X1 H0) change by
   less than ``tol`` between consecutive iterates (Sec. 2.2 and the
   "tolerance" of Sec. 2.3; absolute change, no spin factor), or, if
   ``stall_tol`` > 0, when the idempotency error e = Tr X0 - ||X0||_F^2 has
   not decreased over two iterations while below ``stall_tol``.
5. P0 = X0, P1 = X1.

Readings of the paper used here: a tie Tr X0 = N_occ takes the square branch
(the ">=" of Eq. TC2); X1_0 uses the Gershgorin bounds of X0_0 so that X1_n is
exactly the derivative of X0_n; truncation follows each update and never
touches H0, H1 or the initial matrices.  The paper does not say what TC2 does
when the filter pushes eigenvalues out of [0, 1] (idempotency error below
zero): with the trace test alone the iteration then diverges for large
thresholds (1e-5 and 1e-4 on the synthetic clusters); here the branch
alternates with the previous one whenever e < -1e-10 N_occ, a level that
rounding at tau = 0 never reaches.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np


def gershgorin_bounds(h: np.ndarray, n: Optional[int] = None):
    """(eps_min, eps_max) from Gershgorin discs: every eigenvalue of the
    symmetric matrix h lies in some [h_ii - r_i, h_ii + r_i] with
    r_i = sum_{j != i} |h_ij|.  Only the first ``n`` rows are used."""
    h = np.asarray(h, dtype=np.float64)
    n = h.shape[0] if n is None else n
    d = np.diag(h)[:n]
    r = np.abs(h[:n, :n]).sum(axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def block_norms(x: np.ndarray, b: int) -> np.ndarray:
    """Frobenius norm of every b x b block of x (ragged last block included)."""
    n = x.shape[0]
    nb = -(-n // b)
    xp = np.zeros((nb * b, nb * b))
    xp[:n, :n] = x
    return np.sqrt(np.sum(xp.reshape(nb, b, nb, b) ** 2, axis=(1, 3)))


def block_truncate(x: np.ndarray, b: int, tau: float) -> np.ndarray:
    """Zero every b x b block whose Frobenius norm is below tau."""
    if tau <= 0:
        return x
    n = x.shape[0]
    nb = -(-n // b)
    keep = block_norms(x, b) >= tau
    mask = np.repeat(np.repeat(keep, b, axis=0), b, axis=1)[:n, :n]
    return np.where(mask, x, 0.0)


def count_blocks(x: np.ndarray, b: int) -> int:
    return int(np.count_nonzero(block_norms(x, b) > 0))


@dataclass
class Tc2Result:
    p0: np.ndarray
    p1s: List[np.ndarray]
    eps_min: float
    eps_max: float
    iterations: int
    converged: bool
    branches: List[int] = field(default_factory=list)
    log: List[dict] = field(default_factory=list)


def tc2_response(h0: np.ndarray, h1s: Sequence[np.ndarray], n_occ: int, b: int,
                 tau: float = 0.0, tau_x1: Optional[float] = None, tol: float = 1e-10,
                 max_iter: int = 100, stall_tol: float = 0.0,
                 force_branches: Optional[Sequence[int]] = None,
                 min_iter: int = 1) -> Tc2Result:
    """Dense TC2 + first-order recursion (Eqs. TC2 and TC2-CPSCF).

    ``force_branches[n]`` (1 = square, 2 = 2X - X^2) overrides the trace test
    at iteration n; iterations beyond its length use the trace test.
    ``tol = 0`` disables the band-energy stop (exactly ``max_iter`` steps
    unless the stall rule fires).
    """
    h0 = np.asarray(h0, dtype=np.float64)
    tau_x1 = tau if tau_x1 is None else tau_x1
    n = h0.shape[0]
    emin, emax = gershgorin_bounds(h0)
    w = emax - emin
    x0 = (emax * np.eye(n) - h0) / w
    x1s = [-np.asarray(h1, dtype=np.float64) / w for h1 in h1s]

    res = Tc2Result(x0, x1s, emin, emax, 0, False)
    e_hist: List[float] = []
    eb_prev = None
    for it in range(max_iter):
        t = float(np.trace(x0))
        idem = t - float(np.sum(x0 * x0))
        e_hist.append(idem)
        if force_branches is not None and it < len(force_branches):
            branch = int(force_branches[it])
        else:
            branch = 1 if t >= n_occ else 2
            # an idempotency error clearly below zero means eigenvalues outside
            # [0, 1] (the filter moves them); the trace test alone would then
            # square an eigenvalue above 1 again and again, so the branch
            # alternates with the previous one and both edges contract
            if it > 0 and idem < -1e-10 * max(1.0, float(n_occ)):
                branch = 2 if res.branches[-1] == 1 else 1
        x0sq = x0 @ x0
        if branch == 1:
            x0n = x0sq
            x1n = [x1 @ x0 + x0 @ x1 for x1 in x1s]
        else:
            x0n = 2.0 * x0 - x0sq
            x1n = [2.0 * x1 - x1 @ x0 - x0 @ x1 for x1 in x1s]
        x0n = block_truncate(x0n, b, tau)
        x1n = [block_truncate(m, b, tau_x1) for m in x1n]
        eb0 = float(np.sum(x0n * h0))
        eb1 = [float(np.sum(m * h0)) for m in x1n]
        res.log.append({"iter": it, "branch": branch, "trace": t, "idempotency": idem,
                        "eb0": eb0, "eb1": eb1, "nnzb0": count_blocks(x0n, b),
                        "nnzb1": [count_blocks(m, b) for m in x1n]})
        res.branches.append(branch)
        x0, x1s = x0n, x1n
        res.iterations = it + 1
        if tol > 0 and eb_prev is not None and it + 1 >= min_iter:
            d0 = abs(eb0 - eb_prev[0])
            d1 = max([abs(a - c) for a, c in zip(eb1, eb_prev[1])], default=0.0)
            if d0 < tol and d1 < tol:
                res.converged = True
                break
        eb_prev = (eb0, eb1)
        if stall_tol > 0 and it >= 2:
            e_new = float(np.trace(x0)) - float(np.sum(x0 * x0))
            if e_new >= e_hist[-2] and e_new < stall_tol:
                res.converged = True
                break
    res.p0, res.p1s = x0, x1s
    return res

