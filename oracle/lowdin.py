"""Oracle for a non-orthogonal basis (overlap S): the Loewdin route of Sec. 2.2.

Test infrastructure only (see the package docstring).  Dense FP64 NumPy.

The paper solves the generalized problem H C = S C E (Eq. KS-matrix) in the
orthogonal basis obtained with S^(-1/2): H_orth = S^(-1/2) H S^(-1/2)
(Sec. 2.2), runs TC2 there and transforms the density matrices back,
P = S^(-1/2) P_orth S^(-1/2).  A perturbation that leaves S unchanged (an
electric field) transforms like H.  Here S^(-1/2) comes from the eigenpairs
of S, H_orth and H1_orth are formed literally, Oracle A gives P0_orth and
P1_orth, and both are transformed back.  The polarizability is basis
independent: Tr(P1 H1) = Tr(P1_orth H1_orth) (Eq. polar).
"""

from __future__ import annotations

from typing import Sequence

import numpy as np

from .dense import exact_response


def inverse_sqrt(s: np.ndarray) -> np.ndarray:
    """S^(-1/2) of a symmetric positive definite S from its eigenpairs."""
    w, u = np.linalg.eigh(np.asarray(s, dtype=np.float64))
    if not np.all(w > 0):
        raise ValueError("S is not positive definite")
    return (u / np.sqrt(w)) @ u.T


def lowdin_response(h0: np.ndarray, h1s: Sequence[np.ndarray], s: np.ndarray, n_occ: int):
    """(P0, [P1_gamma], Z) in the non-orthogonal basis, Z = S^(-1/2)."""
    z = inverse_sqrt(s)
    h0o = z @ np.asarray(h0, dtype=np.float64) @ z
    h1o = [z @ np.asarray(h1, dtype=np.float64) @ z for h1 in h1s]
    p0o, p1o, _, _ = exact_response(h0o, h1o, n_occ)
    return z @ p0o @ z, [z @ p @ z for p in p1o], z
