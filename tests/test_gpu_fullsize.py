"""The full-size workload, in the launch configuration of the bench (mixed
fp16 ladder, tau = 1e-6, tol = 1e-9, 32 x 32 blocks): the 24-system batch of
84,131 atoms (N = 673,048).  The dense oracle cannot hold it, so the checks
are (a) the outputs the oracle can compute one by one: the polarizability of
the batch's smallest system against the exact sum-over-states value of oracle
A, and (b) properties that hold at any size, for every system: convergence,
Tr P0 = N_occ, idempotency, a symmetric positive polarizability, and a
response of zero trace (Tr P1 = 0).
"""

import numpy as np
import pytest

from oracle import exact_response, polarizability
from synth import make_batch_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def test_full_batch_sampled_against_the_oracle_and_invariants(rdm):
    systems = make_batch_config(24, b=32)
    sol = rdm.Solver(0)
    try:
        sol.set_params(tau=1e-6, tol=1e-9, mode="mixed_fp16", max_iter=100, block_size=32, autotune=0)
        sol.load(systems)
        code, info = sol.solve()
        assert code == rdm.RDM_OK and info.converged
        for k, s in enumerate(systems):
            ik = sol.info(k)
            assert ik.converged
            assert abs(ik.trace_error) < 1e-8 * s.n_occ
            assert abs(ik.idempotency) < 1e-8 * s.n_occ
            a = sol.alpha(k)
            assert np.all(np.diag(a) > 0)
            assert np.max(np.abs(a - a.T)) <= 1e-6 * np.max(np.abs(a))
        # the smallest system: alpha against the exact sum-over-states value
        k = int(np.argmin([s.n for s in systems]))
        s = systems[k]
        h0 = s.h0.to_dense()
        h1s = [m.to_dense() for m in s.h1]
        _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
        ao = polarizability(p1s, h1s)
        assert np.max(np.abs(sol.alpha(k) - ao)) / np.max(np.abs(ao)) <= 1e-6
        # every system's response has zero trace (Tr P1 = 0: the field does not
        # move the electron count), from the diagonal blocks alone
        for k, s in enumerate(systems):
            for d in range(3):
                p1 = sol.p1(k, d)
                rows = np.repeat(np.arange(p1.nb), np.diff(p1.row_ptr))
                diag = p1.vals[rows == p1.col_idx]
                tr = float(np.einsum("kii->", diag))
                assert abs(tr) <= 1e-7 * np.max(np.abs(p1.vals)) * s.n
    finally:
        sol.close()
