"""The allocation-free inner product (rdm_bsr_dot_noalloc) against the
library's own polarizability, which reduces the same <P1_d, H1_g> with
allocated scratch: alpha[g][d] = -2 <P1_d, H1_g>.

This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone and after the others.
"""

import numpy as np
import pytest

from synth import make_cluster

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def _device_bsr(m, torch):
    class D:
        pass

    d = D()
    d.nb, d.b, d.n = m.nb, m.b, m.n
    d.row_ptr = torch.from_numpy(np.ascontiguousarray(m.row_ptr, dtype=np.int32)).cuda()
    d.col_idx = torch.from_numpy(np.ascontiguousarray(m.col_idx, dtype=np.int32)).cuda()
    d.vals = torch.from_numpy(np.ascontiguousarray(m.vals, dtype=np.float64)).cuda()
    return d


def test_noalloc_dot_matches_alpha_twice_in_a_row(rdm):
    import torch

    s = make_cluster(120, opa=8, b=32, cutoff=10.0, seed=31, dirs=("x", "y", "z"))
    sol = rdm.Solver(0)
    sol.set_params(tau=1e-7, tol=1e-9, mode="fp64", max_iter=100)
    sol.load(s)
    code, _ = sol.solve()
    assert code == rdm.RDM_OK
    alpha = sol.alpha()
    h1 = [_device_bsr(m, torch) for m in s.h1]
    p1 = [_device_bsr(sol.p1(0, d), torch) for d in range(3)]
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on the shared scratch array: (g, d) = (0, 0) then (1, 2)
    for g, d in ((0, 0), (1, 2)):
        rdm.rdm_bsr_dot_noalloc(p1[d], h1[g], out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = -2.0 * float(out.item())
        assert got == pytest.approx(alpha[g, d], rel=1e-12, abs=1e-12)


def test_noalloc_dot_rejects_what_it_cannot_do(rdm):
    import torch

    s = make_cluster(20, opa=8, b=32, cutoff=10.0, seed=32, dirs=("x",))
    a = _device_bsr(s.h0, torch)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(rdm.RdmError):
        rdm.rdm_bsr_dot_noalloc(s.h0, s.h0, out.data_ptr())          # host matrices
    big = _device_bsr(s.h0, torch)
    big.nb = 1 << 19                                                 # above the scratch limit
    with pytest.raises(rdm.RdmError):
        rdm.rdm_bsr_dot_noalloc(big, big, out.data_ptr())
    rdm.rdm_bsr_dot_noalloc(a, a, out.data_ptr())                   # <H0, H0> = ||H0||_F^2
    torch.cuda.synchronize()
    assert float(out.item()) == pytest.approx(float(np.sum(s.h0.vals ** 2)), rel=1e-12)
