"""C-ABI checks that need no GPU: the library loads, exports every function
include/rdm.h declares, and the ctypes structures of the binding have the
layout a C compiler gives the header's structs."""

import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rdm.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rdm_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def rdm():
    from paper_2009_03551_gb300 import build as b
    b.build()
    from paper_2009_03551_gb300 import rdm as mod
    return mod


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rdm_create", "rdm_destroy", "rdm_set_params", "rdm_upload_h0", "rdm_upload_h1",
                     "rdm_solve", "rdm_get_p0", "rdm_get_p1", "rdm_get_alpha", "rdm_batch_create",
                     "rdm_force_branches", "rdm_get_log", "rdm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(rdm):
    lib = rdm._lib
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", str(rdm._LIB_PATH)], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (rdm_[a-z0-9_]+)", out.stdout))
    assert set(declared_functions()) <= exported
    assert set(rdm.EXPORTED) <= exported


def test_struct_layout_matches_c(rdm):
    import ctypes as C
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "rdm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(rdm_bsr), sizeof(rdm_bsr_out), sizeof(rdm_params),
         sizeof(rdm_info), sizeof(rdm_iter_log));
  printf("%zu %zu %zu %zu\n", offsetof(rdm_bsr, nnzb), offsetof(rdm_params, max_iter),
         offsetof(rdm_info, eps_min), offsetof(rdm_iter_log, nnzb0));
  printf("%zu %zu %zu %zu\n", sizeof(rdm_test_knobs), offsetof(rdm_test_knobs, tc_hold),
         offsetof(rdm_test_knobs, tc_window_cols), offsetof(rdm_test_knobs, tc_block_copies));
  printf("%zu %zu %zu %zu %zu\n", offsetof(rdm_params, split_directions), offsetof(rdm_params, correct),
         offsetof(rdm_info, oz_launches), offsetof(rdm_info, correction_ms), offsetof(rdm_params, correct_tau));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [C.sizeof(rdm.rdm_bsr), C.sizeof(rdm.rdm_bsr_out), C.sizeof(rdm.rdm_params),
                     C.sizeof(rdm.rdm_info), C.sizeof(rdm.rdm_iter_log)]
    assert offs == [rdm.rdm_bsr.nnzb.offset, rdm.rdm_params.max_iter.offset,
                    rdm.rdm_info.eps_min.offset, rdm.rdm_iter_log.nnzb0.offset]
    knobs = [int(x) for x in lines[2].split()]
    assert knobs == [C.sizeof(rdm.rdm_test_knobs), rdm.rdm_test_knobs.tc_hold.offset,
                     rdm.rdm_test_knobs.tc_window_cols.offset, rdm.rdm_test_knobs.tc_block_copies.offset]
    tail = [int(x) for x in lines[3].split()]
    assert tail == [rdm.rdm_params.split_directions.offset, rdm.rdm_params.correct.offset,
                    rdm.rdm_info.oz_launches.offset, rdm.rdm_info.correction_ms.offset,
                    rdm.rdm_params.correct_tau.offset]


def test_default_params_without_gpu(rdm):
    p = rdm.rdm_default_params()
    assert p.tau == 1e-6 and p.max_iter == 100 and p.mode == rdm.MODE_FP64 and p.spin_factor == 2.0


def test_create_fails_loudly_without_gpu(rdm):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(rdm.RdmError) as e:
        rdm.rdm_create(0)
    assert e.value.code == rdm.RDM_ECUDA


def test_null_handle_is_rejected(rdm):
    import ctypes as C
    assert rdm._lib.rdm_solve(None, None) == rdm.RDM_EINVAL
    assert rdm._lib.rdm_set_params(None, None) == rdm.RDM_EINVAL
    assert rdm._lib.rdm_destroy(None) == rdm.RDM_OK
    assert rdm._lib.rdm_default_params(None) == rdm.RDM_EINVAL
    n = C.c_int()
    assert rdm._lib.rdm_get_log(None, None, 0, C.byref(n)) == rdm.RDM_EINVAL


def _fake_getter(rdm, nb, b, nnz):
    """A stand-in for rdm_get_p0/p1 that follows the C contract (size query
    with row_ptr == NULL, then a copy into the caller's buffers)."""
    import ctypes as C
    import numpy as np

    def getter(h, *args):
        out = C.cast(args[-1], C.POINTER(rdm.rdm_bsr_out)).contents
        if not out.row_ptr:
            out.nb, out.b, out.n, out.nnzb = nb, b, nb * b, nnz
            return 0
        assert out.nnzb >= nnz
        def view(addr, ctype, n):
            return np.ctypeslib.as_array(C.cast(addr, C.POINTER(ctype)), shape=(n,))
        view(out.row_ptr, C.c_int32, nb + 1)[:] = np.linspace(0, nnz, nb + 1).astype(np.int32)
        if nnz:
            view(out.col_idx, C.c_int32, nnz)[:] = np.arange(nnz) % nb
            view(out.vals, C.c_double, nnz * b * b)[:] = np.arange(nnz * b * b)
        out.n = nb * b
        return 0
    return getter


def test_getter_fills_fresh_or_caller_buffers(rdm):
    """The binding's getters copy once: into fresh arrays, or into the
    caller's (e.g. pinned) buffers, returning views of exactly the result."""
    import numpy as np
    nb, b, nnz = 5, 4, 7
    g = _fake_getter(rdm, nb, b, nnz)
    r = rdm._fetch(None, g, 0)
    assert r.row_ptr.shape == (nb + 1,) and r.col_idx.shape == (nnz,) and r.vals.shape == (nnz, b, b)
    assert np.array_equal(r.vals.reshape(-1), np.arange(nnz * b * b))
    bufs = (np.zeros(nb + 1, np.int32), np.zeros(nnz + 3, np.int32), np.zeros((nnz + 3) * b * b))
    r2 = rdm._fetch(None, g, 0, out=bufs)
    assert np.shares_memory(r2.vals, bufs[2]) and np.shares_memory(r2.col_idx, bufs[1])
    assert r2.vals.shape == (nnz, b, b) and np.array_equal(r2.vals, r.vals)
    assert np.array_equal(r2.col_idx, r.col_idx) and np.array_equal(r2.row_ptr, r.row_ptr)
    with pytest.raises(ValueError):
        rdm._fetch(None, g, 0, out=(bufs[0], bufs[1][: nnz - 1], bufs[2]))
    with pytest.raises(ValueError):
        rdm._fetch(None, g, 0, out=(bufs[0], bufs[1], bufs[2].astype(np.float32)))
    empty = rdm._fetch(None, _fake_getter(rdm, nb, b, 0), 0)
    assert empty.col_idx.shape == (0,) and empty.vals.shape == (0, b, b)
