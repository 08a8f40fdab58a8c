"""The allocation-free selection statistics (stmf_selection_stats_noalloc).

Some callers may not allocate device memory when they call: a process whose
device-memory budget is fixed at start-up, or a loop that cannot pay for the
synchronisation and allocator work of cudaMalloc.  For them the library
offers one entry point whose scratch is a fixed device array inside the
library.  This test calls it through the C ABI twice in a row, on different
inputs, and checks each result against stmf_selection_stats (which grows a
workspace with cudaMalloc) within the tolerance of the other statistics
tests; it also checks that a problem too large for the fixed array is
rejected before anything is launched.  The file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _inputs(m, n, r, obs, seed):
    R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=seed)
    rng = np.random.default_rng(seed)
    U = rng.random((m, r)).astype(np.float32)
    V = rng.random((r, n)).astype(np.float32) - 0.5
    return R, M, U, V


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2205_06619_gb300 import api
    for (m, n, r, obs, seed) in [(300, 517, 7, 0.8, 1), (129, 2050, 12, 0.5, 2)]:
        R, M, U, V = _inputs(m, n, r, obs, seed)
        Rg, Ug, Vg, Mw = _tg(R), _tg(U), _tg(V), api.pack_mask(M)
        td_ref, ch_ref, f_ref = api.selection_stats(Rg, Ug, Vg, Mw)
        td = torch.full((n,), float("nan"), device="cuda", dtype=torch.float64)
        ch = torch.full((n, r), -1, device="cuda", dtype=torch.int32)
        td, ch, f = api.selection_stats_noalloc(Rg, Ug, Vg, Mw, td_col=td, colhist=ch)
        torch.cuda.synchronize()
        assert torch.equal(ch, ch_ref)
        assert torch.allclose(td, td_ref, rtol=1e-12, atol=0.0)
        assert abs(f - f_ref) <= 1e-12 * abs(f_ref)


def test_noalloc_rejects_problems_above_its_scratch():
    from paper_2205_06619_gb300 import api
    L = api.load()
    ctx = api.context()
    f = ctypes.c_double()
    # 4000 x 20000 at rank 20 needs far more than the fixed scratch; the sizes
    # are checked before any pointer is used or any work is launched
    st = L.stmf_selection_stats_noalloc(ctx.h, 4000, 20000, 20, ctypes.c_void_p(16), 20000, None, 0,
                                        ctypes.c_void_p(16), 20, ctypes.c_void_p(16), 20000, None, None,
                                        ctypes.byref(f))
    assert st == 1
    assert b"scratch" in L.stmf_last_error(ctx.h)
