"""The allocation-free selection statistics (stmf_selection_stats_noalloc).

Some callers may not allocate device memory when they call: a process whose
device-memory budget is fixed at start-up, or a loop that cannot pay for the
synchronisation and allocator work of cudaMalloc.  For them the library
offers one entry point whose scratch is a fixed device array inside the
library.  This test calls it through the C ABI twice in a row, on different
inputs, and checks each result against stmf_selection_stats (which grows a
workspace with cudaMalloc): the same kernels and summation orders, so the
results must be identical.  It checks both against the oracle's statistics of
the ByRow strategy (td_col within 1e-12 relative, the histograms exactly), and
that the device's free memory is the same before and after the two calls.  It
also checks that a problem too large for the fixed array is rejected before
anything is launched.  The file is named so that pytest collects it last.
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
    import oracle as orc
    from paper_2205_06619_gb300 import api
    cases = [(300, 517, 7, 0.8, 1), (129, 2050, 12, 0.5, 2)]
    data = []
    for (m, n, r, obs, seed) in cases:
        R, M, U, V = _inputs(m, n, r, obs, seed)
        Rg, Ug, Vg, Mw = _tg(R), _tg(U), _tg(V), api.pack_mask(M)
        td_ref, ch_ref, f_ref = api.selection_stats(Rg, Ug, Vg, Mw)
        td = torch.full((n,), float("nan"), device="cuda", dtype=torch.float64)
        ch = torch.full((n, r), -1, device="cuda", dtype=torch.int32)
        data.append((R, M, U, V, Rg, Ug, Vg, Mw, td_ref, ch_ref, f_ref, td, ch))
    # the first call of the process may load the library's device code (lazy
    # module loading), which is not an allocation of the call itself
    api.selection_stats_noalloc(data[0][4], data[0][5], data[0][6], data[0][7], td_col=data[0][11],
                                colhist=data[0][12])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    results = []
    for (R, M, U, V, Rg, Ug, Vg, Mw, td_ref, ch_ref, f_ref, td, ch) in data:
        td.fill_(float("nan")); ch.fill_(-1)
        torch.cuda.synchronize()
        results.append(api.selection_stats_noalloc(Rg, Ug, Vg, Mw, td_col=td, colhist=ch))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for (R, M, U, V, Rg, Ug, Vg, Mw, td_ref, ch_ref, f_ref, _, _), (td, ch, f) in zip(data, results):
        assert torch.equal(ch, ch_ref) and torch.equal(td, td_ref) and f == f_ref
        etd, ech, _ = orc.row_stats(R, M, U.astype(np.float64), V.astype(np.float64), 0)
        assert np.array_equal(ch.cpu().numpy(), ech)
        tdn = td.cpu().numpy()
        assert np.all(np.abs(tdn - etd) <= 1e-12 * np.maximum(np.abs(etd), 1e-300))
        ef = orc.error(R, M, U.astype(np.float64), V.astype(np.float64))
        assert abs(f - ef) <= 1e-12 * ef


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
