"""Parity of the selections of (j, k) within a row (Section "The ByRow
strategy": TD_B, TD and SEQ; TD_A, the published method, is covered by
test_gpu_parity.py) between the CUDA path and the oracle: every row visit's
decision is replayed against the oracle's step with the same selection, the
factors must be bit-exact and the errors within 1e-6 relative.
"""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6
SELS = ["TD_B", "TD", "SEQ"]


def api():
    from paper_2205_06619_gb300 import api as a
    return a


def tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def run_and_replay(R, M, r, sweeps, seed, selection, window=0, divergences=1):
    from tests.replay import replay
    U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=r, sweeps=sweeps, seed=seed, window=window,
                                       trace_cap=5000, selection=selection)
    assert len(trace) == rep["trace_records"] and rep["trace_records"] < 5000
    out = replay(R, M, r, trace, seed=seed, selection=selection)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"]), selection
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"]), selection
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= divergences
    return rep, trace


@pytest.mark.parametrize("selection", SELS)
@pytest.mark.parametrize("window", [2, 64])
def test_selection_small_replay(selection, window):
    """36 x 52, rank 3, 80 % given, 3 sweeps; the window size must not change
    any decision."""
    R, M, _, _ = synth.uniform_planted(36, 52, 3, 0.01, 0.8, seed=21)
    rep, _ = run_and_replay(R, M, 3, 3, 4, selection, window=window)
    assert rep["accepted"] > 0


@pytest.mark.parametrize("selection", SELS)
def test_selection_ragged_tall_and_degenerate_shapes(selection):
    for (m, n, r, obs, seed) in [(1, 9, 1, 1.0, 1), (9, 1, 2, 1.0, 2), (17, 33, 1, 0.5, 3), (33, 17, 5, 0.9, 4),
                                 (2, 2, 2, 1.0, 5), (70, 40, 4, 0.6, 6)]:
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=seed)
        run_and_replay(R, M, r, 2, seed, selection)


@pytest.mark.parametrize("selection", SELS)
def test_selection_sparse_wide_replay(selection):
    """10 % given, n = 301 (not a multiple of 32), rank 4: long rows of
    positions with few candidates, several windows per row."""
    R, M, _, _ = synth.uniform_planted(24, 301, 4, 0.01, 0.1, seed=33)
    run_and_replay(R, M, 4, 2, 7, selection)


@pytest.mark.parametrize("selection", SELS)
def test_selection_lognormal_replay(selection):
    """Gene-expression-like values (planted rank 6, 0.5 log2(1 + LogNormal))."""
    R, M, _, _ = synth.lognormal_planted(40, 96, 6, 0.05, 0.8, seed=35)
    run_and_replay(R, M, 6, 2, 8, selection)


@pytest.mark.parametrize("selection", SELS)
def test_selection_graph_and_host_driven_loops_agree(selection, monkeypatch):
    R, M, _, _ = synth.uniform_planted(40, 50, 3, 0.01, 0.8, seed=41)
    a = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=200, selection=selection)
    monkeypatch.setenv("STMF_NO_GRAPH", "1")
    b = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=200, selection=selection)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]


def test_selections_in_the_batched_form():
    """Each selection in one batched launch gives the factors of the single
    calls."""
    probs = []
    for q, (m, n, r) in enumerate([(30, 60, 3), (50, 20, 2), (25, 90, 5)]):
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.7, seed=50 + q)
        probs.append(dict(R=tg(R), mask_words=api().pack_mask(M), rank=r, sweeps=2, seed=q))
    for sel in ["TD_A"] + SELS:
        outs, tuned = api().factorize_batched(probs, selection=sel)
        for pr, (U, V, rep), w in zip(probs, outs, tuned):
            U1, V1, _, _ = api().factorize(pr["R"], pr["mask_words"], rank=pr["rank"], sweeps=2, seed=pr["seed"],
                                           window=w, selection=sel)
            assert torch.equal(U, U1) and torch.equal(V, V1), sel


def test_rank_one_td_a_and_td_b_agree():
    """With r = 1 every k is 0 and TD_A, TD_B order the same columns: the
    same decisions on the device."""
    R, M, _, _ = synth.uniform_planted(30, 45, 1, 0.01, 0.8, seed=61)
    a = api().factorize(tg(R), api().pack_mask(M), rank=1, sweeps=2, seed=3, trace_cap=200, selection="TD_A")
    b = api().factorize(tg(R), api().pack_mask(M), rank=1, sweeps=2, seed=3, trace_cap=200, selection="TD_B")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]


def test_unknown_selection_rejected_by_the_library():
    """An out-of-range value reaching the C ABI is STMF_ERR_INVALID."""
    import ctypes as C
    a = api()
    R, M, _, _ = synth.uniform_planted(8, 10, 2, 0.01, 1.0, seed=1)
    Rg = tg(R)
    o, keep = a._options(1)
    o.selection = 7
    U = torch.empty((8, 2), device="cuda"); V = torch.empty((2, 10), device="cuda")
    ctx = a.context()
    st = a.load().stmf_factorize(ctx.h, 8, 10, 2, Rg.data_ptr(), 10, None, 0, C.byref(o), U.data_ptr(),
                                 V.data_ptr(), None)
    assert st == 1 and b"selection" in a.load().stmf_last_error(ctx.h)


@pytest.mark.parametrize("kw", [dict(selection="TD_B"), dict(selection="TD"), dict(selection="SEQ"),
                                dict(strategy="ByElement"), dict(strategy="ByMatrix")])
def test_fp16_screen_keeps_the_decisions_of_every_variant(kw):
    """The FP16 screen drops only candidates that provably do not improve, so
    with any selection or strategy precision 1 keeps precision 0's updates."""
    R, M, _, _ = synth.uniform_planted(40, 64, 3, 0.01, 0.8, seed=71)
    sweeps = 12 if kw.get("strategy") == "ByMatrix" else 2
    a = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=sweeps, seed=5, trace_cap=4000, precision=0, **kw)
    b = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=sweeps, seed=5, trace_cap=4000, precision=1, **kw)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]
