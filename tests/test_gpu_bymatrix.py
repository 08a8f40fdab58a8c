"""Parity of the ByMatrix method (STMF_ByMatrix_NoPerm_TD_W; Section "The
ByMatrix strategy") between the CUDA path and the oracle: every iteration's
outcome (the kept element's position in the err order, its update, or
nothing) is replayed against the oracle's iteration, the factors must be
bit-exact and the errors within 1e-6 relative.  Sizes cover one sort tile
and many (global merge passes).
"""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


def api():
    from paper_2205_06619_gb300 import api as a
    return a


def tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def run_and_replay(R, M, r, iters, seed, window=0, divergences=1):
    from tests.replay import replay_bymatrix
    U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=r, sweeps=iters, seed=seed, window=window,
                                       trace_cap=iters + 1, strategy="ByMatrix")
    assert rep["sweeps_done"] == iters and len(trace) == iters
    assert [t[0] for t in trace] == list(range(iters))
    assert sum(1 for t in trace if t[2] >= 0) == rep["accepted"]
    out = replay_bymatrix(R, M, r, trace, seed=seed)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= divergences
    return rep, trace


@pytest.mark.parametrize("window", [2, 64])
def test_bymatrix_small_replay(window):
    R, M, _, _ = synth.uniform_planted(36, 52, 3, 0.01, 0.8, seed=21)
    rep, trace = run_and_replay(R, M, 3, 30, 4, window=window)
    assert rep["accepted"] > 20
    assert any(t[2] > 0 for t in trace)          # some iterations keep a later element of the order


def test_bymatrix_many_sort_tiles_replay():
    """100 x 500 (50,000 elements, a 65,536-pair sort: 32 tiles and global
    merge passes)."""
    R, M, _, _ = synth.uniform_planted(100, 500, 4, 0.01, 0.8, seed=23)
    run_and_replay(R, M, 4, 6, 5)


def test_bymatrix_ragged_tall_and_degenerate_shapes():
    for (m, n, r, obs, seed) in [(1, 9, 1, 1.0, 1), (9, 1, 2, 1.0, 2), (17, 33, 1, 0.5, 3), (33, 17, 5, 0.9, 4),
                                 (2, 2, 2, 1.0, 5), (70, 40, 4, 0.6, 6)]:
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=seed)
        run_and_replay(R, M, r, 12, seed)


def test_bymatrix_sparse_wide_and_lognormal_replay():
    R, M, _, _ = synth.uniform_planted(24, 301, 4, 0.01, 0.1, seed=33)
    run_and_replay(R, M, 4, 15, 7)
    R, M, _, _ = synth.lognormal_planted(40, 96, 6, 0.05, 0.8, seed=35)
    run_and_replay(R, M, 6, 15, 8)


def test_bymatrix_graph_and_host_driven_loops_agree(monkeypatch):
    R, M, _, _ = synth.uniform_planted(40, 50, 3, 0.01, 0.8, seed=41)
    a = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=10, seed=2, trace_cap=20, strategy="ByMatrix")
    monkeypatch.setenv("STMF_NO_GRAPH", "1")
    b = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=10, seed=2, trace_cap=20, strategy="ByMatrix")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]


def test_bymatrix_in_the_batched_form():
    probs = []
    for q, (m, n, r) in enumerate([(30, 60, 3), (50, 20, 2), (25, 90, 5)]):
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.7, seed=50 + q)
        probs.append(dict(R=tg(R), mask_words=api().pack_mask(M), rank=r, sweeps=8, seed=q))
    outs, tuned = api().factorize_batched(probs, strategy="ByMatrix")
    for pr, (U, V, rep), w in zip(probs, outs, tuned):
        U1, V1, _, _ = api().factorize(pr["R"], pr["mask_words"], rank=pr["rank"], sweeps=8, seed=pr["seed"],
                                       window=w, strategy="ByMatrix")
        assert torch.equal(U, U1) and torch.equal(V, V1)


def test_bymatrix_rejects_row_permutation_and_selection():
    a = api()
    R, M, _, _ = synth.uniform_planted(8, 10, 2, 0.01, 1.0, seed=1)
    with pytest.raises(a.StmfError):
        a.factorize(tg(R), a.pack_mask(M), rank=2, sweeps=1, strategy="ByMatrix", perm=np.arange(8))
    with pytest.raises(a.StmfError):
        a.factorize(tg(R), a.pack_mask(M), rank=2, sweeps=1, strategy="ByMatrix", selection="TD_B")
