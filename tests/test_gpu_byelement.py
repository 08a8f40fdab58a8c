"""Parity of the ByElement method (STMF_ByElement_PermC_TD_W; Section "The
ByElement strategy") between the CUDA path and the oracle: every kept update
and every end of a sweep is replayed against the oracle's element scan, the
factors must be bit-exact and the errors within 1e-6 relative.
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


def run_and_replay(R, M, r, sweeps, seed, window=0, divergences=1):
    from tests.replay import replay_byelement
    U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=r, sweeps=sweeps, seed=seed, window=window,
                                       trace_cap=20000, strategy="ByElement")
    assert len(trace) == rep["trace_records"] and rep["trace_records"] < 20000
    assert sum(1 for t in trace if t[1] < 0) == rep["sweeps_done"]          # one end record per sweep
    assert sum(1 for t in trace if t[1] >= 0) == rep["accepted"]
    out = replay_byelement(R, M, r, trace, seed=seed)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= divergences
    return rep, trace


@pytest.mark.parametrize("window", [2, 64])
def test_byelement_small_replay(window):
    R, M, _, _ = synth.uniform_planted(36, 52, 3, 0.01, 0.8, seed=21)
    rep, trace = run_and_replay(R, M, 3, 3, 4, window=window)
    assert rep["accepted"] > 0
    # within a sweep the kept positions increase
    for sw in range(3):
        q = [t[2] for t in trace if t[0] == sw and t[1] >= 0]
        assert q == sorted(q) and len(set(q)) == len(q)


def test_byelement_ragged_tall_and_degenerate_shapes():
    for (m, n, r, obs, seed) in [(1, 9, 1, 1.0, 1), (9, 1, 2, 1.0, 2), (17, 33, 1, 0.5, 3), (33, 17, 5, 0.9, 4),
                                 (2, 2, 2, 1.0, 5), (70, 40, 4, 0.6, 6)]:
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=seed)
        run_and_replay(R, M, r, 2, seed)


def test_byelement_sparse_wide_and_lognormal_replay():
    R, M, _, _ = synth.uniform_planted(24, 301, 4, 0.01, 0.1, seed=33)
    run_and_replay(R, M, 4, 2, 7)
    R, M, _, _ = synth.lognormal_planted(40, 96, 6, 0.05, 0.8, seed=35)
    run_and_replay(R, M, 6, 2, 8)


def test_byelement_graph_and_host_driven_loops_agree(monkeypatch):
    R, M, _, _ = synth.uniform_planted(40, 50, 3, 0.01, 0.8, seed=41)
    a = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=2000, strategy="ByElement")
    monkeypatch.setenv("STMF_NO_GRAPH", "1")
    b = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=2000, strategy="ByElement")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]


def test_byelement_in_the_batched_form():
    probs = []
    for q, (m, n, r) in enumerate([(30, 60, 3), (50, 20, 2), (25, 90, 5)]):
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.7, seed=50 + q)
        probs.append(dict(R=tg(R), mask_words=api().pack_mask(M), rank=r, sweeps=2, seed=q))
    outs, tuned = api().factorize_batched(probs, strategy="ByElement")
    for pr, (U, V, rep), w in zip(probs, outs, tuned):
        U1, V1, _, _ = api().factorize(pr["R"], pr["mask_words"], rank=pr["rank"], sweeps=2, seed=pr["seed"],
                                       window=w, strategy="ByElement")
        assert torch.equal(U, U1) and torch.equal(V, V1)


def test_byelement_rejects_row_permutation_and_selection():
    a = api()
    R, M, _, _ = synth.uniform_planted(8, 10, 2, 0.01, 1.0, seed=1)
    with pytest.raises(a.StmfError):
        a.factorize(tg(R), a.pack_mask(M), rank=2, sweeps=1, strategy="ByElement", perm=np.arange(8))
    with pytest.raises(a.StmfError):
        a.factorize(tg(R), a.pack_mask(M), rank=2, sweeps=1, strategy="ByElement", selection="TD")
    U, V, rep, _ = a.factorize(tg(R), a.pack_mask(M), rank=2, sweeps=1)     # the context stays usable
    assert rep["sweeps_done"] == 1


def test_permc_order_with_ties_signed_zeros_and_negative_minima():
    """PermC (Section "The ByElement strategy": columns by increasing minimum
    given entry), computed on the device by rank counting: equal minima keep
    the smaller column first, -0 and +0 count as equal, a smaller entry that
    is not given does not count.  Checked through the replay of two sweeps,
    whose start depends on the column order (Acol draws its picks over the
    permuted columns) and whose every decision follows it."""
    rng = np.random.default_rng(61)
    m, n = 24, 700                       # more columns than one rank chunk of 512
    R = rng.integers(0, 40, size=(m, n)).astype(np.float64) / 8.0 - 2.0
    M = rng.random((m, n)) < 0.85
    M[0, :] = True
    mins = rng.integers(-6, 6, size=n).astype(np.float64) / 4.0    # many ties, negatives
    mins[5] = -0.0; mins[9] = 0.0; mins[600] = -0.0                # signed zeros tie with 0.0
    R = np.maximum(R, mins[None, :] + 0.125)
    R[0, :] = mins                                                 # row 0 holds each column's minimum
    R[1, 7] = -50.0; M[1, 7] = False                               # not given: no effect on the minimum
    assert np.signbit(R[0, 5]) and not np.signbit(R[0, 9])
    run_and_replay(R.astype(np.float32), M, 3, 2, 8, window=16, divergences=2)
