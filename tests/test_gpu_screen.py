"""FP16 screening with FP32 re-check (precision 1).

The screen may only drop candidates whose FP32 change is provably >= 0, and
the survivors are evaluated in FP32 by the same kernels as in precision 0, so
every decision, factor and reported error must be bit-identical to the FP32
path, in both selection modes and in the batched form.
"""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def api():
    from paper_2205_06619_gb300 import api as a
    return a


def tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _case(kind, m, n, r, obs, seed):
    if kind == "uniform":
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed)
    elif kind == "lognormal":
        R, M, _, _ = synth.lognormal_planted(m, n, r, 0.05, obs, seed)
    elif kind == "dyadic":
        R, M = synth.dyadic_noise(m, n, obs, seed)
    else:
        raise ValueError(kind)
    return R, M


def _run(R, M, r, precision, **kw):
    return api().factorize(tg(R), api().pack_mask(M), rank=r, precision=precision, trace_cap=5000, **kw)


def _same(a, b):
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[3] == b[3]                    # trace records, including the error after each row
    for key in ("f_init", "f_final", "candidates_tried", "candidates_issued", "accepted", "windows"):
        assert a[2][key] == b[2][key], key


CASES = [("uniform", 36, 52, 3, 0.8, 21), ("uniform", 200, 100, 3, 0.8, 0), ("uniform", 33, 17, 5, 0.9, 4),
         ("uniform", 1, 9, 1, 1.0, 1), ("lognormal", 130, 300, 10, 0.8, 7), ("dyadic", 70, 90, 4, 0.6, 3),
         ("uniform", 260, 530, 20, 0.5, 11)]


@pytest.mark.parametrize("kind,m,n,r,obs,seed", CASES)
def test_screen_keeps_the_fp32_decisions(kind, m, n, r, obs, seed):
    R, M = _case(kind, m, n, r, obs, seed)
    a = _run(R, M, r, 0, sweeps=3, seed=seed)
    b = _run(R, M, r, 1, sweeps=3, seed=seed)
    _same(a, b)
    assert a[2]["candidates_screened"] == 0
    assert 0 <= b[2]["candidates_screened"] <= b[2]["candidates_issued"]


@pytest.mark.parametrize("window", [2, 16, 64])
def test_screen_windows_and_best_mode(window):
    R, M = _case("uniform", 120, 90, 4, 0.7, 5)
    for select in (0, 1):
        a = _run(R, M, 4, 0, sweeps=2, seed=3, window=window, select=select)
        b = _run(R, M, 4, 1, sweeps=2, seed=3, window=window, select=select)
        _same(a, b)


def test_screen_drops_candidates_early():
    """Right after the random initialisation many candidates move the error
    up by far more than the bound, and the screen removes them."""
    R, M = _case("uniform", 400, 600, 8, 0.8, 2)
    a = _run(R, M, 8, 0, sweeps=1, seed=1)
    b = _run(R, M, 8, 1, sweeps=1, seed=1)
    _same(a, b)
    assert b[2]["candidates_screened"] > 0


def test_screen_replays_against_oracle():
    from tests.replay import replay
    R, M, _, _ = synth.uniform_planted(36, 52, 3, 0.01, 0.8, seed=21)
    U, V, rep, trace = _run(R, M, 3, 1, sweeps=3, seed=4)
    out = replay(R, M, 3, trace, seed=4)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert len(out["divergences"]) <= 1


def test_screen_host_driven_loop(monkeypatch):
    R, M = _case("uniform", 40, 50, 3, 0.8, 41)
    a = _run(R, M, 3, 1, sweeps=2, seed=2)
    monkeypatch.setenv("STMF_NO_GRAPH", "1")
    b = _run(R, M, 3, 1, sweeps=2, seed=2)
    _same(a, b)
    assert a[2]["candidates_screened"] == b[2]["candidates_screened"]


def test_screen_batched():
    probs = []
    for q, (m, n, r) in enumerate([(50, 80, 3), (120, 40, 5), (7, 300, 2)]):
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.7, 100 + q)
        probs.append(dict(R=tg(R), mask_words=api().pack_mask(M), rank=r, sweeps=2, seed=q))
    a, _ = api().factorize_batched(probs, window=8, precision=0)
    b, _ = api().factorize_batched(probs, window=8, precision=1)
    for (Ua, Va, ra), (Ub, Vb, rb) in zip(a, b):
        assert torch.equal(Ua, Ub) and torch.equal(Va, Vb)
        assert ra["f_final"] == rb["f_final"] and ra["candidates_tried"] == rb["candidates_tried"]


def test_unknown_precision_is_rejected():
    R, M = _case("uniform", 10, 12, 2, 1.0, 1)
    with pytest.raises(api().StmfError, match="precision"):
        _run(R, M, 2, 2, sweeps=1)
