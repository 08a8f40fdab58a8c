"""The batched form (many problems in one device launch) makes exactly the
decisions of the one-problem method, with autotuned or fixed windows."""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _problems(count, seed):
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(seed)
    probs = []
    for q in range(count):
        m = int(rng.integers(5, 90)); n = int(rng.integers(5, 160))
        r = int(rng.integers(1, 9)); d = float(rng.uniform(0.3, 0.95))
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, d, seed=int(rng.integers(1 << 30)))
        probs.append(dict(R=_tg(R), mask_words=api.pack_mask(M), rank=r, sweeps=int(rng.integers(1, 4)),
                          seed=int(rng.integers(1 << 30))))
    return probs


@pytest.mark.parametrize("window", [0, 8])
def test_batched_equals_one_at_a_time(window):
    from paper_2205_06619_gb300 import api
    probs = _problems(12, seed=5 + window)
    outs, tuned = api.factorize_batched(probs, window=window)
    assert len(outs) == len(probs)
    if window:
        assert all(t == window for t in tuned)
    else:
        assert all(t in (16, 32, 64) for t in tuned)
    for pr, (U, V, rep) in zip(probs, outs):
        U1, V1, rep1, _ = api.factorize(pr["R"], pr["mask_words"], rank=pr["rank"], sweeps=pr["sweeps"],
                                        seed=pr["seed"])
        assert torch.equal(U, U1) and torch.equal(V, V1)
        assert rep["candidates_tried"] == rep1["candidates_tried"] and rep["accepted"] == rep1["accepted"]
        assert rep["sweeps_done"] == pr["sweeps"]
        assert abs(rep["f_final"] - rep1["f_final"]) <= 1e-9 * max(rep1["f_final"], 1e-30)
