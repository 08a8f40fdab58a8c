"""RMSE-A / RMSE-P on the device (stmf_rmse; Section "Evaluation metrics",
with the held-out test set of Section "Evaluation") against the oracle: the
per-entry terms are the same FP32 residuals on both sides, so only the
summation order differs (1e-12 relative); the counts are exact."""
import numpy as np
import pytest

import oracle as orc
from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _check(R, M, U, V, mask=True):
    from paper_2205_06619_gb300 import api
    got = api.rmse(_tg(R), _tg(U), _tg(V), api.pack_mask(M) if mask else None)
    Me = M if mask else np.ones_like(M)
    exp = orc.rmse(R, Me, U.astype(np.float64), V.astype(np.float64))
    assert got[2:] == exp[2:]
    for g, e in zip(got[:2], exp[:2]):
        if np.isnan(e):
            assert np.isnan(g)
        else:
            assert abs(g - e) <= 1e-12 * max(e, 1e-300), (got, exp)
    return got


@pytest.mark.parametrize("m,n,r,obs", [(1, 1, 1, 1.0), (7, 300, 3, 0.8), (257, 513, 10, 0.5), (64, 2000, 32, 0.9)])
def test_rmse_matches_oracle(m, n, r, obs):
    R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=m + n)
    rng = np.random.default_rng(m)
    U = rng.random((m, r)).astype(np.float32)
    V = (rng.random((r, n)) - 0.3).astype(np.float32)
    _check(R, M, U, V)
    a, p, na, np_ = _check(R, M, U, V, mask=False)
    assert np_ == 0 and np.isnan(p)


def test_rmse_skips_held_out_entries_without_truth():
    R, M, _, _ = synth.uniform_planted(40, 90, 4, 0.01, 0.7, seed=9)
    R = R.copy()
    hid = np.argwhere(~M)
    for q in hid[::3]:
        R[tuple(q)] = np.nan
    rng = np.random.default_rng(9)
    U = rng.random((40, 4)).astype(np.float32)
    V = rng.random((4, 90)).astype(np.float32)
    a, p, na, np_ = _check(R, M, U, V)
    assert np_ == len(hid) - len(hid[::3])


def test_rmse_of_a_gene_scale_factorization():
    """The 1000 x 5000 rank-10 workload after two sweeps: training error
    (RMSE-A) and prediction error on the 20% held out (RMSE-P)."""
    from paper_2205_06619_gb300 import api
    w = synth.workload_gene(seed=0)
    U, V, rep, _ = api.factorize(_tg(w["R"]), api.pack_mask(w["mask"]), rank=10, sweeps=2, seed=0)
    a, p, na, np_ = _check(w["R"], w["mask"], U.cpu().numpy(), V.cpu().numpy())
    assert na == int(w["mask"].sum()) and np_ == w["mask"].size - na
    assert 0.0 < a < p * 10 and np.isfinite(p)
