"""Parity at the benchmark sizes, on samples the oracle computes one by one and
on properties that hold at any size."""
import numpy as np
import pytest

import oracle as orc
from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,n,r", [(1000, 5000, 10), (4000, 20000, 20)])
def test_product_full_size_sampled_rows(m, n, r):
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(m + r)
    U = (0.5 * np.log2(1 + rng.lognormal(3, 2, size=(m, r)))).astype(np.float32)
    V = (0.5 * np.log2(1 + rng.lognormal(3, 2, size=(r, n)))).astype(np.float32)
    P1, A, P2 = api.maxplus(_tg(U), _tg(V))
    rows = rng.choice(m, size=12, replace=False)
    e1, ea, e2 = orc.maxplus(U[rows], V, "fp32")
    assert np.array_equal(P1[rows].cpu().numpy().astype(np.float64), e1)
    assert np.array_equal(A[rows].cpu().numpy().astype(np.int32), ea)
    assert np.array_equal(P2[rows].cpu().numpy().astype(np.float64), e2)


def test_gene_scale_sweep_properties_and_first_rows():
    """One sweep of the 1000 x 5000 rank-10 workload: the reported errors never
    increase, the final error equals the oracle's recomputation from the
    returned factors (1e-6 relative), U (x) V <= R on given entries up to the
    FP32 roundings of the residuations, and the first rows' decisions equal
    the oracle's (replayed from the same start)."""
    from paper_2205_06619_gb300 import api
    from tests.replay import replay
    w = synth.workload_gene(seed=0)
    R, M = w["R"], w["mask"]
    Rg, Mw = _tg(R), api.pack_mask(M)
    fz = api.Factorization(Rg, Mw, rank=10, seed=0, trace_cap=2000)
    rep = fz.run(1)
    U, V = fz.result()
    trace = fz.trace_records()
    assert len(trace) == 1000
    fs = [t[6] for t in trace]
    assert all(b <= a * (1 + 1e-7) for a, b in zip(fs, fs[1:]))
    Un, Vn = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    f_or = orc.error(R, M, Un, Vn)
    assert abs(rep["f_final"] - f_or) <= 1e-6 * f_or
    P1, _, _ = api.maxplus(U, V)
    P = P1.cpu().numpy().astype(np.float64)
    mag = np.abs(R.astype(np.float64)) + np.abs(Un).max() + np.abs(Vn).max()
    assert np.all((P - R)[M] <= (mag * 2.0 ** -22)[M])
    # decisions of the first 3 rows of sweep 0, replayed by the oracle
    out = replay(R, M, 10, trace[:3], seed=0)
    assert len(out["divergences"]) == 0
