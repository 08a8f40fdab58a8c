"""Pins of the oracle's ByMatrix method (STMF_ByMatrix_NoPerm_TD_W; Section
"The ByMatrix strategy" and its pseudocode in the Supplement): the err order
on a hand-computed example (tests/golden/bymatrix_2x3.txt), the order's
defining properties on random dyadic data, the coin against the published
SplitMix64, brute force of an iteration, and invariants of the whole method.
"""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth
from test_oracle_pins import _consistent_state, load_golden


def test_matrix_order_hand_example(orc):
    g = load_golden("bymatrix_2x3.txt")
    M = g["M"].astype(bool)
    for mode in ("fp64", "fp32"):
        qs, ks, ty, errs = orc.matrix_order(g["R"], M, g["U"], g["V"], seed=3, it=0, mode=mode)
        assert qs.tolist() == g["order_q"][0].astype(int).tolist()
        assert errs.tolist() == g["order_err"][0].tolist()
        assert not ks.any()


def test_matrix_coin_is_the_published_generator(orc):
    """The coin is the top bit of SplitMix64 (pinned against its published
    outputs elsewhere) keyed by seed ^ 0x5A..5A at counter it*m*n + q, and it
    is fair."""
    m, n, seed = 7, 9, 11
    draws = []
    for it in range(3):
        for q in range(m * n):
            c = orc.matrix_coin(seed, it, m, n, q)
            assert c == orc.splitmix64(seed ^ 0x5A5A5A5A5A5A5A5A, it * m * n + q) >> 63
            draws.append(c)
    assert 0.4 < np.mean(draws) < 0.6


def _seq_sum(values):
    s = 0.0
    for v in values:
        s += float(v)
    return s


def test_matrix_order_follows_its_definition(orc):
    for seed in range(5):
        R, M = synth.dyadic_noise(6, 9, 0.8, seed=500 + seed, levels=8)     # few levels: ties in err
        R = R.astype(float)
        U, V = _consistent_state(orc, R, M, 3, seed)
        m, n = R.shape
        P1, A, _ = orc.maxplus(U, V, "fp32")
        td = np.where(M, np.abs((R - P1).astype(np.float32)).astype(float), 0.0)
        tdr = [_seq_sum(td[i][M[i]]) for i in range(m)]
        tdc = [_seq_sum(td[:, j][M[:, j]]) for j in range(n)]
        for it in (0, 4):
            qs, ks, ty, errs = orc.matrix_order(R, M, U, V, seed=seed, it=it)
            assert sorted(qs.tolist()) == np.flatnonzero(M.ravel()).tolist()
            for a, q in enumerate(qs):
                i, j = divmod(int(q), n)
                assert errs[a] == (tdr[i] + tdc[j]) - td[i, j]
                assert ks[a] == A[i, j] and ty[a] == orc.matrix_coin(seed, it, m, n, int(q))
            assert np.all(errs[:-1] >= errs[1:])
            assert all(qs[a] < qs[a + 1] for a in range(len(qs) - 1) if errs[a] == errs[a + 1])


def test_matrix_step_brute_force(orc):
    """An iteration keeps the first element, in the err order, whose update
    (F-ULF or F-URF by its coin) lowers the error, and counts its tries."""
    checked = 0
    for seed in range(10):
        R, M = synth.dyadic_noise(5, 6, 0.8, seed=600 + seed, levels=32)
        R = R.astype(float)
        U, V = _consistent_state(orc, R, M, 2, seed)
        f = orc.error(R, M, U, V)
        n = R.shape[1]
        for it in (0, 1, 7):
            qs, ks, ty, _ = orc.matrix_order(R, M, U, V, seed=seed, it=it)
            expected, tried = None, 0
            for a, (q, k, t) in enumerate(zip(qs, ks, ty)):
                i, j = divmod(int(q), n)
                tried += 1
                _, _, fn_ = (orc.fulf if t == 0 else orc.furf)(R, M, U, V, i, j, int(k))
                if fn_ < f:
                    expected = ((a, i, j, int(k), int(t)), fn_)
                    break
            U2, V2 = U.copy(), V.copy()
            kept, f2, out, ntried = orc.matrix_step(R, M, U2, V2, seed, it, f)
            assert ntried == tried
            if expected is None:
                assert not kept and f2 == f and np.array_equal(U2, U)
            else:
                assert kept and out == expected[0] and f2 == expected[1]
                checked += 1
    assert checked > 10


def test_bymatrix_whole_method_invariants(orc):
    R, M = synth.dyadic_noise(8, 12, 0.8, seed=61, levels=64)
    a = orc.factorize(R, M, 3, sweeps=25, seed=5, strategy="ByMatrix", trace_cap=100)
    b = orc.factorize(R, M, 3, sweeps=25, seed=5, strategy="ByMatrix", trace_cap=100)
    assert np.all(np.diff(a["f_hist"]) <= 0) and a["f_hist"][-1] < a["f_hist"][0]
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["trace"], b["trace"])
    P = np.max(a["U"][:, :, None] + a["V"][None, :, :], axis=1)
    assert np.all(P[M] <= R[M])
    fin = np.abs(R.astype(float) - P.astype(np.float32))[M].sum()
    assert abs(fin - a["f_hist"][-1]) <= 1e-9 * fin
    assert len(a["trace"]) == 25 and a["trace"][:, 0].tolist() == list(range(25))
    assert a["kept"] == int(np.sum(a["trace"][:, 1] >= 0))


def test_bymatrix_transpose_and_shift(orc):
    R, M = synth.dyadic_noise(7, 11, 1.0, seed=63, levels=64)
    a = orc.factorize(R, M, 2, sweeps=10, p=4, seed=3, strategy="ByMatrix", trace_cap=100)
    b = orc.factorize(R.T.copy(), M.T.copy(), 2, sweeps=10, p=4, seed=3, strategy="ByMatrix", trace_cap=100)
    assert np.array_equal(b["U"], a["V"].T) and np.array_equal(b["V"], a["U"].T)
    assert np.array_equal(a["trace"], b["trace"])
    c = orc.factorize(R + 3.5, M, 2, sweeps=10, p=4, seed=3, strategy="ByMatrix", trace_cap=100)
    assert np.array_equal(a["trace"], c["trace"]) and np.array_equal(a["f_hist"], c["f_hist"])
    assert np.array_equal(c["U"], a["U"] + 3.5) and np.array_equal(c["V"], a["V"])


def test_bymatrix_rejects_perm_and_selection(orc):
    R, M = synth.dyadic_noise(4, 5, 1.0, seed=1)
    with pytest.raises(ValueError):
        orc.factorize(R, M, 2, sweeps=1, strategy="ByMatrix", selection="TD")
