"""Pins of the oracle's selections of (j, k) within a row (Section "The ByRow
strategy": SEQ, TD, TD_A, TD_B) against a hand-computed example
(tests/golden/selections_3x4.txt), against the defining properties of each
order on random dyadic inputs, against brute force over the candidates of a
row, and against invariants of the whole method.
"""
import numpy as np
import pytest

from paper_2205_06619_gb300 import synth
from test_oracle_pins import _consistent_state, load_golden

SELECTIONS = ("TD_A", "TD_B", "TD", "SEQ")


def test_selection_golden(orc):
    g = load_golden("selections_3x4.txt")
    R, U, V = g["R"], g["U"], g["V"]
    M = g["M"].astype(bool)
    for mode in ("fp64", "fp32"):
        for sel in SELECTIONS:
            for i in range(3):
                js, ks = orc.row_order(R, M, U, V, i, mode=mode, selection=sel)
                assert js.tolist() == g["%s_row%d_js" % (sel, i)][0].astype(int).tolist(), (sel, i)
                assert ks.tolist() == g["%s_row%d_ks" % (sel, i)][0].astype(int).tolist(), (sel, i)


def _state(orc, seed, m=7, n=11, r=3, density=0.75):
    R, M = synth.dyadic_noise(m, n, density, seed=seed, levels=16)   # few levels: many ties
    U, V = _consistent_state(orc, R.astype(float), M, r, seed)
    return R.astype(float), M, U, V


def test_selection_orders_follow_their_definitions(orc):
    """Each order, checked against the property that defines it."""
    for seed in range(6):
        R, M, U, V = _state(orc, 200 + seed)
        m, n = R.shape
        r = U.shape[1]
        P1, A, _ = orc.maxplus(U, V, "fp32")
        td = np.where(M, np.abs(R - P1), -1.0)          # -1 marks entries not given
        for i in range(m):
            given = np.flatnonzero(M[i])
            # SEQ: given j in increasing order, each with k = 0..r-1
            js, ks = orc.row_order(R, M, U, V, i, selection="SEQ")
            assert js.tolist() == np.repeat(given, r).tolist()
            assert ks.tolist() == np.tile(np.arange(r), len(given)).tolist()
            # TD: a permutation of the given j, td(i, j) non-increasing, equal
            # td in increasing j; k = f(i, j)
            js, ks = orc.row_order(R, M, U, V, i, selection="TD")
            assert sorted(js.tolist()) == given.tolist()
            d = td[i, js]
            assert np.all(d[:-1] >= d[1:])
            assert all(js[a] < js[a + 1] for a in range(len(js) - 1) if d[a] == d[a + 1])
            assert ks.tolist() == A[i, js].tolist()
            # TD_B: the columns of TD_A; k from the worst entries of row i and
            # of column j
            ja, _ = orc.row_order(R, M, U, V, i, selection="TD_A")
            js, ks = orc.row_order(R, M, U, V, i, selection="TD_B")
            assert js.tolist() == ja.tolist()
            j0 = int(given[np.argmax(td[i, given])])              # first maximum: smaller t
            for j, k in zip(js, ks):
                col = np.flatnonzero(M[:, j])
                i0 = int(col[np.argmax(td[col, j])])
                want = A[i, j0] if P1[i, j0] >= P1[i0, j] else A[i0, j]
                assert k == want


@pytest.mark.parametrize("selection", ["TD_B", "TD", "SEQ"])
def test_selection_step_keeps_first_improving(orc, selection):
    """Over all candidates of the row in the selection's order (F-ULF then
    F-URF for each pair), the step keeps exactly the first one whose error is
    strictly below the current one, and counts the candidates it tried."""
    checked = 0
    for seed in range(8):
        R, M = synth.dyadic_noise(5, 6, 0.8, seed=300 + seed, levels=32)
        U, V = _consistent_state(orc, R.astype(float), M, 2, seed)
        f = orc.error(R, M, U, V)
        for i in range(5):
            js, ks = orc.row_order(R, M, U, V, i, selection=selection)
            expected, tried = None, 0
            for pos, (j, k) in enumerate(zip(js, ks)):
                for typ, fn in ((0, orc.fulf), (1, orc.furf)):
                    tried += 1
                    _, _, fn_ = fn(R, M, U, V, i, j, k)
                    if fn_ < f:
                        expected = (pos, int(j), int(k), typ, fn_, tried)
                        break
                if expected:
                    break
            U2, V2 = U.copy(), V.copy()
            kept, f2, out, ntried = orc.row_step(R, M, U2, V2, i, f, selection=selection)
            if expected is None:
                assert not kept and f2 == f and ntried == tried
                assert np.array_equal(U2, U) and np.array_equal(V2, V)
            else:
                assert kept and out == expected[:4] and f2 == expected[4] and ntried == expected[5]
                checked += 1
    assert checked > 5


def test_selection_rank_one_cases(orc):
    """With r = 1 every k is 0: TD_A and TD_B order the same columns the same
    way and so take identical decisions; SEQ then tries the given columns in
    increasing j."""
    R, M = synth.dyadic_noise(9, 13, 0.7, seed=17, levels=32)
    a = orc.factorize(R, M, 1, sweeps=2, seed=4, selection="TD_A", trace_cap=100)
    b = orc.factorize(R, M, 1, sweeps=2, seed=4, selection="TD_B", trace_cap=100)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["U"], b["U"])
    st = orc.prepare(R, M, 1, seed=4)
    for i in range(st["R"].shape[0]):
        js, ks = orc.row_order(st["R"], st["M"], st["U"], st["V"], i, selection="SEQ")
        assert js.tolist() == np.flatnonzero(st["M"][i]).tolist() and not ks.any()


@pytest.mark.parametrize("selection", SELECTIONS)
def test_selection_whole_method_invariants(orc, selection):
    """Monotone error, U (x) V <= R on given entries, determinism, and
    equivariance under R + c with dyadic c (same decisions, U + c)."""
    R, M = synth.dyadic_noise(8, 12, 1.0, seed=21, levels=64)
    a = orc.factorize(R, M, 3, sweeps=3, p=4, seed=6, selection=selection, trace_cap=100)
    b = orc.factorize(R + 2.5, M, 3, sweeps=3, p=4, seed=6, selection=selection, trace_cap=100)
    c = orc.factorize(R, M, 3, sweeps=3, p=4, seed=6, selection=selection, trace_cap=100)
    assert np.all(np.diff(a["f_hist"]) <= 0) and a["f_hist"][-1] < a["f_hist"][0]
    P = np.max(a["U"][:, :, None] + a["V"][None, :, :], axis=1)
    assert np.all(P[M] <= R[M])
    assert np.array_equal(a["trace"], c["trace"]) and np.array_equal(a["U"], c["U"])
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["f_hist"], b["f_hist"])
    assert np.array_equal(b["U"], a["U"] + 2.5) and np.array_equal(b["V"], a["V"])
    assert a["kept"] > 0


def test_selection_unknown_name_rejected(orc):
    R, M = synth.dyadic_noise(4, 5, 1.0, seed=1)
    with pytest.raises(ValueError):
        orc.factorize(R, M, 2, sweeps=1, selection="BEST")
