"""Pins of the oracle's ByElement method (STMF_ByElement_PermC_TD_W; Section
"The ByElement strategy" and its pseudocode in the Supplement): the PermC
column order on a hand-computed example, the element scan against brute
force over every element and both updates, the err = 0 skip rule, and
invariants of the whole method (monotone error, U (x) V <= R, the output
frame, transpose equivalence, shift equivariance).
"""
import numpy as np

from paper_2205_06619_gb300 import synth
from test_oracle_pins import _consistent_state


def test_colmin_perm_hand_example(orc):
    # column minima over GIVEN entries: col0 3 (the -10 is not given), col1 1,
    # col2 1, col3 -2, col4 5  ->  increasing, ties to the smaller column:
    # 3, 1, 2, 0, 4
    R = np.array([[3.0, 1.0, 4.0, -2.0, 5.0],
                  [-10.0, 2.0, 1.0, 0.0, 6.0]])
    M = np.array([[1, 1, 1, 1, 1],
                  [0, 1, 1, 1, 1]], dtype=bool)
    assert orc.colmin_perm(R, M).tolist() == [3, 1, 2, 0, 4]


def test_element_scan_brute_force(orc):
    """From several start positions, the scan stops at the first element (in
    row-major order, given, td > 0) whose F-ULF or F-URF lowers the error,
    tries F-ULF first, and counts exactly the candidates tried."""
    checked = 0
    for seed in range(10):
        R, M = synth.dyadic_noise(5, 6, 0.8, seed=400 + seed, levels=32)
        R = R.astype(float)
        U, V = _consistent_state(orc, R, M, 2, seed)
        f = orc.error(R, M, U, V)
        m, n = R.shape
        for q0 in (0, 7, 19):
            P1, A, _ = orc.maxplus(U, V, "fp32")
            expected, tried = None, 0
            for q in range(q0, m * n):
                i, j = divmod(q, n)
                if not M[i, j] or abs(np.float32(R[i, j] - P1[i, j])) == 0.0:
                    continue
                k = int(A[i, j])
                for typ, fn in ((0, orc.fulf), (1, orc.furf)):
                    tried += 1
                    _, _, fn_ = fn(R, M, U, V, i, j, k)
                    if fn_ < f:
                        expected = (q, (i, j, k, typ), fn_)
                        break
                if expected:
                    break
            U2, V2 = U.copy(), V.copy()
            q, f2, out, ntried = orc.element_scan(R, M, U2, V2, q0, f)
            assert ntried == tried
            if expected is None:
                assert q == -1 and f2 == f and np.array_equal(U2, U) and np.array_equal(V2, V)
            else:
                assert q == expected[0] and out == expected[1] and f2 == expected[2]
                checked += 1
    assert checked > 10


def test_element_scan_skips_exact_entries(orc):
    """err = td(i,j) = 0 is skipped: from an exact factorization nothing is
    tried; with one entry perturbed only elements with td > 0 are tried."""
    R, M, Us, Vs = synth.dyadic_planted(6, 9, 2, 0.8, seed=31)
    U, V = Us.astype(float).copy(), Vs.astype(float).copy()
    q, f2, _, tried = orc.element_scan(R, M, U, V, 0, 0.0)
    assert q == -1 and tried == 0
    R2 = R.astype(float).copy()
    i, j = np.argwhere(M)[3]
    R2[i, j] += 0.5                      # one entry above the exact fit: td > 0 there only
    V2 = np.stack([orc.residuate_v(R2, M, U[:, l])[0] for l in range(2)])
    P1, _, _ = orc.maxplus(U, V2, "fp32")
    td = np.where(M, np.abs(R2 - P1), 0.0)
    f = orc.error(R2, M, U, V2)
    q, f3, _, tried = orc.element_scan(R2, M, U.copy(), V2.copy(), 0, f)
    positive = int(np.count_nonzero(td))
    assert tried <= 2 * positive
    if q < 0:
        assert tried == 2 * positive


def test_byelement_whole_method_invariants(orc):
    R, M = synth.dyadic_noise(9, 14, 0.8, seed=41, levels=64)
    a = orc.factorize(R, M, 3, sweeps=3, seed=5, strategy="ByElement", trace_cap=2000)
    b = orc.factorize(R, M, 3, sweeps=3, seed=5, strategy="ByElement", trace_cap=2000)
    assert np.all(np.diff(a["f_hist"]) <= 0) and a["f_hist"][-1] < a["f_hist"][0]
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["trace"], b["trace"])
    # the output is in the caller's frame: its error is the reported one
    P = np.max(a["U"][:, :, None] + a["V"][None, :, :], axis=1)
    fin = np.abs(R.astype(float) - P.astype(np.float32))[M].sum()
    assert abs(fin - a["f_hist"][-1]) <= 1e-9 * fin
    assert np.all(P[M] <= R[M])
    # trace: kept updates at increasing positions within a sweep, one end record per sweep
    tr = a["trace"]
    ends = tr[tr[:, 1] < 0]
    assert ends[:, 0].tolist() == list(range(a["sweeps"]))
    for sw in range(a["sweeps"]):
        q = tr[(tr[:, 0] == sw) & (tr[:, 1] >= 0), 2]
        assert np.all(np.diff(q) > 0)
    assert a["kept"] == int(np.sum(tr[:, 1] >= 0))


def test_byelement_transpose_equivalence(orc):
    """A tall input runs as its wide transpose: factorize(R^T) returns the
    transposed factors of factorize(R)."""
    R, M = synth.dyadic_noise(8, 13, 0.75, seed=43, levels=64)
    a = orc.factorize(R, M, 2, sweeps=2, seed=3, strategy="ByElement", trace_cap=500)
    b = orc.factorize(R.T.copy(), M.T.copy(), 2, sweeps=2, seed=3, strategy="ByElement", trace_cap=500)
    assert np.array_equal(b["U"], a["V"].T) and np.array_equal(b["V"], a["U"].T)
    assert np.array_equal(a["trace"], b["trace"])


def test_byelement_shift_equivariance(orc):
    """R + c (dyadic c) keeps the column order, the decisions and V, and
    shifts U by c (full mask, 4 picks: exact Acol means)."""
    R, M = synth.dyadic_noise(7, 11, 1.0, seed=45, levels=64)
    a = orc.factorize(R, M, 3, sweeps=2, p=4, seed=5, strategy="ByElement", trace_cap=500)
    b = orc.factorize(R + 3.5, M, 3, sweeps=2, p=4, seed=5, strategy="ByElement", trace_cap=500)
    assert np.array_equal(orc.colmin_perm(R, M), orc.colmin_perm(R + 3.5, M))
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["f_hist"], b["f_hist"])
    assert np.array_equal(b["U"], a["U"] + 3.5) and np.array_equal(b["V"], a["V"])
