"""Pins of the oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: they use hand-computed
examples (tests/golden), algebraic identities of the (max,+) semiring, the
optimality of residuation, exact recovery of noiseless tropical low-rank
data, brute force over all candidates on tiny inputs, and equivariances.
Each block names the definition or algorithm it pins.
"""
import itertools
import os

import numpy as np

from paper_2205_06619_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NEG = -np.inf


def load_golden(name):
    blocks, key = {}, None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            key = line
            blocks[key] = []
        else:
            blocks[key].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


# --------------------------------------------------------------------------
# Tropical product (Section "Related work"; f(i,j) of Section "The ByRow
# strategy")

def test_maxplus_golden(orc):
    g = load_golden("maxplus_3x2x3.txt")
    for mode in ("fp64", "fp32"):
        P1, A, P2 = orc.maxplus(g["U"], g["V"], mode)
        assert np.array_equal(P1, g["P1"])
        assert np.array_equal(A, g["A"].astype(np.int32))
        assert np.array_equal(P2, g["P2"])


def test_maxplus_identity_and_neutral(orc):
    rng = np.random.default_rng(1)
    X = rng.integers(-20, 20, size=(5, 4)).astype(float)
    I = np.full((4, 4), NEG)
    np.fill_diagonal(I, 0.0)
    P1, A, _ = orc.maxplus(X, I, "fp64")
    assert np.array_equal(P1, X)
    assert np.array_equal(A, np.tile(np.arange(4), (5, 1)))
    # -inf is the neutral element of (+) = max: an extra all -inf component
    # changes neither the product nor the argmax.
    Y = rng.integers(-20, 20, size=(4, 6)).astype(float)
    Xe = np.concatenate([X, np.full((5, 1), NEG)], axis=1)
    Ye = np.concatenate([Y, rng.integers(-5, 5, size=(1, 6)).astype(float)], axis=0)
    assert np.array_equal(orc.maxplus(Xe, Ye, "fp64")[0], orc.maxplus(X, Y, "fp64")[0])
    assert np.array_equal(orc.maxplus(Xe, Ye, "fp64")[1], orc.maxplus(X, Y, "fp64")[1])


def test_maxplus_associative_distributive_transpose(orc):
    rng = np.random.default_rng(2)
    A = rng.integers(-50, 50, size=(6, 5)) / 4.0
    B = rng.integers(-50, 50, size=(5, 7)) / 4.0
    C = rng.integers(-50, 50, size=(7, 3)) / 4.0
    B2 = rng.integers(-50, 50, size=(5, 7)) / 4.0
    for mode in ("fp64", "fp32"):
        AB = orc.maxplus(A, B, mode)[0]
        BC = orc.maxplus(B, C, mode)[0]
        assert np.array_equal(orc.maxplus(AB, C, mode)[0], orc.maxplus(A, BC, mode)[0])
        lhs = orc.maxplus(A, np.maximum(B, B2), mode)[0]
        rhs = np.maximum(AB, orc.maxplus(A, B2, mode)[0])
        assert np.array_equal(lhs, rhs)
        # (U (x) V)^T = V^T (x) U^T (used by the wide transpose of Algorithm 3)
        assert np.array_equal(AB.T, orc.maxplus(B.T, A.T, mode)[0])


def test_maxplus_argmax_runner_up_brute(orc):
    rng = np.random.default_rng(3)
    for r in (1, 2, 3, 7):
        U = rng.integers(0, 4, size=(6, r)).astype(float)   # many ties
        V = rng.integers(0, 4, size=(r, 5)).astype(float)
        P1, A, P2 = orc.maxplus(U, V, "fp32")
        for i, j in itertools.product(range(6), range(5)):
            s = [U[i, l] + V[l, j] for l in range(r)]
            best = max(s)
            assert P1[i, j] == best
            assert A[i, j] == s.index(best)                  # smaller l on ties
            rest = [x for l, x in enumerate(s) if l != A[i, j]]
            assert P2[i, j] == (max(rest) if rest else NEG)


def test_fp32_mode_rounds_each_add(orc):
    # 1 + 2^-30 is not a float: fp32 mode must round it away, fp64 must not.
    U = np.array([[1.0]])
    V = np.array([[2.0 ** -30]])
    assert orc.maxplus(U, V, "fp32")[0][0, 0] == 1.0
    assert orc.maxplus(U, V, "fp64")[0][0, 0] == 1.0 + 2.0 ** -30
    # and a float-exact sum must not change
    x = np.float32(0.1)
    y = np.float32(0.2)
    got = orc.maxplus(np.array([[float(x)]]), np.array([[float(y)]]), "fp32")[0][0, 0]
    assert got == float(np.float32(x + y))


# --------------------------------------------------------------------------
# Residuation (Section "Related work", (min,+) over given entries)

def test_residuation_golden(orc):
    g = load_golden("residuation_2x3.txt")
    M = g["M"].astype(bool)
    v, e = orc.residuate_v(g["R"], M, g["u"][0])
    assert e == 0 and np.array_equal(v, g["v"][0])
    u2, e = orc.residuate_u(g["R"], M, v)
    assert e == 0 and np.array_equal(u2, g["u2"][0])
    Mb = g["M_b"].astype(bool)
    v, _ = orc.residuate_v(g["R"], Mb, g["u_b"][0])
    assert np.array_equal(v, g["v_b"][0])
    u2, _ = orc.residuate_u(g["R"], Mb, v)
    assert np.array_equal(u2, g["u2_b"][0])


def test_residuation_principal_solution(orc):
    """v = (-u)^T (x)* R is the greatest v with u_s + v_t <= R_st on given
    entries: it satisfies the inequality, attains equality in every column,
    and raising any entry breaks it."""
    rng = np.random.default_rng(4)
    R, M = synth.dyadic_noise(9, 13, 0.6, seed=4)
    R = R.astype(float)
    u = rng.integers(0, 40, size=9) / 8.0
    v, e = orc.residuate_v(R, M, u)
    assert e == 0
    lhs = u[:, None] + v[None, :]
    assert np.all(lhs[M] <= R[M])
    for t in range(13):
        col = M[:, t]
        assert np.any(lhs[col, t] == R[col, t])
        vv = v.copy(); vv[t] += 0.125
        assert np.any((u[:, None] + vv[None, :])[M] > R[M])
    # row version
    w = rng.integers(0, 40, size=13) / 8.0
    uu, _ = orc.residuate_u(R, M, w)
    lhs = uu[:, None] + w[None, :]
    assert np.all(lhs[M] <= R[M])
    for s in range(9):
        assert np.any(lhs[s, M[s]] == R[s, M[s]])


def test_residuation_closure(orc):
    """Galois closure: after u' = R (x)* (-v)^T with v = (-u)^T (x)* R,
    residuating again gives v back exactly."""
    R, M = synth.dyadic_noise(8, 11, 0.7, seed=5)
    R = R.astype(float)
    u = np.random.default_rng(5).integers(0, 40, size=8) / 8.0
    v, _ = orc.residuate_v(R, M, u)
    u2, _ = orc.residuate_u(R, M, v)
    v2, _ = orc.residuate_v(R, M, u2)
    assert np.array_equal(v, v2)
    assert np.all(u2 >= u)


def test_exact_recovery(orc):
    """If R = U* (x) V* (any mask), then V = (-U*)^T (x)* R gives zero error."""
    for seed in range(3):
        R, M, Us, Vs = synth.dyadic_planted(12, 17, 3, 0.7, seed)
        Us = Us.astype(float)
        V = np.stack([orc.residuate_v(R, M, Us[:, l])[0] for l in range(3)])
        for mode in ("fp64", "fp32"):
            assert orc.error(R, M, Us, V, mode) == 0.0
        assert orc.error(R, M, Us, Vs, "fp32") == 0.0


# --------------------------------------------------------------------------
# b-norm error (Section "Evaluation metrics")

def test_bnorm_golden(orc):
    g = load_golden("bnorm_2x3.txt")
    assert orc.error(g["R"], g["M_all"].astype(bool), g["U"], g["V"]) == g["f_all"][0][0]
    assert orc.error(g["R"], g["M_part"].astype(bool), g["U"], g["V"]) == g["f_part"][0][0]


def test_bnorm_matches_definition_on_random(orc):
    R, M = synth.dyadic_noise(7, 9, 0.5, seed=6)
    rng = np.random.default_rng(6)
    U = rng.integers(0, 16, size=(7, 2)) / 8.0
    V = rng.integers(0, 16, size=(2, 9)) / 8.0
    P = np.max(U[:, :, None] + V[None, :, :], axis=1)
    assert orc.error(R, M, U, V, "fp64") == np.abs(R.astype(float) - P)[M].sum()


# --------------------------------------------------------------------------
# F-ULF / F-URF (Algorithms 1 and 2)

def test_fulf_furf_golden(orc):
    g = load_golden("fulf_furf_2x2.txt")
    M = np.ones((2, 2), bool)
    U0, V0 = g["U0"], g["V0"]
    assert orc.error(g["R"], M, U0, V0) == g["f0"][0][0]
    U, V, f = orc.fulf(g["R"], M, U0, V0, 0, 1, 0)
    assert np.array_equal(U, g["ulf_01_U"]) and np.array_equal(V, g["ulf_01_V"]) and f == g["ulf_01_f"][0][0]
    U, V, f = orc.furf(g["R"], M, U0, V0, 1, 0, 0)
    assert np.array_equal(U, g["urf_10_U"]) and np.array_equal(V, g["urf_10_V"]) and f == g["urf_10_f"][0][0]
    U, V, f = orc.fulf(g["R"], M, U0, V0, 1, 0, 0)
    assert np.array_equal(U, g["ulf_10_U"]) and np.array_equal(V, g["ulf_10_V"]) and f == g["ulf_10_f"][0][0]


def _consistent_state(orc, R, M, r, seed):
    rng = np.random.default_rng(seed)
    U = rng.integers(0, 40, size=(R.shape[0], r)) / 8.0
    V = np.stack([orc.residuate_v(R, M, U[:, l])[0] for l in range(r)])
    U = np.stack([orc.residuate_u(R, M, V[l])[0] for l in range(r)], axis=1)
    return U, V


def test_fulf_equals_full_ulf(orc):
    """The paper states F-ULF gives the same U, V as the whole-matrix ULF
    (Section "Our contribution").  Whole-matrix ULF from a consistent state:
    U_ik <- R_ij - V_kj, then V <- (-U)^T (x)* R and U <- R (x)* (-V)^T on
    all components.  Written here with numpy min-reductions."""
    R, M = synth.dyadic_noise(7, 10, 0.7, seed=7)
    Rf = R.astype(float)
    big = np.where(M, Rf, np.inf)
    U, V = _consistent_state(orc, Rf, M, 3, 7)
    for (i, j, k) in [(0, 1, 0), (3, 4, 2), (6, 9, 1)]:
        if not M[i, j]:
            continue
        Uf = U.copy()
        Uf[i, k] = Rf[i, j] - V[k, j]
        Vf = np.min(big[None, :, :] - Uf.T[:, :, None], axis=1)          # (-U)^T (x)* R
        Uf = np.min(big[:, None, :] - Vf[None, :, :], axis=2)            # R (x)* (-V)^T
        U2, V2, _ = orc.fulf(Rf, M, U, V, i, j, k, "fp64")
        assert np.array_equal(U2, Uf) and np.array_equal(V2, Vf)
        # and whole-matrix URF
        Vg = V.copy()
        Vg[k, j] = Rf[i, j] - U[i, k]
        Ug = np.min(big[:, None, :] - Vg[None, :, :], axis=2)
        Vg = np.min(big[None, :, :] - Ug.T[:, :, None], axis=1)
        U3, V3, _ = orc.furf(Rf, M, U, V, i, j, k, "fp64")
        assert np.array_equal(U3, Ug) and np.array_equal(V3, Vg)
        # closure (exact on dyadic data): the updated U_.k reproduces V_k.
        assert np.array_equal(orc.residuate_v(Rf, M, U2[:, k], "fp64")[0], V2[k])
        assert np.array_equal(orc.residuate_u(Rf, M, V3[k], "fp64")[0], U3[:, k])


def test_updates_touch_only_component_k_and_keep_invariant(orc):
    R, M, _, _ = synth.uniform_planted(10, 14, 3, 0.01, 0.8, seed=8)
    U, V = _consistent_state(orc, R.astype(float), M, 3, 8)
    U = U.astype(np.float32).astype(float); V = V.astype(np.float32).astype(float)
    for fn in (orc.fulf, orc.furf):
        for (i, j, k) in [(2, 3, 1), (9, 13, 0)]:
            if not M[i, j]:
                continue
            U2, V2, f = fn(R, M, U, V, i, j, k)
            others = [l for l in range(3) if l != k]
            assert np.array_equal(U2[:, others], U[:, others])
            assert np.array_equal(V2[others], V[others])
            P = orc.maxplus(U2, V2)[0]
            # U (x) V <= R on given entries, up to the fp32 roundings of
            # R - V and U + V, whose size scales with the intermediates
            mag = np.abs(R.astype(float)) + np.abs(U2).max() + np.abs(V2).max()
            slack = mag * 2.0 ** -23
            assert np.all(P[M] <= R.astype(float)[M] + slack[M])
            assert f == orc.error(R, M, U2, V2)


# --------------------------------------------------------------------------
# Selection statistics, order and the ByRow step (Algorithm 3; TD, TD_A)

def test_row_stats_and_order_brute(orc):
    R, M = synth.dyadic_noise(6, 9, 0.7, seed=9)
    U, V = _consistent_state(orc, R.astype(float), M, 3, 9)
    Rf = R.astype(float)
    P1, A, _ = orc.maxplus(U, V, "fp32")
    for i in range(6):
        td, ch, rh = orc.row_stats(R, M, U, V, i)
        td_b = np.where(M, np.abs(Rf - P1), 0.0).sum(axis=0)
        assert np.array_equal(td, td_b)
        for t in range(9):
            for l in range(3):
                assert ch[t, l] == np.sum(M[:, t] & (A[:, t] == l))
        for l in range(3):
            assert rh[l] == np.sum(M[i] & (A[i] == l))
        js, ks = orc.row_order(R, M, U, V, i)
        cand = np.flatnonzero(M[i])
        order = cand[np.argsort(-td[cand], kind="stable")]     # decreasing td_col, then smaller j
        assert np.array_equal(js, order)
        for j, k in zip(js, ks):
            counts = rh + ch[j]
            assert k == int(np.argmax(counts))                 # argmax takes the first (smaller l)


def test_row_step_brute_force_first_improving(orc):
    """Over all candidates of a row (every given j, both F-ULF and F-URF with
    the TD_A component k_j), the step keeps exactly the first one, in the
    order of Algorithm 3, whose error is strictly below the current one."""
    checked = 0
    for seed in range(12):
        R, M = synth.dyadic_noise(5, 6, 0.8, seed=100 + seed, levels=32)
        U, V = _consistent_state(orc, R.astype(float), M, 2, seed)
        f = orc.error(R, M, U, V)
        for i in range(5):
            js, ks = orc.row_order(R, M, U, V, i)
            expected = None
            tried = 0
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
            kept, f2, out, ntried = orc.row_step(R, M, U2, V2, i, f)
            if expected is None:
                assert not kept and f2 == f and ntried == tried
                assert np.array_equal(U2, U) and np.array_equal(V2, V)
            else:
                assert kept and out == expected[:4] and f2 == expected[4] and ntried == expected[5]
                checked += 1
    assert checked > 5


# --------------------------------------------------------------------------
# Initialisation and random draws

def test_splitmix64_published_vector(orc):
    # SplitMix64 seeded with 0: the published first outputs.
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64(0, 2) == 0x06C45D188009454F


def test_randperm_and_picks_valid(orc):
    for m in (1, 2, 17, 200):
        p = orc.randperm(m, 12345)
        assert sorted(p.tolist()) == list(range(m))
    pk = orc.acol_picks(50, 7, 5, 99)
    for row in pk:
        assert len(set(row.tolist())) == 5 and row.min() >= 0 and row.max() < 50
    # first position of a random permutation is roughly uniform
    counts = np.bincount([orc.randperm(8, s)[0] for s in range(4000)], minlength=8)
    assert counts.min() > 380 and counts.max() < 620


def test_acol_init_golden(orc):
    # R (2 x 4), picks for 2 components; row 1 misses both picks of component 1
    R = np.array([[1.0, 2.0, 4.0, 8.0], [3.0, 5.0, 7.0, 9.0]])
    M = np.array([[1, 1, 1, 0], [1, 0, 1, 1]], bool)
    picks = np.array([[0, 2], [1, 3]], np.int32)
    U = orc.acol_init(R, M, picks)
    # comp 0: row0 (1+4)/2 = 2.5, row1 (3+7)/2 = 5; comp 1: row0 only col1 -> 2,
    # row1 only col3 -> 9
    assert np.array_equal(U, np.array([[2.5, 2.0], [5.0, 9.0]]))
    picks = np.array([[1, 1]], np.int32)
    U = orc.acol_init(R, M, picks)
    # row1 has col1 missing twice: falls back to its row mean (3+7+9)/3
    assert U[0, 0] == 2.0 and U[1, 0] == np.float32(19.0 / 3.0)


# --------------------------------------------------------------------------
# The whole method (Algorithm 3)

def test_factorize_monotone_and_deterministic(orc):
    w = synth.workload_small(seed=3)
    R, M = w["R"][:40, :30], w["mask"][:40, :30]
    a = orc.factorize(R, M, 3, sweeps=4, seed=7)
    b = orc.factorize(R, M, 3, sweeps=4, seed=7)
    assert np.all(np.diff(a["f_hist"]) <= 0)
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["V"], b["V"])
    assert a["f_hist"][-1] < a["f_hist"][0]
    P = np.max(a["U"][:, :, None] + a["V"][None, :, :], axis=1)
    fin = np.abs(R.astype(float) - P.astype(np.float32))[M].sum()
    assert abs(fin - a["f_hist"][-1]) <= 1e-9 * fin


def test_factorize_transpose_equivalence(orc):
    """A tall input is transposed into the same wide problem (Algorithm 3):
    factorize(R^T) returns (V^T, U^T) of factorize(R)."""
    R, M = synth.dyadic_noise(8, 12, 0.75, seed=11, levels=64)
    perm = orc.randperm(8, 3)
    a = orc.factorize(R, M, 2, sweeps=2, perm=perm, seed=3)
    b = orc.factorize(R.T.copy(), M.T.copy(), 2, sweeps=2, perm=perm, seed=3)
    assert np.array_equal(b["U"], a["V"].T) and np.array_equal(b["V"], a["U"].T)
    assert np.array_equal(a["f_hist"], b["f_hist"])


def test_factorize_shift_equivariance(orc):
    """R + c (dyadic c) gives the same decisions, the same errors and U + c.
    Exactness needs exact Acol means, hence a full mask with 4 picks; the
    masked variant starts both runs from a given U0 (shifted by c)."""
    R, M = synth.dyadic_noise(7, 11, 1.0, seed=12, levels=64)
    a = orc.factorize(R, M, 3, sweeps=2, p=4, seed=5, trace_cap=100)
    b = orc.factorize(R + 3.5, M, 3, sweeps=2, p=4, seed=5, trace_cap=100)
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["f_hist"], b["f_hist"])
    assert np.array_equal(b["U"], a["U"] + 3.5) and np.array_equal(b["V"], a["V"])
    R, M = synth.dyadic_noise(7, 11, 0.7, seed=13, levels=64)
    U0 = np.random.default_rng(13).integers(0, 64, size=(7, 3)) / 8.0
    perm = np.arange(7, dtype=np.int32)
    a = orc.factorize(R, M, 3, sweeps=2, perm=perm, U0=U0, trace_cap=100)
    b = orc.factorize(R + 3.5, M, 3, sweeps=2, perm=perm, U0=U0 + 3.5, trace_cap=100)
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["f_hist"], b["f_hist"])
    assert np.array_equal(b["U"], a["U"] + 3.5) and np.array_equal(b["V"], a["V"])


def test_factorize_exact_start_stays_exact(orc):
    R, M, Us, Vs = synth.dyadic_planted(9, 14, 3, 0.8, seed=13)
    out = orc.factorize(R, M, 3, sweeps=2, perm=np.arange(9, dtype=np.int32), U0=Us.astype(float))
    assert np.all(out["f_hist"] == 0.0) and out["kept"] == 0


def test_factorize_modes_agree_on_dyadic_data(orc):
    # full mask: with a missing pick the row-mean fallback divides by a
    # count that is not a power of two, which is not exact
    R, M, _, _ = synth.dyadic_planted(8, 12, 2, 1.0, seed=14)
    R = R + np.random.default_rng(14).integers(0, 4, size=R.shape) / 8.0   # not exactly low-rank
    perm = np.arange(8, dtype=np.int32)
    picks = np.array([[0], [5]], np.int32)
    a = orc.factorize(R, M, 2, sweeps=2, perm=perm, picks=picks, p=1, mode="fp64", trace_cap=50)
    b = orc.factorize(R, M, 2, sweeps=2, perm=perm, picks=picks, p=1, mode="fp32", trace_cap=50)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["f_hist"], b["f_hist"])


def test_factorize_tropical_data_fits_well(orc):
    """On noiseless tropical data (lambda = 1) the TD methods come close to a
    perfect fit (Section "Comparing selections"); a statistical check."""
    R, M = synth.r_lambda(30, 40, 3, 1.0, 0.8, seed=15)
    out = orc.factorize(R, M, 3, sweeps=8, seed=1)
    assert out["f_hist"][-1] < 0.25 * out["f_hist"][0]


def test_fp32_mode_outputs_are_floats(orc):
    w = synth.workload_small(seed=4)
    R, M = w["R"][:30, :20], w["mask"][:30, :20]
    out = orc.factorize(R, M, 3, sweeps=1, seed=2)
    assert np.array_equal(out["U"], out["U"].astype(np.float32).astype(float))
    assert np.array_equal(out["V"], out["V"].astype(np.float32).astype(float))


def test_oracle_results_do_not_depend_on_host_threads(orc):
    """The parallel loops of the oracle sum in a fixed order: one thread and
    all host threads give the same decisions, factors and errors bit for bit."""
    w = synth.workload_small(seed=5)
    R, M = w["R"][:50, :40], w["mask"][:50, :40]
    try:
        orc.set_threads(1)
        a = orc.factorize(R, M, 3, sweeps=3, seed=9, trace_cap=200)
        orc.set_threads(0)
        b = orc.factorize(R, M, 3, sweeps=3, seed=9, trace_cap=200)
    finally:
        orc.set_threads(0)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["f_hist"], b["f_hist"])
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["V"], b["V"])


def eps_stop_case(f_hist, min_stop=2):
    """A threshold for the convergence rule (Section "Comparison of
    strategies": stop when a sweep changes the error by less than eps) that
    the run with these errors crosses first at sweep s*, with a factor of at
    least 2 between eps and every change it is compared with up to s*.
    Returns (s*, eps) or None."""
    d = np.abs(np.diff(np.asarray(f_hist, dtype=float)))   # d[s-1]: change of sweep s
    for s in range(min_stop, len(d) + 1):
        before = d[:s - 1].min()
        if d[s - 1] * 4.0 <= before:
            eps = np.sqrt(d[s - 1] * before) if d[s - 1] > 0 else before / 2.0
            return s, float(eps)
    return None


def test_factorize_eps_stop(orc):
    """Convergence rule (Section "Comparison of strategies"): the sweep loop
    ends after the first sweep whose change of the error is below eps; that
    sweep is kept, and nothing else about the run changes.  Checked against
    the changes of a run without the rule, and on an exact start, where the
    first sweep changes nothing and ends the run."""
    R, M, _, _ = synth.uniform_planted(30, 44, 3, 0.01, 0.8, seed=31)
    full = orc.factorize(R, M, 3, sweeps=10, seed=2, trace_cap=1000)
    case = eps_stop_case(full["f_hist"])
    assert case is not None
    s_star, eps = case
    stop = orc.factorize(R, M, 3, sweeps=10, eps=eps, seed=2, trace_cap=1000)
    assert stop["sweeps"] == s_star
    assert np.array_equal(stop["f_hist"], full["f_hist"][:s_star + 1])
    short = orc.factorize(R, M, 3, sweeps=s_star, seed=2)
    assert np.array_equal(stop["U"], short["U"]) and np.array_equal(stop["V"], short["V"])
    # a larger threshold that every change falls below stops after sweep 1
    one = orc.factorize(R, M, 3, sweeps=10, eps=10.0 * full["f_hist"][0], seed=2)
    assert one["sweeps"] == 1
    R2, M2, Us, _ = synth.dyadic_planted(9, 14, 3, 0.8, seed=13)
    ex = orc.factorize(R2, M2, 3, sweeps=5, eps=1e-12, perm=np.arange(9, dtype=np.int32), U0=Us.astype(float))
    assert ex["sweeps"] == 1 and np.all(ex["f_hist"] == 0.0)
