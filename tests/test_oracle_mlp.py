"""Pins of the FP64 MLP / sketch reference and of the gauge fixing of targets."""
import numpy as np

from oracle import mlp as om
from paper_2205_06619_gb300 import learned_init


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    r = 5
    p = learned_init.init_params(r, seed=1).astype(np.float64)
    p[-(2 * om.HID + r):] = rng.normal(0, 0.1, size=2 * om.HID + r)      # non-zero biases
    X = rng.normal(size=(7, om.SK)); T = rng.normal(size=(7, r))
    loss, g = om.loss_and_grad(p, X, T, r)
    idx = rng.choice(p.size, size=60, replace=False)
    for q in idx:
        h = 1e-6
        pp = p.copy(); pp[q] += h
        pm = p.copy(); pm[q] -= h
        fd = (om.loss_and_grad(pp, X, T, r)[0] - om.loss_and_grad(pm, X, T, r)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 + 1e-5 * abs(fd), (q, fd, g[q])


def test_mlp_zero_weights_give_bias():
    r = 3
    p = np.zeros(om.SK * om.HID + om.HID * om.HID + om.HID * r + 2 * om.HID + r)
    p[-r:] = [1.0, -2.0, 0.5]
    Y, _ = om.forward(p, np.ones((4, om.SK)), r)
    assert np.array_equal(Y, np.tile([1.0, -2.0, 0.5], (4, 1)))


def test_sketch_definition_and_shift():
    rng = np.random.default_rng(1)
    R = rng.normal(size=(5, 77)); M = rng.random((5, 77)) < 0.6
    sk, med = om.row_sketch(R, M)
    for s in range(5):
        v = np.sort(R[s][M[s]]); c = v.size
        assert med[s] == v[c // 2]
        for q in range(32):
            assert sk[s, q] == v[min(int((q + 0.5) * c / 32), c - 1)] - v[c // 2]
    sk2, med2 = om.row_sketch(R + 3.25, M)
    assert np.allclose(sk2, sk) and np.allclose(med2, med + 3.25)


def _dyadic(rng, shape, lo=-64, hi=64):
    """Multiples of 1/8 of modest size: every FP32 sum below is exact."""
    return (rng.integers(lo, hi, size=shape) / 8.0).astype(np.float32)


def test_targets_are_gauge_invariant():
    """Shifting each component (U_.l + c, V_l. - c) and renumbering the
    components leave the targets unchanged (exact on dyadic data)."""
    rng = np.random.default_rng(2)
    U = _dyadic(rng, (9, 4)); V = _dyadic(rng, (4, 11))
    U[:, 0] += 20.0; U[:, 2] -= 20.0            # well-separated component sums
    med = _dyadic(rng, 9)
    c = _dyadic(rng, 4, -16, 16)
    perm = np.array([2, 0, 3, 1])
    for srt in (False, True):
        a = om.targets(U, V, med, srt)
        b = om.targets((U + c)[:, perm], (V - c[:, None])[perm], med, srt)
        assert np.array_equal(a, b)


def test_targets_keep_the_product_and_order_components():
    """The canonical rows (plus the median) and V shifted to max 0 in the same
    component order give the same max-plus product; components come in
    decreasing order of their row sums; sorted rows are the canonical rows
    sorted."""
    rng = np.random.default_rng(5)
    U = _dyadic(rng, (7, 3)); V = _dyadic(rng, (3, 10))
    U[:, 1] += 30.0; U[:, 2] += 10.0          # sums: component 1 > 2 > 0
    med = _dyadic(rng, 7)
    T = om.targets(U, V, med)
    Vs = V - V.max(axis=1, keepdims=True)
    order = [1, 2, 0]
    P = np.max(U[:, :, None] + V[None, :, :], axis=1)
    Pc = np.max((T + med[:, None])[:, :, None] + Vs[order][None, :, :], axis=1)
    assert np.array_equal(P, Pc)
    assert np.array_equal(T[:, 0] + med, U[:, 1] + V[1].max())
    Ts = om.targets(U, V, med, sorted_rows=True)
    assert np.array_equal(Ts, -np.sort(-T, axis=1))


def test_assign_by_rank_hand_case_and_brute_force():
    Y = np.array([[3.0, 1.0, 2.0], [5.0, 5.0, -1.0]], np.float32)
    Ur = np.array([[0.0, 9.0, 4.0], [2.0, 2.0, 7.0]], np.float32)
    # row 0: U_ref order 1, 2, 0 gets 3, 2, 1; row 1: order 2, 0, 1 (tie: 0 first) gets 5, 5, -1
    assert np.array_equal(om.assign_by_rank(Y, Ur), [[1.0, 3.0, 2.0], [5.0, -1.0, 5.0]])
    rng = np.random.default_rng(4)
    Y = rng.normal(size=(6, 5)).astype(np.float32)
    Ur = rng.integers(0, 3, size=(6, 5)).astype(np.float32)       # many ties
    out = om.assign_by_rank(Y, Ur)
    for s in range(6):
        assert sorted(out[s].tolist()) == sorted(Y[s].tolist())
        for l in range(5):
            for q in range(5):
                if Ur[s, l] > Ur[s, q] or (Ur[s, l] == Ur[s, q] and l < q):
                    assert out[s, l] > out[s, q]


def test_bf16_rounding_and_operand_mode():
    """bf16(): round to nearest even on the FP32 value (hand-checked cases);
    with bf16_operands the reference's products see exactly the rounded
    operands: the first layer equals the product of the rounded input."""
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -9, -3.0 - 2.0 ** -7 - 2.0 ** -9, 0.0])
    assert np.array_equal(om.bf16(x), [1.0, 1.0, 1.0 + 2.0 ** -7, 1.0, -3.0 - 2.0 ** -6, 0.0])
    r = 2
    rng = np.random.default_rng(3)
    p = np.zeros(om.SK * om.HID + om.HID * om.HID + om.HID * r + 2 * om.HID + r)
    p[:om.SK * om.HID] = om.bf16(rng.normal(size=om.SK * om.HID))
    X = rng.normal(size=(3, om.SK))
    _, (_, h1, _) = om.forward(p, X, r, bf16_operands=True)
    W1 = p[:om.SK * om.HID].reshape(om.SK, om.HID)
    assert np.array_equal(h1, np.maximum(om.bf16(X) @ W1, 0.0))
    _, (_, h1x, _) = om.forward(p, X, r)
    assert not np.array_equal(h1, h1x)
