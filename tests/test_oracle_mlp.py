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


def test_canonical_targets_are_gauge_invariant():
    rng = np.random.default_rng(2)
    U = rng.normal(size=(9, 4)); V = rng.normal(size=(4, 11))
    c = rng.normal(size=4)
    perm = np.array([2, 0, 3, 1])
    a = learned_init.canonical_U(U, V)
    b = learned_init.canonical_U((U + c)[:, perm], (V - c[:, None])[perm])
    assert np.allclose(a, b)
    # the product is the same in the canonical gauge
    Vc = V - V.max(axis=1, keepdims=True)
    order = np.argsort(-(U + V.max(axis=1)).mean(axis=0), kind="stable")
    P = np.max(U[:, :, None] + V[None, :, :], axis=1)
    Pc = np.max(a[:, :, None] + Vc[order][None, :, :], axis=1)
    assert np.allclose(P, Pc)
