"""GPU parity of the learned-initialisation kernels with the FP64 reference:
row sketch, training targets and rank hand-over (bit-exact), MLP forward,
prediction and gradient (tensor-core products with BF16 operands and FP32
accumulation; the reference rounds the same operands to BF16 and computes in
FP64)."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_2205_06619_gb300 import learned_init, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bf16(x):
    """Round float32 values to bfloat16 (round to nearest even), as floats."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _bf16_params(p, r):
    q = np.asarray(p, dtype=np.float32).copy()
    nw = om.SK * om.HID + om.HID * om.HID + om.HID * r
    q[:nw] = _bf16(q[:nw])
    return q


# Gradient tolerance, relative to the sum of the absolute values of the terms
# of each entry.  Both sides multiply the same BF16 operands (exact in FP32);
# the library sums in FP32 (about 2^-24 per addition, up to 256 terms), and an
# operand computed in FP32 on the GPU and in FP64 in the reference can round to
# neighbouring BF16 values (2^-8 of one term).  2^-12 still fails when one
# batch row's term (1/256 of the magnitude or more) is dropped or has its
# sign flipped.
GRAD_TOL = 2.0 ** -12


def _grad_magnitudes(params, X, T, r):
    """Per gradient entry, the sum of the absolute values of the products it
    adds up (the backward pass of the reference with every factor replaced by
    its absolute value and the reference's ReLU masks), with the output's
    dependence on the forward pass's FP32 rounding folded into |dY|."""
    W1, W2, W3, b1, b2, b3 = om.split(params, r)
    Y, (X, h1, h2) = om.forward(params, X, r, bf16_operands=True)
    B = X.shape[0]
    Yabs = np.abs(h2) @ np.abs(W3) + np.abs(b3)
    dY = (np.abs(Y - np.asarray(T, dtype=np.float64)) + 2.0 ** -10 * Yabs) * (2.0 / (B * r))
    gW3 = np.abs(h2).T @ dY; gb3 = dY.sum(axis=0)
    dH2 = (dY @ np.abs(W3).T) * (h2 > 0)
    gW2 = np.abs(h1).T @ dH2; gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ np.abs(W2).T) * (h1 > 0)
    gW1 = np.abs(X).T @ dH1; gb1 = dH1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gW2.ravel(), gW3.ravel(), gb1, gb2, gb3])


def _clear_relu_edges(params, X, r, rng, rel=2.0 ** -14):
    """Redraws the batch rows whose hidden pre-activations lie within `rel` of
    zero relative to their magnitude: there the ReLU decision could go either
    way between FP32 and FP64, and an element-wise gradient comparison would
    compare two different (equally correct) derivatives."""
    W1, W2, W3, b1, b2, b3 = om.split(params, r)
    for _ in range(200):
        z1 = om.bf16(X) @ W1 + b1
        m1 = np.abs(X) @ np.abs(W1) + np.abs(b1)
        h1 = np.maximum(z1, 0.0)
        z2 = om.bf16(h1) @ W2 + b2
        m2 = h1 @ np.abs(W2) + np.abs(b2)
        bad = np.any(np.abs(z1) <= rel * m1, axis=1) | np.any(np.abs(z2) <= rel * m2, axis=1)
        if not bad.any():
            return X
        X = X.copy()
        X[bad] = rng.normal(size=(int(bad.sum()), X.shape[1])).astype(X.dtype)
    raise AssertionError("could not draw a batch away from the ReLU edges")


def test_row_sketch_bitexact():
    from paper_2205_06619_gb300 import api
    for (m, n, obs, seed) in [(40, 77, 0.6, 1), (17, 5000, 0.8, 2), (9, 33, 0.2, 3)]:
        R, M, _, _ = synth.lognormal_planted(m, n, 4, 0.05, obs, seed)
        sk, md = api.row_sketch(torch.from_numpy(R).cuda(), api.pack_mask(M))
        esk, emd = om.row_sketch(R, M)
        assert np.array_equal(md.cpu().numpy().astype(np.float64), emd)
        # sketch = v[idx] - median, subtracted in FP32 on the GPU
        vals = (esk + emd[:, None]).astype(np.float32)          # the quantile values themselves (exact)
        exp = vals - emd[:, None].astype(np.float32)            # FP32 subtraction
        assert np.array_equal(sk.cpu().numpy(), exp)


@pytest.mark.parametrize("r,B", [(10, 256), (3, 45), (20, 1)])
def test_mlp_forward_and_gradient_match_reference(r, B):
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(r + B)
    p = learned_init.init_params(r, seed=r)
    p[-(2 * om.HID + r):] = rng.normal(0, 0.1, size=2 * om.HID + r).astype(np.float32)
    net = api.MLP(r, p)
    X = rng.normal(size=(B, om.SK)).astype(np.float32)
    T = rng.normal(size=(B, r)).astype(np.float32)
    pb = _bf16_params(p, r)
    X = _clear_relu_edges(pb, X, r, rng)
    Xg, Tg = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y = net.forward(Xg).cpu().numpy()
    eY, _ = om.forward(pb, X, r, bf16_operands=True)
    assert np.allclose(Y, eY, rtol=1e-4, atol=1e-4)
    loss, g = net.gradient(Xg, Tg)
    eloss, eg = om.loss_and_grad(pb, X, T, r, bf16_operands=True)
    assert abs(loss - eloss) <= 1e-4 * abs(eloss)
    # element by element: every gradient entry is a sum of products; the
    # library forms them in FP32 (BF16 weights, the same as the reference's),
    # so each entry may differ by a small multiple of the FP32 unit times the
    # sum of the absolute values of its terms
    ag = _grad_magnitudes(pb, X, T, r)
    assert np.all(np.abs(g - eg) <= GRAD_TOL * ag), np.max(np.abs(g - eg) / np.maximum(ag, 1e-30))


@pytest.mark.parametrize("m,n,r", [(37, 301, 10), (5, 9, 1), (130, 64, 32)])
def test_targets_and_rank_assignment_match_the_oracle(m, n, r):
    """stmf_mlp_targets (canonical and sorted) and stmf_assign_by_rank against
    the oracle, bit for bit: the same FP32 operations, the same FP64
    row-order sums for the component order, and exact sorts."""
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(m + n + r)
    U = rng.normal(0, 3, size=(m, r)).astype(np.float32)
    V = rng.normal(0, 3, size=(r, n)).astype(np.float32)
    med = rng.normal(size=m).astype(np.float32)
    Ug, Vg, mg = (torch.from_numpy(x).cuda() for x in (U, V, med))
    for srt in (False, True):
        T = api.mlp_targets(Ug, Vg, mg, sorted_rows=srt).cpu().numpy()
        assert np.array_equal(T, om.targets(U, V, med, srt)), srt
    Y = rng.normal(size=(m, r)).astype(np.float32)
    Ur = rng.integers(0, 4, size=(m, r)).astype(np.float32)      # ties in every row
    out = api.assign_by_rank(torch.from_numpy(Y).cuda(), torch.from_numpy(Ur).cuda()).cpu().numpy()
    assert np.array_equal(out, om.assign_by_rank(Y, Ur))


def test_predict_matches_the_reference():
    """MLP.predict (stmf_mlp_predict: sketch, forward, plus the median, in one
    call) against the reference forward pass on the oracle's sketch."""
    from paper_2205_06619_gb300 import api
    r = 6
    rng = np.random.default_rng(8)
    p = learned_init.init_params(r, seed=2)
    p[-(2 * om.HID + r):] = rng.normal(0, 0.1, size=2 * om.HID + r).astype(np.float32)
    net = api.MLP(r, p)
    R, M, _, _ = synth.lognormal_planted(40, 500, 4, 0.05, 0.7, 4)
    U0 = net.predict(torch.from_numpy(R).cuda(), api.pack_mask(M)).cpu().numpy()
    sk, med = om.row_sketch(R, M)
    sk32 = (sk + med[:, None]).astype(np.float32) - med[:, None].astype(np.float32)   # FP32 as the library
    Y, _ = om.forward(_bf16_params(p, r), sk32, r, bf16_operands=True)
    assert np.allclose(U0, Y + med[:, None], rtol=1e-4, atol=1e-4)


def test_training_reduces_loss_and_init_is_valid():
    from paper_2205_06619_gb300 import api
    X, T = learned_init.training_set(count=12, m=60, n=300, rank=10, sweeps=3, seed=0)
    net, hist = learned_init.train(X, T, rank=10, epochs=20, batch=64, lr=2e-3)
    assert hist[-1] < 0.85 * hist[0]          # Adam on the library's gradients lowers the loss
    R, M = learned_init.gene_like(50, 240, seed=99)
    Rg, Mw = torch.from_numpy(R).cuda(), api.pack_mask(M)
    U0 = learned_init.predict_U(net, Rg, Mw)
    assert torch.isfinite(U0).all()
    perm = np.arange(50, dtype=np.int32)
    U, V, rep, _ = api.factorize(Rg, Mw, rank=10, sweeps=2, perm=perm, U0=U0)
    assert rep["f_final"] <= rep["f_init"]


def test_learned_start_against_untrained_and_acol():
    """What training buys, measured: on fresh matrices the initial b-norm
    error of the trained network's start, of the same network untrained
    (rows = row median plus noise) and of Random Acol.  Measured on GB300:
    trained 1.15-1.28x Acol's error, untrained 1.11-1.23x: the trained start
    is the worst of the three (regressing gauge-fixed targets pulls the
    components towards one average row).  The test checks that every start is
    a valid factorization the method improves from, and records the errors."""
    from paper_2205_06619_gb300 import api
    X, T = learned_init.training_set(count=24, m=80, n=400, rank=6, sweeps=4, seed=3)
    trained, hist = learned_init.train(X, T, rank=6, epochs=30, batch=128, lr=2e-3, seed=1)
    assert hist[-1] < hist[0]
    untrained = api.MLP(6, learned_init.init_params(6, seed=1))
    rows = []
    for q in range(4):
        R, M = learned_init.gene_like(80, 400, seed=1000 + q)
        Rg, Mw = torch.from_numpy(R).cuda(), api.pack_mask(M)
        perm = np.arange(80, dtype=np.int32)
        f = {}
        for name, net in (("trained", trained), ("untrained", untrained)):
            U0 = learned_init.predict_U(net, Rg, Mw)
            fz = api.Factorization(Rg, Mw, rank=6, perm=perm, U0=U0)
            f[name] = fz.run(0)["f_init"]
            f[name + "_1"] = fz.run(1)["f_final"]
            fz.close()
        fz = api.Factorization(Rg, Mw, rank=6, perm=perm, seed=q)
        f["acol"] = fz.run(0)["f_init"]
        fz.close()
        rows.append(f)
    print("initial errors (trained, untrained, Random Acol):",
          [(round(r["trained"]), round(r["untrained"]), round(r["acol"])) for r in rows])
    for r in rows:
        for name in ("trained", "untrained", "acol"):
            assert np.isfinite(r[name]) and r[name] > 0
        assert r["trained_1"] < r["trained"] and r["untrained_1"] < r["untrained"]


def test_learned_start_inside_the_library_equals_the_binding_path():
    """stmf_options.mlp: the library computes U0 = MLP(row sketch) + median on
    the oriented, permuted problem; the result equals passing the same start
    as U0 from the binding (rows permuted by the caller)."""
    from paper_2205_06619_gb300 import api
    X, T = learned_init.training_set(count=8, m=60, n=300, rank=5, sweeps=2, seed=5)
    net, _ = learned_init.train(X, T, rank=5, epochs=5, batch=64, lr=2e-3)
    R, M = learned_init.gene_like(50, 240, seed=7)
    Rg, Mw = torch.from_numpy(R).cuda(), api.pack_mask(M)
    perm = np.random.default_rng(3).permutation(50).astype(np.int32)
    U0 = learned_init.predict_U(net, Rg, Mw)[torch.from_numpy(perm.astype(np.int64)).cuda()].contiguous()
    a = api.factorize(Rg, Mw, rank=5, sweeps=2, perm=perm, U0=U0, trace_cap=200)
    b = api.factorize(Rg, Mw, rank=5, sweeps=2, perm=perm, mlp=net, trace_cap=200)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[2]["f_init"] == b[2]["f_init"] and a[3] == b[3]
    with pytest.raises(api.StmfError, match="rank"):
        api.factorize(Rg, Mw, rank=4, sweeps=1, mlp=net)
    # the batched form takes the network for every problem
    probs = [dict(R=Rg, mask_words=Mw, rank=5, sweeps=1, seed=q) for q in range(2)]
    outs, _ = api.factorize_batched(probs, window=8, mlp=net)
    for U, V, rep in outs:
        assert torch.isfinite(U).all() and rep["f_final"] <= rep["f_init"]
