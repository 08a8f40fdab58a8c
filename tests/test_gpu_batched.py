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


def test_batched_chains_gpu_filling_problems():
    """Problems whose phase 2 fills every SM alone (here 800 x 2048: 800
    tiles for 760 resident blocks) run one after another inside the batched
    graph, the small ones beside them; every problem still makes the decisions
    of its single call."""
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(17)
    probs = []
    for q, (m, n, r) in enumerate([(800, 2048, 3), (40, 60, 2), (2048, 800, 4), (800, 2100, 2), (30, 90, 3)]):
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.7, seed=int(rng.integers(1 << 30)))
        probs.append(dict(R=_tg(R), mask_words=api.pack_mask(M), rank=r, sweeps=1, seed=q))
    outs, _ = api.factorize_batched(probs, window=16)
    for pr, (U, V, rep) in zip(probs, outs):
        U1, V1, rep1, _ = api.factorize(pr["R"], pr["mask_words"], rank=pr["rank"], sweeps=1, seed=pr["seed"],
                                        window=16)
        assert torch.equal(U, U1) and torch.equal(V, V1)
        assert rep["candidates_tried"] == rep1["candidates_tried"]


def _ragged_problems(seed, count, sweeps):
    """Problems of uneven shape (tall and wide), rank and density, with their
    host copies for the oracle."""
    from paper_2205_06619_gb300 import api
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        m = int(rng.integers(6, 70)); n = int(rng.integers(6, 90))
        r = int(rng.integers(1, 6)); d = float(rng.uniform(0.4, 0.95))
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, d, seed=int(rng.integers(1 << 30)))
        out.append(dict(R=_tg(R), mask_words=api.pack_mask(M), rank=r, sweeps=sweeps,
                        seed=int(rng.integers(1 << 30)), R_np=R, M_np=M))
    return out


def test_batched_replays_every_problem_against_the_oracle():
    """Each problem of one batched launch exposes its trace; the replay
    harness checks every row visit of every problem against the oracle's
    ByRow step (Algorithm 3) and the final factors bit for bit."""
    from paper_2205_06619_gb300 import api
    from tests.replay import replay
    probs = _ragged_problems(41, 10, 3)
    for pr in probs:
        pr["trace_cap"] = 3 * max(pr["R_np"].shape) + 8
    outs, _ = api.factorize_batched(probs, window=8)
    for pr, (U, V, rep) in zip(probs, outs):
        tr = rep["trace"]
        assert len(tr) == rep["trace_records"] == 3 * min(pr["R_np"].shape)
        out = replay(pr["R_np"], pr["M_np"], pr["rank"], tr, seed=pr["seed"])
        assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
        assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
        assert abs(rep["f_final"] - out["f"]) <= 1e-6 * max(out["f"], 1e-30)
        assert len(out["divergences"]) <= 3       # near-ties within 1e-6 relative, adopted by the replay


def test_batched_eps_stop_matches_the_oracle():
    """The device-driven sweep loop of the batched form (k_sweep_end) applies
    the convergence rule of Section "Comparison of strategies" per problem:
    each problem's decisions replay against the oracle (near-ties adopted),
    and it stops after the first sweep whose change of the replayed error is
    below eps; eps is chosen 1.5x or more away from every change."""
    import oracle as orc
    from paper_2205_06619_gb300 import api
    from tests.replay import replay
    from tests.test_oracle_pins import eps_stop_case
    cands = _ragged_problems(43, 24, 10)
    chosen = []
    for pr in cands:
        full = orc.factorize(pr["R_np"], pr["M_np"], pr["rank"], sweeps=10, seed=pr["seed"])
        case = eps_stop_case(full["f_hist"])
        if case is not None:
            chosen.append((pr, case, np.abs(np.diff(full["f_hist"]))))
    # one eps for the whole batch: keep the problems with no change within 1.5x of it
    eps = float(np.median([c[1] for _, c, _ in chosen]))
    batch = [pr for pr, _, d in chosen if np.all(np.abs(np.log(d[d > 0] / eps)) > np.log(1.5))]
    assert len(batch) >= 4
    for pr in batch:
        pr["trace_cap"] = 10 * max(pr["R_np"].shape) + 8
    outs, _ = api.factorize_batched(batch, window=8, eps=eps)
    stopped_early = 0
    for pr, (U, V, rep) in zip(batch, outs):
        tr = rep["trace"]
        out = replay(pr["R_np"], pr["M_np"], pr["rank"], tr, seed=pr["seed"])
        assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
        assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
        # the rule on the replayed errors: f after each sweep = f of its last record
        st = orc.prepare(pr["R_np"], pr["M_np"], pr["rank"], seed=pr["seed"])
        f_hist = [orc.error(st["R"], st["M"], st["U"], st["V"])]
        for sw in range(rep["sweeps_done"]):
            f_hist.append([t[6] for t in tr if t[0] == sw][-1])
        d = np.abs(np.diff(f_hist))
        stop = next((s + 1 for s in range(len(d)) if d[s] < eps), 10)
        assert rep["sweeps_done"] == stop
        stopped_early += stop < 10
    assert stopped_early >= 4
