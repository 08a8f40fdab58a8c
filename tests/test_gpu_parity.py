"""Parity of the CUDA path (through the C ABI) with the oracle.

Bars: the max-plus product, argmax and runner-up bit-exact against the
oracle's FP32 mode; F-ULF / F-URF factors bit-exact; b-norm errors within
1e-6 relative (FP32 terms are identical on both sides, only the summation
order differs); decisions identical except where the replay harness shows a
near-tie within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2205_06619_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


def api():
    from paper_2205_06619_gb300 import api as a
    return a


def tg(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


# ----------------------------------------------------------------- product

@pytest.mark.parametrize("m,n,r", [(1, 1, 1), (7, 5, 1), (33, 130, 3), (130, 257, 10), (64, 300, 20),
                                   (5, 1000, 32), (300, 97, 7), (129, 129, 2)])
def test_maxplus_bitexact(m, n, r):
    rng = np.random.default_rng(m * 1000 + n * 10 + r)
    U = rng.standard_normal((m, r)).astype(np.float32)
    V = rng.standard_normal((r, n)).astype(np.float32)
    P1, A, P2 = api().maxplus(tg(U), tg(V))
    e1, ea, e2 = orc.maxplus(U, V, "fp32")
    assert np.array_equal(P1.cpu().numpy().astype(np.float64), e1)
    assert np.array_equal(A.cpu().numpy().astype(np.int32), ea)
    assert np.array_equal(P2.cpu().numpy().astype(np.float64), e2)


@pytest.mark.parametrize("r", [1, 2, 5, 32])
def test_maxplus_ties_take_smaller_index(r):
    rng = np.random.default_rng(r)
    U = rng.integers(0, 3, size=(70, r)).astype(np.float32)
    V = rng.integers(0, 3, size=(r, 90)).astype(np.float32)
    P1, A, P2 = api().maxplus(tg(U), tg(V))
    e1, ea, e2 = orc.maxplus(U, V, "fp32")
    assert np.array_equal(A.cpu().numpy().astype(np.int32), ea)
    assert np.array_equal(P2.cpu().numpy().astype(np.float64), e2)


def test_maxplus_masked_entries_marked():
    rng = np.random.default_rng(9)
    U = rng.standard_normal((40, 4)).astype(np.float32)
    V = rng.standard_normal((4, 77)).astype(np.float32)
    M = rng.random((40, 77)) < 0.6
    P1, A, P2 = api().maxplus(tg(U), tg(V), api().pack_mask(M))
    e1, ea, e2 = orc.maxplus(U, V, "fp32")
    P1 = P1.cpu().numpy(); A = A.cpu().numpy(); P2 = P2.cpu().numpy()
    assert np.array_equal(P1[M].astype(np.float64), e1[M]) and np.all(np.isnan(P1[~M]))
    assert np.array_equal(A[M].astype(np.int32), ea[M]) and np.all(A[~M] == 255)
    assert np.array_equal(P2[M].astype(np.float64), e2[M]) and np.all(np.isnan(P2[~M]))


@pytest.mark.parametrize("m,n,r,obs", [(50, 70, 3, 0.8), (200, 513, 10, 0.5), (31, 33, 1, 0.3)])
def test_selection_stats(m, n, r, obs):
    R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=m + n)
    rng = np.random.default_rng(m)
    U = rng.random((m, r)).astype(np.float32)
    V = rng.random((r, n)).astype(np.float32) - 0.5
    td, ch, f = api().selection_stats(tg(R), tg(U), tg(V), api().pack_mask(M))
    e_td, e_ch, _ = orc.row_stats(R, M, U, V, 0)
    assert np.array_equal(ch.cpu().numpy(), e_ch)
    td = td.cpu().numpy()
    assert np.all(np.abs(td - e_td) <= 1e-12 * np.maximum(e_td, 1e-300))
    e_f = orc.error(R, M, U, V)
    assert rel(f, e_f) <= 1e-12


# ------------------------------------------------------- single updates

def _consistent(R, M, r, seed):
    rng = np.random.default_rng(seed)
    U0 = rng.random((R.shape[0], r)).astype(np.float32)
    V = np.stack([orc.residuate_v(R, M, U0[:, l])[0] for l in range(r)])
    return U0, V


@pytest.mark.parametrize("m,n,r", [(20, 30, 3), (130, 300, 5), (64, 700, 10)])
def test_update_unconditional_matches_oracle(m, n, r):
    """F-ULF / F-URF applied unconditionally: factors bit-exact, f' within 1e-6."""
    R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, 0.8, seed=3 * m + n)
    U0, V0 = _consistent(R, M, r, seed=m)
    prob = api().Problem(tg(R), api().pack_mask(M), rank=r, U0=tg(U0))
    Ug, Vg, fg = prob.get()
    assert np.array_equal(Vg.cpu().numpy().astype(np.float64), V0)
    U, V = U0.astype(np.float64), V0
    f = orc.error(R, M, U, V)
    assert rel(fg, f) <= TOL
    rng = np.random.default_rng(7)
    given = np.argwhere(M)
    for step in range(12):
        i, j = given[rng.integers(len(given))]
        k = int(rng.integers(r))
        typ = step % 2
        fn, kept = (prob.update_U if typ == 0 else prob.update_V)(int(i), int(j), k, commit_if_decreases=False)
        U, V, fo = (orc.fulf if typ == 0 else orc.furf)(R, M, U, V, int(i), int(j), k)
        assert kept
        assert rel(fn, fo) <= TOL, (step, fn, fo)
        Ug, Vg, fg = prob.get()
        assert np.array_equal(Ug.cpu().numpy().astype(np.float64), U), step
        assert np.array_equal(Vg.cpu().numpy().astype(np.float64), V), step
        assert rel(fg, fo) <= TOL


def test_update_commit_if_decreases_follows_the_paper():
    """commit_if_decreases keeps the update exactly when f' < f (Algorithm 3)."""
    R, M, _, _ = synth.uniform_planted(40, 90, 3, 0.01, 0.8, seed=11)
    U0, V0 = _consistent(R, M, 3, seed=11)
    prob = api().Problem(tg(R), api().pack_mask(M), rank=3, U0=tg(U0))
    U, V = U0.astype(np.float64), V0
    f = orc.error(R, M, U, V)
    rng = np.random.default_rng(12)
    given = np.argwhere(M)
    n_kept = 0
    for step in range(30):
        i, j = (int(x) for x in given[rng.integers(len(given))])
        k = int(rng.integers(3))
        typ = step % 2
        fn, kept = (prob.update_U if typ == 0 else prob.update_V)(i, j, k, commit_if_decreases=True)
        U2, V2, fo = (orc.fulf if typ == 0 else orc.furf)(R, M, U, V, i, j, k)
        assert rel(fn, fo) <= TOL
        if abs(fo - f) > TOL * f:
            assert kept == (fo < f)
        if kept:
            U, V, f = U2, V2, fo
            n_kept += 1
        Ug, Vg, _ = prob.get()
        assert np.array_equal(Ug.cpu().numpy().astype(np.float64), U)
        assert np.array_equal(Vg.cpu().numpy().astype(np.float64), V)
    assert n_kept > 0


def test_update_rejects_bad_indices():
    R, M, _, _ = synth.uniform_planted(10, 12, 2, 0.01, 0.7, seed=2)
    prob = api().Problem(tg(R), api().pack_mask(M), rank=2)
    i, j = np.argwhere(~M)[0]
    with pytest.raises(api().StmfError):
        prob.update_U(int(i), int(j), 0)
    with pytest.raises(api().StmfError):
        prob.update_V(0, 0, 5)


def test_problem_rejects_empty_column():
    R = np.ones((6, 8), np.float32)
    M = np.ones((6, 8), bool)
    M[:, 3] = False
    with pytest.raises(api().StmfError):
        api().Problem(tg(R), api().pack_mask(M), rank=2)


def test_rejects_given_entries_beyond_the_magnitude_limit():
    """Given entries must be finite and below 2^60 in magnitude (entries that
    are not given sit at a sentinel of 2^126 in the evaluation's planes)."""
    R = np.ones((6, 8), np.float32)
    M = np.ones((6, 8), bool)
    R[2, 3] = 2.0 ** 61
    with pytest.raises(api().StmfError, match="2\\^60"):
        api().factorize(tg(R), api().pack_mask(M), rank=2)
    with pytest.raises(api().StmfError, match="2\\^60"):
        api().Problem(tg(R), api().pack_mask(M), rank=2)
    M[2, 3] = False                       # not given: its value is never read
    api().factorize(tg(R), api().pack_mask(M), rank=2, sweeps=1)
    R[2, 3] = 2.0 ** 59
    M[2, 3] = True
    api().factorize(tg(R), api().pack_mask(M), rank=2, sweeps=1)


# ------------------------------------------------------------ factorize

@pytest.mark.parametrize("shape,transposed", [((40, 70), False), ((70, 40), True)])
def test_factorize_init_matches_oracle(shape, transposed):
    """Orientation, RandPerm (SplitMix64), Random Acol and V by residuation."""
    m, n = shape
    R, M, _, _ = synth.uniform_planted(m, n, 4, 0.01, 0.8, seed=m)
    U, V, rep, _ = api().factorize(tg(R), api().pack_mask(M), rank=4, sweeps=0, seed=123)
    ref = orc.factorize(R, M, 4, sweeps=0, seed=123)
    assert rep["transposed"] == int(transposed)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), ref["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), ref["V"])
    assert rel(rep["f_init"], ref["f_hist"][0]) <= TOL


@pytest.mark.parametrize("window", [2, 8, 64])
def test_factorize_small_replay(window):
    """Decisions of every row visit replayed against the oracle; the window
    size must not change any decision."""
    from tests.replay import replay
    R, M, _, _ = synth.uniform_planted(36, 52, 3, 0.01, 0.8, seed=21)
    U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=3, seed=4, window=window,
                                       trace_cap=1000)
    out = replay(R, M, 3, trace, seed=4)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= 1


def test_factorize_workload_small_replay():
    """The 200 x 100 rank-3 workload (runs as 100 x 200), 10 sweeps."""
    from tests.replay import replay
    w = synth.workload_small(seed=0)
    U, V, rep, trace = api().factorize(tg(w["R"]), api().pack_mask(w["mask"]), rank=3, sweeps=10, seed=0,
                                       trace_cap=2000)
    assert rep["transposed"] == 1
    out = replay(w["R"], w["mask"], 3, trace, seed=0)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= 2
    # the error never increases (reported values carry ~1e-9 summation noise)
    f_hist = [t[6] for t in trace]
    assert all(b <= a * (1 + 1e-7) for a, b in zip(f_hist, f_hist[1:]))


def test_factorize_ragged_and_degenerate_shapes():
    from tests.replay import replay
    for (m, n, r, obs, seed) in [(1, 9, 1, 1.0, 1), (9, 1, 2, 1.0, 2), (17, 33, 1, 0.5, 3), (33, 17, 5, 0.9, 4),
                                 (2, 2, 2, 1.0, 5)]:
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, obs, seed=seed)
        U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=r, sweeps=2, seed=seed, trace_cap=100)
        out = replay(R, M, r, trace, seed=seed)
        assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"]), (m, n, r)
        assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"]), (m, n, r)


@pytest.mark.parametrize("obs,r", [(0.05, 3), (0.5, 20), (1.0, 32)])
def test_factorize_density_and_rank_extremes_replay(obs, r):
    """Sparse (5% given), half and fully given matrices at ranks 3, 20 and 32,
    with n not a multiple of 32: decisions replayed against the oracle."""
    from tests.replay import replay
    R, M, _, _ = synth.uniform_planted(45, 301, r, 0.01, obs, seed=int(obs * 100) + r)
    U, V, rep, trace = api().factorize(tg(R), api().pack_mask(M), rank=r, sweeps=2, seed=3, trace_cap=500)
    out = replay(R, M, r, trace, seed=3)
    assert np.array_equal(U.cpu().numpy().astype(np.float64), out["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), out["V"])
    assert rel(rep["f_final"], out["f"]) <= TOL
    assert len(out["divergences"]) <= 1


def test_factorize_in_pieces_equals_one_call():
    """Sweeps run in pieces on a live problem give the same run as one call."""
    R, M, _, _ = synth.uniform_planted(30, 64, 3, 0.01, 0.8, seed=31)
    U1, V1, rep1, tr1 = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=3, seed=9, trace_cap=200)
    fz = api().Factorization(tg(R), api().pack_mask(M), rank=3, seed=9, trace_cap=200)
    fz.run(2)
    rep2 = fz.run(1)
    U2, V2 = fz.result()
    assert torch.equal(U1, U2) and torch.equal(V1, V2)
    assert rep1["candidates_tried"] == rep2["candidates_tried"] and rep1["accepted"] == rep2["accepted"]
    assert [t[:6] for t in tr1] == [t[:6] for t in fz.trace_records()]


@pytest.mark.parametrize("window", [4, 64])
def test_graph_and_host_driven_loops_agree(monkeypatch, window):
    """The device-driven sweep (one CUDA graph with conditional nodes, the
    evaluation of window t beside the decision of window t-1) and the
    host-driven loop (the same steps one after another) make the same
    decisions and do the same work, including the windows evaluated ahead
    and dropped at the end of a row (at most one per row visit; none for a
    row run short, whose first windows are each followed by an empty
    placeholder instead)."""
    R, M, _, _ = synth.uniform_planted(40, 50, 3, 0.01, 0.8, seed=41)
    a = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=200, window=window)
    monkeypatch.setenv("STMF_NO_GRAPH", "1")
    b = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=2, seed=2, trace_cap=200, window=window)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert [t[:6] for t in a[3]] == [t[:6] for t in b[3]]
    for key in ("candidates_tried", "candidates_issued", "windows", "accepted", "candidates_discarded",
                "eval_launches", "eval_candidates"):
        assert a[2][key] == b[2][key], key
    rows = 2 * 40
    assert 0 <= a[2]["candidates_discarded"] <= rows * window
    assert a[2]["windows"] >= a[2]["eval_launches"]          # placeholders are decided, not evaluated


def test_launch_shapes_never_change_a_decision():
    """Phase 1's column chunk and phase 2's blocks per SM (the shapes the
    batched form's autotuner picks) change the grouping of the work, never a
    decision: the same trace and factors for every shape tried, and the
    reports name the shapes used."""
    R, M, _, _ = synth.uniform_planted(70, 900, 4, 0.01, 0.8, seed=43)
    runs = []
    for shapes in (None, (32, 1), (40, 3), (128, 5), (0, 3, 8), (48, 4, 8), (0, 1, 8)):
        runs.append(api().factorize(tg(R), api().pack_mask(M), rank=4, sweeps=2, seed=6, trace_cap=300,
                                    window=16, shapes=shapes))
        if shapes is not None:
            assert runs[-1][2]["eval_res_chunk"] == (shapes[0] or runs[0][2]["eval_res_chunk"])
            assert runs[-1][2]["eval_delta_rows"] == (shapes[2] if len(shapes) > 2 else 4)
    for U, V, rep, tr in runs[1:]:
        assert torch.equal(U, runs[0][0]) and torch.equal(V, runs[0][1])
        assert [t[:6] for t in tr] == [t[:6] for t in runs[0][3]]
    with pytest.raises(api().StmfError, match="res_chunk"):
        api().factorize(tg(R), api().pack_mask(M), rank=4, sweeps=1, shapes=(36, 0))
    with pytest.raises(api().StmfError, match="delta_tile_rows"):
        api().factorize(tg(R), api().pack_mask(M), rank=4, sweeps=1, shapes=(0, 0, 6))


# ------------------------------------------------------ checkpoint / faults

def test_resume_from_saved_state_equals_the_uninterrupted_run():
    """Checkpoint / resume: the factors and permutation after sweep 1, passed
    back as U0, V0 and perm, continue exactly as the uninterrupted run."""
    R, M, _, _ = synth.uniform_planted(40, 90, 4, 0.01, 0.8, seed=12)
    Rg, Mw = tg(R), api().pack_mask(M)
    perm = np.random.default_rng(5).permutation(40).astype(np.int32)
    full = api().factorize(Rg, Mw, rank=4, sweeps=3, seed=1, perm=perm, trace_cap=500)
    fz = api().Factorization(Rg, Mw, rank=4, seed=1, perm=perm)
    fz.run(1)
    U1, V1 = fz.result()
    fz.close()
    U0 = U1[torch.from_numpy(perm.astype(np.int64)).cuda()].contiguous()    # oriented, permuted rows
    res = api().factorize(Rg, Mw, rank=4, sweeps=2, perm=perm, U0=U0, V0=V1.contiguous(), trace_cap=500)
    assert torch.equal(res[0], full[0]) and torch.equal(res[1], full[1])
    assert res[2]["f_final"] == full[2]["f_final"]
    later = [t[1:] for t in full[3] if t[0] >= 1]
    assert [t[1:] for t in res[3]] == later
    with pytest.raises(api().StmfError, match="V0 needs U0"):
        api().factorize(Rg, Mw, rank=4, sweeps=1, V0=V1.contiguous())


def test_injected_allocation_failures_leave_the_context_usable(monkeypatch):
    """Host-side fault injection (STMF_TEST_FAIL_ALLOC=N fails the N-th device
    allocation of a problem): the call returns STMF_ERR_OOM, frees what it had
    allocated and the next call works."""
    R, M, _, _ = synth.uniform_planted(30, 50, 3, 0.01, 0.8, seed=2)
    Rg, Mw = tg(R), api().pack_mask(M)
    ref = api().factorize(Rg, Mw, rank=3, sweeps=1, seed=0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n in (1, 2, 7, 13, 20):
        monkeypatch.setenv("STMF_TEST_FAIL_ALLOC", str(n))
        with pytest.raises(api().StmfError) as ei:
            api().factorize(Rg, Mw, rank=3, sweeps=1, seed=0)
        assert ei.value.status == 3          # STMF_ERR_OOM
    monkeypatch.delenv("STMF_TEST_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 * 1024 * 1024
    again = api().factorize(Rg, Mw, rank=3, sweeps=1, seed=0)
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])


def test_factorize_eps_stop_matches_the_oracle():
    """Convergence rule (Section "Comparison of strategies"): with eps > 0 the
    host-driven sweep loop of stmf_factorize stops after the same sweep as the
    oracle, with the oracle's factors and error; eps is chosen a factor of 2
    or more away from every change it is compared with."""
    from tests.test_oracle_pins import eps_stop_case
    R, M, _, _ = synth.uniform_planted(40, 56, 3, 0.01, 0.8, seed=32)
    full = orc.factorize(R, M, 3, sweeps=10, seed=6)
    s_star, eps = eps_stop_case(full["f_hist"])
    ref = orc.factorize(R, M, 3, sweeps=10, eps=eps, seed=6)
    assert ref["sweeps"] == s_star
    U, V, rep, _ = api().factorize(tg(R), api().pack_mask(M), rank=3, sweeps=10, eps=eps, seed=6)
    assert rep["sweeps_done"] == s_star
    assert np.array_equal(U.cpu().numpy().astype(np.float64), ref["U"])
    assert np.array_equal(V.cpu().numpy().astype(np.float64), ref["V"])
    assert rel(rep["f_final"], ref["f_hist"][-1]) <= TOL


@pytest.mark.parametrize("graph", [True, False])
def test_loop_bound_stops_cleanly_with_timeout(monkeypatch, graph):
    """The device-driven loops are bounded.  A test-only bound of one window
    per row (STMF_TEST_WINDOW_CAP=1) is passed by the first row that needs a
    second window: every loop stops, nothing of that window is committed, the
    call returns STMF_ERR_TIMEOUT, and the context then runs the same
    factorization normally.  Single calls (graph- and host-driven) and the
    batched form."""
    from tests.replay import replay
    if not graph:
        monkeypatch.setenv("STMF_NO_GRAPH", "1")
    R, M, _, _ = synth.uniform_planted(40, 64, 3, 0.01, 0.8, seed=33)
    Rg, Mw = tg(R), api().pack_mask(M)
    ref = api().factorize(Rg, Mw, rank=3, sweeps=2, seed=1, window=2, trace_cap=500)
    assert ref[2]["windows"] > ref[2]["trace_records"]        # some row needed a second window
    monkeypatch.setenv("STMF_TEST_WINDOW_CAP", "1")
    with pytest.raises(api().StmfError) as ei:
        api().factorize(Rg, Mw, rank=3, sweeps=2, seed=1, window=2)
    assert ei.value.status == 4          # STMF_ERR_TIMEOUT
    with pytest.raises(api().StmfError) as ei:
        api().factorize_batched([dict(R=Rg, mask_words=Mw, rank=3, sweeps=2, seed=1)], window=2)
    assert ei.value.status == 4
    # the rows before the stop are the method's own: a run resumed in pieces
    fz = api().Factorization(Rg, Mw, rank=3, seed=1, window=2, trace_cap=500)
    with pytest.raises(api().StmfError):
        fz.run(2)
    fz.result()
    part = fz.trace_records()
    fz.close()
    out = replay(R, M, 3, part, seed=1)
    assert len(out["divergences"]) == 0
    monkeypatch.delenv("STMF_TEST_WINDOW_CAP")
    again = api().factorize(Rg, Mw, rank=3, sweeps=2, seed=1, window=2)
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])
