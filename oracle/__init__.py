"""Oracle for FastSTMF (arXiv 2205.06619) -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``stmf_oracle.c``: a plain, slow, single-threaded CPU
restatement of the paper's definitions and algorithms in FP64 (mode "fp64")
or in FP64 with every elementary add/sub/div rounded to FP32 (mode "fp32",
which reproduces IEEE fp32 arithmetic bit for bit).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the CUDA library never does.  It shares no code with the CUDA path.

Every function cites the passage of the paper it follows; see the C file.
Parity is pinned by ``tests/test_oracle_pins.py`` (closed forms, tropical
identities, residuation optimality, exact recovery, brute force on tiny
inputs, equivariances), ``tests/test_oracle_selections.py`` (the TD_B, TD and
SEQ selections), ``tests/test_oracle_byelement.py`` and
``tests/test_oracle_bymatrix.py`` (the ByElement and ByMatrix strategies),
with hand-computed examples under ``tests/golden/``.  The quality of the final factorization against the
paper's own experiments is "parity unpinned": the paper prints no absolute
errors for reproducible inputs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stmf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

MODES = {"fp64": 0, "fp32": 1}
# selections of (j, k) within a row (Section "The ByRow strategy")
SELECTIONS = {"TD_A": 0, "TD_B": 1, "TD": 2, "SEQ": 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liborc.so`` (portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        # -ffp-contract=off: no fused multiply-add may merge the rounded steps.
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, u64, i64 = C.c_double, C.c_int, C.c_uint64, C.c_int64
        P = C.c_void_p
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64, u64]
        L.orc_randperm.argtypes = [i, u64, P]
        L.orc_acol_picks.argtypes = [i, i, i, u64, P]
        L.orc_maxplus.argtypes = [i, i, i, i, P, P, P, P, P]
        L.orc_residuate_v.argtypes = [i, i, i, P, P, P, P]
        L.orc_residuate_u.argtypes = [i, i, i, P, P, P, P]
        L.orc_error.restype = d
        L.orc_error.argtypes = [i, i, i, i, P, P, P, P]
        L.orc_fulf.restype = d
        L.orc_fulf.argtypes = [i, i, i, i, P, P, P, P, i, i, i]
        L.orc_furf.restype = d
        L.orc_furf.argtypes = [i, i, i, i, P, P, P, P, i, i, i]
        L.orc_row_stats.argtypes = [i, i, i, i, P, P, P, P, i, P, P, P]
        L.orc_row_order.restype = i
        L.orc_row_order.argtypes = [i, i, i, i, P, P, P, P, i, P, P]
        L.orc_row_step.restype = i
        L.orc_row_step.argtypes = [i, i, i, i, P, P, P, P, i, P, P, P]
        L.orc_row_order_sel.restype = i
        L.orc_row_order_sel.argtypes = [i, i, i, i, i, P, P, P, P, i, P, P]
        L.orc_row_step_sel.restype = i
        L.orc_row_step_sel.argtypes = [i, i, i, i, i, P, P, P, P, i, P, P, P]
        L.orc_acol_init.argtypes = [i, i, i, i, P, P, P, i, P]
        L.orc_prepare.restype = i
        L.orc_prepare.argtypes = [i, i, i, i, P, P, P, P, i, u64, P, P, P, P, P, P, P]
        L.orc_finish.argtypes = [i, i, i, i, P, P, P, P, P]
        L.orc_factorize.restype = i
        L.orc_factorize.argtypes = [i, i, i, i, P, P, i, d, P, P, i, u64, P, P, P, P, P, i64, P]
        L.orc_factorize_sel.restype = i
        L.orc_factorize_sel.argtypes = [i, i, i, i, i, P, P, i, d, P, P, i, u64, P, P, P, P, P, i64, P]
        L.orc_colmin_perm.argtypes = [i, i, P, P, P]
        L.orc_element_scan.restype = i
        L.orc_element_scan.argtypes = [i, i, i, i, P, P, P, P, i, P, P, P]
        L.orc_factorize_byelement.restype = i
        L.orc_factorize_byelement.argtypes = [i, i, i, i, P, P, i, d, P, i, u64, P, P, P, P, P, i64, P]
        L.orc_matrix_coin.restype = i
        L.orc_matrix_coin.argtypes = [u64, i64, i, i, i]
        L.orc_matrix_order.restype = i
        L.orc_matrix_order.argtypes = [i, i, i, i, P, P, P, P, u64, i64, P, P, P, P]
        L.orc_matrix_step.restype = i
        L.orc_matrix_step.argtypes = [i, i, i, i, P, P, P, P, u64, i64, P, P, P]
        L.orc_factorize_bymatrix.restype = i
        L.orc_factorize_bymatrix.argtypes = [i, i, i, i, P, P, i, d, P, i, u64, P, P, P, P, P, i64, P]
        L.orc_rmse.argtypes = [i, i, i, i, P, P, P, P, P]
        L.orc_set_threads.argtypes = [i]
        L.orc_max_threads.restype = i
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _m(mask):
    return np.ascontiguousarray(mask, dtype=np.uint8)


def _mode(mode):
    return MODES[mode]


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's parallel loops (0: all cores); returns
    the count now in use.  Results do not depend on it (fixed sum orders)."""
    L = lib()
    L.orc_set_threads(int(n))
    return L.orc_max_threads()


def max_threads() -> int:
    return lib().orc_max_threads()


def splitmix64(key: int, c: int) -> int:
    return int(lib().orc_splitmix64(key, c))


def randperm(m: int, seed: int) -> np.ndarray:
    out = np.empty(m, np.int32)
    lib().orc_randperm(m, seed, _p(out))
    return out


def acol_picks(n: int, r: int, p: int, seed: int) -> np.ndarray:
    out = np.empty((r, p), np.int32)
    lib().orc_acol_picks(n, r, p, seed, _p(out))
    return out


def maxplus(U, V, mode="fp32"):
    """(U (x) V, argmax, runner-up) -- tropical product, ties to smaller l."""
    U, V = _d(U), _d(V)
    m, r = U.shape
    n = V.shape[1]
    P1 = np.empty((m, n)); A = np.empty((m, n), np.int32); P2 = np.empty((m, n))
    lib().orc_maxplus(_mode(mode), m, n, r, _p(U), _p(V), _p(P1), _p(A), _p(P2))
    return P1, A, P2


def residuate_v(R, M, u, mode="fp32"):
    """v = (-u)^T (x)* R over given entries."""
    R, M, u = _d(R), _m(M), _d(u)
    m, n = R.shape
    v = np.empty(n)
    empty = lib().orc_residuate_v(_mode(mode), m, n, _p(R), _p(M), _p(u), _p(v))
    return v, empty


def residuate_u(R, M, v, mode="fp32"):
    """u = R (x)* (-v)^T over given entries."""
    R, M, v = _d(R), _m(M), _d(v)
    m, n = R.shape
    u = np.empty(m)
    empty = lib().orc_residuate_u(_mode(mode), m, n, _p(R), _p(M), _p(v), _p(u))
    return u, empty


def error(R, M, U, V, mode="fp32") -> float:
    """b-norm of R - U (x) V over the given entries."""
    R, M, U, V = _d(R), _m(M), _d(U), _d(V)
    m, n = R.shape
    r = U.shape[1]
    return float(lib().orc_error(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V)))


def fulf(R, M, U, V, i, j, k, mode="fp32"):
    """F-ULF (Algorithm 1) on copies; returns (U', V', f')."""
    R, M = _d(R), _m(M)
    U, V = _d(U).copy(), _d(V).copy()
    m, n = R.shape
    r = U.shape[1]
    f = lib().orc_fulf(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), i, j, k)
    return U, V, float(f)


def furf(R, M, U, V, i, j, k, mode="fp32"):
    """F-URF (Algorithm 2) on copies; returns (U', V', f')."""
    R, M = _d(R), _m(M)
    U, V = _d(U).copy(), _d(V).copy()
    m, n = R.shape
    r = U.shape[1]
    f = lib().orc_furf(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), i, j, k)
    return U, V, float(f)


def rmse(R, M, U, V, mode="fp32"):
    """(RMSE-A over the given entries, RMSE-P over the held-out entries with a
    known value, |S_A|, |S_P|) of R against U (x) V (Section "Evaluation
    metrics").  R holds the true values of the held-out entries (NaN: none)."""
    R, M, U, V = _d(R), _m(M), _d(U), _d(V)
    m, n = R.shape
    out = np.empty(4)
    lib().orc_rmse(_mode(mode), m, n, U.shape[1], _p(R), _p(M), _p(U), _p(V), _p(out))
    return float(out[0]), float(out[1]), int(out[2]), int(out[3])


def row_stats(R, M, U, V, i, mode="fp32"):
    R, M, U, V = _d(R), _m(M), _d(U), _d(V)
    m, n = R.shape
    r = U.shape[1]
    td = np.empty(n); ch = np.empty((n, r), np.int32); rh = np.empty(r, np.int32)
    lib().orc_row_stats(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), i, _p(td), _p(ch), _p(rh))
    return td, ch, rh


def _sel(selection):
    if selection not in SELECTIONS:
        raise ValueError("selection must be one of %s" % sorted(SELECTIONS))
    return SELECTIONS[selection]


def row_order(R, M, U, V, i, mode="fp32", selection="TD_A"):
    """The (j, k) pairs of row i in the order the selection tries them."""
    R, M, U, V = _d(R), _m(M), _d(U), _d(V)
    m, n = R.shape
    r = U.shape[1]
    cap = n * r if selection == "SEQ" else n
    js = np.empty(cap, np.int32); ks = np.empty(cap, np.int32)
    c = lib().orc_row_order_sel(_mode(mode), _sel(selection), m, n, r, _p(R), _p(M), _p(U), _p(V), i,
                                _p(js), _p(ks))
    return js[:c].copy(), ks[:c].copy()


def row_step(R, M, U, V, i, f, mode="fp32", selection="TD_A"):
    """One ByRow row step in place on U, V (float64 arrays).

    Returns (kept, f_new, (pos, j, k, type), tried)."""
    R, M = _d(R), _m(M)
    assert U.dtype == np.float64 and V.dtype == np.float64 and U.flags.c_contiguous and V.flags.c_contiguous
    m, n = R.shape
    r = U.shape[1]
    fb = C.c_double(f)
    out = np.full(4, -1, np.int32)
    tried = C.c_int64(0)
    kept = lib().orc_row_step_sel(_mode(mode), _sel(selection), m, n, r, _p(R), _p(M), _p(U), _p(V), i,
                                  C.byref(fb), _p(out), C.byref(tried))
    return bool(kept), fb.value, tuple(int(x) for x in out), tried.value


def acol_init(R, M, picks, mode="fp32"):
    R, M = _d(R), _m(M)
    picks = np.ascontiguousarray(picks, np.int32)
    m, n = R.shape
    r, p = picks.shape
    U = np.empty((m, r))
    lib().orc_acol_init(_mode(mode), m, n, r, _p(R), _p(M), _p(picks), p, _p(U))
    return U


def prepare(R0, M0, r, perm=None, picks=None, p=5, seed=0, U0=None, mode="fp32"):
    """Orientation, permutation, init and V (Algorithm 3 before the loop)."""
    R0, M0 = _d(R0), _m(M0)
    m0, n0 = R0.shape
    tr = m0 > n0
    m, n = (n0, m0) if tr else (m0, n0)
    p = min(p, n)
    Ri = np.empty((m, n)); Mi = np.empty((m, n), np.uint8)
    Ui = np.empty((m, r)); Vi = np.empty((r, n)); perm_out = np.empty(m, np.int32)
    trb = C.c_int(0)
    perm = None if perm is None else np.ascontiguousarray(perm, np.int32)
    picks = None if picks is None else np.ascontiguousarray(picks, np.int32)
    U0 = None if U0 is None else _d(U0)
    empty = lib().orc_prepare(_mode(mode), m0, n0, r, _p(R0), _p(M0), _p(perm), _p(picks), p, seed,
                              _p(U0), _p(Ri), _p(Mi), _p(Ui), _p(Vi), _p(perm_out), C.byref(trb))
    return dict(R=Ri, M=Mi.astype(bool), U=Ui, V=Vi, perm=perm_out, transposed=bool(trb.value),
                empty=int(empty))


def finish(m0, n0, transposed, Ui, Vi, perm):
    Ui, Vi = _d(Ui), _d(Vi)
    r = Ui.shape[1]
    U = np.empty((m0, r)); V = np.empty((r, n0))
    lib().orc_finish(m0, n0, r, int(transposed), _p(Ui), _p(Vi),
                     _p(np.ascontiguousarray(perm, np.int32)), _p(U), _p(V))
    return U, V


def colmin_perm(R, M):
    """PermC: columns by increasing minimum of their given entries (stable)."""
    R, M = _d(R), _m(M)
    m, n = R.shape
    cp = np.empty(n, np.int32)
    lib().orc_colmin_perm(m, n, _p(R), _p(M), _p(cp))
    return cp


def element_scan(R, M, U, V, q0, f, mode="fp32"):
    """The ByElement scan from element position q0, in place on U, V.

    Returns (q or -1, f_new, (i, j, k, type), tried)."""
    R, M = _d(R), _m(M)
    assert U.dtype == np.float64 and V.dtype == np.float64 and U.flags.c_contiguous and V.flags.c_contiguous
    m, n = R.shape
    r = U.shape[1]
    fb = C.c_double(f)
    out = np.full(5, -1, np.int32)
    tried = C.c_int64(0)
    q = lib().orc_element_scan(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), q0, C.byref(fb), _p(out),
                               C.byref(tried))
    return int(q), fb.value, tuple(int(x) for x in out[1:]), tried.value


def matrix_coin(seed, it, m, n, q):
    """ByMatrix's coin for iteration it and element q: 0 = F-ULF, 1 = F-URF."""
    return int(lib().orc_matrix_coin(seed, it, m, n, q))


def matrix_order(R, M, U, V, seed, it, mode="fp32"):
    """ByMatrix order of iteration it: (q, k, type, err) arrays."""
    R, M, U, V = _d(R), _m(M), _d(U), _d(V)
    m, n = R.shape
    r = U.shape[1]
    qs = np.empty(m * n, np.int32); ks = np.empty(m * n, np.int32); ty = np.empty(m * n, np.int32)
    errs = np.empty(m * n)
    c = lib().orc_matrix_order(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), seed, it, _p(qs), _p(ks),
                               _p(ty), _p(errs))
    return qs[:c].copy(), ks[:c].copy(), ty[:c].copy(), errs[:c].copy()


def matrix_step(R, M, U, V, seed, it, f, mode="fp32"):
    """One ByMatrix iteration in place on U, V.

    Returns (kept, f_new, (pos, i, j, k, type), tried)."""
    R, M = _d(R), _m(M)
    assert U.dtype == np.float64 and V.dtype == np.float64 and U.flags.c_contiguous and V.flags.c_contiguous
    m, n = R.shape
    r = U.shape[1]
    fb = C.c_double(f)
    out = np.full(5, -1, np.int32)
    tried = C.c_int64(0)
    kept = lib().orc_matrix_step(_mode(mode), m, n, r, _p(R), _p(M), _p(U), _p(V), seed, it, C.byref(fb),
                                 _p(out), C.byref(tried))
    return bool(kept), fb.value, tuple(int(x) for x in out), tried.value


def _factorize_bymatrix(R0, M0, r, sweeps, eps, picks, p, seed, U0, mode, trace_cap):
    m0, n0 = R0.shape
    U = np.empty((m0, r)); V = np.empty((r, n0))
    f_hist = np.full(sweeps + 1, np.nan)
    trace = np.empty((max(trace_cap, 1), 6), np.int32)
    counters = np.zeros(4, np.int64)
    empty = lib().orc_factorize_bymatrix(_mode(mode), m0, n0, r, _p(R0), _p(M0), sweeps, eps, _p(picks), p,
                                         seed, _p(U0), _p(U), _p(V), _p(f_hist),
                                         _p(trace) if trace_cap else None, trace_cap, _p(counters))
    if empty:
        raise ValueError("oracle: %d rows/columns without a given entry" % empty)
    done = int(counters[0])
    return dict(U=U, V=V, f_hist=f_hist[:done + 1], sweeps=done, tried=int(counters[1]),
                kept=int(counters[2]), trace=trace[:int(counters[3])].copy() if trace_cap else None)


def _factorize_byelement(R0, M0, r, sweeps, eps, picks, p, seed, U0, mode, trace_cap):
    m0, n0 = R0.shape
    U = np.empty((m0, r)); V = np.empty((r, n0))
    f_hist = np.full(sweeps + 1, np.nan)
    trace = np.empty((max(trace_cap, 1), 6), np.int32)
    counters = np.zeros(4, np.int64)
    empty = lib().orc_factorize_byelement(_mode(mode), m0, n0, r, _p(R0), _p(M0), sweeps, eps, _p(picks), p,
                                          seed, _p(U0), _p(U), _p(V), _p(f_hist),
                                          _p(trace) if trace_cap else None, trace_cap, _p(counters))
    if empty:
        raise ValueError("oracle: %d rows/columns without a given entry" % empty)
    done = int(counters[0])
    return dict(U=U, V=V, f_hist=f_hist[:done + 1], sweeps=done, tried=int(counters[1]),
                kept=int(counters[2]), trace=trace[:int(counters[3])].copy() if trace_cap else None)


def factorize(R0, M0, r, sweeps, eps=0.0, perm=None, picks=None, p=5, seed=0, U0=None,
              mode="fp32", trace_cap=0, selection="TD_A", strategy="ByRow"):
    """FastSTMF (Algorithm 3) with the row's selection of (j, k) (TD_A as
    published; TD_B, TD, SEQ of Section "The ByRow strategy"), or, with
    strategy="ByElement", STMF_ByElement_PermC_TD_W (Section "The ByElement
    strategy"; perm and selection do not apply, U0 is in the frame of the
    oriented, column-permuted matrix), or with strategy="ByMatrix",
    STMF_ByMatrix_NoPerm_TD_W (Section "The ByMatrix strategy"; `sweeps`
    counts its iterations, each keeping at most one update).
    Returns dict(U, V, f_hist, sweeps, tried, kept, trace)."""
    if strategy not in ("ByRow", "ByElement", "ByMatrix"):
        raise ValueError("strategy must be ByRow, ByElement or ByMatrix")
    if strategy != "ByRow":
        if perm is not None or selection != "TD_A":
            raise ValueError("%s takes no row permutation and no selection" % strategy)
        R0, M0 = _d(R0), _m(M0)
        p = min(p, max(R0.shape))
        picks = None if picks is None else np.ascontiguousarray(picks, np.int32)
        U0 = None if U0 is None else _d(U0)
        fn = _factorize_byelement if strategy == "ByElement" else _factorize_bymatrix
        return fn(R0, M0, r, sweeps, eps, picks, p, seed, U0, mode, trace_cap)
    R0, M0 = _d(R0), _m(M0)
    m0, n0 = R0.shape
    p = min(p, max(m0, n0))  # the oriented matrix is wide: n = max(m0, n0)
    U = np.empty((m0, r)); V = np.empty((r, n0))
    f_hist = np.full(sweeps + 1, np.nan)
    trace = np.empty((max(trace_cap, 1), 6), np.int32)
    counters = np.zeros(4, np.int64)
    perm = None if perm is None else np.ascontiguousarray(perm, np.int32)
    picks = None if picks is None else np.ascontiguousarray(picks, np.int32)
    U0 = None if U0 is None else _d(U0)
    empty = lib().orc_factorize_sel(_mode(mode), _sel(selection), m0, n0, r, _p(R0), _p(M0), sweeps, eps,
                                    _p(perm), _p(picks), p, seed, _p(U0), _p(U), _p(V), _p(f_hist),
                                    _p(trace) if trace_cap else None, trace_cap, _p(counters))
    if empty:
        raise ValueError("oracle: %d rows/columns without a given entry" % empty)
    done = int(counters[0])
    return dict(U=U, V=V, f_hist=f_hist[:done + 1], sweeps=done, tried=int(counters[1]),
                kept=int(counters[2]), trace=trace[:int(counters[3])].copy() if trace_cap else None)
