"""Python binding of the C ABI in ``include/stmf.h`` (argument marshalling only).

Every computation runs in ``libstmf.so``'s CUDA kernels.  Tensors are torch
CUDA tensors (device memory and streams come from PyTorch); the functions
take and return them, pass raw pointers and the current stream to the
library, and raise :class:`StmfError` on any non-OK status.  There is no CPU
fallback: if the library is missing or no GPU is present, calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import struct

import numpy as np

from . import build as _build

STMF_MAX_RANK = 32
STMF_TRACE_INTS = 8
STATUS = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "INTERNAL"}

EXPORTS = ["stmf_create", "stmf_destroy", "stmf_last_error", "stmf_set_stream", "stmf_maxplus",
           "stmf_selection_stats", "stmf_problem_create", "stmf_problem_destroy", "stmf_update_U",
           "stmf_update_V", "stmf_problem_get", "stmf_factorize", "stmf_factorize_begin",
           "stmf_factorize_run", "stmf_factorize_end", "stmf_default_options", "stmf_struct_sizes",
           "stmf_peak_addmax", "stmf_rmse",
           "stmf_selection_stats_noalloc", "stmf_factorize_batched", "stmf_row_sketch", "stmf_mlp_param_count",
           "stmf_mlp_create", "stmf_mlp_destroy", "stmf_mlp_get_params", "stmf_mlp_forward", "stmf_mlp_gradient",
           "stmf_mlp_train_step", "stmf_mlp_targets", "stmf_assign_by_rank",
           "stmf_mlp_predict"]


class StmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("stmf status %s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Options(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("eps", C.c_double), ("window", C.c_int), ("select", C.c_int),
                ("precision", C.c_int), ("acol_p", C.c_int), ("seed", C.c_uint64),
                ("perm", C.c_void_p), ("picks", C.c_void_p), ("U0", C.c_void_p),
                ("trace", C.c_void_p), ("trace_cap", C.c_int64), ("V0", C.c_void_p), ("mlp", C.c_void_p),
                ("selection", C.c_int), ("strategy", C.c_int), ("res_chunk", C.c_int),
                ("delta_blocks_per_sm", C.c_int), ("delta_tile_rows", C.c_int)]


# selections of (j, k) within a row (Section "The ByRow strategy"; stmf.h STMF_SEL_*)
SELECTIONS = {"TD_A": 0, "TD_B": 1, "TD": 2, "SEQ": 3}


# update strategies (stmf.h STMF_STRATEGY_*): Algorithm 3, and the ByElement method
STRATEGIES = {"ByRow": 0, "ByElement": 1, "ByMatrix": 2}


def _strategy(name):
    if name not in STRATEGIES:
        raise ValueError("strategy must be one of %s" % sorted(STRATEGIES))
    return STRATEGIES[name]


def _selection(name):
    if name not in SELECTIONS:
        raise ValueError("selection must be one of %s" % sorted(SELECTIONS))
    return SELECTIONS[name]


class BatchProblem(C.Structure):
    _fields_ = [("m", C.c_int), ("n", C.c_int), ("r", C.c_int), ("R", C.c_void_p), ("ldr", C.c_int),
                ("mask", C.c_void_p), ("ldm_words", C.c_int), ("U_out", C.c_void_p), ("V_out", C.c_void_p),
                ("seed", C.c_uint64), ("sweeps", C.c_int), ("trace", C.c_void_p), ("trace_cap", C.c_int64)]


class Report(C.Structure):
    _fields_ = [("f_init", C.c_double), ("f_final", C.c_double), ("sweeps_done", C.c_int),
                ("transposed", C.c_int), ("candidates_tried", C.c_int64),
                ("candidates_issued", C.c_int64), ("accepted", C.c_int64), ("refreshes", C.c_int64),
                ("windows", C.c_int64), ("trace_records", C.c_int64), ("eval_ns", C.c_int64),
                ("eval_launches", C.c_int64), ("eval_candidates", C.c_int64), ("seconds", C.c_double),
                ("candidates_screened", C.c_int64), ("eval_res_ns", C.c_int64), ("eval_delta_ns", C.c_int64),
                ("candidates_discarded", C.c_int64), ("eval_res_chunk", C.c_int64),
                ("eval_delta_blocks", C.c_int64), ("eval_delta_rows", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(build_if_missing: bool = True):
    """Loads libstmf.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libstmf.so is not built (run paper_2205_06619_gb300.build.build())")
        _build.build()
    L = C.CDLL(path)
    P, i, d = C.c_void_p, C.c_int, C.c_double
    L.stmf_create.argtypes = [C.POINTER(P), i, P]
    L.stmf_destroy.argtypes = [P]
    L.stmf_destroy.restype = None
    L.stmf_last_error.argtypes = [P]
    L.stmf_last_error.restype = C.c_char_p
    L.stmf_set_stream.argtypes = [P, P]
    L.stmf_maxplus.argtypes = [P, i, i, i, P, i, P, i, P, i, P, i, P, i, P]
    L.stmf_selection_stats.argtypes = [P, i, i, i, P, i, P, i, P, i, P, i, P, P, C.POINTER(d)]
    L.stmf_selection_stats_noalloc.argtypes = [P, i, i, i, P, i, P, i, P, i, P, i, P, P, C.POINTER(d)]
    L.stmf_rmse.argtypes = [P, i, i, i, P, i, P, i, P, i, P, i, C.POINTER(d)]
    L.stmf_problem_create.argtypes = [P, i, i, i, P, i, P, i, P, C.POINTER(Options), C.POINTER(P)]
    L.stmf_problem_destroy.argtypes = [P]
    L.stmf_problem_destroy.restype = None
    L.stmf_update_U.argtypes = [P, i, i, i, i, C.POINTER(d), C.POINTER(i)]
    L.stmf_update_V.argtypes = [P, i, i, i, i, C.POINTER(d), C.POINTER(i)]
    L.stmf_problem_get.argtypes = [P, P, P, C.POINTER(d)]
    L.stmf_factorize.argtypes = [P, i, i, i, P, i, P, i, C.POINTER(Options), P, P, C.POINTER(Report)]
    L.stmf_factorize_begin.argtypes = [P, i, i, i, P, i, P, i, C.POINTER(Options), C.POINTER(P)]
    L.stmf_factorize_run.argtypes = [P, i, d, C.POINTER(Report)]
    L.stmf_factorize_end.argtypes = [P, P, P, P, C.c_int64]
    L.stmf_factorize_batched.argtypes = [P, i, C.POINTER(BatchProblem), C.POINTER(Options), C.POINTER(Report),
                                         C.POINTER(i)]
    L.stmf_row_sketch.argtypes = [P, i, i, P, i, P, i, P, P]
    L.stmf_mlp_param_count.argtypes = [i]
    L.stmf_mlp_create.argtypes = [P, i, P, C.POINTER(P)]
    L.stmf_mlp_destroy.argtypes = [P]
    L.stmf_mlp_destroy.restype = None
    L.stmf_mlp_get_params.argtypes = [P, P]
    L.stmf_mlp_forward.argtypes = [P, i, P, P]
    L.stmf_mlp_gradient.argtypes = [P, i, P, P, C.POINTER(d), P]
    L.stmf_mlp_train_step.argtypes = [P, i, P, P, C.c_float, C.POINTER(d)]
    L.stmf_mlp_predict.argtypes = [P, i, i, P, i, P, i, P]
    L.stmf_mlp_targets.argtypes = [P, i, i, i, P, i, P, i, P, i, P]
    L.stmf_assign_by_rank.argtypes = [P, i, i, P, i, P, i, P, i]
    L.stmf_default_options.argtypes = [C.POINTER(Options)]
    L.stmf_default_options.restype = None
    L.stmf_struct_sizes.argtypes = [C.POINTER(C.c_size_t)] * 3
    L.stmf_struct_sizes.restype = None
    L.stmf_peak_addmax.argtypes = [P, i, i, C.POINTER(d)]
    for name in EXPORTS:
        if name not in ("stmf_destroy", "stmf_last_error", "stmf_problem_destroy", "stmf_default_options",
                        "stmf_mlp_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("stmf needs a CUDA GPU; none is available")
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_f32(t, name):
    torch = _torch()
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError("%s must be a float32 CUDA tensor" % name)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s must be 2-D with unit column stride" % name)


def pack_mask(mask):
    """Boolean mask (m x n; torch or numpy) -> bit-packed uint32 words (m x ceil(n/32)),
    bit t%32 of word t/32 set when entry t is given.  Returns a CUDA int32 tensor."""
    torch = _torch()
    if isinstance(mask, torch.Tensor):
        mask = mask.detach().cpu().numpy()
    mask = np.ascontiguousarray(mask, dtype=bool)
    m, n = mask.shape
    words = (n + 31) // 32
    padded = np.zeros((m, words * 32), dtype=bool)
    padded[:, :n] = mask
    bits = np.packbits(padded.reshape(m, words, 4, 8)[:, :, :, ::-1], axis=-1).reshape(m, words, 4)
    packed = bits.astype(np.uint32)
    w = packed[:, :, 0] | (packed[:, :, 1] << 8) | (packed[:, :, 2] << 16) | (packed[:, :, 3] << 24)
    return torch.from_numpy(w.view(np.int32).copy()).cuda()


class Context:
    """A library context bound to a CUDA device and (by default) the current stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        st = L.stmf_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st != 0:
            raise StmfError(st, "stmf_create(device=%d) failed" % device)
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            load().stmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        if st != 0:
            raise StmfError(st, load().stmf_last_error(self.h).decode())

    def use_current_stream(self):
        torch = _torch()
        s = torch.cuda.current_stream(self.device)
        if s is not self.stream:
            self.stream = s
            self.check(load().stmf_set_stream(self.h, C.c_void_p(s.cuda_stream)))


_default_ctx = None


def context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(0)
    _default_ctx.use_current_stream()
    return _default_ctx


def maxplus(U, V, mask_words=None, with_argmax=True, with_runner_up=True):
    """P1 = U (x) V (max-plus), A = argmax (uint8, smaller l on ties), P2 = runner-up."""
    torch = _torch()
    _check_f32(U, "U"); _check_f32(V, "V")
    m, r = U.shape
    n = V.shape[1]
    ctx = context()
    P1 = torch.empty((m, n), device=U.device, dtype=torch.float32)
    A = torch.empty((m, n), device=U.device, dtype=torch.uint8) if with_argmax else None
    P2 = torch.empty((m, n), device=U.device, dtype=torch.float32) if with_runner_up else None
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_maxplus(ctx.h, m, n, r, _ptr(U), U.stride(0), _ptr(V), V.stride(0), _ptr(mask_words),
                                  ldm, _ptr(P1), n, _ptr(A), n, _ptr(P2)))
    return P1, A, P2


def selection_stats(R, U, V, mask_words=None):
    """(td_col float64[n], colhist int32[n, r], f) over the given entries."""
    torch = _torch()
    _check_f32(R, "R"); _check_f32(U, "U"); _check_f32(V, "V")
    m, n = R.shape
    r = U.shape[1]
    ctx = context()
    td = torch.empty(n, device=R.device, dtype=torch.float64)
    ch = torch.empty((n, r), device=R.device, dtype=torch.int32)
    f = C.c_double()
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_selection_stats(ctx.h, m, n, r, _ptr(R), R.stride(0), _ptr(mask_words), ldm,
                                          _ptr(U), U.stride(0), _ptr(V), V.stride(0), _ptr(td), _ptr(ch),
                                          C.byref(f)))
    return td, ch, f.value


def rmse(R, U, V, mask_words=None):
    """(RMSE-A, RMSE-P, |S_A|, |S_P|) of R against U (x) V on the device
    (stmf_rmse): the given entries, and the held-out ones whose true value R
    holds (NaN: none)."""
    _check_f32(R, "R"); _check_f32(U, "U"); _check_f32(V, "V")
    m, n = R.shape
    ctx = context()
    out = (C.c_double * 4)()
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_rmse(ctx.h, m, n, U.shape[1], _ptr(R), R.stride(0), _ptr(mask_words), ldm, _ptr(U),
                               U.stride(0), _ptr(V), V.stride(0), out))
    return out[0], out[1], int(out[2]), int(out[3])


def selection_stats_noalloc(R, U, V, mask_words=None, td_col=None, colhist=None):
    """Same results as :func:`selection_stats`, computed without any device
    allocation inside the library (its scratch is a fixed static array; see
    stmf_selection_stats_noalloc in include/stmf.h).  Output tensors may be
    passed in so that this call allocates nothing either."""
    torch = _torch()
    _check_f32(R, "R"); _check_f32(U, "U"); _check_f32(V, "V")
    m, n = R.shape
    r = U.shape[1]
    ctx = context()
    td = td_col if td_col is not None else torch.empty(n, device=R.device, dtype=torch.float64)
    ch = colhist if colhist is not None else torch.empty((n, r), device=R.device, dtype=torch.int32)
    f = C.c_double()
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_selection_stats_noalloc(ctx.h, m, n, r, _ptr(R), R.stride(0), _ptr(mask_words), ldm,
                                                  _ptr(U), U.stride(0), _ptr(V), V.stride(0), _ptr(td), _ptr(ch),
                                                  C.byref(f)))
    return td, ch, f.value


def _options(sweeps=1, eps=0.0, window=0, select=0, precision=0, acol_p=5, seed=0, perm=None, picks=None,
             U0=None, trace=None, mlp=None, V0=None, selection="TD_A", strategy="ByRow", shapes=None):
    """shapes: (res_chunk, delta_blocks_per_sm[, delta_tile_rows]), the window
    evaluation's launch shapes (0: the library's choice)."""
    o = Options()
    load().stmf_default_options(C.byref(o))
    o.sweeps, o.eps, o.window, o.select, o.precision, o.acol_p, o.seed = (
        sweeps, eps, window, select, precision, acol_p, seed)
    o.selection = _selection(selection)
    o.strategy = _strategy(strategy)
    if shapes is not None:
        o.res_chunk, o.delta_blocks_per_sm = int(shapes[0]), int(shapes[1])
        o.delta_tile_rows = int(shapes[2]) if len(shapes) > 2 else 0
    keep = []
    if perm is not None:
        a = np.ascontiguousarray(perm, dtype=np.int32); keep.append(a); o.perm = a.ctypes.data
    if picks is not None:
        a = np.ascontiguousarray(picks, dtype=np.int32); keep.append(a); o.picks = a.ctypes.data
    if U0 is not None:
        _check_f32(U0, "U0"); keep.append(U0); o.U0 = U0.data_ptr()
    if trace is not None:
        keep.append(trace); o.trace = trace.ctypes.data; o.trace_cap = trace.shape[0]
    if mlp is not None:
        keep.append(mlp); o.mlp = mlp.h.value
    if V0 is not None:
        _check_f32(V0, "V0"); keep.append(V0); o.V0 = V0.data_ptr()
    return o, keep


class Problem:
    """A problem on the device: F-ULF / F-URF single updates (Algorithms 1, 2)."""

    def __init__(self, R, mask_words=None, rank=3, U0=None, seed=0, acol_p=5, picks=None):
        _check_f32(R, "R")
        self.ctx = context()
        m, n = R.shape
        self.m, self.n, self.r = m, n, rank
        o, keep = _options(seed=seed, acol_p=acol_p, picks=picks)
        h = C.c_void_p()
        ldm = mask_words.shape[1] if mask_words is not None else 0
        self.ctx.check(load().stmf_problem_create(self.ctx.h, m, n, rank, _ptr(R), R.stride(0), _ptr(mask_words),
                                                  ldm, _ptr(U0), C.byref(o), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().stmf_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _update(self, fn, i, j, k, commit_if_decreases):
        f = C.c_double()
        acc = C.c_int()
        self.ctx.check(fn(self.h, i, j, k, int(commit_if_decreases), C.byref(f), C.byref(acc)))
        return f.value, bool(acc.value)

    def update_U(self, i, j, k, commit_if_decreases=True):
        """F-ULF(i, j, k); returns (f', kept)."""
        return self._update(load().stmf_update_U, i, j, k, commit_if_decreases)

    def update_V(self, i, j, k, commit_if_decreases=True):
        """F-URF(i, j, k); returns (f', kept)."""
        return self._update(load().stmf_update_V, i, j, k, commit_if_decreases)

    def get(self):
        torch = _torch()
        U = torch.empty((self.m, self.r), device="cuda", dtype=torch.float32)
        V = torch.empty((self.r, self.n), device="cuda", dtype=torch.float32)
        f = C.c_double()
        self.ctx.check(load().stmf_problem_get(self.h, _ptr(U), _ptr(V), C.byref(f)))
        return U, V, f.value


def decode_trace(trace: np.ndarray):
    """Trace records -> list of (sweep, row, pos, j, k, type, f)."""
    out = []
    for rec in trace:
        f = struct.unpack("<d", struct.pack("<ii", int(rec[6]), int(rec[7])))[0]
        out.append((int(rec[0]), int(rec[1]), int(rec[2]), int(rec[3]), int(rec[4]), int(rec[5]), f))
    return out


def sweep_log(trace):
    """Per-sweep summary of trace records (one JSON-ready dict per sweep, in
    sweep order): records ("rows": the rows visited for ByRow; the kept
    updates plus the end-of-sweep record for ByElement; 1 per iteration for
    ByMatrix, whose "sweep" is an iteration), updates kept, the b-norm error
    after the sweep, and the mean position of the kept candidates (in their
    row's order; ByElement: element positions i*n + j; ByMatrix: positions in
    the err order)."""
    acc = {}
    for (sw, row, pos, j, k, typ, f) in trace:
        d = acc.setdefault(sw, {"sweep": sw, "rows": 0, "accepted": 0, "f": f, "pos_sum": 0})
        d["rows"] += 1
        d["f"] = f
        if pos >= 0:
            d["accepted"] += 1
            d["pos_sum"] += pos
    return [{"sweep": d["sweep"], "rows": d["rows"], "accepted": d["accepted"], "f": d["f"],
             "mean_kept_position": d["pos_sum"] / d["accepted"] if d["accepted"] else None}
            for _, d in sorted(acc.items())]


def factorize(R, mask_words=None, rank=3, sweeps=1, eps=0.0, window=0, select=0, precision=0, acol_p=5,
              seed=0, perm=None, picks=None, U0=None, trace_cap=0, mlp=None, V0=None, selection="TD_A",
              strategy="ByRow", shapes=None):
    """FastSTMF (Algorithm 3) on the device.  R: float32 CUDA (m x n).
    shapes: (res_chunk, delta_blocks_per_sm[, delta_tile_rows]) launch shapes, or None.
    mlp: an MLP (learned initialisation on the device) or None (Random Acol).
    selection: "TD_A" (the method as published), "TD_B", "TD" or "SEQ"
    (Section "The ByRow strategy").  strategy: "ByRow" (Algorithm 3),
    "ByElement" (STMF_ByElement_PermC_TD_W; trace records per kept update) or
    "ByMatrix" (STMF_ByMatrix_NoPerm_TD_W; `sweeps` counts its iterations).

    Returns (U m x r, V r x n, report dict, trace list or None)."""
    torch = _torch()
    _check_f32(R, "R")
    m, n = R.shape
    ctx = context()
    trace = np.zeros((trace_cap, STMF_TRACE_INTS), np.int32) if trace_cap else None
    o, keep = _options(sweeps, eps, window, select, precision, acol_p, seed, perm, picks, U0, trace, mlp, V0,
                       selection, strategy, shapes)
    U = torch.empty((m, rank), device=R.device, dtype=torch.float32)
    V = torch.empty((rank, n), device=R.device, dtype=torch.float32)
    rep = Report()
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_factorize(ctx.h, m, n, rank, _ptr(R), R.stride(0), _ptr(mask_words), ldm, C.byref(o),
                                    _ptr(U), _ptr(V), C.byref(rep)))
    tr = None
    if trace is not None:
        tr = decode_trace(trace[:min(trace_cap, rep.trace_records)])
    return U, V, rep.as_dict(), tr


def factorize_batched(problems, window=0, select=0, eps=0.0, precision=0, mlp=None, selection="TD_A",
                      strategy="ByRow"):
    """Many independent problems in one device launch (stmf_factorize_batched).

    problems: list of dicts with R (float32 CUDA m x n), mask_words (or None),
    rank, sweeps, seed and optionally trace_cap.  window=0 lets the library's
    autotuner choose each problem's window.  Returns (list of (U, V, report
    dict), tuned windows); a problem with trace_cap > 0 gets its decoded trace
    records in report["trace"]."""
    torch = _torch()
    ctx = context()
    n = len(problems)
    arr = (BatchProblem * max(n, 1))()
    outs = []
    for q, pr in enumerate(problems):
        R = pr["R"]
        _check_f32(R, "R")
        m, nn = R.shape
        r = pr["rank"]
        U = torch.empty((m, r), device=R.device, dtype=torch.float32)
        V = torch.empty((r, nn), device=R.device, dtype=torch.float32)
        mw = pr.get("mask_words")
        cap = int(pr.get("trace_cap", 0))
        tr = np.zeros((cap, STMF_TRACE_INTS), np.int32) if cap else None
        arr[q] = BatchProblem(m, nn, r, R.data_ptr(), R.stride(0), 0 if mw is None else mw.data_ptr(),
                              0 if mw is None else mw.shape[1], U.data_ptr(), V.data_ptr(), pr.get("seed", 0),
                              pr.get("sweeps", 1), 0 if tr is None else tr.ctypes.data, cap)
        outs.append((U, V, tr))
    o, keep = _options(0, eps, window, select, precision, mlp=mlp, selection=selection, strategy=strategy)
    reps = (Report * max(n, 1))()
    tuned = (C.c_int * max(n, 1))()
    ctx.check(load().stmf_factorize_batched(ctx.h, n, arr, C.byref(o), reps, tuned))
    res = []
    for q, (U, V, tr) in enumerate(outs):
        rep = reps[q].as_dict()
        if tr is not None:
            rep["trace"] = decode_trace(tr[:min(len(tr), rep["trace_records"])])
        res.append((U, V, rep))
    return res, [tuned[q] for q in range(n)]


def row_sketch(R, mask_words=None):
    """(sketch m x 32, median m): nearest-rank quantiles of each row's given
    entries, centred on the row median (stmf_row_sketch)."""
    torch = _torch()
    _check_f32(R, "R")
    m, n = R.shape
    ctx = context()
    sk = torch.empty((m, 32), device=R.device, dtype=torch.float32)
    md = torch.empty(m, device=R.device, dtype=torch.float32)
    ldm = mask_words.shape[1] if mask_words is not None else 0
    ctx.check(load().stmf_row_sketch(ctx.h, m, n, _ptr(R), R.stride(0), _ptr(mask_words), ldm, _ptr(sk), _ptr(md)))
    return sk, md


def mlp_targets(U, V, median, sorted_rows=False):
    """Training targets (m x r) of the learned initialisation from a
    factorization U (m x r), V (r x n) and the row medians (stmf_mlp_targets):
    gauge fixed by max_t V_lt = 0, components in decreasing order of their
    row sums; sorted_rows: each row's values in decreasing order instead."""
    torch = _torch()
    _check_f32(U, "U")
    _check_f32(V, "V")
    if median.dtype != torch.float32 or not median.is_cuda or median.dim() != 1 or median.stride(0) != 1:
        raise TypeError("median must be a contiguous 1-D float32 CUDA tensor")
    m, r = U.shape
    if V.shape[0] != r or median.shape[0] != m:
        raise ValueError("U, V and median disagree in shape")
    ctx = context()
    T = torch.empty((m, r), device=U.device, dtype=torch.float32)
    ctx.check(load().stmf_mlp_targets(ctx.h, m, V.shape[1], r, _ptr(U), U.stride(0), _ptr(V), V.stride(0),
                                      _ptr(median), int(bool(sorted_rows)), _ptr(T)))
    return T


def assign_by_rank(Y, U_ref):
    """out[s][l] = the value of Y[s] whose rank in its row (decreasing) is the
    rank of U_ref[s][l] in its row (decreasing, equal values: smaller index
    first) (stmf_assign_by_rank)."""
    torch = _torch()
    _check_f32(Y, "Y")
    _check_f32(U_ref, "U_ref")
    if Y.shape != U_ref.shape:
        raise ValueError("Y and U_ref differ in shape")
    m, r = Y.shape
    ctx = context()
    out = torch.empty((m, r), device=Y.device, dtype=torch.float32)
    ctx.check(load().stmf_assign_by_rank(ctx.h, m, r, _ptr(Y), Y.stride(0), _ptr(U_ref), U_ref.stride(0),
                                         _ptr(out), r))
    return out


class MLP:
    """The learned-initialisation network on the device (stmf_mlp_*)."""

    def __init__(self, rank, params):
        self.ctx = context()
        self.r = rank
        self.np = load().stmf_mlp_param_count(rank)
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.np
        h = C.c_void_p()
        self.ctx.check(load().stmf_mlp_create(self.ctx.h, rank, p.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().stmf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.np, np.float32)
        self.ctx.check(load().stmf_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, X):
        torch = _torch()
        X = X.contiguous()
        Y = torch.empty((X.shape[0], self.r), device=X.device, dtype=torch.float32)
        self.ctx.check(load().stmf_mlp_forward(self.h, X.shape[0], _ptr(X), _ptr(Y)))
        return Y

    def predict(self, R, mask_words=None):
        """U0 (m x r) = MLP(row sketch of R) + row median (stmf_mlp_predict)."""
        torch = _torch()
        _check_f32(R, "R")
        m, n = R.shape
        U0 = torch.empty((m, self.r), device=R.device, dtype=torch.float32)
        ldm = mask_words.shape[1] if mask_words is not None else 0
        self.ctx.check(load().stmf_mlp_predict(self.h, m, n, _ptr(R), R.stride(0), _ptr(mask_words), ldm,
                                               _ptr(U0)))
        return U0

    def gradient(self, X, T):
        g = np.empty(self.np, np.float32)
        loss = C.c_double()
        X, T = X.contiguous(), T.contiguous()
        self.ctx.check(load().stmf_mlp_gradient(self.h, X.shape[0], _ptr(X), _ptr(T), C.byref(loss),
                                                g.ctypes.data_as(C.c_void_p)))
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = C.c_double()
        self.ctx.check(load().stmf_mlp_train_step(self.h, X.shape[0], _ptr(X), _ptr(T), C.c_float(lr),
                                                  C.byref(loss)))
        return loss.value


class Factorization:
    """FastSTMF on one live problem, run in pieces (stmf_factorize_begin / _run / _end).

    ``run(sweeps)`` adds sweeps; ``result()`` returns (U, V) in the caller's
    orientation; ``report`` holds the cumulative counters."""

    def __init__(self, R, mask_words=None, rank=3, window=0, select=0, precision=0, acol_p=5, seed=0,
                 perm=None, picks=None, U0=None, trace_cap=0, mlp=None, V0=None, selection="TD_A",
                 strategy="ByRow", shapes=None):
        _check_f32(R, "R")
        self.ctx = context()
        self.m, self.n, self.r = R.shape[0], R.shape[1], rank
        self.trace = np.zeros((trace_cap, STMF_TRACE_INTS), np.int32) if trace_cap else None
        o, self._keep = _options(0, 0.0, window, select, precision, acol_p, seed, perm, picks, U0, self.trace,
                                 mlp, V0, selection, strategy, shapes)
        h = C.c_void_p()
        ldm = mask_words.shape[1] if mask_words is not None else 0
        self.ctx.check(load().stmf_factorize_begin(self.ctx.h, self.m, self.n, rank, _ptr(R), R.stride(0),
                                                   _ptr(mask_words), ldm, C.byref(o), C.byref(h)))
        self.h = h
        self.report = None

    def run(self, sweeps, eps=0.0):
        rep = Report()
        self.ctx.check(load().stmf_factorize_run(self.h, sweeps, eps, C.byref(rep)))
        self.report = rep.as_dict()
        return self.report

    def result(self):
        torch = _torch()
        U = torch.empty((self.m, self.r), device="cuda", dtype=torch.float32)
        V = torch.empty((self.r, self.n), device="cuda", dtype=torch.float32)
        cap = 0 if self.trace is None else self.trace.shape[0]
        tp = None if self.trace is None else C.c_void_p(self.trace.ctypes.data)
        self.ctx.check(load().stmf_factorize_end(self.h, _ptr(U), _ptr(V), tp, cap))
        return U, V

    def trace_records(self):
        if self.trace is None or self.report is None:
            return []
        return decode_trace(self.trace[:min(self.trace.shape[0], self.report["trace_records"])])

    def close(self):
        if getattr(self, "h", None):
            load().stmf_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def peak_addmax(mode=0, iters=4096):
    """Measured FP32 add+max issue rate in Gop/s (see stmf_peak_addmax)."""
    ctx = context()
    g = C.c_double()
    ctx.check(load().stmf_peak_addmax(ctx.h, mode, iters, C.byref(g)))
    return g.value
