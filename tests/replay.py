"""Decision-replay harness: runs the oracle in lockstep with a GPU trace.

At each row visit the oracle takes its own ByRow step from the same state.
Where its decision differs from the GPU's, the difference is accepted only
when floating-point order can explain it: the two kept candidates' errors
agree within ``tol`` relative, or either one lies within ``tol`` relative of
the error before the row (a near-tie with "f decreases").  The oracle then
adopts the GPU's decision (it applies the same F-ULF / F-URF itself, which in
FP32 mode reproduces the GPU's factors bit for bit) and continues.
"""

import oracle as orc


def replay(R, M, r, gpu_trace, seed=0, perm=None, picks=None, p=5, tol=1e-6, U0=None, selection="TD_A",
           state=None):
    """state (optional): (U, V) in the caller's frame, the factors the GPU held
    before its first traced row visit (a run resumed mid-way); the oracle
    starts from them instead of its own initialisation.  The result's
    "tried" lists the candidates the oracle tried at each row visit."""
    st = orc.prepare(R, M, r, perm=perm, picks=picks, p=p, seed=seed, U0=U0)
    Ri, Mi, Ui, Vi = st["R"], st["M"], st["U"], st["V"]
    if state is not None:
        import numpy as np
        Us, Vs = (np.asarray(x, dtype=np.float64) for x in state)
        if st["transposed"]:
            Us, Vs = Vs.T, Us.T
        Ui = np.ascontiguousarray(Us[st["perm"]])
        Vi = np.ascontiguousarray(Vs)
    f = orc.error(Ri, Mi, Ui, Vi)
    divergences, tried = [], []
    for rec in gpu_trace:
        sweep, i, pos, j, k, typ, f_gpu = rec
        U0_, V0_ = Ui.copy(), Vi.copy()
        kept, fn, out, nt = orc.row_step(Ri, Mi, Ui, Vi, i, f, selection=selection)
        tried.append(nt)
        gpu_kept = pos >= 0
        same = (kept == gpu_kept) and (not kept or tuple(out) == (pos, j, k, typ))
        if same:
            f = fn
            assert abs(f_gpu - f) <= tol * max(f, 1e-30), (rec, f)
            continue
        f_old = f
        f_orc = fn if kept else f_old
        if gpu_kept:
            fun = orc.fulf if typ == 0 else orc.furf
            Ug, Vg, f_g = fun(Ri, Mi, U0_, V0_, i, j, k)
        else:
            Ug, Vg, f_g = U0_, V0_, f_old
        scale = tol * max(f_old, 1e-30)
        ok = abs(f_g - f_orc) <= scale or abs(f_g - f_old) <= scale or abs(f_orc - f_old) <= scale
        assert ok, ("decision differs beyond tolerance", rec, out, kept, f_old, f_orc, f_g)
        divergences.append((rec, out, f_old, f_orc, f_g))
        Ui, Vi, f = Ug, Vg, f_g
    U, V = orc.finish(R.shape[0], R.shape[1], st["transposed"], Ui, Vi, st["perm"])
    return dict(U=U, V=V, f=f, divergences=divergences, perm=st["perm"], transposed=st["transposed"], tried=tried)


def replay_byelement(R, M, r, gpu_trace, seed=0, picks=None, p=5, tol=1e-6):
    """The same lockstep replay for the ByElement method: at each GPU record
    (a kept update, or the end of a sweep) the oracle scans from its own
    position to its first kept update; a different outcome is accepted only
    as a near-tie within ``tol`` relative, and the oracle then adopts the
    GPU's outcome."""
    import numpy as np
    R = np.asarray(R, dtype=np.float64)
    M = np.asarray(M, dtype=bool)
    tr = R.shape[0] > R.shape[1]
    Ro, Mo = (R.T.copy(), M.T.copy()) if tr else (R, M)
    cp = orc.colmin_perm(Ro, Mo)
    Rc, Mc = Ro[:, cp].copy(), Mo[:, cp].copy()
    m = Rc.shape[0]
    st = orc.prepare(Rc, Mc, r, perm=np.arange(m, dtype=np.int32), picks=picks, p=p, seed=seed)
    Ri, Mi, Ui, Vi = st["R"], st["M"], st["U"], st["V"]
    f = orc.error(Ri, Mi, Ui, Vi)
    q = 0
    divergences = []
    for rec in gpu_trace:
        sweep, i, pos, j, k, typ, f_gpu = rec
        U0_, V0_ = Ui.copy(), Vi.copy()
        got, fn, out, _ = orc.element_scan(Ri, Mi, Ui, Vi, q, f)
        gpu_kept = i >= 0
        same = (got >= 0) == gpu_kept and (not gpu_kept or (got == pos and out == (i, j, k, typ)))
        if same:
            f = fn
            assert abs(f_gpu - f) <= tol * max(f, 1e-30), (rec, f)
            q = got + 1 if gpu_kept else 0
            continue
        f_old = f
        f_orc = fn if got >= 0 else f_old
        if gpu_kept:
            fun = orc.fulf if typ == 0 else orc.furf
            Ug, Vg, f_g = fun(Ri, Mi, U0_, V0_, i, j, k)
        else:
            Ug, Vg, f_g = U0_, V0_, f_old
        scale = tol * max(f_old, 1e-30)
        ok = abs(f_g - f_orc) <= scale or abs(f_g - f_old) <= scale or abs(f_orc - f_old) <= scale
        assert ok, ("decision differs beyond tolerance", rec, got, out, f_old, f_orc, f_g)
        divergences.append((rec, got, out, f_old, f_orc, f_g))
        Ui, Vi, f = Ug, Vg, f_g
        q = pos + 1 if gpu_kept else 0
    Vo = np.empty_like(Vi)
    Vo[:, cp] = Vi
    U, V = (Vo.T.copy(), Ui.T.copy()) if tr else (Ui, Vo)
    return dict(U=U, V=V, f=f, divergences=divergences, transposed=tr, cperm=cp)


def replay_bymatrix(R, M, r, gpu_trace, seed=0, picks=None, p=5, tol=1e-6):
    """The lockstep replay for the ByMatrix method: one GPU record per
    iteration (the kept element's position in the err order, or none); the
    oracle runs the same iteration from its own state."""
    import numpy as np
    R = np.asarray(R, dtype=np.float64)
    M = np.asarray(M, dtype=bool)
    m0, n0 = R.shape
    tr = m0 > n0
    m = n0 if tr else m0
    st = orc.prepare(R, M, r, perm=np.arange(m, dtype=np.int32), picks=picks, p=p, seed=seed)
    Ri, Mi, Ui, Vi = st["R"], st["M"], st["U"], st["V"]
    f = orc.error(Ri, Mi, Ui, Vi)
    divergences = []
    for rec in gpu_trace:
        it, i, pos, j, k, typ, f_gpu = rec
        U0_, V0_ = Ui.copy(), Vi.copy()
        kept, fn, out, _ = orc.matrix_step(Ri, Mi, Ui, Vi, seed, it, f)
        gpu_kept = pos >= 0
        same = kept == gpu_kept and (not kept or tuple(out) == (pos, i, j, k, typ))
        if same:
            f = fn
            assert abs(f_gpu - f) <= tol * max(f, 1e-30), (rec, f)
            continue
        f_old = f
        f_orc = fn if kept else f_old
        if gpu_kept:
            fun = orc.fulf if typ == 0 else orc.furf
            Ug, Vg, f_g = fun(Ri, Mi, U0_, V0_, i, j, k)
        else:
            Ug, Vg, f_g = U0_, V0_, f_old
        scale = tol * max(f_old, 1e-30)
        ok = abs(f_g - f_orc) <= scale or abs(f_g - f_old) <= scale or abs(f_orc - f_old) <= scale
        assert ok, ("decision differs beyond tolerance", rec, out, kept, f_old, f_orc, f_g)
        divergences.append((rec, out, f_old, f_orc, f_g))
        Ui, Vi, f = Ug, Vg, f_g
    U, V = orc.finish(m0, n0, st["transposed"], Ui, Vi, st["perm"])
    return dict(U=U, V=V, f=f, divergences=divergences)
