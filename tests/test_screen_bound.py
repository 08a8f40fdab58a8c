"""CPU pins of two arithmetic facts the GPU path relies on, checked on the
oracle's own F-ULF / F-URF candidates (no GPU code is involved).

1. Residuation keeps U (x) V <= R on given entries, so a candidate's change
   of an entry's b-norm term, |R - P'| - |R - P1|, equals P1 - P'.  In FP32
   the two forms may differ by a few ulps (a value can round an ulp above R);
   an entry the candidate leaves unchanged gives exactly 0 in both.
2. The FP16 screen: with R, P1, P2 and x = fl32(u' + v') rounded to nearest
   half, the half term |R_h - max(E_h, x_h)| - |R_h - P1_h| (each operation
   rounded to half) is within 6.01 u_h M + 2^-22 of the exact term, and every
   entry whose term is non-zero in either form lies in S = {A = k} u
   {x_h >= E_h}.
"""
import numpy as np

from paper_2205_06619_gb300 import synth

UH = 2.0 ** -11


def half(x):
    """Round to nearest half (from exact float64 values)."""
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def _cases(orc):
    out = []
    for name, (R, M), r in [("uniform", synth.uniform_planted(60, 90, 3, 0.01, 0.8, 3)[:2], 3),
                            ("lognormal", synth.lognormal_planted(50, 120, 6, 0.05, 0.7, 4)[:2], 6),
                            ("dyadic", synth.dyadic_noise(40, 70, 0.6, 5), 4)]:
        st = orc.prepare(R, M, r, seed=1)
        Ri, Mi, U, V = st["R"], st["M"], st["U"], st["V"]
        rng = np.random.default_rng(7)
        for _ in range(12):
            i = int(rng.integers(Ri.shape[0]))
            j = int(rng.choice(np.nonzero(Mi[i])[0]))
            k = int(rng.integers(r))
            for fn in (orc.fulf, orc.furf):
                U2, V2, _ = fn(Ri, Mi, U, V, i, j, k, "fp32")
                out.append((name, Ri, Mi, U, V, U2[:, k], V2[k], k))
    return out


def _planes(orc, U, V, k, u, v):
    P1, A, P2 = orc.maxplus(U, V, "fp32")
    x = (u.astype(np.float32)[:, None] + v.astype(np.float32)[None, :]).astype(np.float64)   # fl32(u + v)
    E = np.where(A == k, P2, P1)
    return P1, A, P2, x, E


def test_change_identity_under_residuation(orc):
    for name, R, M, U, V, u, v, k in _cases(orc):
        P1, A, P2, x, E = _planes(orc, U, V, k, u, v)
        Pp = np.maximum(E, x)
        f32 = np.float32
        lit = (np.abs(R.astype(f32) - Pp.astype(f32)) - np.abs(R.astype(f32) - P1.astype(f32))).astype(np.float64)
        new = (P1.astype(f32) - Pp.astype(f32)).astype(np.float64)
        mag = np.abs(R) + np.abs(Pp) + np.abs(P1)
        diff = np.abs(lit - new)[M]
        assert np.all(diff <= 4.0 * 2.0 ** -23 * mag[M]), name
        same = (Pp == P1) & M
        assert np.all(lit[same] == 0) and np.all(new[same] == 0)
        # the summed change moves by far less than the 1e-6 tolerance
        assert abs(np.sum(lit[M]) - np.sum(new[M])) <= 1e-6 * max(np.sum(np.abs(lit[M])), 1e-30)


def test_half_screen_term_within_bound_and_support(orc):
    worst = 0.0
    for name, R, M, U, V, u, v, k in _cases(orc):
        P1, A, P2, x, E = _planes(orc, U, V, k, u, v)
        given = M
        Pp = np.maximum(E, x)
        exact = np.abs(R - Pp) - np.abs(R - P1)
        Rh, P1h, P2h, xh = half(R), half(P1), half(P2), half(x)
        Eh = np.where(A == k, P2h, P1h)
        Pph = np.maximum(Eh, xh)
        assert np.array_equal(Pph, half(Pp))             # rn is monotone: max commutes with it
        ah = np.abs(half(Rh - Pph))
        t0h = np.abs(half(Rh - P1h))
        dh = half(ah - t0h)
        finite_p2 = np.isfinite(P2)
        Mbound = np.abs(R[given]).max() + max(np.abs(P1[given]).max(), np.abs(P2[given & finite_p2]).max(),
                                             np.abs(u).max() + np.abs(v).max())
        bound = 6.01 * UH * Mbound + 2.0 ** -22
        err = np.abs(dh - exact)[given]
        assert np.all(err <= bound), (name, err.max(), bound)
        worst = max(worst, float(err.max() / bound))
        S = given & ((A == k) | (xh >= Eh))
        nonzero = given & ((exact != 0) | (dh != 0))
        assert not np.any(nonzero & ~S), name
    # the bound is not vacuous: the worst entry reaches about a tenth of it
    # (0.63 u_h M observed against 6.01 u_h M)
    assert worst > 0.05
