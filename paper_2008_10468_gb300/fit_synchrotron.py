"""Offline generator of the binary32 tables used by the CUDA library.

Writes ``csrc/synchro_coeffs.h``.  Run once when the approximation scheme
changes:  ``python -m paper_2008_10468_gb300.fit_synchrotron``.

1. Synchrotron functions (Sec. 3.2.1).  The paper approximates
   G(x) = x K_{2/3}(x) by a series for small x, by x^{1/3} M~ - x^{5/3} P~ for
   medium x and by x^{1/2} e^{-x} L~(1/x) for large x, with minimax (Remez)
   polynomials (Sec. 3.2.1, Table 1); it states the scheme carries over to
   F(x) = x int_x^inf K_{5/3}.  In binary32 the medium-range difference
   x^{1/3} M - x^{5/3} P cancels badly (a factor ~10^3 at x = 4), so here both
   functions use one branch-free form on every octave of x:

       F(x) = x^{1/3} * exp(-lam_k x) * sum_j c_{k,j} t^j,
       t = log2(x) - k  for x in [2^k, 2^(k+1)),  k = KMIN .. KMAX,

   with lam_k = 0 below x = 1/2 (where F / x^{1/3} is a power series in
   x^{2/3}, the paper's M and P parts) and lam_k = 1 from x = 1/2 (the paper's
   e^{-x} envelope).  In the log variable the nearest singularity of F(e^s) is
   at Im s = +-pi, so a degree-5 polynomial per octave reaches ~1e-7.  Below
   x = 2^KMIN one extra piece uses t = x^{2/3} (the paper's small-x series).
   Coefficients are discrete Remez (minimax relative error) fits, rounded to
   binary32.

2. Rejection squeeze.  The acceptance test y < P(x) of Algorithms 1 and 2
   only needs P when y is below an upper bound of P over all x.  For each
   octave of b = 3 chi / 2 we store H = 1.02 * max over the octave of
   sup_x P(x; b) / (c b^{2/3}).

The target values come from mpmath: G from the modified Bessel functions I_nu
of the paper's definition (Sec. 3.2.1), F from F = 2G - (pi/sqrt3) x +
x int_0^x K_{1/3} with the K_{1/3} series integrated term by term, both at a
working precision that absorbs the cancellation of the series for large x.
"""
import math
import os
import sys

import numpy as np

try:
    import mpmath as mp
except ImportError:  # pragma: no cover
    mp = None

KMIN, KMAX = -14, 6            # octaves [2^k, 2^(k+1)), k = KMIN..KMAX
LAMBDA_FROM = -1               # lam_k = 1 for k >= LAMBDA_FROM (x >= 1/2)
DEG = 5
NPIECE = KMAX - KMIN + 2       # + the small-x piece
T_LO, T_HI = -0.02, 1.02       # fit range of t (covers log2 rounding at edges)
GRID = 401

# squeeze tables
B_OCT_MIN_E, B_OCT_MAX_E = -40, 16
B_OCT_MIN_P, B_OCT_MAX_P = -8, 16
SQUEEZE_MARGIN = 1.02

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "synchro_coeffs.h")


# --------------------------------------------------------------------------
# Targets in extended precision
# --------------------------------------------------------------------------
def _dps_for(x):
    return int(40 + 0.9 * float(x))


def G_mp(x):
    """G(x) = (pi x / 2) (I_{-2/3}(x) - I_{2/3}(x)) / sin(2 pi / 3)."""
    with mp.workdps(_dps_for(x)):
        x = mp.mpf(x)
        a = mp.mpf(2) / 3
        return +(mp.pi * x / 2 * (mp.besseli(-a, x) - mp.besseli(a, x)) / mp.sin(2 * mp.pi / 3))


def _int_I(alpha, x):
    """int_0^x I_alpha(t) dt = sum_n (1/2)^(2n+alpha) x^(2n+alpha+1) / ((2n+alpha+1) n! Gamma(n+alpha+1))."""
    s = mp.mpf(0)
    n = 0
    while True:
        e = 2 * n + alpha
        term = (x / 2) ** e * x / ((e + 1) * mp.factorial(n) * mp.gamma(n + alpha + 1))
        s += term
        if n > 5 and abs(term) < abs(s) * mp.mpf(10) ** (-mp.mp.dps):
            return s
        n += 1


def F_mp(x):
    """F(x) = x int_x^inf K_{5/3} = 2 G(x) - (pi/sqrt3) x + x int_0^x K_{1/3}."""
    with mp.workdps(_dps_for(x)):
        x = mp.mpf(x)
        third = mp.mpf(1) / 3
        k13 = mp.pi / (2 * mp.sin(mp.pi / 3)) * (_int_I(-third, x) - _int_I(third, x))
        return +(2 * G_mp(x) - mp.pi / mp.sqrt(3) * x + x * k13)


def _self_check():
    """Cross-check the series targets against mpmath's K_nu and quadrature."""
    for x in (1e-5, 0.3, 2.0, 17.0, 90.0):
        g_ref = mp.mpf(x) * mp.besselk(mp.mpf(2) / 3, x)
        assert abs(G_mp(x) / g_ref - 1) < 1e-20, x
    for x in (1e-3, 0.7, 5.0):
        with mp.workdps(30):
            f_ref = x * mp.quad(lambda t: mp.besselk(mp.mpf(5) / 3, t), [x, x + 2, mp.inf])
        assert abs(F_mp(x) / f_ref - 1) < 1e-15, x


# --------------------------------------------------------------------------
# Discrete Remez for minimax relative error
# --------------------------------------------------------------------------
def remez_relative(t, q, deg, iters=60):
    """Coefficients c (power basis in t) minimising max |p(t)/q - 1| over the grid."""
    n = deg + 1
    m = len(t)
    # initial reference: Chebyshev-like points
    idx = np.unique(np.round((1 - np.cos(np.linspace(0, np.pi, n + 1))) / 2 * (m - 1)).astype(int))
    while len(idx) < n + 1:
        idx = np.unique(np.concatenate([idx, [m // 2 + len(idx)]]))
    best = None
    for _ in range(iters):
        A = np.zeros((n + 1, n + 1))
        for r, i in enumerate(idx):
            A[r, :n] = t[i] ** np.arange(n)
            A[r, n] = (-1) ** r * q[i]
        sol = np.linalg.solve(A, q[idx])
        c = sol[:n]
        err = (np.polyval(c[::-1], t) - q) / q
        emax = np.max(np.abs(err))
        if best is None or emax < best[1]:
            best = (c.copy(), emax)
        # exchange: extrema of alternating-sign runs
        sgn = np.sign(err)
        sgn[sgn == 0] = 1
        runs = []
        start = 0
        for i in range(1, m + 1):
            if i == m or sgn[i] != sgn[start]:
                j = start + int(np.argmax(np.abs(err[start:i])))
                runs.append(j)
                start = i
        while len(runs) > n + 1:
            # drop the smaller end or merge the smallest pair
            a = [abs(err[j]) for j in runs]
            if a[0] <= a[-1]:
                runs.pop(0)
            else:
                runs.pop()
        if len(runs) < n + 1:
            break
        new = np.array(runs)
        if np.array_equal(new, idx):
            break
        idx = new
    return best


def fit_piece(k):
    """Return (coef[2][DEG+1], lam, max_rel_err_fp32) for piece k (None -> small-x)."""
    if k is None:
        vmax = (2.0 ** KMIN) ** (2.0 / 3.0) * 1.02
        t = np.linspace(0.0, vmax, GRID)
        x = np.maximum(t, 1e-300) ** 1.5
        lam = 0.0
    else:
        t = np.linspace(T_LO, T_HI, GRID)
        x = 2.0 ** (k + t)
        lam = 1.0 if k >= LAMBDA_FROM else 0.0
    coefs, errs = [], []
    for fun in (F_mp, G_mp):
        q = []
        for xv, tv in zip(x, t):
            if k is None and tv == 0.0:
                xv = 1e-40
            with mp.workdps(_dps_for(xv)):
                val = fun(mp.mpf(xv)) * mp.exp(lam * mp.mpf(xv)) / mp.cbrt(mp.mpf(xv))
            q.append(float(val))
        q = np.array(q)
        c, _ = remez_relative(t, q, DEG)
        c32 = c.astype(np.float32).astype(np.float64)
        e32 = np.max(np.abs(np.polyval(c32[::-1], t) / q - 1))
        coefs.append(c.astype(np.float32))
        errs.append(e32)
    return coefs, lam, max(errs)


# --------------------------------------------------------------------------
# Squeeze tables: sup over x of the acceptance functions divided by c
# --------------------------------------------------------------------------
def _eval_fit(coef_table, lam_table, x):
    """F, G from the fitted pieces in float64 (used only to locate maxima)."""
    x = np.asarray(x, dtype=np.float64)
    F = np.zeros_like(x)
    G = np.zeros_like(x)
    ok = (x > 0) & (x < 700)
    xv = x[ok]
    kraw = np.floor(np.log2(xv)).astype(int)
    small = kraw < KMIN
    piece = np.where(small, 0, np.clip(kraw, KMIN, KMAX) - KMIN + 1)
    t = np.where(small, np.cbrt(xv) ** 2, np.log2(xv) - np.clip(kraw, KMIN, KMAX))
    lam = lam_table[piece]
    env = np.cbrt(xv) * np.exp(-lam * xv)
    for which, out in ((0, F), (1, G)):
        c = coef_table[piece, which, :].astype(np.float64)
        acc = c[:, DEG]
        for j in range(DEG - 1, -1, -1):
            acc = acc * t + c[:, j]
        out[ok] = env * acc
    return F, G


def _sup_emission(b, ev):
    x = np.concatenate([np.logspace(-12, -1, 400), np.linspace(0.1, 1 - 1e-9, 1600)])
    d = x ** 3
    z = d / (b * (1 - d))
    F, G = ev(z)
    P = (b / x) * ((1 - d) * F + d * d * G)
    i = int(np.argmax(P))
    # refine around the grid maximum
    lo, hi = x[max(i - 1, 0)], x[min(i + 1, len(x) - 1)]
    xs = np.linspace(lo, hi, 401)
    d = xs ** 3
    z = d / (b * (1 - d))
    F, G = ev(z)
    return max(float(P[i]), float(np.max((b / xs) * ((1 - d) * F + d * d * G))))


def _sup_pair(b, ev):
    d = np.concatenate([np.logspace(-12, -1, 300), np.linspace(0.1, 0.5, 1200)])
    dd = d * (1 - d)
    z = 1.0 / (b * dd)
    F, G = ev(z)
    P = (b / 3) * (G - dd * F)
    i = int(np.argmax(P))
    lo, hi = d[max(i - 1, 0)], d[min(i + 1, len(d) - 1)]
    ds = np.linspace(lo, hi, 401)
    dd = ds * (1 - ds)
    z = 1.0 / (b * dd)
    F, G = ev(z)
    return max(float(P[i]), float(np.max((b / 3) * (G - dd * F))))


def squeeze_table(sup, oct_min, oct_max, ev):
    H = []
    for j in range(oct_min, oct_max):
        bs = 2.0 ** (j + np.linspace(0.0, 1.0, 65))
        h = max(sup(b, ev) / b ** (2.0 / 3.0) for b in bs)
        h32 = np.float32(h * SQUEEZE_MARGIN)
        if float(h32) < h * SQUEEZE_MARGIN:
            h32 = np.nextafter(h32, np.float32(np.inf))
        H.append(h32)
    return np.array(H, dtype=np.float32)


# --------------------------------------------------------------------------
def _c_float(v):
    v = float(v)
    if v == 0.0:
        return "0.0f"
    return "%.9ef" % v


def main():
    if mp is None:
        raise SystemExit("mpmath is required to regenerate the tables")
    mp.mp.dps = 40
    _self_check()
    coef = np.zeros((NPIECE, 2, DEG + 1), dtype=np.float32)
    lam = np.zeros(NPIECE, dtype=np.float32)
    report = []
    c, l, e = fit_piece(None)
    coef[0] = np.array(c)
    lam[0] = l
    report.append(("x < 2^%d" % KMIN, e))
    for k in range(KMIN, KMAX + 1):
        c, l, e = fit_piece(k)
        coef[k - KMIN + 1] = np.array(c)
        lam[k - KMIN + 1] = l
        report.append(("[2^%d, 2^%d)" % (k, k + 1), e))
        print("piece", k, "max rel err (binary32 coefficients) %.2e" % e, file=sys.stderr)
    ev = lambda z: _eval_fit(coef, lam, z)
    He = squeeze_table(_sup_emission, B_OCT_MIN_E, B_OCT_MAX_E, ev)
    Hp = squeeze_table(_sup_pair, B_OCT_MIN_P, B_OCT_MAX_P, ev)
    # small-b limit of sup_x 3x^2 P(x^3) / (c b^{2/3}): the x -> 0 value
    c_small = 4 * math.pi / (math.sqrt(3) * math.gamma(1 / 3) * 2 ** (1 / 3))

    L = []
    L.append("/* Generated by paper_2008_10468_gb300/fit_synchrotron.py.  Do not edit.")
    L.append(" *")
    L.append(" * Synchrotron functions F(x) = x int_x^inf K_{5/3} and G(x) = x K_{2/3}(x)")
    L.append(" * (Sec. 3.2.1) as x^{1/3} exp(-lam x) poly(t), one degree-%d polynomial per" % DEG)
    L.append(" * octave of x (t = log2 x - k), plus a small-x piece in t = x^{2/3}.")
    L.append(" * Max relative error of each piece with these binary32 coefficients,")
    L.append(" * evaluated exactly (the kernel adds its own rounding):")
    for name, e in report:
        L.append(" *   %-18s %.2e" % (name, e))
    L.append(" */")
    L.append("#pragma once")
    L.append("#ifndef QED_TABLE_ATTR")
    L.append("#define QED_TABLE_ATTR /* __device__ when compiled for the GPU */")
    L.append("#endif")
    L.append("#define QED_SYN_KMIN (%d)" % KMIN)
    L.append("#define QED_SYN_KMAX (%d)" % KMAX)
    L.append("#define QED_SYN_DEG %d" % DEG)
    L.append("#define QED_SYN_NPIECE %d" % NPIECE)
    L.append("/* piece 0: x < 2^KMIN; piece k - KMIN + 1: x in [2^k, 2^(k+1)) */")
    L.append("/* row layout: F coefficients c0..c5, G coefficients c0..c5, lam, 3 pad */")
    L.append("QED_TABLE_ATTR static const float qed_syn_table[QED_SYN_NPIECE][16] = {")
    for i in range(NPIECE):
        row = list(coef[i, 0]) + list(coef[i, 1]) + [lam[i], 0.0, 0.0, 0.0]
        L.append("  {" + ", ".join(_c_float(v) for v in row) + "},")
    L.append("};")
    L.append("")
    L.append("/* Rejection squeeze: sup_x of the acceptance function of Algorithm 1 (emission)")
    L.append(" * or Algorithm 2 (pair) divided by c b^{2/3}, maximised over each octave")
    L.append(" * [2^j, 2^(j+1)) of b = 3 chi / 2 and multiplied by %.2f. */" % SQUEEZE_MARGIN)
    L.append("#define QED_SQZ_E_JMIN (%d)" % B_OCT_MIN_E)
    L.append("#define QED_SQZ_E_JMAX (%d)" % B_OCT_MAX_E)
    L.append("#define QED_SQZ_P_JMIN (%d)" % B_OCT_MIN_P)
    L.append("#define QED_SQZ_P_JMAX (%d)" % B_OCT_MAX_P)
    L.append("#define QED_SQZ_E_SMALL %sf  /* b below the table: 1.02 x small-b limit */"
             % ("%.9e" % (c_small * SQUEEZE_MARGIN)))
    L.append("QED_TABLE_ATTR static const float qed_sqz_emission[%d] = {" % len(He))
    L.append("  " + ", ".join(_c_float(v) for v in He))
    L.append("};")
    L.append("QED_TABLE_ATTR static const float qed_sqz_pair[%d] = {" % len(Hp))
    L.append("  " + ", ".join(_c_float(v) for v in Hp))
    L.append("};")
    with open(OUT, "w") as f:
        f.write("\n".join(L) + "\n")
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
