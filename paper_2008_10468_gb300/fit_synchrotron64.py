"""Offline generator of the binary64 synchrotron tables (``csrc/synchro_coeffs64.h``).

Run once when the scheme changes:
``python -m paper_2008_10468_gb300.fit_synchrotron64``.

The double-precision companion of the binary32 functions (Sec. 3.2.1: the
paper fits its F and G forms to 1e-8 and to 1e-14 relative error, Table 1).
Its medium-range form x^{1/3} M - x^{5/3} P still cancels by ~10^3 near x = 4
in binary64, so this scheme, like the binary32 one, avoids the difference:

    x = m 2^k, m in [1, 2);  [1, 1.25), [1.25, 1.5), [1.5, 2) of an octave are pieces
    F(x) = 2^{k/3} * exp(-lam_k x) * sum_j c_j u^j,   u = (m - centre) / halfwidth in [-1, 1)

with lam_k = 0 below x = 1/2 and 1 from there (the large-x e^{-x} envelope).
The factor x^{1/3} of the small- and medium-x behaviour is split into the
per-octave constant 2^{k/3} and a part m^{1/3} that the polynomial absorbs, so
the evaluation needs neither a logarithm nor a cube root; u is exact in
binary64 (dyadic centres and half-widths).  The pieces are narrower near m = 1,
where the branch point of m^{1/3} at m = 0 is closest.  Below x = 2^KMIN one more piece is the small-x series
F = x^{1/3} * sum_j a_j v^j in v = x^{2/3} (the paper's S(x)).  Above 2^(KMAX+1)
the functions are below 1e-220 and the kernel returns 0.

Coefficients interpolate the target at Chebyshev nodes of u (solved at 60
digits), then are rounded to binary64; with degree 11 the evaluation error in
binary64 is a few units in the last place.  The targets are the binary32
generator's extended-precision series (this module does not use the oracle).
"""
import math
import os
import sys

import numpy as np

from . import fit_synchrotron as fs

try:
    import mpmath as mp
except ImportError:  # pragma: no cover
    mp = None

KMIN, KMAX = -14, 8        # octaves [2^k, 2^(k+1)), k = KMIN..KMAX
PARTS = ((1.125, 0.125), (1.375, 0.125), (1.75, 0.25))   # (centre, half-width) in m
LAMBDA_FROM = -1           # lam_k = 1 for k >= LAMBDA_FROM (x >= 1/2)
DEG = 11
SMALL_DEG = 6
NPIECE = 1 + len(PARTS) * (KMAX - KMIN + 1)

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "synchro_coeffs64.h")


def _nodes(n):
    return [mp.cos(mp.pi * (2 * i + 1) / (2 * n)) for i in range(n)]


def _interp(us, vals, deg):
    with mp.workdps(60):
        A = mp.matrix(deg + 1, deg + 1)
        b = mp.matrix(deg + 1, 1)
        for i, (u, v) in enumerate(zip(us, vals)):
            for j in range(deg + 1):
                A[i, j] = mp.mpf(u) ** j
            b[i] = v
        c = mp.lu_solve(A, b)
        return [float(c[j]) for j in range(deg + 1)]


def piece_target(fun, k, part, u):
    """fun(x) * exp(lam x) / 2^(k/3) at x = (centre + halfwidth u) 2^k."""
    centre, half = (mp.mpf(v) for v in PARTS[part])
    lam = 1 if k >= LAMBDA_FROM else 0
    with mp.workdps(60):
        x = (centre + half * mp.mpf(u)) * mp.power(2, k)
    xf = float(x)
    with mp.workdps(fs._dps_for(xf)):
        return fun(x) * mp.exp(lam * x) / mp.power(2, mp.mpf(k) / 3)


def fit_piece(k, part):
    us = _nodes(DEG + 1)
    return [_interp(us, [piece_target(fun, k, part, u) for u in us], DEG)
            for fun in (fs.F_mp, fs.G_mp)]


def fit_small():
    """F, G = x^{1/3} * sum_j a_j v^j, v = x^{2/3} in (0, 2^(2 KMIN / 3)]."""
    vmax = mp.power(2, mp.mpf(2 * KMIN) / 3)
    us = _nodes(SMALL_DEG + 1)
    out = []
    for fun in (fs.F_mp, fs.G_mp):
        vals, ts = [], []
        for u in us:
            with mp.workdps(60):
                v = vmax * (u + 1) / 2
                x = v ** mp.mpf(1.5)
            with mp.workdps(60):
                vals.append(fun(x) / mp.cbrt(x))
            ts.append(u)
        # polynomial in u, converted to the power basis in v
        cu = _interp(ts, vals, SMALL_DEG)
        with mp.workdps(60):
            # u = 2 v / vmax - 1: expand sum cu_j (2 v / vmax - 1)^j
            cv = [mp.mpf(0)] * (SMALL_DEG + 1)
            for j, c in enumerate(cu):
                for i in range(j + 1):
                    cv[i] += mp.mpf(c) * mp.binomial(j, i) * (2 / vmax) ** i * (-1) ** (j - i)
        out.append([float(c) for c in cv])
    return out


def eval64(table, x):
    """The kernel's evaluation in binary64 (numpy), for the fit check."""
    small, pieces = table
    x = float(x)
    if not (x > 0.0) or x >= 2.0 ** (KMAX + 1):
        return 0.0, 0.0
    m, e = math.frexp(x)          # x = m 2^e, m in [0.5, 1)
    k = e - 1
    m = 2.0 * m
    if k < KMIN:
        r = x ** (1.0 / 3.0)
        v = r * r
        res = []
        for f in range(2):
            p = 0.0
            for a in reversed(small[f]):
                p = p * v + a
            res.append(r * p)
        return tuple(res)
    part = 0 if m < 1.25 else (1 if m < 1.5 else 2)
    centre, half = PARTS[part]
    u = (m - centre) / half
    cf = pieces[(k - KMIN) * len(PARTS) + part]
    s = 2.0 ** (k / 3.0) * (math.exp(-x) if k >= LAMBDA_FROM else 1.0)
    res = []
    for f in range(2):
        p = 0.0
        for a in reversed(cf[f]):
            p = p * u + a
        res.append(s * p)
    return tuple(res)


def write_header(table, path=OUT):
    small, pieces = table
    lines = ["// Generated by paper_2008_10468_gb300/fit_synchrotron64.py -- do not edit.",
             "// Binary64 synchrotron functions F(x) = x int_x^inf K_{5/3}, G(x) = x K_{2/3}(x)",
             "// (Sec. 3.2.1): per piece [1, 1.25), [1.25, 1.5), [1.5, 2) of m in x = m 2^k,",
             "// F = 2^{k/3} exp(-lam x) sum_j c_j u^j with u = (m - centre) / halfwidth;",
             "// below 2^KMIN, F = x^{1/3} sum_j a_j (x^{2/3})^j.",
             "#pragma once",
             "#define QED_SYN64_KMIN (%d)" % KMIN,
             "#define QED_SYN64_KMAX %d" % KMAX,
             "#define QED_SYN64_LAMBDA_FROM (%d)" % LAMBDA_FROM,
             "#define QED_SYN64_DEG %d" % DEG,
             "#define QED_SYN64_SMALL_DEG %d" % SMALL_DEG,
             "#define QED_SYN64_NPIECE %d" % (len(pieces)),
             "// [piece][F coefficients 0..DEG, G coefficients 0..DEG], piece = 3 (k - KMIN) + part",
             "static __device__ const double qed_syn64_table[QED_SYN64_NPIECE][2 * (QED_SYN64_DEG + 1)] = {"]
    for cf in pieces:
        vals = cf[0] + cf[1]
        lines.append("    {" + ", ".join("%.17g" % v for v in vals) + "},")
    lines.append("};")
    lines.append("static __device__ const double qed_syn64_small[2][QED_SYN64_SMALL_DEG + 1] = {")
    for f in range(2):
        lines.append("    {" + ", ".join("%.17g" % v for v in small[f]) + "},")
    lines.append("};")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main():
    if mp is None:
        sys.exit("mpmath is required")
    mp.mp.dps = 50
    fs._self_check()
    pieces = []
    for k in range(KMIN, KMAX + 1):
        for part in range(len(PARTS)):
            pieces.append(fit_piece(k, part))
            print("piece k=%d part=%d" % (k, part), flush=True)
    table = (fit_small(), pieces)
    # check: random points per piece against the targets
    rng = np.random.default_rng(20081046)
    worst = 0.0
    for k in range(KMIN - 3, KMAX + 1):
        for _ in range(12):
            x = float(2.0 ** (k + rng.random()))
            F, G = eval64(table, x)
            with mp.workdps(fs._dps_for(x)):
                rf = float(fs.F_mp(mp.mpf(x)))
                rg = float(fs.G_mp(mp.mpf(x)))
            worst = max(worst, abs(F / rf - 1), abs(G / rg - 1))
    print("max relative error of the binary64 evaluation: %.3e" % worst)
    write_header(table)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
