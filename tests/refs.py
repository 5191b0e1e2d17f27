"""Independent references for the oracle pins: scipy library routines and
closed forms from the literature.  Nothing here calls the oracle."""
import numpy as np
from scipy import integrate, special

SQRT3 = np.sqrt(3.0)


def F2_ref(x):
    """G(x) = x K_{2/3}(x) (Sec. 3.2.1) via scipy.special.kv."""
    x = np.asarray(x, dtype=np.float64)
    return x * special.kv(2.0 / 3.0, x)


def F1_ref(x):
    """F(x) = x int_x^inf K_{5/3}: with K_{1/3} + K_{5/3} = -2 K'_{2/3},
    int_x^inf K_{5/3} = 2 K_{2/3}(x) - int_x^inf K_{1/3}; the last integrand is
    integrable at 0, so scipy.integrate.quad is accurate."""
    out = []
    for v in np.atleast_1d(np.asarray(x, dtype=np.float64)):
        tail, _ = integrate.quad(lambda t: special.kv(1.0 / 3.0, t), v, np.inf,
                                 epsabs=0.0, epsrel=1e-13, limit=400)
        out.append(v * (2.0 * special.kv(2.0 / 3.0, v) - tail))
    return np.array(out)


def emission_integrand(b, x):
    """3x^2 P(x^3) / c with delta = x^3 (Eq. 1 in the form of Algorithm 1)."""
    d = x ** 3
    z = d / (b * (1.0 - d))
    return (b / x) * ((1.0 - d) * F1_ref(z) + d * d * F2_ref(z))


def pair_integrand(b, d):
    """P_p(delta) / c (Eq. 2, positive bracket)."""
    dd = d * (1.0 - d)
    z = 1.0 / (b * dd)
    return (b / 3.0) * (F2_ref(z) - dd * F1_ref(z))


def gl_integral(fun, a, b, panels=24, order=24):
    xs, ws = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, panels + 1)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        xx = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xs
        tot += 0.5 * (hi - lo) * float(np.dot(ws, fun(xx)))
    return tot


def codata():
    """(alpha, hbar/(m c^2) in s, c in m/s) from scipy.constants."""
    from scipy import constants as k
    alpha = k.physical_constants["fine-structure constant"][0]
    tau_c = k.hbar / (k.m_e * k.c ** 2)
    return alpha, tau_c, k.c
