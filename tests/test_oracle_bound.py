"""Pins of the oracle's refined emission bound f(b) (Sec. 3.1.1) and of the
sub-step counts it plans, with values fixed by something other than the
printed formula:

* the per-sub-step emission probability itself (the integral that f bounds),
  from scipy's Bessel functions (``tests/refs.py``) and its classical limit
  5 pi / 9 at b -> 0;
* where the bound is tightest and how loose it gets: above the rate by 4.7%
  at its tightest point near b = 2.1 and by 36% at b = 1e3, each of the four
  pieces within 10% of the rate somewhere on its range, and neighbouring
  pieces agreeing within 3% where they meet (a bound built to be tight on
  both sides of an edge cannot jump by more than its own slack there);
* the planned sub-step counts of the synthetic workloads, computed once from
  the printed bound independently of this code: uniform-field electrons
  (gamma 1e2..1e4, chi 0.1..10): mean 736, median 201, 99th percentile 7308;
  clumped population: hot e+- median 303 and 99th percentile 1685, hot
  photons median 52 and 99th percentile 376, cold e+- mean 4.9 and maximum 29.

The last test plants each plausible misprint of the four coefficients and
four exponents in the oracle and checks that one of these pins fails.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_10468_gb300 import inputs as I
from tests import refs

PRINTED_A = (0.56, 0.45, 0.42, 0.55)
PRINTED_E = (1.0, 11.0 / 12.0, 19.0 / 24.0, 2.0 / 3.0)
EDGES = (0.1, 0.5, 10.0)


def _margins(bs):
    return np.array([O.bound_emission(b, 1.0) / O.total_per_c(0, b) for b in bs])


@pytest.mark.parametrize("b", [1e-3, 0.1, 1.0, 2.1, 10.0, 150.0])
def test_rate_against_scipy(b):
    # the integral f bounds: 3x^2 P(x^3) / c over x in [0, 1]
    ref = refs.gl_integral(lambda x: refs.emission_integrand(b, x), 0.0, 1.0, 64, 24)
    assert O.total_per_c(0, b, 256, 32) == pytest.approx(ref, rel=1e-7)
    assert O.total_per_c(0, b) == pytest.approx(ref, rel=3e-6)   # the default rule


def test_rate_classical_limit():
    # W / (c b) -> 5 pi / 9 as b -> 0 (the classical photon number rate)
    assert O.total_per_c(0, 1e-7) / 1e-7 == pytest.approx(5 * math.pi / 9, rel=1e-6)


def _pin_failures(samples):
    """Every pin of the bound that fails for the oracle as it is now."""
    fail = []
    bs = np.logspace(-3, 3, 121)
    m = _margins(bs)
    if not np.all(m > 1.0):
        fail.append("f does not bound the rate at b = %g" % bs[np.argmin(m)])
    i = int(np.argmin(m))
    if not (1.044 <= m[i] <= 1.050 and 1.7 <= bs[i] <= 2.6):
        fail.append("tightest point %.4f at b = %.3g" % (m[i], bs[i]))
    m3 = O.bound_emission(1e3, 1.0) / O.total_per_c(0, 1e3)
    if abs(m3 - 1.36) > 0.005:
        fail.append("margin at b = 1e3: %.4f" % m3)
    for lo, hi in ((1e-3, 0.1), (0.1, 0.5), (0.5, 10.0), (10.0, 1e3)):
        sel = (bs >= lo) & (bs < hi)
        if not m[sel].min() <= 1.09:
            fail.append("piece [%g, %g) loose: min margin %.4f" % (lo, hi, m[sel].min()))
    for e in EDGES:
        r = O.bound_emission(e * (1 + 1e-12), 1.0) / O.bound_emission(e * (1 - 1e-12), 1.0)
        if abs(r - 1.0) > 0.03:
            fail.append("pieces meet at b = %g with a jump of %.3f" % (e, r - 1.0))
    n1, hot_e, hot_p, cold_e = (_counts(*s) for s in samples)
    if abs(n1.mean() / 736.0 - 1.0) > 0.005 or abs(np.median(n1) - 201) > 1 \
            or abs(np.percentile(n1, 99) / 7308.0 - 1.0) > 0.03:
        fail.append("uniform-field counts: mean %.1f median %g p99 %.0f"
                    % (n1.mean(), np.median(n1), np.percentile(n1, 99)))
    if abs(np.median(hot_e) - 303) > 1 or abs(np.percentile(hot_e, 99) / 1685.0 - 1) > 0.01:
        fail.append("hot e+- counts: median %g p99 %.0f"
                    % (np.median(hot_e), np.percentile(hot_e, 99)))
    if abs(np.median(hot_p) - 52) > 1 or abs(np.percentile(hot_p, 99) / 376.0 - 1) > 0.01:
        fail.append("hot photon counts: median %g p99 %.0f"
                    % (np.median(hot_p), np.percentile(hot_p, 99)))
    if abs(cold_e.mean() - 4.9) > 0.05 or cold_e.max() != 29:
        fail.append("cold e+- counts: mean %.3f max %d" % (cold_e.mean(), cold_e.max()))
    return fail


def _counts(cf, arr, rows, photon):
    out = []
    for i in rows:
        if (arr["type"][i] == 2) != photon:
            continue
        p = (arr["px"][i], arr["py"][i], arr["pz"][i])
        E = (arr["Ex"][i], arr["Ey"][i], arr["Ez"][i])
        B = (arr["Bx"][i], arr["By"][i], arr["Bz"][i])
        out.append(O.plan(cf, p, E, B, 0.1, photon=photon)[0])
    return np.array(out)


@pytest.fixture(scope="module")
def samples():
    cf = O.make_config(1, process_mask=3)
    uni = I.uniform_field_electrons(100_000, 20081047)
    n = 1 << 20
    clump = I.clumped_mixed(n, 20081049)
    n_hot = int(round(n * 0.01))
    h0 = (n - n_hot) // 2
    hot = range(h0, h0 + n_hot)
    return ((cf, uni, range(100_000), False), (cf, clump, hot, False),
            (cf, clump, hot, True), (cf, clump, range(100_000), False))


def test_printed_bound_meets_every_pin(samples):
    fail = _pin_failures(samples)
    assert not fail, fail


MISPRINTS = [
    ("0.56 -> 0.55", (0.55, 0.45, 0.42, 0.55), PRINTED_E),
    ("0.56 -> 0.57", (0.57, 0.45, 0.42, 0.55), PRINTED_E),
    ("0.56 -> 0.65", (0.65, 0.45, 0.42, 0.55), PRINTED_E),
    ("0.45 -> 0.44", (0.56, 0.44, 0.42, 0.55), PRINTED_E),
    ("0.45 -> 0.46", (0.56, 0.46, 0.42, 0.55), PRINTED_E),
    ("0.45 <-> 0.42", (0.56, 0.42, 0.45, 0.55), PRINTED_E),
    ("0.42 -> 0.43", (0.56, 0.45, 0.43, 0.55), PRINTED_E),
    ("0.42 -> 0.41", (0.56, 0.45, 0.41, 0.55), PRINTED_E),
    ("0.55 -> 0.54", (0.56, 0.45, 0.42, 0.54), PRINTED_E),
    ("0.55 -> 0.56", (0.56, 0.45, 0.42, 0.56), PRINTED_E),
    ("0.55 <-> 0.56", (0.55, 0.45, 0.42, 0.56), PRINTED_E),
    ("11/12 <-> 19/24", PRINTED_A, (1.0, 19 / 24, 11 / 12, 2 / 3)),
    ("11/12 -> 12/11", PRINTED_A, (1.0, 12 / 11, 19 / 24, 2 / 3)),
    ("19/24 -> 17/24", PRINTED_A, (1.0, 11 / 12, 17 / 24, 2 / 3)),
    ("19/24 -> 24/19", PRINTED_A, (1.0, 11 / 12, 24 / 19, 2 / 3)),
    ("2/3 -> 3/4", PRINTED_A, (1.0, 11 / 12, 19 / 24, 3 / 4)),
    ("2/3 -> 3/2", PRINTED_A, (1.0, 11 / 12, 19 / 24, 3 / 2)),
    ("2/3 -> 1/3", PRINTED_A, (1.0, 11 / 12, 19 / 24, 1 / 3)),
]


@pytest.mark.parametrize("name,A,e", MISPRINTS, ids=[m[0] for m in MISPRINTS])
def test_misprinted_bound_fails_a_pin(samples, name, A, e):
    with O.planted_emission_bound(A, e):
        fail = _pin_failures(samples)
    assert fail, name
    print(name, "->", fail[0])


def test_misprinted_linear_term_fails_a_pin(samples):
    with O.planted_emission_bound(PRINTED_A, PRINTED_E, lin=0.01):
        fail = _pin_failures(samples)
    assert fail
