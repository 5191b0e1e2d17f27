"""Pins of the oracle's event generator (Algorithms 1 and 2) against
independent quantities: total rates and spectra integrated with scipy, the
exact sub-step survival probability, and bookkeeping invariants.  CPU only."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2008_10468_gb300 import inputs as I
from tests import refs

SQRT3 = math.sqrt(3.0)


def _identical_particles(M, p, E0, ptype):
    """M copies of one particle (distinct ids) in the crossed field E0 y^, E0 z^."""
    f32 = np.float32
    return {
        "px": np.full(M, p[0], f32), "py": np.full(M, p[1], f32), "pz": np.full(M, p[2], f32),
        "Ex": np.zeros(M, f32), "Ey": np.full(M, E0, f32), "Ez": np.zeros(M, f32),
        "Bx": np.zeros(M, f32), "By": np.zeros(M, f32), "Bz": np.full(M, E0, f32),
        "w": np.ones(M, f32), "id": np.arange(1000, 1000 + M, dtype=np.uint64),
        "type": np.full(M, ptype, np.uint8),
    }


def _setup(chi_target, gamma, photon=False):
    # particle moving along -x: eps - p_x = eps + |p|, chi = E0 (eps + |p|) / E_s
    pm = gamma if photon else math.sqrt(gamma * gamma - 1.0)
    p = (np.float32(-pm), np.float32(0.0), np.float32(0.0))
    E0 = np.float32(chi_target * O.schwinger_field() / (gamma + pm))
    return p, E0


def _chi_gamma(p, E0, photon):
    return O.chi(tuple(float(v) for v in p), (0.0, float(E0), 0.0), (0.0, 0.0, float(E0)),
                 photon=photon)


@pytest.mark.parametrize("p_max", [0.01, 0.002])
def test_emission_count_equals_rate_times_dt_without_recoil(p_max):
    # Without recoil the state never changes, each sub-step of length h has
    # event probability W h, so the expected count over the step is W dt,
    # independent of how the step is divided (Sec. 3.1.1, Algorithm 1).
    M, gamma = 3000, 1000.0
    p, E0 = _setup(1.0, gamma)
    chi, g = _chi_gamma(p, E0, False)
    b = 1.5 * chi
    Rdt = O.rate_unit() * 0.1
    W_dt = SQRT3 / math.pi * Rdt / g * refs.gl_integral(
        lambda x: refs.emission_integrand(b, x), 0.0, 1.0, 16, 24)
    cf = O.make_config(77, p_max=p_max, process_mask=1, recoil=0, cascade=0)
    arr = _identical_particles(M, p, E0, 0)
    _, st, ev, _ = O.event_step(cf, arr, 5, capacity=M + 4 * M * 4)
    mean = st["emissions"] / M
    assert abs(mean - W_dt) < 4.0 * math.sqrt(W_dt / M)
    assert st["substeps"] >= M


def test_emission_spectrum_ks_against_scipy_cdf():
    M, gamma, chi_t = 2000, 2000.0, 2.0
    p, E0 = _setup(chi_t, gamma)
    chi, g = _chi_gamma(p, E0, False)
    b = 1.5 * chi
    cf = O.make_config(99, process_mask=1, recoil=0, cascade=0)
    _, st, ev, _ = O.event_step(cf, _identical_particles(M, p, E0, 0), 2, capacity=20 * M)
    x_ev = np.cbrt(ev["delta"])
    # reference CDF in x = delta^{1/3}
    edges = np.linspace(0.0, 1.0, 121)
    xs, ws = np.polynomial.legendre.leggauss(8)
    cum = [0.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        xx = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xs
        cum.append(cum[-1] + 0.5 * (hi - lo) * float(np.dot(ws, refs.emission_integrand(b, xx))))
    cum = np.array(cum) / cum[-1]
    res = stats.kstest(x_ev, lambda v: np.interp(v, edges, cum))
    assert len(x_ev) > 1000
    assert res.pvalue > 0.01


def test_pair_decay_probability_and_spectrum():
    # A photon is removed at its first pair event (Algorithm 2).  With
    # a fixed plan of N sub-steps of probability q each, it survives with
    # probability (1 - q)^N.
    M, gamma, chi_t = 4000, 1500.0, 3.0
    p, E0 = _setup(chi_t, gamma, photon=True)
    chi, g = _chi_gamma(p, E0, True)
    b = 1.5 * chi
    cf = O.make_config(123, process_mask=2, recoil=1, cascade=0)
    N, _, _, _ = O.plan(cf, tuple(float(v) for v in p), (0.0, float(E0), 0.0),
                        (0.0, 0.0, float(E0)), 0.1, photon=True)
    h = 0.1 / N
    c_h = SQRT3 / math.pi * O.rate_unit() * h / g
    q = c_h * refs.gl_integral(lambda d: refs.pair_integrand(b, d), 0.0, 1.0, 16, 24)
    p_decay = 1.0 - (1.0 - q) ** N
    res, st, ev, _ = O.event_step(cf, _identical_particles(M, p, E0, 2), 1, capacity=4 * M)
    k = st["pairs"]
    assert abs(k - M * p_decay) < 4.0 * math.sqrt(M * p_decay * (1 - p_decay))
    assert int(np.sum(res["type"][:M] == 3)) == k
    # electron energy fraction against the pair spectrum, and its symmetry
    edges = np.linspace(0.0, 1.0, 161)
    xs, ws = np.polynomial.legendre.leggauss(8)
    cum = [0.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        xx = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xs
        cum.append(cum[-1] + 0.5 * (hi - lo) * float(np.dot(ws, refs.pair_integrand(b, xx))))
    cum = np.array(cum) / cum[-1]
    d = ev["delta"]
    assert stats.kstest(d, lambda v: np.interp(v, edges, cum)).pvalue > 0.01
    assert stats.ks_2samp(d, 1.0 - d).pvalue > 0.01


def test_children_bookkeeping():
    # Every event has its children in the store with the predicted ids and
    # types, and they carry the parent's fields and weight.
    arr = I.clumped_mixed(400, 5, hot_fraction=0.25)
    cf = O.make_config(2024, process_mask=3, cascade=1)
    res, st, ev, _ = O.event_step(cf, arr, 9, capacity=200000)
    assert st["status"] == 0
    n0 = 400
    assert len(res["px"]) == n0 + st["children"]
    row_of = {int(i): r for r, i in enumerate(res["id"])}
    assert len(row_of) == len(res["id"])          # ids are unique
    decayed = {int(e["parent_id"]) for e in ev if e["kind"] == 2}
    for e in ev:
        pid = int(e["parent_id"])
        c0, c1 = O.child_ids(2024, pid, 9, int(e["s"]))
        assert int(e["child0"]) == c0
        assert c0 in row_of
        r0 = row_of[c0]
        if e["kind"] == 1:
            # the photon may itself have decayed later in the same step
            assert res["type"][r0] == (3 if c0 in decayed else 2)
        else:
            assert res["type"][r0] == 0
        if e["kind"] == 2:
            assert int(e["child1"]) == c1 and c1 in row_of
            assert res["type"][row_of[c1]] == 1
        r_parent = row_of[pid]
        for f in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "w"):
            assert res[f][r0] == res[f][r_parent]
    assert st["emissions"] + 2 * st["pairs"] == st["children"]
    assert st["pairs"] > 0 and st["emissions"] > 0


def test_threaded_oracle_matches_sequential():
    arr = I.clumped_mixed(300, 11, hot_fraction=0.2)
    cf = O.make_config(31, process_mask=3, cascade=1)
    r1, s1, _, _ = O.event_step(cf, arr, 4, capacity=100000, log=False)
    cf4 = O.make_config(31, process_mask=3, cascade=1, threads=4)
    r4, s4 = O.event_step_mt(cf4, arr, 4, capacity=100000)
    for k in ("substeps", "emissions", "pairs", "children"):
        assert s1[k] == s4[k]
    o1 = np.argsort(r1["id"])
    o4 = np.argsort(r4["id"])
    for f in ("px", "py", "pz", "type", "id", "w"):
        np.testing.assert_array_equal(r1[f][o1], r4[f][o4])


def test_memoised_synchrotron_table_matches_quadrature():
    # the CPU baseline's table form of F and G: within 1e-10 of the
    # quadrature over its whole range (ln F interpolated between nodes)
    x = np.exp(np.random.default_rng(8).uniform(np.log(1e-8), np.log(700.0), 20000))
    q1, q2 = O.F1F2(x)
    with O.memoised_F1F2():
        t1, t2 = O.F1F2(x)
    assert np.max(np.abs(t1 / q1 - 1)) < 1e-10 and np.max(np.abs(t2 / q2 - 1)) < 1e-10
    # outside the table range the quadrature is used
    with O.memoised_F1F2():
        e1, e2 = O.F1F2(np.array([1e-9, 710.0]))
    r1, r2 = O.F1F2(np.array([1e-9, 710.0]))
    np.testing.assert_array_equal(e1, r1)
    np.testing.assert_array_equal(e2, r2)


def test_memoised_event_step_equals_quadrature_step():
    arr = I.clumped_mixed(600, 17, hot_fraction=0.05)
    cf = O.make_config(5, process_mask=3, cascade=1, threads=4)
    a, sa = O.event_step_mt(cf, arr, 3, capacity=600 * 60)
    with O.memoised_F1F2(threads=4):
        b, sb = O.event_step_mt(cf, arr, 3, capacity=600 * 60)
    for k in ("substeps", "emissions", "pairs", "children", "plans"):
        assert sa[k] == sb[k], k
    oa, ob = np.argsort(a["id"]), np.argsort(b["id"])
    for k in a:
        np.testing.assert_array_equal(a[k][oa], b[k][ob])
