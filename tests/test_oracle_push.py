"""Pins of the oracle's Boris push (Algorithm 1 moves the momentum by a Boris
step at the start of every sub-step, before the draw) and of the push mode
of its event step.  CPU only.

The binary64 push is pinned to the Lorentz force itself: the exact solution
in a pure electric field, the exact rotation angle and sense in a pure
magnetic field, and second-order convergence to a high-accuracy ODE solution
in general fields.  The binary32 form used on the particle state is pinned
to the binary64 one.  The push-mode step is pinned by two invariants: a
photon's momentum never moves, and with E = 0 and p perpendicular to B the
push only rotates p about B, so chi, and with it every event, is that of the
step without the push."""
import math

import numpy as np
import pytest

import oracle as O

TWO_PI = 2.0 * math.pi


@pytest.mark.parametrize("charge", [-1, 1])
def test_pure_electric_field_is_exact(charge):
    # B = 0: dp/dt = 2 pi q E, so p(t) = p0 + 2 pi q E t exactly
    p0, E = np.array([3.0, -1.0, 0.5]), np.array([0.2, 0.7, -0.4])
    h, n = 0.003, 500
    p = O.boris64(charge, h, p0, E, (0.0, 0.0, 0.0), steps=n)
    np.testing.assert_allclose(p, p0 + TWO_PI * charge * E * h * n, rtol=0, atol=1e-12)


@pytest.mark.parametrize("charge", [-1, 1])
def test_pure_magnetic_field_rotates_by_the_boris_angle(charge):
    # E = 0: |p| and p.B are constant, and each step rotates p_perp about B
    # by 2 atan(|a| |B| / gamma), a = pi q h, in the sense of q (p x B)
    p0, B = np.array([40.0, -10.0, 7.0]), np.array([0.0, 300.0, 400.0])
    h, n = 1e-4, 2000
    g = math.sqrt(1.0 + p0 @ p0)
    theta = 2.0 * math.atan(math.pi * h * np.linalg.norm(B) / g)
    bh = B / np.linalg.norm(B)
    p = p0.copy()
    for _ in range(n):
        q = O.boris64(charge, h, p, (0.0, 0.0, 0.0), B)
        a_perp, b_perp = p - (p @ bh) * bh, q - (q @ bh) * bh
        c = np.cross(a_perp, b_perp) @ bh
        ang = math.atan2(c, a_perp @ b_perp)
        # the force q (p x B) turns p_perp clockwise about B for q > 0
        assert ang * charge < 0
        assert abs(abs(ang) - theta) < 1e-12
        p = q
    assert abs(np.linalg.norm(p) / np.linalg.norm(p0) - 1.0) < 1e-13
    assert abs(p @ bh - p0 @ bh) < 1e-10


def _lorentz_reference(charge, p0, E, B, T):
    integrate = pytest.importorskip("scipy.integrate")

    def rhs(_t, p):
        g = math.sqrt(1.0 + p @ p)
        return TWO_PI * charge * (E + np.cross(p, B) / g)

    sol = integrate.solve_ivp(rhs, (0.0, T), p0, method="DOP853", rtol=1e-13, atol=1e-12)
    return sol.y[:, -1]


def test_second_order_convergence_in_general_fields():
    # Boris is a second-order method: halving h divides the error by ~4
    charge = -1
    p0 = np.array([3.0, -1.0, 2.0])
    E = np.array([0.3, -0.2, 0.5])
    B = np.array([0.1, 0.7, -0.4])
    T = 0.5
    ref = _lorentz_reference(charge, p0, E, B, T)
    errs = []
    for n in (200, 400, 800):
        p = O.boris64(charge, T / n, p0, E, B, steps=n)
        errs.append(np.linalg.norm(p - ref))
    assert errs[0] < 1e-3
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 < e1 / e2 < 4.4, errs


def test_binary32_push_follows_binary64():
    rng = np.random.default_rng(5)
    worst1 = worst_n = 0.0
    for _ in range(200):
        charge = int(rng.choice([-1, 1]))
        p = rng.normal(0.0, 1.0, 3) * 10.0 ** rng.uniform(0, 4)
        E = rng.normal(0.0, 1.0, 3) * 10.0 ** rng.uniform(0, 3)
        B = rng.normal(0.0, 1.0, 3) * 10.0 ** rng.uniform(0, 3)
        h = 10.0 ** rng.uniform(-6, -3)
        p32, E32, B32 = (np.asarray(v, np.float32) for v in (p, E, B))
        h32 = float(np.float32(h))
        scale = np.linalg.norm(p32) + TWO_PI * h32 * np.linalg.norm(E32)
        a = O.boris32(charge, h32, p32, E32, B32)
        b = O.boris64(charge, h32, p32, E32, B32)
        worst1 = max(worst1, np.max(np.abs(a - b)) / scale)
        a = O.boris32(charge, h32, p32, E32, B32, steps=100)
        b = O.boris64(charge, h32, p32, E32, B32, steps=100)
        scale = np.linalg.norm(p32) + 100 * TWO_PI * h32 * (np.linalg.norm(E32) + 1.0)
        worst_n = max(worst_n, np.max(np.abs(a - b)) / scale)
    # one push: a few binary32 roundings of |p|; 100 pushes: at most 100 times that
    assert worst1 < 8 * 2.0 ** -24, worst1
    assert worst_n < 800 * 2.0 ** -24, worst_n


def _population(n, seed, photons=False, perpendicular=False):
    rng = np.random.default_rng(seed)
    f32 = np.float32
    gamma = np.exp(rng.uniform(math.log(200.0), math.log(5000.0), n))
    u = rng.normal(size=(n, 3))
    B = np.zeros((n, 3))
    B[:, 2] = rng.uniform(100.0, 1500.0, n)
    if perpendicular:
        u[:, 2] = 0.0
    u /= np.linalg.norm(u, axis=1)[:, None]
    p = u * np.sqrt(gamma * gamma - 1.0)[:, None]
    E = np.zeros((n, 3)) if perpendicular else rng.normal(0.0, 300.0, (n, 3))
    return {
        "px": p[:, 0].astype(f32), "py": p[:, 1].astype(f32), "pz": p[:, 2].astype(f32),
        "Ex": E[:, 0].astype(f32), "Ey": E[:, 1].astype(f32), "Ez": E[:, 2].astype(f32),
        "Bx": B[:, 0].astype(f32), "By": B[:, 1].astype(f32), "Bz": B[:, 2].astype(f32),
        "w": np.ones(n, f32), "id": np.arange(5000, 5000 + n, dtype=np.uint64),
        "type": np.full(n, 2 if photons else 0, np.uint8) if photons else
        rng.integers(0, 2, n).astype(np.uint8),
    }


def test_push_leaves_photons_alone():
    arr = _population(300, 1, photons=True)
    for k in ("px", "py", "pz"):
        arr[k] = arr[k] * np.float32(3.0)
    # (children stay unprocessed: the pairs' e+- would be pushed)
    a, sa, ea, _ = O.event_step(O.make_config(21, push=0, cascade=0), arr, 3)
    b, sb, eb, _ = O.event_step(O.make_config(21, push=1, cascade=0), arr, 3)
    assert sa == sb and sa["pairs"] > 0
    assert np.array_equal(ea, eb)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_push_in_a_pure_magnetic_field_keeps_every_event():
    # p perpendicular to B, E = 0: the push rotates p about B, |p| and chi stay
    # (up to binary32 rounding), so the events are those of the unpushed step
    arr = _population(400, 2, perpendicular=True)
    cf0 = O.make_config(33, push=0, cascade=0)
    cf1 = O.make_config(33, push=1, cascade=0)
    a, sa, ea, ta = O.event_step(cf0, arr, 4)
    b, sb, eb, tb = O.event_step(cf1, arr, 4)
    assert sa["emissions"] > 100
    tied = {int(t["id"]) for t in ta} | {int(t["id"]) for t in tb}
    keep_a = np.array([int(e["parent_id"]) not in tied for e in ea], bool)
    keep_b = np.array([int(e["parent_id"]) not in tied for e in eb], bool)
    ka, kb = ea[keep_a], eb[keep_b]
    assert len(ka) == len(kb) and len(ka) > 0.9 * len(ea)
    for f in ("parent_id", "child0", "s", "kind"):
        assert np.array_equal(ka[f], kb[f]), f
    np.testing.assert_allclose(kb["delta"], ka["delta"], rtol=1e-12)
    np.testing.assert_allclose(kb["chi"], ka["chi"], rtol=1e-5)
    # the same |p| (rows of untied parents), a different direction
    n = len(arr["px"])
    ids = np.array([int(v) for v in a["id"][:n]])
    ok = np.array([i not in tied for i in ids], bool)
    pa = np.stack([a[k][:n] for k in ("px", "py", "pz")], 1).astype(np.float64)[ok]
    pb = np.stack([b[k][:n] for k in ("px", "py", "pz")], 1).astype(np.float64)[ok]
    na, nb = np.linalg.norm(pa, axis=1), np.linalg.norm(pb, axis=1)
    np.testing.assert_allclose(nb, na, rtol=2e-5)
    assert np.median(np.linalg.norm(pb - pa, axis=1) / na) > 1e-2
    assert np.all(b["pz"][:n] == 0.0)


def test_push_moves_the_momentum_by_the_lorentz_force():
    # the push is part of the sub-step loop of the processed particles: with
    # no process enabled nothing is drawn and nothing moves
    arr = _population(64, 3)
    cf = O.make_config(9, push=1, process_mask=0)
    a, st, ev, _ = O.event_step(cf, arr, 1)
    assert st["substeps"] == 0 and len(ev) == 0
    for k in ("px", "py", "pz"):
        assert np.array_equal(a[k], arr[k])
    # with recoil off, an e+-'s momentum after the step is the binary32 push
    # of its plan's sub-steps: one plan per particle (no re-plan after events)
    cf = O.make_config(9, push=1, recoil=0, cascade=0, process_mask=1)
    a, st, ev, _ = O.event_step(cf, arr, 1)
    checked = 0
    for j in range(len(arr["px"])):
        N, _, _, _ = O.plan(cf, (arr["px"][j], arr["py"][j], arr["pz"][j]),
                            (arr["Ex"][j], arr["Ey"][j], arr["Ez"][j]),
                            (arr["Bx"][j], arr["By"][j], arr["Bz"][j]), 0.1)
        s_events = [int(e["s"]) for e in ev if int(e["parent_id"]) == int(arr["id"][j])]
        if s_events:
            continue   # re-planned after an event
        charge = -1 if arr["type"][j] == 0 else 1
        want = O.boris32(charge, 0.1 / N, (arr["px"][j], arr["py"][j], arr["pz"][j]),
                         (arr["Ex"][j], arr["Ey"][j], arr["Ez"][j]),
                         (arr["Bx"][j], arr["By"][j], arr["Bz"][j]), steps=N)
        got = np.array([a[k][j] for k in ("px", "py", "pz")], np.float32)
        assert np.array_equal(got, want), (j, got, want)
        assert np.linalg.norm(got - arr_p(arr, j)) > 1e-3 * np.linalg.norm(got)
        checked += 1
    assert checked >= 10


def arr_p(arr, j):
    return np.array([arr[k][j] for k in ("px", "py", "pz")], np.float32)


@pytest.mark.parametrize("charge", [-1, 1])
def test_crossed_fields_drift_at_e_cross_b(charge):
    # |E| < |B|, E perpendicular to B: the velocity averaged over many
    # gyrations is the drift E x B / B^2, whatever the charge (a kick with the
    # wrong sign relative to the rotation would reverse or spoil it)
    E = np.array([0.0, 150.0, 0.0])
    B = np.array([0.0, 0.0, 300.0])
    h, n = 2e-5, 40000
    p = np.array([0.0, 0.0, 0.0])
    v = np.zeros(3)
    for _ in range(n):
        p = O.boris64(charge, h, p, E, B)
        v += p / math.sqrt(1.0 + p @ p)
    v /= n
    drift = np.cross(E, B) / (B @ B)
    np.testing.assert_allclose(v, drift, atol=2e-3)
