"""FP64 CPU oracle for the QED event generator (arXiv:2008.10468).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

What it computes (each function cites the passage it follows):

* ``F1``/``F2``: the synchrotron functions F(x) = x int_x^inf K_{5/3} and
  G(x) = x K_{2/3}(x) of Sec. 3.2.1, by trapezoidal quadrature of the integral
  representation of K_nu (C code in ``qed_oracle.c``); ``F1F2_double_reference``
  adds G from mpmath's K_nu for the binary64 routine's 1e-14 level.
* ``philox``/``draw``/``child_ids``: Philox4x32-10 (Salmon et al., SC'11) and
  the per-sub-step draw x, y of Algorithms 1 and 2.
* ``chi``/``plan``: the quantum parameter of Sec. 2.2 and the sub-step count
  from the rate bounds of Sec. 3.1.1.
* ``Pm``/``Pp``: the acceptance functions 3x^2 P(x^3) (Eq. 1, Algorithm 1) and
  P_p (Eq. 2 with the bracket sign corrected, Algorithm 2).
* ``total_per_c``: the per-sub-step event probability divided by c
  (the integral bounded by f(b) in Sec. 3.1.1).
* ``plan_cells``: the sub-step count per cell with which Algorithms 1 and 2
  start (the largest count of the cell's particles).
* ``event_step``: Algorithms 1 and 2 for a particle store over one global step,
  optionally with the Boris push of Algorithm 1 before every e+- draw.
* ``boris64``/``boris32``: that push (the Lorentz force in code units), in
  binary64 and on the binary32 particle state.

Parity is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, u32, u64, i64, i32 = C.c_double, C.c_uint32, C.c_uint64, C.c_int64, C.c_int
        P = C.POINTER
        L.orc_F1.restype = d; L.orc_F1.argtypes = [d]
        L.orc_F2.restype = d; L.orc_F2.argtypes = [d]
        L.orc_F1F2.restype = None
        L.orc_F1F2.argtypes = [i64, P(d), P(d), P(d), i32]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.orc_uniform.restype = d; L.orc_uniform.argtypes = [u32]
        L.orc_draw.restype = None
        L.orc_draw.argtypes = [u64, u64, u32, u32, P(d), P(d)]
        L.orc_child_ids.restype = None
        L.orc_child_ids.argtypes = [u64, u64, u32, u32, P(u64)]
        L.orc_chi.restype = d
        L.orc_chi.argtypes = [i32] + [d] * 10 + [P(d)]
        L.orc_bound_emission.restype = d; L.orc_bound_emission.argtypes = [d, d]
        L.orc_set_emission_bound.restype = None
        L.orc_set_emission_bound.argtypes = [P(d), P(d), d]
        L.orc_bound_pair.restype = d; L.orc_bound_pair.argtypes = [d, d, d]
        L.orc_Pm.restype = d; L.orc_Pm.argtypes = [d, d, d]
        L.orc_Pp.restype = d; L.orc_Pp.argtypes = [d, d, d]
        L.orc_total_per_c.restype = d; L.orc_total_per_c.argtypes = [i32, d, i32, i32]
        L.orc_rate_unit.restype = d; L.orc_rate_unit.argtypes = [d]
        L.orc_schwinger_field.restype = d; L.orc_schwinger_field.argtypes = [d]
        L.orc_event_step.restype = i32
        L.orc_event_step.argtypes = [P(Config), P(Particles), u32, P(Stats), P(Log)]
        L.orc_table_build.restype = None
        L.orc_table_build.argtypes = [i32]
        L.orc_table_off.restype = None
        L.orc_table_off.argtypes = []
        L.orc_event_step_mt.restype = i32
        L.orc_event_step_mt.argtypes = [P(Config), P(Particles), u32, P(Stats)]
        L.orc_log_free.restype = None; L.orc_log_free.argtypes = [P(Log)]
        L.orc_plan.restype = u32
        L.orc_boris64.restype = None
        L.orc_boris64.argtypes = [i32, d, P(d), P(d), P(d)]
        L.orc_boris32.restype = None
        L.orc_boris32.argtypes = [i32, C.c_float, P(C.c_float), P(C.c_float), P(C.c_float)]
        L.orc_plan.argtypes = [P(Config), i32] + [d] * 10 + [P(d), P(d), P(d)]
        _lib = L
    return _lib


class Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("dt", C.c_double), ("R", C.c_double),
                ("E_s", C.c_double), ("p_max", C.c_double), ("pair_coeff", C.c_double),
                ("tie_draw", C.c_double), ("tie_plan", C.c_double),
                ("process_mask", C.c_uint32), ("cascade", C.c_int32),
                ("recoil", C.c_int32), ("threads", C.c_int32), ("push", C.c_int32),
                ("first_N", C.POINTER(C.c_uint32)), ("first_N_rows", C.c_int64)]


class Particles(C.Structure):
    _fields_ = [(n, C.POINTER(C.c_float)) for n in
                ("px", "py", "pz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "w")] + [
                ("id", C.POINTER(C.c_uint64)), ("type", C.POINTER(C.c_uint8)),
                ("count", C.c_int64), ("capacity", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("substeps", C.c_uint64), ("emissions", C.c_uint64), ("pairs", C.c_uint64),
                ("children", C.c_uint64), ("guard_hits", C.c_uint64), ("plans", C.c_uint64),
                ("max_N", C.c_uint32), ("status", C.c_int32),
                ("required_capacity", C.c_int64)]


class Event(C.Structure):
    _fields_ = [("parent_id", C.c_uint64), ("child_id", C.c_uint64 * 2), ("s", C.c_uint32),
                ("kind", C.c_uint32), ("delta", C.c_double), ("chi", C.c_double)]


class Tie(C.Structure):
    _fields_ = [("id", C.c_uint64), ("s", C.c_uint32), ("kind", C.c_uint32)]


class Log(C.Structure):
    _fields_ = [("ev", C.POINTER(Event)), ("n_ev", C.c_int64), ("cap_ev", C.c_int64),
                ("tie", C.POINTER(Tie)), ("n_tie", C.c_int64), ("cap_tie", C.c_int64)]


FIELDS = ("px", "py", "pz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "w")

# Tie bands.  A draw y with |y - P| <= TIE_DRAW * P is a near-tie: from that
# sub-step on the particle is exempt from the event-by-event comparison.  The
# stated tolerance exempts draws within 1e-5 of P; as a fraction of P
# (P < 0.3 on every path) the band is narrower and the comparison stricter.
# A plan is a near-tie when N changes as f / P_max and b move by TIE_PLAN
# relative: the kernels take every count whose binary32 value is not
# certain again in binary64, so counts agree unless f / P_max sits within
# about 1e-13 of an integer.
TIE_DRAW = 1e-5
TIE_PLAN = 1e-12


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def rate_unit(lambda_m=1e-6):
    """R = alpha m c^2 / hbar in 1/laser period (the bracket of Eq. 1 is R dt)."""
    return lib().orc_rate_unit(lambda_m)


def schwinger_field(lambda_m=1e-6):
    """Schwinger field m^2 c^3/(e hbar) in units of m c omega / e."""
    return lib().orc_schwinger_field(lambda_m)


def F1F2(x, threads=None):
    """F(x) = x int_x^inf K_{5/3} and G(x) = x K_{2/3}(x) (Sec. 3.2.1), FP64."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    f1 = np.empty_like(x)
    f2 = np.empty_like(x)
    if threads is None:
        threads = min(os.cpu_count() or 1, max(1, x.size // 256))
    lib().orc_F1F2(x.size, _dp(x), _dp(f1), _dp(f2), int(threads))
    return f1, f2


def F1F2_double_reference(x):
    """Reference values for the binary64 routine: F from the quadrature above
    (FP64 rounding level, ~2e-15), G = x K_{2/3}(x) from mpmath's K_nu at 30
    digits (the definition of Sec. 3.2.1).  Slow: for up to ~10^4 points."""
    import mpmath as mp
    x = np.asarray(x, dtype=np.float64).ravel()
    f1, _ = F1F2(x)
    f2 = np.empty_like(x)
    with mp.workdps(30):
        nu = mp.mpf(2) / 3
        for i, v in enumerate(x):
            f2[i] = float(mp.mpf(v) * mp.besselk(nu, mp.mpf(v))) if v > 0 else 0.0
    return f1, f2


def F1(x):
    return F1F2(x)[0]


def F2(x):
    return F1F2(x)[1]


def philox(ctr, key):
    """Philox4x32-10 of one 128-bit counter under one 64-bit key."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(r):
    return lib().orc_uniform(int(r) & 0xffffffff)


def draw(seed, pid, step, s):
    """(x, y) of sub-step s of particle pid in global step `step`."""
    x = C.c_double()
    y = C.c_double()
    lib().orc_draw(int(seed), int(pid), int(step), int(s), C.byref(x), C.byref(y))
    return x.value, y.value


def child_ids(seed, pid, step, s):
    o = (C.c_uint64 * 2)()
    lib().orc_child_ids(int(seed), int(pid), int(step), int(s), o)
    return int(o[0]), int(o[1])


def chi(p, E, B, photon=False, E_s=None):
    """chi (Sec. 2.2) and gamma (or |k| for a photon) of one particle."""
    if E_s is None:
        E_s = schwinger_field()
    g = C.c_double()
    v = lib().orc_chi(int(photon), *[float(a) for a in (*p, *E, *B)], float(E_s), C.byref(g))
    return v, g.value


def bound_emission(b, c):
    """f(b) of Sec. 3.1.1 for photon emission."""
    return lib().orc_bound_emission(float(b), float(c))


class planted_emission_bound:
    """Context manager for tests of the pins: inside it the oracle's emission
    bound uses coefficients A (4), exponents e (4) and linear term lin instead
    of the printed ones of Sec. 3.1.1; they are restored on exit."""

    def __init__(self, A, e, lin=0.1):
        self.A = (C.c_double * 4)(*[float(v) for v in A])
        self.e = (C.c_double * 4)(*[float(v) for v in e])
        self.lin = float(lin)

    def __enter__(self):
        lib().orc_set_emission_bound(self.A, self.e, self.lin)
        return self

    def __exit__(self, *exc):
        lib().orc_set_emission_bound(None, None, 0.0)
        return False


def bound_pair(b, c, coeff=0.1):
    """f = 0.1 c b of Sec. 3.1.1 for pair production."""
    return lib().orc_bound_pair(float(b), float(c), float(coeff))


def Pm(b, c, x):
    """3 x^2 P(x^3) of Algorithm 1 (Eq. 1)."""
    return lib().orc_Pm(float(b), float(c), float(x))


def Pp(b, c, delta):
    """P_p(delta) of Algorithm 2 (Eq. 2, bracket sign corrected)."""
    return lib().orc_Pp(float(b), float(c), float(delta))


def total_per_c(kind, b, panels=64, order=16):
    """int_0^1 of the acceptance function divided by c: kind 0 emission, 1 pair."""
    return lib().orc_total_per_c(int(kind), float(b), int(panels), int(order))


def make_config(seed, dt=0.1, lambda_m=1e-6, p_max=0.01, pair_coeff=0.1,
                process_mask=3, cascade=1, recoil=1, threads=1,
                tie_draw=TIE_DRAW, tie_plan=TIE_PLAN, push=0):
    cf = Config()
    cf.seed = int(seed)
    cf.dt = float(dt)
    cf.R = rate_unit(lambda_m)
    cf.E_s = schwinger_field(lambda_m)
    # the library's configuration holds these two in binary32
    cf.p_max = float(np.float32(p_max))
    cf.pair_coeff = float(np.float32(pair_coeff))
    cf.tie_draw = float(tie_draw)
    cf.tie_plan = float(tie_plan)
    cf.process_mask = int(process_mask)
    cf.cascade = int(cascade)
    cf.recoil = int(recoil)
    cf.threads = int(threads)
    cf.push = int(push)
    return cf


def boris64(charge, h, p, E, B, steps=1):
    """`steps` Boris pushes of length h (periods) in binary64; returns p."""
    pa = (C.c_double * 3)(*[float(v) for v in p])
    Ea = (C.c_double * 3)(*[float(v) for v in E])
    Ba = (C.c_double * 3)(*[float(v) for v in B])
    for _ in range(int(steps)):
        lib().orc_boris64(int(charge), float(h), pa, Ea, Ba)
    return np.array(list(pa), dtype=np.float64)


def boris32(charge, h, p, E, B, steps=1):
    """`steps` Boris pushes on the binary32 state; returns p (float32)."""
    f = C.c_float
    pa = (f * 3)(*[float(np.float32(v)) for v in p])
    Ea = (f * 3)(*[float(np.float32(v)) for v in E])
    Ba = (f * 3)(*[float(np.float32(v)) for v in B])
    for _ in range(int(steps)):
        lib().orc_boris32(int(charge), float(np.float32(h)), pa, Ea, Ba)
    return np.array(list(pa), dtype=np.float32)


def plan(cf, p, E, B, t_rem, photon=False):
    """Sub-step count N of the planning step of Algorithms 1/2, with chi, gamma and f."""
    ch, g, f = C.c_double(), C.c_double(), C.c_double()
    N = lib().orc_plan(C.byref(cf), int(photon), *[float(a) for a in (*p, *E, *B)],
                       float(t_rem), C.byref(ch), C.byref(g), C.byref(f))
    return int(N), ch.value, g.value, f.value


def plan_cells(cf, arrs, cell, ncells):
    """Per-cell sub-step counts (Algorithms 1 and 2 start by fixing one
    sub-step per cell): for each cell the largest planned N
    (``plan`` over a full global step) of its rows whose process is enabled
    (0 for a cell without one).  Rows with a cell index >= ncells are left out."""
    out = np.zeros(int(ncells), dtype=np.int64)
    for i in range(len(arrs["px"])):
        t = int(arrs["type"][i])
        c = int(cell[i])
        if t > 2 or c >= ncells:
            continue
        photon = t == 2
        if not (cf.process_mask & (2 if photon else 1)):
            continue
        p = (arrs["px"][i], arrs["py"][i], arrs["pz"][i])
        if photon and not any(float(v) != 0.0 for v in p):
            continue   # a photon without momentum has no plan
        N, _, _, _ = plan(cf, p, (arrs["Ex"][i], arrs["Ey"][i], arrs["Ez"][i]),
                          (arrs["Bx"][i], arrs["By"][i], arrs["Bz"][i]), cf.dt, photon=photon)
        out[c] = max(out[c], N)
    return out


def _store(arrs, capacity):
    """Copy a particle dict into capacity-sized contiguous arrays."""
    n = int(arrs["px"].shape[0])
    out = {}
    for k in FIELDS:
        a = np.zeros(capacity, dtype=np.float32)
        a[:n] = arrs[k]
        out[k] = a
    out["id"] = np.zeros(capacity, dtype=np.uint64)
    out["id"][:n] = arrs["id"]
    out["type"] = np.full(capacity, 3, dtype=np.uint8)
    out["type"][:n] = arrs["type"]
    P = Particles()
    for k in FIELDS:
        setattr(P, k, out[k].ctypes.data_as(C.POINTER(C.c_float)))
    P.id = out["id"].ctypes.data_as(C.POINTER(C.c_uint64))
    P.type = out["type"].ctypes.data_as(C.POINTER(C.c_uint8))
    P.count = n
    P.capacity = int(capacity)
    return out, P


def _stats_dict(st):
    return {k: int(getattr(st, k)) for k, _ in Stats._fields_}


def event_step(cf, arrs, step, capacity=None, log=True, first_N=None):
    """One global step of Algorithms 1 and 2 on a copy of `arrs`.

    first_N (optional, one count per row of `arrs`): the first plan of each
    of these rows takes at least this many sub-steps (one sub-step per cell:
    pass each row its cell's ``plan_cells`` count).

    Returns (arrays, stats, events, ties): arrays truncated to the final count,
    stats as a dict, events as a structured array (parent_id, child0, child1,
    s, kind, delta, chi) and ties as a structured array (id, s, kind).
    """
    n = int(arrs["px"].shape[0])
    if capacity is None:
        capacity = 4 * n + 1024
    out, P = _store(arrs, capacity)
    st = Stats()
    L = Log()
    fN = None
    if first_N is not None:
        fN = np.ascontiguousarray(first_N, dtype=np.uint32)
        cf.first_N = fN.ctypes.data_as(C.POINTER(C.c_uint32))
        cf.first_N_rows = len(fN)
    else:
        cf.first_N = None
        cf.first_N_rows = 0
    try:
        if log:
            lib().orc_event_step(C.byref(cf), C.byref(P), int(step), C.byref(st), C.byref(L))
        else:
            lib().orc_event_step(C.byref(cf), C.byref(P), int(step), C.byref(st), None)
    finally:
        # the counts live only for this call
        cf.first_N = None
        cf.first_N_rows = 0
    cnt = int(P.count)
    res = {k: v[:cnt].copy() for k, v in out.items()}
    ev_dt = np.dtype([("parent_id", np.uint64), ("child0", np.uint64), ("child1", np.uint64),
                      ("s", np.uint32), ("kind", np.uint32), ("delta", np.float64),
                      ("chi", np.float64)])
    tie_dt = np.dtype([("id", np.uint64), ("s", np.uint32), ("kind", np.uint32)])
    ev = np.zeros(int(L.n_ev), dtype=ev_dt)
    for j in range(int(L.n_ev)):
        e = L.ev[j]
        ev[j] = (e.parent_id, e.child_id[0], e.child_id[1], e.s, e.kind, e.delta, e.chi)
    ties = np.zeros(int(L.n_tie), dtype=tie_dt)
    for j in range(int(L.n_tie)):
        t = L.tie[j]
        ties[j] = (t.id, t.s, t.kind)
    if log:
        lib().orc_log_free(C.byref(L))
    return res, _stats_dict(st), ev, ties


class memoised_F1F2:
    """Context manager: inside it F1 and F2 come from a table of the
    quadrature (8192 nodes uniform in ln x over [1e-8, 700], Lagrange
    interpolation through the 8 nearest nodes), as a production CPU code would
    evaluate them; used to time the CPU baseline.  Outside it, the quadrature."""

    def __init__(self, threads=None):
        self.threads = int(threads or os.cpu_count() or 1)

    def __enter__(self):
        lib().orc_table_build(self.threads)
        return self

    def __exit__(self, *exc):
        lib().orc_table_off()
        return False


def event_step_mt(cf, arrs, step, capacity=None):
    """Multi-threaded event step (no log); used to time the oracle."""
    n = int(arrs["px"].shape[0])
    if capacity is None:
        capacity = 4 * n + 1024
    out, P = _store(arrs, capacity)
    st = Stats()
    lib().orc_event_step_mt(C.byref(cf), C.byref(P), int(step), C.byref(st))
    cnt = int(P.count)
    return {k: v[:cnt].copy() for k, v in out.items()}, _stats_dict(st)
