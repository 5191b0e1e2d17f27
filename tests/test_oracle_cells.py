"""Pins of the oracle's per-cell planning (one sub-step per cell, with which
Algorithms 1 and 2 start).  CPU only.

A cell's count must be the largest per-particle count of its members: equal
to a lone member's plan, at least every member's, and attained by one of
them.  Empty cells, removed rows, disabled processes and out-of-range cell
indices contribute nothing."""
import numpy as np

import oracle as O
from paper_2008_10468_gb300 import inputs as I


def _row_N(cf, arr, i):
    photon = arr["type"][i] == 2
    return O.plan(cf, (arr["px"][i], arr["py"][i], arr["pz"][i]),
                  (arr["Ex"][i], arr["Ey"][i], arr["Ez"][i]),
                  (arr["Bx"][i], arr["By"][i], arr["Bz"][i]), cf.dt, photon=photon)[0]


def test_cell_count_is_the_largest_member_count():
    arr = I.clumped_mixed(600, 5, hot_fraction=0.1)
    cf = O.make_config(1)
    rng = np.random.default_rng(2)
    ncells = 80
    # cells 0..9 hold one row each; the rest share cells 10..79, some out of range
    cell = rng.integers(10, ncells + 5, len(arr["px"])).astype(np.uint32)
    cell[:10] = np.arange(10)
    got = O.plan_cells(cf, arr, cell, ncells)
    rowN = np.array([_row_N(cf, arr, i) for i in range(len(arr["px"]))])
    for c in range(ncells):
        members = np.nonzero(cell == c)[0]
        if len(members) == 0:
            assert got[c] == 0
            continue
        assert np.all(got[c] >= rowN[members])          # no member exceeds it
        assert got[c] in set(rowN[members].tolist())     # and one member attains it
    # a lone member: its own plan
    lone = [c for c in range(ncells) if np.sum(cell == c) == 1]
    assert lone
    for c in lone:
        assert got[c] == rowN[np.nonzero(cell == c)[0][0]]


def test_removed_rows_and_disabled_processes_do_not_count():
    arr = I.clumped_mixed(64, 9, hot_fraction=0.5)
    cell = np.zeros(64, np.uint32)
    cf = O.make_config(1, process_mask=1)   # emission only: photons do not count
    got = O.plan_cells(cf, arr, cell, 1)
    lep = [i for i in range(64) if arr["type"][i] < 2]
    assert got[0] == max(_row_N(cf, arr, i) for i in lep)
    arr2 = dict(arr)
    arr2["type"] = np.full(64, 3, np.uint8)   # all removed
    assert O.plan_cells(cf, arr2, cell, 1)[0] == 0


def test_one_row_per_cell_is_the_plain_step():
    arr = I.clumped_mixed(300, 3, hot_fraction=0.1)
    n = len(arr["px"])
    for push in (0, 1):
        cf = O.make_config(5, push=push)
        cell = np.arange(n, dtype=np.uint32)
        Nc = O.plan_cells(cf, arr, cell, n)
        a = O.event_step(cf, arr, 0)
        b = O.event_step(cf, arr, 0, first_N=Nc[cell])
        assert a[1] == b[1] and np.array_equal(a[2], b[2])
        for k in a[0]:
            assert np.array_equal(a[0][k], b[0][k]), k


def test_a_finer_cell_sub_step_keeps_the_emission_rate():
    # Without recoil each sub-step of length h has event probability W h, so
    # the expected count over the step is W dt whatever the count N: identical
    # particles sharing a cell with one that needs many more sub-steps emit
    # at the rate of Sec. 3.1.1, with more sub-steps.
    import math
    from tests import refs
    M, gamma = 3000, 1000.0
    pm = math.sqrt(gamma * gamma - 1.0)
    E0 = np.float32(1.0 * O.schwinger_field() / (gamma + pm))
    f32 = np.float32
    arr = {"px": np.full(M + 1, -pm, f32), "py": np.zeros(M + 1, f32), "pz": np.zeros(M + 1, f32),
           "Ex": np.zeros(M + 1, f32), "Ey": np.full(M + 1, E0, f32), "Ez": np.zeros(M + 1, f32),
           "Bx": np.zeros(M + 1, f32), "By": np.zeros(M + 1, f32), "Bz": np.full(M + 1, E0, f32),
           "w": np.ones(M + 1, f32), "id": np.arange(1000, 1001 + M, dtype=np.uint64),
           "type": np.zeros(M + 1, np.uint8)}
    arr["Ey"][M] = arr["Bz"][M] = np.float32(40.0 * E0)   # the cell's demanding particle
    cf = O.make_config(77, process_mask=1, recoil=0, cascade=0)
    cell = np.zeros(M + 1, np.uint32)
    Nc = O.plan_cells(cf, arr, cell, 1)
    own, chi, g, _ = O.plan(cf, (arr["px"][0], 0.0, 0.0), (0.0, E0, 0.0), (0.0, 0.0, E0), 0.1)
    assert Nc[0] > 5 * own
    _, st, ev, _ = O.event_step(cf, arr, 5, capacity=(M + 1) * 40, first_N=Nc[cell])
    count = sum(1 for e in ev if int(e["parent_id"]) < 1000 + M)
    b = 1.5 * chi
    W_dt = math.sqrt(3.0) / math.pi * O.rate_unit() * 0.1 / g * refs.gl_integral(
        lambda x: refs.emission_integrand(b, x), 0.0, 1.0, 16, 24)
    assert abs(count / M - W_dt) < 4.0 * math.sqrt(W_dt / M), (count / M, W_dt)
    # the first plans take the cell's count (re-plans after events their own)
    assert st["substeps"] > 2 * M * own
