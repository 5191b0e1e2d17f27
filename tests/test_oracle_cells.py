"""Pins of the oracle's per-cell planning (one sub-step per cell, as the
first line of Algorithms 1 and 2 plans it).  CPU only.

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
