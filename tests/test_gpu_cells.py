"""The event step with one sub-step per cell for the first plans
(qed_event_step_cells), against the oracle given the same first-plan counts,
through the C ABI.  GPU only.

Algorithms 1 and 2 start by fixing the sub-step of the particle's cell: each
row present at the start of the step makes its first plan with its cell's
count (the largest count of the cell's rows, qed_plan_cells) when that is
larger than its own; re-plans and children plan per particle.  Same protocol
as the other parity tests (tests/parity.py)."""
import numpy as np
import pytest

import oracle as O
from paper_2008_10468_gb300 import inputs as I
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402
from tests.test_gpu_parity import _oracle_plans  # noqa: E402


def _cell_tensor(cell):
    return torch.from_numpy(cell.astype(np.uint32).view(np.int32)).cuda()


def _by_id(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items()}


def test_event_step_cells_parity():
    n = 4133
    arr = I.clumped_mixed(n, 20081049, hot_fraction=0.02)
    cell = (np.arange(n) // 16).astype(np.uint32)
    cell[::97] = 10 ** 6    # out of range: these rows keep their own count
    ncells = (n + 15) // 16
    seed, step, cap = 20081049, 3, n * 20
    ctx = qed.Context(seed=seed, process_mask=3, cascade=True)
    ctx.set_event_log(1 << 20)
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    g_st = ctx.event_step_cells(store, step, _cell_tensor(cell), ncells)
    g_ev, _ = ctx.read_event_log()
    g_store = store.to_numpy()
    cf = O.make_config(seed, process_mask=3, cascade=1)
    Nc = O.plan_cells(cf, arr, cell, ncells)
    first = np.where(cell < ncells, Nc[np.minimum(cell, ncells - 1)], 0)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=cap, first_N=first)
    # a cell whose count may differ (a member's own count is a near-tie) is
    # exempt as a whole: its rows are marked tied from their first sub-step
    _, n_own, tie = _oracle_plans(cf, arr, np.arange(n))
    bad_cells = set(cell[tie].tolist())
    extra = [(int(arr["id"][i]), 0, 2) for i in range(n) if int(cell[i]) in bad_cells]
    ties = np.concatenate([o_ties, np.array(extra, dtype=o_ties.dtype)]) if extra else o_ties
    rep = parity.compare(g_ev, o_ev, ties, g_store, o_store, arr["id"])
    print("cells parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "gpu", g_st, "oracle", o_st)
    assert g_st["status"] == 0 and o_st["status"] == 0
    assert not rep["mismatches"], rep["mismatches"][:5]
    assert rep["exempt"] <= 1e-3 * rep["particles"] + 16 * len(bad_cells)
    assert rep["final_checked"] > 0.5 * rep["particles"]
    if not len(ties):
        for k in ("substeps", "emissions", "pairs", "children", "plans"):
            assert g_st[k] == o_st[k], k
    # the comparison is not vacuous: the cells' counts raise many first plans
    assert (first > n_own).sum() > n // 4


def test_one_row_per_cell_is_the_plain_step():
    n = 5000
    arr = I.clumped_mixed(n, 31, hot_fraction=0.05)
    a_ctx = qed.Context(seed=9)
    b_ctx = qed.Context(seed=9)
    a = qed.ParticleStore.from_numpy(arr, capacity=n * 30)
    b = qed.ParticleStore.from_numpy(arr, capacity=n * 30)
    sa = a_ctx.event_step(a, 1)
    sb = b_ctx.event_step_cells(b, 1, _cell_tensor(np.arange(n)), n)
    for k in ("substeps", "emissions", "pairs", "children", "plans", "max_N", "count", "status"):
        assert sa[k] == sb[k], k
    A, B = a.to_numpy(), b.to_numpy()
    for k in A:   # initial rows in place, children by id
        np.testing.assert_array_equal(A[k][:n], B[k][:n], err_msg=k)
    CA = _by_id({k: v[n:] for k, v in A.items()})
    CB = _by_id({k: v[n:] for k, v in B.items()})
    for k in CA:
        np.testing.assert_array_equal(CA[k], CB[k], err_msg=k)


def test_cells_tail_pass_equals_generations():
    # the first-plan rule is applied wherever a first plan is made (thread
    # pass, both hot-pass modes, the tail pass): the step gives the same
    # result with and without the tail pass
    n = 40000
    arr = I.clumped_mixed(n, 71, hot_fraction=0.01)
    cell = torch.from_numpy((np.arange(n) // 64).astype(np.int32)).cuda()
    ncells = (n + 63) // 64
    out = []
    for tail in (0, None):
        ctx = qed.Context(seed=13)
        if tail is not None:
            ctx.set_tail(tail)
        store = qed.ParticleStore.from_numpy(arr, capacity=n * 40)
        st = ctx.event_step_cells(store, 4, cell, ncells)
        out.append((st, store.to_numpy()))
    (g, a), (t, b) = out
    assert g["status"] == 0 and t["status"] == 0 and g["tail"] == 0 and t["tail"] == 1
    for k in ("substeps", "emissions", "pairs", "children", "plans", "max_N", "count"):
        assert g[k] == t[k], (k, g[k], t[k])
    A, B = _by_id(a), _by_id(b)
    for k in A:
        np.testing.assert_array_equal(A[k], B[k], err_msg=k)


def test_cells_rejects_bad_arguments():
    ctx = qed.Context()
    store = qed.ParticleStore.from_numpy(I.clumped_mixed(100, 3), capacity=1000)
    cell = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(qed.QEDError):
        ctx.event_step_cells(store, 0, cell, 0)
    sctx = qed.Context(sampler=True)
    with pytest.raises(qed.QEDError):
        sctx.event_step_cells(store, 0, cell, 1)
