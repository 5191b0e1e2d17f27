"""Parity of the push-mode event step (Algorithm 1 with the Boris push before
every e+- draw) with the oracle's push mode, through the C ABI.  GPU only.

Same protocol as the other event-step parity tests (tests/parity.py): events
identical per particle up to the oracle's first near-tie, energy fractions
within binary32 rounding, final momenta within p_rtol of |p|.  The push is
the same binary32 evaluation on both sides, so the momenta differ only where
the recoil's rounding differs (a few ulps, carried on by later pushes)."""
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


def _run_gpu(arr, step, capacity, log_cap=1 << 20, push=True, **cfg):
    ctx = qed.Context(**cfg)
    ctx.set_event_log(log_cap)
    store = qed.ParticleStore.from_numpy(arr, capacity=capacity)
    st = ctx.event_step(store, step, push=push)
    ev, nev = ctx.read_event_log()
    assert nev <= log_cap
    return store.to_numpy(), st, ev


def _check(arr, step, capacity, seed, mask=3, cascade=True, recoil=True, max_exempt=1e-3):
    g_store, g_st, g_ev = _run_gpu(arr, step, capacity, seed=seed, process_mask=mask,
                                   cascade=cascade, recoil=recoil)
    cf = O.make_config(seed, process_mask=mask, cascade=int(cascade), recoil=int(recoil), push=1)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=capacity)
    assert g_st["status"] == 0 and o_st["status"] == 0
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
    print("push parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "gpu", g_st, "oracle", o_st)
    assert not rep["mismatches"], rep["mismatches"][:5]
    print("exempt fraction %.2e" % (rep["exempt"] / max(rep["particles"], 1)))
    assert rep["exempt"] <= max_exempt * rep["particles"]
    assert rep["final_checked"] > 0.5 * rep["particles"]
    if len(o_ties) == 0:
        for k in ("substeps", "emissions", "pairs", "children", "plans"):
            assert g_st[k] == o_st[k], k
    return rep, g_st, o_st, g_store


def test_push_uniform_field_emission():
    arr = I.uniform_field_electrons(300, 20081047)
    rep, g_st, _, g_store = _check(arr, 0, 300 * 200, 20081047, mask=1, cascade=False)
    assert g_st["emissions"] > 100
    # the push moved every electron: no final momentum equals the initial one
    moved = (g_store["px"][:300] != arr["px"]) | (g_store["py"][:300] != arr["py"])
    assert moved.all()


def test_push_clumped_cascade():
    arr = I.clumped_mixed(4133, 20081049, hot_fraction=0.02)
    rep, g_st, _, _ = _check(arr, 3, 4133 * 20, 20081049, mask=3, cascade=True)
    # the cascade runs as one persistent pass that takes children as they come
    assert g_st["pairs"] > 0 and g_st["tail"] == 1 and g_st["passes"] == 1


def test_push_without_recoil():
    # without recoil an e+- of the initial store is moved by the push alone:
    # both sides evaluate the same binary32 operations from the same sub-step
    # length, so its final momentum is bit-identical to the oracle's (the
    # length is the binary32 rounding of t/N from float-float on the GPU and
    # from binary64 in the oracle: they can differ in a rare near-half case)
    arr = I.clumped_mixed(1500, 77, hot_fraction=0.05)
    seed, step, cap = 77, 1, 1500 * 40
    g_store, _, g_ev = _run_gpu(arr, step, cap, seed=seed, process_mask=3, cascade=True,
                                recoil=False)
    cf = O.make_config(seed, process_mask=3, cascade=1, recoil=0, push=1)
    o_store, _, o_ev, o_ties = O.event_step(cf, arr, step, capacity=cap)
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
    assert not rep["mismatches"], rep["mismatches"][:5]
    tied = {int(t["id"]) for t in o_ties}
    lep = [j for j in range(1500) if arr["type"][j] < 2 and int(arr["id"][j]) not in tied]
    same = sum(all(g_store[k][j] == o_store[k][j] for k in ("px", "py", "pz")) for j in lep)
    print("bit-identical e+- momenta: %d of %d" % (same, len(lep)))
    assert len(lep) > 500 and same >= 0.99 * len(lep)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 64])
def test_push_tiny_populations_over_several_steps(n):
    arr = I.clumped_mixed(max(n, 4), 900 + n, hot_fraction=0.5)
    arr = {k: v[:n] for k, v in arr.items()}
    for step in range(3):
        g_store, g_st, g_ev = _run_gpu(arr, step, n * 4000, seed=61 + n, process_mask=3,
                                       cascade=True)
        cf = O.make_config(61 + n, process_mask=3, cascade=1, push=1)
        o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=n * 4000)
        rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
        assert g_st["status"] == 0 and o_st["status"] == 0
        assert not rep["mismatches"], (step, rep["mismatches"][:3])
        arr = g_store


def test_push_leaves_photons_as_the_plain_step():
    arr = I.clumped_mixed(3000, 12, hot_fraction=0.1)
    ph = np.nonzero(arr["type"] == 2)[0]
    arr = I.subset(arr, ph)
    a, sa, ea = _run_gpu(arr, 2, len(ph) * 4, push=False, seed=5, process_mask=2, cascade=False)
    b, sb, eb = _run_gpu(arr, 2, len(ph) * 4, push=True, seed=5, process_mask=2, cascade=False)
    assert sa["pairs"] > 0
    for k in ("substeps", "pairs", "children", "plans"):
        assert sa[k] == sb[k], k
    key = lambda e: (int(e["parent_id"]), int(e["s"]))  # noqa: E731
    assert sorted(map(key, ea)) == sorted(map(key, eb))
    n = len(ph)
    for k in ("px", "py", "pz", "type"):
        assert np.array_equal(a[k][:n], b[k][:n]), k


def test_push_full_size_sampled():
    """The 2^24 clumped population in push mode; 64 sampled roots (24 of the
    hot clump, with their cascades) against the oracle."""
    n = 1 << 24
    arr = I.clumped_mixed(n, 20081049)
    n_hot = int(round(n * 0.01))
    h0 = (n - n_hot) // 2
    rng = np.random.default_rng(13)
    hot = rng.choice(np.arange(h0, h0 + n_hot), 24, replace=False)
    cold = rng.choice(np.concatenate([np.arange(0, h0), np.arange(h0 + n_hot, n)]), 40,
                      replace=False)
    roots = np.sort(np.concatenate([hot, cold]))
    g_store, g_st, g_ev = _run_gpu(arr, 0, n + (1 << 25), log_cap=1 << 25, seed=20081049,
                                   process_mask=3, cascade=True)
    print("push full-size step:", g_st)
    assert g_st["status"] == 0
    sub = I.subset(arr, roots)
    cf = O.make_config(20081049, process_mask=3, cascade=1, push=1)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, sub, 0, capacity=len(roots) * 4000)
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, sub["id"])
    print("sampled push parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "exempt fraction %.2e" % (rep["exempt"] / max(rep["particles"], 1)))
    assert not rep["mismatches"], rep["mismatches"][:5]
    assert rep["events"] > 100
    assert rep["exempt"] <= 1e-3 * rep["particles"]


def test_push_capacity_overflow_reports_required_rows():
    arr = I.uniform_field_electrons(2000, 20081047)
    ctx = qed.Context(process_mask=1, cascade=False)
    store = qed.ParticleStore.from_numpy(arr, capacity=2100)
    st = ctx.event_step(store, 0, push=True)
    assert st["status"] == qed.QED_ERR_CAPACITY
    assert st["required_capacity"] > 2100
    assert store.n() == 2100
    # with the cascade on (one persistent pass) the step reports the overflow too
    store = qed.ParticleStore.from_numpy(arr, capacity=2100)
    ctx2 = qed.Context(process_mask=3, cascade=True)
    st = ctx2.event_step(store, 0, push=True)
    assert st["status"] == qed.QED_ERR_CAPACITY and st["passes"] == 1
    # the context stays usable after the error
    store2 = qed.ParticleStore.from_numpy(I.uniform_field_electrons(100, 1), capacity=100000)
    assert ctx.event_step(store2, 1, push=True)["status"] == 0


def test_push_empty_store_and_bad_arguments():
    ctx = qed.Context()
    store = qed.ParticleStore(1024)
    st = ctx.event_step(store, 0, push=True)
    assert st["status"] == 0 and st["substeps"] == 0
    with pytest.raises(qed.QEDError):
        ctx.event_step(store, 1 << 33, push=True)


def _cells_check(arr, cell, ncells, seed, step=0, cap_mult=20):
    n = len(arr["px"])
    ctx = qed.Context(seed=seed, process_mask=3, cascade=True)
    ctx.set_event_log(1 << 20)
    store = qed.ParticleStore.from_numpy(arr, capacity=n * cap_mult)
    cd = torch.from_numpy(cell.astype(np.uint32).view(np.int32)).cuda()
    g_st = ctx.event_step_push_cells(store, step, cd, ncells)
    g_ev, _ = ctx.read_event_log()
    g_store = store.to_numpy()
    cf = O.make_config(seed, process_mask=3, cascade=1, push=1)
    Nc = O.plan_cells(cf, arr, cell, ncells)
    first = np.where(cell < ncells, Nc[np.minimum(cell, ncells - 1)], 0)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=n * cap_mult,
                                               first_N=first)
    # a cell whose count may differ (a member's own count is a near-tie) is
    # exempt as a whole: its rows are marked tied from their first sub-step
    from tests.test_gpu_parity import _oracle_plans
    _, _, tie = _oracle_plans(cf, arr, np.arange(n))
    bad_cells = set(cell[tie].tolist())
    extra = [(int(arr["id"][i]), 0, 2) for i in range(n) if int(cell[i]) in bad_cells]
    ties = np.concatenate([o_ties, np.array(extra, dtype=o_ties.dtype)]) if extra else o_ties
    rep = parity.compare(g_ev, o_ev, ties, g_store, o_store, arr["id"])
    print("push cells parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "gpu", g_st, "oracle", o_st)
    assert g_st["status"] == 0 and o_st["status"] == 0
    assert not rep["mismatches"], rep["mismatches"][:5]
    assert rep["final_checked"] > 0.5 * rep["particles"]
    return g_st, o_st


def test_push_cells_parity():
    arr = I.clumped_mixed(4133, 20081049, hot_fraction=0.02)
    cell = (np.arange(4133) // 16).astype(np.uint32)
    cell[::97] = 10 ** 6    # out of range: these rows keep their own count
    g_st, o_st = _cells_check(arr, cell, (4133 + 15) // 16, 20081049, step=3)
    plain = qed.Context(seed=20081049, process_mask=3, cascade=True)
    store = qed.ParticleStore.from_numpy(arr, capacity=4133 * 20)
    assert g_st["substeps"] > plain.event_step(store, 3, push=True)["substeps"]


def test_push_one_row_per_cell_is_the_push_step():
    arr = I.clumped_mixed(2000, 31, hot_fraction=0.05)
    n = 2000
    a_ctx = qed.Context(seed=9, process_mask=3, cascade=True)
    b_ctx = qed.Context(seed=9, process_mask=3, cascade=True)
    a = qed.ParticleStore.from_numpy(arr, capacity=n * 20)
    b = qed.ParticleStore.from_numpy(arr, capacity=n * 20)
    sa = a_ctx.event_step(a, 1, push=True)
    cd = torch.arange(n, dtype=torch.int32, device="cuda")
    sb = b_ctx.event_step_push_cells(b, 1, cd, n)
    for k in ("substeps", "emissions", "pairs", "children", "plans", "count", "status"):
        assert sa[k] == sb[k], k
    # initial rows in place; children (appended in reservation order) by id
    A, B = a.to_numpy(), b.to_numpy()
    ia, ib = np.argsort(A["id"][n:]), np.argsort(B["id"][n:])
    for k in A:
        assert np.array_equal(A[k][:n], B[k][:n]), k
        assert np.array_equal(A[k][n:][ia], B[k][n:][ib]), k
    with pytest.raises(qed.QEDError):
        b_ctx.event_step_push_cells(b, 1, cd, 0)


def _by_id(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items()}


@pytest.mark.parametrize("cells", [False, True])
def test_push_persistent_pass_equals_generations(cells):
    # the whole step in one persistent launch (children taken as soon as they
    # are reserved) against the generation loop (tail_rows 0): the draws are
    # keyed by (id, step, sub-step) and the push is a fixed sequence of
    # binary32 operations, so statistics and store (by id) are equal bit for
    # bit whatever the order in which the lanes take the rows
    n = 30011
    arr = I.clumped_mixed(n, 20081049, hot_fraction=0.01)
    cell = torch.from_numpy((np.arange(n) // 16).astype(np.int32)).cuda()
    out = []
    for tail in (0, None):
        ctx = qed.Context(seed=41, process_mask=3, cascade=True)
        if tail is not None:
            ctx.set_tail(tail)
        store = qed.ParticleStore.from_numpy(arr, capacity=n * 40)
        if cells:
            st = ctx.event_step_push_cells(store, 6, cell, (n + 15) // 16)
        else:
            st = ctx.event_step(store, 6, push=True)
        out.append((st, store.to_numpy()))
    (g, a), (t, b) = out
    assert g["status"] == 0 and t["status"] == 0
    assert g["tail"] == 0 and g["passes"] > 2 and t["tail"] == 1 and t["passes"] == 1
    for k in ("substeps", "emissions", "pairs", "children", "plans", "candidates", "max_N",
              "guard_hits", "count"):
        assert g[k] == t[k], (k, g[k], t[k])
    for k in a:   # initial rows in place, then the children by id
        np.testing.assert_array_equal(a[k][:n], b[k][:n], err_msg=k)
    A, B = _by_id({k: v[n:] for k, v in a.items()}), _by_id({k: v[n:] for k, v in b.items()})
    for k in A:
        np.testing.assert_array_equal(A[k], B[k], err_msg=k)


def test_push_persistent_pass_wait_limit_ends_the_step_with_timeout():
    # failure detection without a fault: with a wait limit of 1 ns the
    # persistent pass's warps give up at their first idle poll (more lanes
    # than rows), the step ends with QED_ERR_TIMEOUT, and at the default limit
    # the context steps as a fresh one does
    n = 3000
    arr = I.clumped_mixed(n, 52, hot_fraction=0.05)
    ctx = qed.Context(seed=8, process_mask=3, cascade=True)
    ctx.set_wait_limit(1)
    store = qed.ParticleStore.from_numpy(arr, capacity=n * 40)
    st = ctx.event_step(store, 2, push=True)
    assert st["status"] == qed.QED_ERR_TIMEOUT and st["tail"] == 1, st
    ctx.set_wait_limit(0)
    again = qed.ParticleStore.from_numpy(arr, capacity=n * 40)
    st = ctx.event_step(again, 2, push=True)
    ref_ctx = qed.Context(seed=8, process_mask=3, cascade=True)
    ref = qed.ParticleStore.from_numpy(arr, capacity=n * 40)
    st_ref = ref_ctx.event_step(ref, 2, push=True)
    assert st["status"] == 0 and st_ref["status"] == 0
    for k in ("substeps", "emissions", "pairs", "children", "plans", "count"):
        assert st[k] == st_ref[k], (k, st[k], st_ref[k])
    a, b = _by_id(again.to_numpy()), _by_id(ref.to_numpy())
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
