"""Store compaction, photon drain and the multi-step CUDA graph.  GPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2008_10468_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402


def _sorted(store_np):
    o = np.argsort(store_np["id"])
    return {k: v[o] for k, v in store_np.items()}


@pytest.mark.parametrize("n,frac", [(0, 0.0), (1, 1.0), (4095, 0.3), (4097, 0.0), (50001, 0.5),
                                    (12288, 1.0)])
def test_compaction_is_stable_and_exact(n, frac):
    ctx = qed.Context()
    arr = I.clumped_mixed(max(n, 1), 6)
    arr = {k: v[:n] for k, v in arr.items()}
    rng = np.random.default_rng(n)
    dead = rng.random(n) < frac
    arr["type"] = np.where(dead, 3, arr["type"]).astype(np.uint8)
    store = qed.ParticleStore.from_numpy(arr, capacity=n + 9000)
    removed = ctx.compact(store)
    assert removed == int(dead.sum())
    got = store.to_numpy()
    keep = ~dead
    for k in arr:
        np.testing.assert_array_equal(got[k], arr[k][keep])


def test_photon_drain_fills_spectrum():
    arr = I.clumped_mixed(20000, 9)
    cf = O.make_config(1)
    chi = np.array([O.chi((arr["px"][i], arr["py"][i], arr["pz"][i]),
                          (arr["Ex"][i], arr["Ey"][i], arr["Ez"][i]),
                          (arr["Bx"][i], arr["By"][i], arr["Bz"][i]), photon=True)[0]
                    for i in range(20000)])
    photon = arr["type"] == 2
    thr = 5e-3
    drained = photon & (chi < thr)
    margin = photon & (np.abs(chi / thr - 1) < 1e-5)   # binary32 chi may fall either side
    ctx = qed.Context(drain_chi=thr)
    store = qed.ParticleStore.from_numpy(arr, capacity=20000)
    ctx.read_spectrum(reset=True)
    removed = ctx.compact(store)
    assert abs(removed - drained.sum()) <= margin.sum()
    spec = ctx.read_spectrum()
    assert spec.sum() == pytest.approx(float(arr["w"][drained].sum()), abs=margin.sum() + 1e-6)
    energy = np.sqrt(arr["px"] ** 2 + arr["py"] ** 2 + arr["pz"] ** 2)[drained]
    h, _ = np.histogram(np.log10(energy), bins=qed.SPECTRUM_BINS,
                        range=(qed.SPECTRUM_LOG10_MIN, qed.SPECTRUM_LOG10_MAX))
    assert np.abs(spec - h).sum() <= 2 * margin.sum() + 2  # bin-edge rounding only


def _eager_steps(arr, cap, first, k, **cfg):
    ctx = qed.Context(**cfg)
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    stats = []
    for j in range(k):
        st = ctx.event_step(store, first + j)
        ctx.compact(store)
        st["count"] = store.n()
        stats.append(st)
    return store.to_numpy(), stats


def _graph_steps(arr, cap, first, k, **cfg):
    ctx = qed.Context(**cfg)
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    ctx.graph_capture(store, first, k)
    ctx.graph_launch()
    stats = ctx.graph_read_stats()
    return store.to_numpy(), stats, ctx, store


def _same(e_stats, g_stats, e_store, g_store):
    for a, b in zip(e_stats, g_stats):
        for k in ("substeps", "emissions", "pairs", "children", "plans", "candidates", "max_N",
                  "passes", "status", "count"):
            assert a[k] == b[k], (k, a[k], b[k])
    e, g = _sorted(e_store), _sorted(g_store)
    for k in e:
        np.testing.assert_array_equal(e[k], g[k])


def test_graph_equals_eager_steps():
    arr = I.clumped_mixed(3000, 21, hot_fraction=0.03)
    cap = 2_000_000
    ectx = qed.Context(seed=99)
    estore = qed.ParticleStore.from_numpy(arr, capacity=cap)

    def eager(first, k):
        stats = []
        for j in range(k):
            st = ectx.event_step(estore, first + j)
            ectx.compact(estore)
            st["count"] = estore.n()
            stats.append(st)
        return stats

    e_stats = eager(50, 5)
    g_store, g_stats, ctx, store = _graph_steps(arr, cap, 50, 5, seed=99)
    _same(e_stats, g_stats, estore.to_numpy(), g_store)
    # a second launch continues from the evolved store with steps 55..59
    e_stats2 = eager(55, 5)
    ctx.graph_launch()
    g_stats2 = ctx.graph_read_stats()
    assert all(s["status"] == 0 for s in g_stats2), [s["status"] for s in g_stats2]
    _same(e_stats2, g_stats2, estore.to_numpy(), store.to_numpy())


def test_graph_capacity_overflow_is_sticky():
    arr = I.uniform_field_electrons(2000, 20081047)
    g_store, stats, ctx, store = _graph_steps(arr, 2300, 0, 4, process_mask=1, cascade=False)
    assert stats[0]["status"] == qed.QED_ERR_CAPACITY
    assert stats[0]["required_capacity"] > 2300
    for s in stats[1:]:
        assert s["status"] == qed.QED_ERR_CAPACITY and s["substeps"] == 0
    # the context is still usable: a new capture on a roomy store works
    store2 = qed.ParticleStore.from_numpy(I.uniform_field_electrons(100, 1), capacity=100000)
    ctx.graph_capture(store2, 0, 2)
    ctx.graph_launch()
    assert all(s["status"] == 0 for s in ctx.graph_read_stats())


def test_cascade_batch_graph_small():
    # the cascade batch grows roughly tenfold per step even with the drain
    arr, cell = I.cascade_cells(128, 20081050, n_max=4096)
    n = len(arr["px"])
    _, stats, ctx, store = _graph_steps(arr, n * 2000, 0, 3, seed=20081050, drain_chi=0.05)
    assert all(s["status"] == 0 for s in stats), stats
    assert stats[-1]["count"] > 0
    assert sum(s["substeps"] for s in stats) > n
    assert ctx.read_spectrum().sum() > 0


def test_host_loop_equals_graph_step():
    # with per-kernel timing the step runs generation by generation from the
    # host; without, as the cached one-step graph: same results
    arr = I.clumped_mixed(30000, 33, hot_fraction=0.03)
    cap = 30000 * 40
    out = []
    for profile in (False, True):
        ctx = qed.Context(seed=17)
        ctx.profile(profile)
        store = qed.ParticleStore.from_numpy(arr, capacity=cap)
        sts = []
        for k in range(2):
            sts.append(ctx.event_step(store, 40 + k))
            assert sts[-1]["count"] == store.n()   # the count after the step's children
        assert sts[0]["children"] > 0
        out.append((sts, _sorted(store.to_numpy())))
    (sa, ga), (sb, gb) = out
    for a, b in zip(sa, sb):
        for k in ("substeps", "emissions", "pairs", "children", "plans", "max_N", "passes",
                  "status", "count"):
            assert a[k] == b[k], (k, a[k], b[k])
    for k in ga:
        np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("n,hot,profile", [(3000, 0.03, False), (30000, 0.01, True),
                                           (200000, 0.01, False)])
def test_tail_pass_equals_generations(n, hot, profile):
    # generations below tail_rows are finished by one thread pass and one
    # persistent kernel; every decision is the generation loop's
    arr = I.clumped_mixed(n, 41, hot_fraction=hot)
    cap = n * 40
    out = []
    for tail in (0, 1 << 30, 4096):
        ctx = qed.Context(seed=23)
        ctx.set_tail(tail)
        ctx.profile(profile)
        store = qed.ParticleStore.from_numpy(arr, capacity=cap)
        sts = []
        for k in range(2):
            sts.append(ctx.event_step(store, 60 + k))
            assert sts[-1]["status"] == 0
            assert sts[-1]["count"] == store.n()
        out.append((sts, _sorted(store.to_numpy())))
    (s0, g0) = out[0]
    assert s0[0]["children"] > 0 and s0[0]["passes"] > 2
    assert all(s["tail"] == 0 for s in s0) and all(s["tail"] == 1 for s in out[1][0])
    for sts, g in out[1:]:
        for a, b in zip(s0, sts):
            # (candidates also count draws past an event, which depend on the
            # launch shape: not compared)
            for k in ("substeps", "emissions", "pairs", "children", "plans", "max_N", "count"):
                assert a[k] == b[k], (k, a[k], b[k])
        for k in g0:
            np.testing.assert_array_equal(g0[k], g[k])
    # with the tail from the second generation on, a step has at most three passes
    assert all(s["passes"] <= 3 for s in out[1][0])


def test_tail_pass_in_multi_step_graph():
    arr = I.clumped_mixed(20000, 43, hot_fraction=0.02)
    cap = 20000 * 40
    res = []
    for tail in (0, 1 << 30):
        ctx = qed.Context(seed=5)
        ctx.set_tail(tail)
        store = qed.ParticleStore.from_numpy(arr, capacity=cap)
        ctx.graph_capture(store, 70, 3)
        ctx.graph_launch()
        res.append((ctx.graph_read_stats(), _sorted(store.to_numpy())))
    (sa, ga), (sb, gb) = res
    for a, b in zip(sa, sb):
        assert a["status"] == 0 and b["status"] == 0
        for k in ("substeps", "emissions", "pairs", "children", "plans", "count"):
            assert a[k] == b[k], (k, a[k], b[k])
    for k in ga:
        np.testing.assert_array_equal(ga[k], gb[k])


@pytest.mark.parametrize("tail", [0, 1 << 30])
def test_capacity_overflow_in_the_cascade(tail):
    # children that do not fit end the step with QED_ERR_CAPACITY and the rows
    # needed.  With room for 80% of the children the overflow comes after the
    # first generation, i.e. inside the tail pass when it is on: there the rows
    # published as removed by a failed reservation are completed like any
    # other, so the step ends (no timeout)
    n = 4000
    arr = I.clumped_mixed(n, 51, hot_fraction=0.05)
    ctx = qed.Context(seed=3)
    ctx.set_tail(tail)
    full = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
    st_full = ctx.event_step(full, 9)
    assert st_full["status"] == 0
    total = st_full["count"]
    cap = n + int(0.8 * (total - n))
    ctx = qed.Context(seed=3)
    ctx.set_tail(tail)
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    st = ctx.event_step(store, 9)
    assert st["status"] == qed.QED_ERR_CAPACITY
    assert st["required_capacity"] > cap
    assert store.n() == cap and st["count"] == cap
    if tail:
        assert st["tail"] == 1


@pytest.mark.parametrize("graph", [False, True])
def test_tail_pass_wait_limit_ends_the_step_with_timeout(graph):
    # failure detection without a fault: every wait of the tail pass is
    # bounded.  With a limit of 1 ns the persistent kernel's warps give up at
    # their first idle poll, so the step ends with QED_ERR_TIMEOUT instead of
    # waiting; in a multi-step graph the following steps do nothing.  Back at
    # the default limit the context steps as a fresh one does.
    n = 4000
    arr = I.clumped_mixed(n, 51, hot_fraction=0.05)
    ctx = qed.Context(seed=3)
    ctx.set_wait_limit(1)
    store = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
    if graph:
        ctx.graph_capture(store, 9, 2)
        ctx.graph_launch()
        stats = ctx.graph_read_stats()
        assert stats[0]["status"] == qed.QED_ERR_TIMEOUT and stats[0]["tail"] == 1, stats[0]
        assert stats[1]["status"] == qed.QED_ERR_TIMEOUT and stats[1]["substeps"] == 0
    else:
        st = ctx.event_step(store, 9)
        assert st["status"] == qed.QED_ERR_TIMEOUT and st["tail"] == 1, st
    ctx.set_wait_limit(0)
    again = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
    st = ctx.event_step(again, 9)
    ref_ctx = qed.Context(seed=3)
    ref = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
    st_ref = ref_ctx.event_step(ref, 9)
    assert st["status"] == 0 and st["tail"] == 1
    for k in ("substeps", "emissions", "pairs", "children", "plans", "count"):
        assert st[k] == st_ref[k], (k, st[k], st_ref[k])
    a, b = _sorted(again.to_numpy()), _sorted(ref.to_numpy())
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_host_store_step_equals_device_step():
    # qed_event_step_host: the store in host memory, copied in, stepped and
    # copied back by the library; the same kernels run on the same rows, so
    # the result equals qed_event_step's bit for bit (initial rows in place,
    # children by id), for page-locked and pageable host arrays
    n = 5000
    arr = I.clumped_mixed(n, 57, hot_fraction=0.03)
    ref_ctx = qed.Context(seed=12)
    ref = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
    st_ref = ref_ctx.event_step(ref, 4)
    assert st_ref["children"] > 0
    R = ref.to_numpy()
    for pinned in (True, False):
        ctx = qed.Context(seed=12)
        h = qed.HostStore.from_numpy(arr, capacity=n * 60, pinned=pinned)
        st = ctx.event_step_host(h, 4)
        assert st["status"] == 0 and h.n() == st_ref["count"]
        for k in ("substeps", "emissions", "pairs", "children", "plans", "count"):
            assert st[k] == st_ref[k], (k, st[k], st_ref[k])
        H = h.to_numpy()
        for k in H:
            np.testing.assert_array_equal(H[k][:n], R[k][:n], err_msg=k)
        a, b = _sorted({k: v[n:] for k, v in H.items()}), _sorted({k: v[n:] for k, v in R.items()})
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        # a second step continues from the updated host store
        st2 = ctx.event_step_host(h, 5)
        st2_ref = ref_ctx.event_step(ref, 5)
        for k in ("substeps", "emissions", "pairs", "children", "count"):
            assert st2[k] == st2_ref[k], (k, st2[k], st2_ref[k])
        ref = qed.ParticleStore.from_numpy(arr, capacity=n * 60)
        ref_ctx.event_step(ref, 4)


def test_host_store_step_leaves_the_store_on_failure():
    n = 2000
    arr = I.uniform_field_electrons(n, 20081047)
    ctx = qed.Context(seed=3, process_mask=1, cascade=False)
    h = qed.HostStore.from_numpy(arr, capacity=2100)
    before = h.to_numpy()
    st = ctx.event_step_host(h, 0)
    assert st["status"] == qed.QED_ERR_CAPACITY and st["required_capacity"] > 2100
    assert h.n() == n
    after = h.to_numpy()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k], err_msg=k)
    # bad arguments
    h.count = 2101
    with pytest.raises(qed.QEDError):
        ctx.event_step_host(h, 0)
    h.count = n
    with pytest.raises(qed.QEDError):
        ctx.event_step_host(h, 1 << 33)
    # empty store
    e = qed.HostStore(16)
    st = ctx.event_step_host(e, 0)
    assert st["status"] == 0 and st["substeps"] == 0 and e.n() == 0
