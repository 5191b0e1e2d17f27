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


def _check(arr, step, capacity, seed, mask=3, cascade=True, recoil=True, max_exempt=0.1):
    g_store, g_st, g_ev = _run_gpu(arr, step, capacity, seed=seed, process_mask=mask,
                                   cascade=cascade, recoil=recoil)
    cf = O.make_config(seed, process_mask=mask, cascade=int(cascade), recoil=int(recoil), push=1)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=capacity)
    assert g_st["status"] == 0 and o_st["status"] == 0
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
    print("push parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "gpu", g_st, "oracle", o_st)
    assert not rep["mismatches"], rep["mismatches"][:5]
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
    assert g_st["pairs"] > 0 and g_st["passes"] > 1


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
    print("sampled push parity:", {k: v for k, v in rep.items() if k != "mismatches"})
    assert not rep["mismatches"], rep["mismatches"][:5]
    assert rep["events"] > 100


def test_push_capacity_overflow_reports_required_rows():
    arr = I.uniform_field_electrons(2000, 20081047)
    ctx = qed.Context(process_mask=1, cascade=False)
    store = qed.ParticleStore.from_numpy(arr, capacity=2100)
    st = ctx.event_step(store, 0, push=True)
    assert st["status"] == qed.QED_ERR_CAPACITY
    assert st["required_capacity"] > 2100
    assert store.n() == 2100
    # with the cascade on, the generations stop at the overflow
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
