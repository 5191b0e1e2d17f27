"""qed_event_step_noalloc, the event step for callers that cannot allocate
device memory (hosts that hand out a fixed memory budget in advance, plug-ins
living inside another program's memory pool), must give the results of
qed_event_step.  It keeps its scratch in a device array built into the
library, so two calls in a row also check that nothing left over from the
first call changes the second.  Both entry points run the same kernels with
the same keyed draws, so the stores must be equal bit for bit.
GPU only; this file is named to run after the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2008_10468_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402

MAX_ROWS = 65536   # QED_NOALLOC_MAX_ROWS


def _noalloc_fn():
    L = qed.lib()
    f = L.qed_event_step_noalloc
    f.argtypes = [C.POINTER(qed.Config), C.POINTER(qed.Particles), C.c_uint64, C.c_void_p,
                  C.POINTER(qed.StepStats)]
    f.restype = C.c_int
    return f


def _config(seed, cascade=True, sampler_mode=0):
    cfg = qed.Config()
    qed.lib().qed_config_default(C.byref(cfg))
    cfg.seed = seed
    cfg.cascade_in_step = 1 if cascade else 0
    cfg.sampler_mode = sampler_mode
    return cfg


def _sorted(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items()}


def _noalloc_step(fn, arr, cap, step, seed, cascade=True):
    got = qed.ParticleStore.from_numpy(arr, capacity=cap)
    out = qed.StepStats()
    status = fn(C.byref(_config(seed, cascade)), C.byref(got.struct()), step,
                C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out))
    return status, qed.stats_dict(out), got


def test_noalloc_matches_event_step_on_two_calls():
    fn = _noalloc_fn()
    seed = 4242
    arr = I.clumped_mixed(5000, 31, hot_fraction=0.03)
    ctx = qed.Context(seed=seed)
    # the second call fills the largest store the entry point accepts, whose
    # long-plan queue is then exactly full
    for call, (step, cap) in enumerate(((7, 60000), (8, MAX_ROWS))):
        ref = qed.ParticleStore.from_numpy(arr, capacity=cap)
        st_ref = ctx.event_step(ref, step)
        status, st, got = _noalloc_step(fn, arr, cap, step, seed)
        assert status == qed.QED_OK, status
        assert st_ref["children"] > 0 and st_ref["tail"] == 1
        for k in ("substeps", "emissions", "pairs", "children", "plans", "candidates", "max_N",
                  "passes", "count", "status", "tail"):
            assert st[k] == st_ref[k], (call, k, st[k], st_ref[k])
        a, b = _sorted(ref.to_numpy()), _sorted(got.to_numpy())
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg="%d %s" % (call, k))


def test_noalloc_capacity_overflow_matches_event_step():
    fn = _noalloc_fn()
    seed = 17
    arr = I.uniform_field_electrons(2000, 20081047)
    # one generation: the rows needed are the same whatever the order of the
    # reservations
    ctx = qed.Context(seed=seed, cascade=False)
    ref = qed.ParticleStore.from_numpy(arr, capacity=2100)
    st_ref = ctx.event_step(ref, 0)
    status, st, got = _noalloc_step(fn, arr, 2100, 0, seed, cascade=False)
    assert st_ref["status"] == qed.QED_ERR_CAPACITY
    assert status == qed.QED_ERR_CAPACITY and st["status"] == qed.QED_ERR_CAPACITY
    assert st["required_capacity"] == st_ref["required_capacity"] > 2100
    assert st["count"] == st_ref["count"] == 2100 == got.n()
    # with the cascade the store is full at the end of the step as well
    arr = I.clumped_mixed(4000, 51, hot_fraction=0.05)
    status, st, got = _noalloc_step(fn, arr, 6000, 9, seed)
    assert status == qed.QED_ERR_CAPACITY and st["required_capacity"] > 6000
    assert st["count"] == 6000 == got.n()
    # and the next call on a roomy store is exact again
    ctx = qed.Context(seed=seed)
    ref = qed.ParticleStore.from_numpy(arr, capacity=MAX_ROWS)
    st_ref = ctx.event_step(ref, 9)
    status, st, got = _noalloc_step(fn, arr, MAX_ROWS, 9, seed)
    assert status == qed.QED_OK
    for k in ("substeps", "emissions", "pairs", "children", "count"):
        assert st[k] == st_ref[k], k
    a, b = _sorted(ref.to_numpy()), _sorted(got.to_numpy())
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_noalloc_rejects_what_it_cannot_do():
    fn = _noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = qed.StepStats()
    big = qed.ParticleStore(MAX_ROWS + 1)
    assert fn(C.byref(_config(1)), C.byref(big.struct()), 0, stream,
              C.byref(out)) == qed.QED_ERR_ARG
    # the learned sampler lives in a context: not available here
    small = qed.ParticleStore(1024)
    assert fn(C.byref(_config(1, sampler_mode=1)), C.byref(small.struct()), 0, stream,
              C.byref(out)) == qed.QED_ERR_ARG
