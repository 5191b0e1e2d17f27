"""qed_event_step_noalloc, the event step for callers that cannot allocate
device memory (code under stream capture, fixed memory budgets, plug-ins in
another program's pool), must give the results of qed_event_step.  It keeps
its scratch in a device array built into the library, so two calls in a row
also check that nothing left over from the first call changes the second.
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

P_RTOL = 2e-5   # momentum tolerance of the parity tests (relative to |p|)


def _noalloc_fn():
    L = qed.lib()
    f = L.qed_event_step_noalloc
    f.argtypes = [C.POINTER(qed.Config), C.POINTER(qed.Particles), C.c_uint64, C.c_void_p,
                  C.POINTER(qed.StepStats)]
    f.restype = C.c_int
    return f


def _config(seed):
    cfg = qed.Config()
    qed.lib().qed_config_default(C.byref(cfg))
    cfg.seed = seed
    return cfg


def _sorted(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items()}


def test_noalloc_matches_event_step_on_two_calls():
    fn = _noalloc_fn()
    seed = 4242
    arr = I.clumped_mixed(5000, 31, hot_fraction=0.03)
    cap = qed_cap = 60000
    assert cap <= 65536
    ctx = qed.Context(seed=seed)
    stream = torch.cuda.current_stream()
    for call, step in enumerate((7, 8)):
        ref = qed.ParticleStore.from_numpy(arr, capacity=cap)
        st_ref = ctx.event_step(ref, step)
        got = qed.ParticleStore.from_numpy(arr, capacity=qed_cap)
        p = got.struct()
        out = qed.StepStats()
        status = fn(C.byref(_config(seed)), C.byref(p), step, C.c_void_p(stream.cuda_stream),
                    C.byref(out))
        assert status == qed.QED_OK, status
        st = qed.stats_dict(out)
        for k in ("substeps", "emissions", "pairs", "children", "plans", "candidates", "max_N",
                  "passes", "count", "status"):
            assert st[k] == st_ref[k], (call, k, st[k], st_ref[k])
        a, b = _sorted(ref.to_numpy()), _sorted(got.to_numpy())
        np.testing.assert_array_equal(a["id"], b["id"])
        np.testing.assert_array_equal(a["type"], b["type"])
        for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "w"):
            np.testing.assert_array_equal(a[k], b[k])
        pa = np.stack([a["px"], a["py"], a["pz"]], 1).astype(np.float64)
        pb = np.stack([b["px"], b["py"], b["pz"]], 1).astype(np.float64)
        scale = np.maximum(np.linalg.norm(pa, axis=1), 1e-30)[:, None]
        assert np.all(np.abs(pa - pb) <= P_RTOL * scale)


def test_noalloc_rejects_stores_beyond_its_limit():
    fn = _noalloc_fn()
    big = qed.ParticleStore(65537)
    out = qed.StepStats()
    status = fn(C.byref(_config(1)), C.byref(big.struct()), 0,
                C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out))
    assert status == qed.QED_ERR_ARG
