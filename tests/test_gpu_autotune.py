"""Launch-setting search: the store is left as it was, the settings change no
result (particles compared by id), and the JSON record is complete.  GPU only."""
import json

import numpy as np
import pytest

from paper_2008_10468_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402


def _by_id(a):
    o = np.argsort(a["id"], kind="stable")
    return {k: v[o] for k, v in a.items()}


def _step(ctx, arr, cap, step):
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    st = ctx.event_step(store, step)
    ctx.compact(store)
    return st, _by_id(store.to_numpy())


def test_autotune_restores_store_and_writes_record(tmp_path):
    arr = I.clumped_mixed(1 << 16, 77, hot_fraction=0.02)
    cap = 3 << 16
    ctx = qed.Context(seed=5)
    store = qed.ParticleStore.from_numpy(arr, capacity=cap)
    out = tmp_path / "tune.json"
    ctx.autotune(store, 3, str(out))
    after = store.to_numpy()
    for k in arr:
        np.testing.assert_array_equal(after[k], arr[k])
    rec = json.loads(out.read_text())
    assert rec["hot_min"] in (16, 32, 64, 128, 256)
    assert rec["long_min"] in (128, 256, 512, 1024, 2048, 1 << 30)
    assert rec["cold_blocks_per_sm"] >= 1 and rec["hot_blocks_per_sm"] >= 1
    assert rec["tail_rows"] in (0, 1 << 14, 1 << 16, 1 << 17, 1 << 18, 1 << 20, 1 << 22)
    assert any(t["tail_rows"] == 0 for t in rec["trials"])
    assert len(rec["trials"]) >= 6 and all(t["ms"] > 0 for t in rec["trials"])


@pytest.mark.parametrize("hot_min,long_min,cold,hot", [(16, 128, 1, 2), (128, 1 << 30, 2, 1),
                                                       (1 << 20, 0, 0, 0), (32, 32, 0, 1)])
def test_launch_settings_change_no_result(hot_min, long_min, cold, hot):
    arr = I.clumped_mixed(20000, 78, hot_fraction=0.03)
    cap = 400000
    ref_st, ref = _step(qed.Context(seed=8), arr, cap, 11)
    ctx = qed.Context(seed=8)
    ctx.set_launch(hot_min, long_min, cold, hot)
    st, got = _step(ctx, arr, cap, 11)
    for k in ("substeps", "emissions", "pairs", "children", "max_N", "status"):
        assert st[k] == ref_st[k], k
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k])
