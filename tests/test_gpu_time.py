"""The float-float remaining-time arithmetic of the event kernels (the global
step split into N sub-steps, t - m h after an event) against exact rational
arithmetic and the oracle's binary64, over the worst cases: plans of up to
2^30 sub-steps, events next to the plan's end, remaining times left by many
earlier events.  GPU only."""
import ctypes as C
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402


def _split(t_hi, t_lo, N, m):
    L = qed.lib()
    f = L.qed_time_split
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)  # noqa: E731
    th, tl = dev(t_hi, torch.float32), dev(t_lo, torch.float32)
    Nd = dev(N.view(np.int32), torch.int32)
    md = dev(m.view(np.int32), torch.int32)
    n = len(N)
    h = torch.empty(n, dtype=torch.float64, device="cuda")
    ta = torch.empty(n, dtype=torch.float64, device="cuda")
    st = f(th.data_ptr(), tl.data_ptr(), Nd.data_ptr(), md.data_ptr(), n, h.data_ptr(),
           ta.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == qed.QED_OK
    return h.cpu().numpy(), ta.cpu().numpy()


def test_float_float_time_against_exact_and_binary64():
    rng = np.random.default_rng(30)
    n = 20000
    # remaining times as the kernels hold them: a binary64 value in (0, 0.1]
    # split into a float-float pair
    t = 0.1 * rng.uniform(1e-6, 1.0, n) ** 3
    t_hi = t.astype(np.float32)
    t_lo = (t - t_hi.astype(np.float64)).astype(np.float32)
    N = np.exp(rng.uniform(0, np.log(2.0 ** 30), n)).astype(np.uint32)
    N = np.maximum(N, 1)
    N[:200] = 1 << 30                    # the cap on the sub-step count
    N[200:400] = np.arange(1, 201)
    frac = rng.uniform(0, 1, n)
    m = np.minimum((frac * N).astype(np.uint64) + 1, N.astype(np.uint64)).astype(np.uint32)
    m[400:1400] = N[400:1400] - 1        # events next to the end of the plan
    m[400:1400] = np.maximum(m[400:1400], 1)
    h, ta = _split(t_hi, t_lo, N, m)
    err_h = err_t = err_o = 0.0
    for i in range(n):
        tt = Fraction(float(t_hi[i])) + Fraction(float(t_lo[i]))
        hx = tt / int(N[i])
        tx = tt - int(m[i]) * hx if m[i] < N[i] else Fraction(0)
        err_h = max(err_h, abs(float(Fraction(h[i]) - hx) / float(hx)))
        err_t = max(err_t, abs(float(Fraction(ta[i]) - tx)) / float(tt))
        # the oracle's binary64: h = t / N, t - m h
        tb = float(t_hi[i]) + float(t_lo[i])
        hb = tb / float(N[i])
        ob = tb - float(m[i]) * hb if m[i] < N[i] else 0.0
        err_o = max(err_o, abs(ob - ta[i]) / tb)
    print("float-float time: max rel err of h %.2e, of t - m h (of t) %.2e, vs binary64 %.2e"
          % (err_h, err_t, err_o))
    assert err_h < 5e-14 and err_t < 5e-14 and err_o < 5e-14
    # the plan's last sub-step ends it exactly
    last = np.nonzero(m >= N)[0]
    assert len(last) > 0 and np.all(ta[last] == 0.0)
