"""ctypes binding of the CUDA library ``csrc/libqed.so`` (C ABI in include/qed.h).

Argument marshalling only: every step of the event generator runs in the
library's kernels.  PyTorch provides device memory and the CUDA stream.  The
binding raises ``QEDError`` if the library is missing (build it with
``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU
fallback.
"""
import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "csrc", "libqed.so")

QED_OK, QED_ERR_ARG, QED_ERR_CUDA, QED_ERR_CAPACITY, QED_ERR_TIMEOUT, QED_ERR_STATE = range(6)
PROC_EMISSION, PROC_PAIR = 1, 2
ELECTRON, POSITRON, PHOTON, REMOVED = 0, 1, 2, 3
FLOAT_FIELDS = ("px", "py", "pz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "w")
KERNEL_KINDS = ("sweep", "generate", "plan", "cold", "hot", "control", "sampler")
SPECTRUM_BINS, SPECTRUM_LOG10_MIN, SPECTRUM_LOG10_MAX = 240, -4, 8
SAMPLER_PARAMS, SAMPLER_BINS = 8577, 64


class QEDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("qed status %d: %s" % (status, msg))
        self.status = status


class Config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("dt_periods", C.c_double), ("lambda_m", C.c_double),
                ("p_max", C.c_float), ("pair_bound_coeff", C.c_float),
                ("process_mask", C.c_uint32), ("cascade_in_step", C.c_int32),
                ("recoil", C.c_int32), ("max_passes", C.c_int32), ("drain_chi", C.c_float),
                ("sampler_mode", C.c_int32), ("sampler_max_err", C.c_float)]


class Particles(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in FLOAT_FIELDS] + [
        ("id", C.c_void_p), ("type", C.c_void_p), ("count", C.c_void_p), ("capacity", C.c_int64)]


class HostParticles(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in FLOAT_FIELDS] + [
        ("id", C.c_void_p), ("type", C.c_void_p), ("count", C.c_int64), ("capacity", C.c_int64)]


class StepStats(C.Structure):
    _fields_ = [("substeps", C.c_uint64), ("emissions", C.c_uint64), ("pairs", C.c_uint64),
                ("children", C.c_uint64), ("guard_hits", C.c_uint64), ("plans", C.c_uint64),
                ("candidates", C.c_uint64), ("max_N", C.c_uint32), ("status", C.c_int32),
                ("required_capacity", C.c_int64), ("count", C.c_int64), ("passes", C.c_int32),
                ("tail", C.c_int32), ("substeps_warp", C.c_uint64),
                ("sampler_events", C.c_uint64), ("sampler_pairs", C.c_uint64)]


EVENT_DTYPE = np.dtype([("parent_id", np.uint64), ("child0", np.uint64), ("child1", np.uint64),
                        ("s", np.uint32), ("kind", np.uint32), ("delta", np.float32),
                        ("chi", np.float32)])

_lib = None


def lib():
    """The loaded library; raises QEDError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QEDError(QED_ERR_STATE, "CUDA library not built: %s is missing" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i64, u64, st = C.c_void_p, C.c_int64, C.c_uint64, C.c_int
        L.qed_config_default.argtypes = [C.POINTER(Config)]
        L.qed_config_default.restype = None
        L.qed_init.argtypes = [C.POINTER(vp), C.POINTER(Config), vp]
        L.qed_init.restype = st
        L.qed_destroy.argtypes = [vp]
        L.qed_destroy.restype = st
        L.qed_last_error.argtypes = [vp]
        L.qed_last_error.restype = C.c_char_p
        L.qed_synchrotron_F1F2.argtypes = [vp, vp, vp, vp, i64]
        L.qed_synchrotron_F1F2.restype = st
        L.qed_synchrotron_F1F2_f64.argtypes = [vp, vp, vp, i64, vp]
        L.qed_synchrotron_F1F2_f64.restype = st
        L.qed_synchrotron_generate.argtypes = [vp, u64, i64, C.c_float, C.c_float, vp, vp, vp, vp]
        L.qed_synchrotron_generate.restype = st
        L.qed_plan.argtypes = [vp, C.POINTER(Particles), i64, vp, vp]
        L.qed_plan.restype = st
        L.qed_event_step.argtypes = [vp, C.POINTER(Particles), u64, C.POINTER(StepStats)]
        L.qed_event_step.restype = st
        L.qed_event_step_push.argtypes = [vp, C.POINTER(Particles), u64, C.POINTER(StepStats)]
        L.qed_event_step_push.restype = st
        L.qed_event_step_host.argtypes = [vp, C.POINTER(HostParticles), u64, C.POINTER(StepStats)]
        L.qed_event_step_host.restype = st
        L.qed_event_step_cells.argtypes = [vp, C.POINTER(Particles), u64, vp, i64,
                                           C.POINTER(StepStats)]
        L.qed_event_step_cells.restype = st
        L.qed_plan_cells.argtypes = [vp, C.POINTER(Particles), i64, vp, i64, vp]
        L.qed_plan_cells.restype = st
        L.qed_event_step_push_cells.argtypes = [vp, C.POINTER(Particles), u64, vp, i64,
                                                C.POINTER(StepStats)]
        L.qed_event_step_push_cells.restype = st
        L.qed_read_stats.argtypes = [vp, C.POINTER(StepStats)]
        L.qed_read_stats.restype = st
        L.qed_set_event_log.argtypes = [vp, vp, i64, vp]
        L.qed_set_event_log.restype = st
        L.qed_compact.argtypes = [vp, C.POINTER(Particles), C.POINTER(i64)]
        L.qed_compact.restype = st
        L.qed_read_spectrum.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.c_int]
        L.qed_read_spectrum.restype = st
        L.qed_graph_capture.argtypes = [vp, C.POINTER(Particles), u64, C.c_int]
        L.qed_graph_capture.restype = st
        L.qed_graph_launch.argtypes = [vp]
        L.qed_graph_launch.restype = st
        L.qed_graph_read_stats.argtypes = [vp, C.POINTER(StepStats), C.c_int]
        L.qed_graph_read_stats.restype = st
        fp = C.POINTER(C.c_float)
        L.qed_sampler_train.argtypes = [vp, u64, i64, C.c_int, C.c_float, fp]
        L.qed_sampler_train.restype = st
        L.qed_sampler_process.argtypes = [vp, C.c_uint32]
        L.qed_sampler_process.restype = st
        L.qed_sampler_evaluate.argtypes = [vp, fp, C.c_int]
        L.qed_sampler_evaluate.restype = st
        L.qed_sampler_gradient.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp]
        L.qed_sampler_gradient.restype = st
        L.qed_sampler_quantile.argtypes = [vp, vp, vp, vp, i64, C.c_int]
        L.qed_sampler_quantile.restype = st
        L.qed_sampler_load.argtypes = [vp, fp, i64]
        L.qed_sampler_load.restype = st
        L.qed_sampler_save.argtypes = [vp, fp, i64]
        L.qed_sampler_save.restype = st
        L.qed_set_launch.argtypes = [vp, C.c_uint32, C.c_uint32, C.c_int, C.c_int]
        L.qed_set_launch.restype = st
        L.qed_set_tail.argtypes = [vp, C.c_int64]
        L.qed_set_tail.restype = st
        L.qed_set_wait_limit.argtypes = [vp, u64]
        L.qed_set_wait_limit.restype = st
        L.qed_autotune.argtypes = [vp, C.POINTER(Particles), u64, C.c_char_p]
        L.qed_autotune.restype = st
        L.qed_profile_enable.argtypes = [vp, C.c_int]
        L.qed_profile_enable.restype = st
        L.qed_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]
        L.qed_profile_read.restype = st
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise QEDError(QED_ERR_ARG, "tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise QEDError(QED_ERR_ARG, "tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def stats_dict(s):
    return {k: int(getattr(s, k)) for k, _ in StepStats._fields_}


PROBE_MUL32, PROBE_FMA32, PROBE_EX2, PROBE_ALU = 0, 1, 2, 3


def peak_probe(kind, iters=1 << 16, stream=None):
    """(operations per second, ms) of one peak probe (qed_peak_probe)."""
    L = lib()
    L.qed_peak_probe.argtypes = [C.c_int, C.c_int64, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.c_void_p]
    L.qed_peak_probe.restype = C.c_int
    r, ms = C.c_double(), C.c_double()
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    st = L.qed_peak_probe(int(kind), int(iters), C.byref(r), C.byref(ms), C.c_void_p(s))
    if st != QED_OK:
        raise QEDError(st, "qed_peak_probe failed")
    return r.value, ms.value


def synchrotron_F1F2_f64(y, F1=None, F2=None, stream=None):
    """F and G in binary64 (float64 CUDA tensors) on `stream` (default: the
    current torch stream); no context needed."""
    import torch
    if y.dtype != torch.float64 or any(t is not None and t.dtype != torch.float64
                                       for t in (F1, F2)):
        raise QEDError(QED_ERR_ARG, "float64 tensors expected")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib().qed_synchrotron_F1F2_f64(_ptr(y), _ptr(F1), _ptr(F2), int(y.numel()),
                                        C.c_void_p(stream.cuda_stream))
    if st != QED_OK:
        raise QEDError(st, "qed_synchrotron_F1F2_f64 failed")
    return F1, F2


class ParticleStore:
    """Caller-owned SoA particle arrays on the GPU (see qed_particles)."""

    def __init__(self, capacity, device="cuda"):
        self.capacity = int(capacity)
        self.device = torch.device(device)
        f = dict(dtype=torch.float32, device=self.device)
        for k in FLOAT_FIELDS:
            setattr(self, k, torch.zeros(self.capacity, **f))
        self.id = torch.zeros(self.capacity, dtype=torch.int64, device=self.device)
        self.type = torch.full((self.capacity,), REMOVED, dtype=torch.uint8, device=self.device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)

    @classmethod
    def from_numpy(cls, arrs, capacity=None, device="cuda"):
        n = int(arrs["px"].shape[0])
        s = cls(capacity if capacity is not None else max(n, 1), device)
        s.load(arrs)
        return s

    def load(self, arrs):
        n = int(arrs["px"].shape[0])
        if n > self.capacity:
            raise QEDError(QED_ERR_ARG, "more rows than capacity")
        for k in FLOAT_FIELDS:
            getattr(self, k)[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs[k], np.float32)))
        self.id[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs["id"]).view(np.int64)))
        self.type[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs["type"], np.uint8)))
        self.type[n:].fill_(REMOVED)
        self.count.fill_(n)

    def n(self):
        return int(self.count.item())

    def to_numpy(self):
        n = self.n()
        out = {k: getattr(self, k)[:n].cpu().numpy() for k in FLOAT_FIELDS}
        out["id"] = self.id[:n].cpu().numpy().view(np.uint64)
        out["type"] = self.type[:n].cpu().numpy()
        return out

    def struct(self):
        p = Particles()
        for k in FLOAT_FIELDS:
            setattr(p, k, _ptr(getattr(self, k)))
        p.id = _ptr(self.id)
        p.type = _ptr(self.type)
        p.count = _ptr(self.count)
        p.capacity = self.capacity
        return p


class HostStore:
    """Caller-owned SoA particle arrays in host memory (see qed_host_particles),
    page-locked by default."""

    def __init__(self, capacity, pinned=True):
        self.capacity = int(capacity)
        kw = dict(pin_memory=bool(pinned))
        for k in FLOAT_FIELDS:
            setattr(self, k, torch.zeros(self.capacity, dtype=torch.float32, **kw))
        self.id = torch.zeros(self.capacity, dtype=torch.int64, **kw)
        self.type = torch.full((self.capacity,), REMOVED, dtype=torch.uint8, **kw)
        self.count = 0

    @classmethod
    def from_numpy(cls, arrs, capacity=None, pinned=True):
        n = int(arrs["px"].shape[0])
        s = cls(capacity if capacity is not None else max(n, 1), pinned)
        s.load(arrs)
        return s

    def load(self, arrs):
        n = int(arrs["px"].shape[0])
        if n > self.capacity:
            raise QEDError(QED_ERR_ARG, "more rows than capacity")
        for k in FLOAT_FIELDS:
            getattr(self, k)[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs[k], np.float32)))
        self.id[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs["id"]).view(np.int64)))
        self.type[:n].copy_(torch.from_numpy(np.ascontiguousarray(arrs["type"], np.uint8)))
        self.type[n:].fill_(REMOVED)
        self.count = n

    def n(self):
        return self.count

    def to_numpy(self):
        n = self.count
        out = {k: getattr(self, k)[:n].numpy().copy() for k in FLOAT_FIELDS}
        out["id"] = self.id[:n].numpy().view(np.uint64).copy()
        out["type"] = self.type[:n].numpy().copy()
        return out

    def struct(self):
        p = HostParticles()
        for k in FLOAT_FIELDS:
            setattr(p, k, getattr(self, k).data_ptr())
        p.id = self.id.data_ptr()
        p.type = self.type.data_ptr()
        p.count = self.count
        p.capacity = self.capacity
        return p


class Context:
    """A library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, seed=20081046, dt=0.1, lambda_m=1e-6, p_max=0.01, pair_coeff=0.1,
                 process_mask=PROC_EMISSION | PROC_PAIR, cascade=True, recoil=True,
                 max_passes=64, drain_chi=0.0, sampler=False, sampler_max_err=1e-3,
                 stream=None):
        L = lib()
        cfg = Config()
        L.qed_config_default(C.byref(cfg))
        cfg.seed = int(seed)
        cfg.dt_periods = float(dt)
        cfg.lambda_m = float(lambda_m)
        cfg.p_max = float(p_max)
        cfg.pair_bound_coeff = float(pair_coeff)
        cfg.process_mask = int(process_mask)
        cfg.cascade_in_step = int(bool(cascade))
        cfg.recoil = int(bool(recoil))
        cfg.max_passes = int(max_passes)
        cfg.drain_chi = float(drain_chi)
        # sampler: False, True (per sub-step) or "event" (event-driven)
        cfg.sampler_mode = 2 if sampler == "event" else int(bool(sampler))
        cfg.sampler_max_err = float(sampler_max_err)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._h = C.c_void_p()
        st = L.qed_init(C.byref(self._h), C.byref(cfg), C.c_void_p(stream.cuda_stream))
        if st != QED_OK:
            raise QEDError(st, "qed_init failed")
        self._log = None

    def _check(self, st):
        if st != QED_OK:
            raise QEDError(st, lib().qed_last_error(self._h).decode(errors="replace"))

    def close(self):
        if self._h:
            lib().qed_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchrotron_F1F2(self, y, F1=None, F2=None):
        n = int(y.numel())
        self._check(lib().qed_synchrotron_F1F2(self._h, _ptr(y), _ptr(F1), _ptr(F2), n))
        return F1, F2

    def synchrotron_generate(self, seed, n, lo=1e-4, hi=50.0, checksum=None, y=None, F1=None,
                             F2=None):
        self._check(lib().qed_synchrotron_generate(self._h, int(seed), int(n), float(lo),
                                                   float(hi), _ptr(checksum), _ptr(y), _ptr(F1),
                                                   _ptr(F2)))

    def plan(self, store, n, chi=None, N=None):
        p = store.struct()
        self._check(lib().qed_plan(self._h, C.byref(p), int(n), _ptr(chi), _ptr(N)))

    def plan_cells(self, store, n, cell, ncells, N_cell=None):
        """Per-cell sub-step counts (max of the rows' N per cell); returns N_cell."""
        if N_cell is None:
            N_cell = torch.empty(int(ncells), dtype=torch.int32, device=store.device)
        p = store.struct()
        self._check(lib().qed_plan_cells(self._h, C.byref(p), int(n), _ptr(cell), int(ncells),
                                         _ptr(N_cell)))
        return N_cell

    def set_event_log(self, capacity):
        """Record events of later steps into a device log of `capacity` records."""
        if capacity <= 0:
            self._check(lib().qed_set_event_log(self._h, None, 0, None))
            self._log = None
            return
        buf = torch.zeros(int(capacity) * EVENT_DTYPE.itemsize, dtype=torch.uint8,
                          device=torch.device("cuda"))
        cnt = torch.zeros(1, dtype=torch.int64, device=buf.device)
        self._check(lib().qed_set_event_log(self._h, _ptr(buf), int(capacity), _ptr(cnt)))
        self._log = (buf, cnt, int(capacity))

    def read_event_log(self):
        buf, cnt, cap = self._log
        n = min(int(cnt.item()), cap)
        raw = buf[:n * EVENT_DTYPE.itemsize].cpu().numpy()
        return raw.view(EVENT_DTYPE).copy(), int(cnt.item())

    def event_step(self, store, step, sync=True, push=False):
        """One global step; returns the statistics dict (sync=True) or None.
        push=True: the step with the Boris push before every e+- draw."""
        fn = lib().qed_event_step_push if push else lib().qed_event_step
        p = store.struct()
        if sync:
            s = StepStats()
            st = fn(self._h, C.byref(p), int(step), C.byref(s))
            if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT):   # step outcomes
                self._check(st)
            return stats_dict(s)
        self._check(fn(self._h, C.byref(p), int(step), None))
        return None

    def event_step_host(self, hstore, step):
        """One global step on a HostStore (qed_event_step_host): its rows go to
        the device, the step runs, the changes come back; returns the
        statistics dict.  On an unsuccessful step the host store is unchanged."""
        p = hstore.struct()
        s = StepStats()
        st = lib().qed_event_step_host(self._h, C.byref(p), int(step), C.byref(s))
        if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT):   # step outcomes
            self._check(st)
        hstore.count = int(p.count)
        return stats_dict(s)

    def event_step_cells(self, store, step, cell, ncells):
        """The event step with one sub-step per cell for the first plans
        (qed_event_step_cells; cell: int32 CUDA tensor of a cell index per row
        in use); returns the statistics dict."""
        p = store.struct()
        s = StepStats()
        st = lib().qed_event_step_cells(self._h, C.byref(p), int(step), _ptr(cell), int(ncells),
                                        C.byref(s))
        if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT):   # step outcomes
            self._check(st)
        return stats_dict(s)

    def event_step_push_cells(self, store, step, cell, ncells):
        """Push-mode step with one sub-step per cell (cell: int32 CUDA tensor of
        a cell index per row in use); returns the statistics dict."""
        p = store.struct()
        s = StepStats()
        st = lib().qed_event_step_push_cells(self._h, C.byref(p), int(step), _ptr(cell),
                                             int(ncells), C.byref(s))
        if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT):   # step outcomes
            self._check(st)
        return stats_dict(s)

    def compact(self, store):
        """Squeeze removed rows out of the store; returns the rows removed."""
        p = store.struct()
        r = C.c_int64()
        self._check(lib().qed_compact(self._h, C.byref(p), C.byref(r)))
        return int(r.value)

    def read_spectrum(self, reset=False):
        out = (C.c_double * SPECTRUM_BINS)()
        self._check(lib().qed_read_spectrum(self._h, out, SPECTRUM_BINS, int(bool(reset))))
        return np.array(out[:])

    def graph_capture(self, store, first_step, nsteps):
        """Record nsteps global steps on `store` as one CUDA graph."""
        self._graph_store = store
        p = store.struct()
        self._check(lib().qed_graph_capture(self._h, C.byref(p), int(first_step), int(nsteps)))
        self._graph_steps = int(nsteps)

    def graph_launch(self):
        self._check(lib().qed_graph_launch(self._h))

    def graph_read_stats(self):
        """Per-step statistics of the last graph launch (list of dicts)."""
        n = self._graph_steps
        out = (StepStats * n)()
        st = lib().qed_graph_read_stats(self._h, out, n)
        if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT, QED_ERR_STATE):
            self._check(st)
        return [stats_dict(out[k]) for k in range(n)]

    def sampler_process(self, process):
        """Address the emission (PROC_EMISSION) or the pair (PROC_PAIR) network
        with the sampler_* calls that follow."""
        self._check(lib().qed_sampler_process(self._h, int(process)))

    def sampler_train(self, seed, samples, batch=4096, lr=3e-3):
        loss = C.c_float()
        self._check(lib().qed_sampler_train(self._h, int(seed), int(samples), int(batch),
                                            float(lr), C.byref(loss)))
        return float(loss.value)

    def sampler_evaluate(self):
        err = (C.c_float * SAMPLER_BINS)()
        self._check(lib().qed_sampler_evaluate(self._h, err, SAMPLER_BINS))
        return np.array(err[:])

    def sampler_gradient(self, params, v, target, grad, loss=None, weight=None):
        self._check(lib().qed_sampler_gradient(self._h, _ptr(params), _ptr(v), _ptr(target),
                                               _ptr(weight), int(target.numel()), _ptr(grad),
                                               _ptr(loss)))

    def sampler_quantile(self, log10chi, u, x, use_net=True):
        """use_net: False the exact table inverse, True the network (FP32
        activations), "mma" the network on the tensor cores."""
        mode = 2 if use_net == "mma" else int(bool(use_net))
        self._check(lib().qed_sampler_quantile(self._h, _ptr(log10chi), _ptr(u), _ptr(x),
                                               int(x.numel()), mode))

    def sampler_load(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        self._check(lib().qed_sampler_load(self._h, a.ctypes.data_as(C.POINTER(C.c_float)),
                                           a.size))

    def sampler_save(self):
        a = np.empty(SAMPLER_PARAMS, dtype=np.float32)
        self._check(lib().qed_sampler_save(self._h, a.ctypes.data_as(C.POINTER(C.c_float)),
                                           a.size))
        return a

    def set_launch(self, hot_min=0, long_min=0, cold_blocks_per_sm=0, hot_blocks_per_sm=0):
        self._check(lib().qed_set_launch(self._h, int(hot_min), int(long_min),
                                         int(cold_blocks_per_sm), int(hot_blocks_per_sm)))

    def set_tail(self, tail_rows):
        """Generations below tail_rows rows go to the tail pass (0: off)."""
        self._check(lib().qed_set_tail(self._h, int(tail_rows)))

    def set_wait_limit(self, ns):
        """Longest bounded wait of the tail pass in ns (0: the 1 s default)."""
        self._check(lib().qed_set_wait_limit(self._h, int(ns)))

    def autotune(self, store, step, out_json=None):
        """Pick the fastest launch settings for `store` (left unchanged)."""
        p = store.struct()
        path = out_json.encode() if out_json else None
        self._check(lib().qed_autotune(self._h, C.byref(p), int(step), path))

    def profile(self, enable=True):
        self._check(lib().qed_profile_enable(self._h, int(bool(enable))))

    def profile_read(self):
        """{kind: (ms, launches)} since the last read, for kinds in KERNEL_KINDS."""
        ms = (C.c_double * 8)()
        ln = (C.c_int64 * 8)()
        self._check(lib().qed_profile_read(self._h, ms, ln, 8))
        return {name: (float(ms[i]), int(ln[i])) for i, name in enumerate(KERNEL_KINDS)}

    def read_stats(self):
        s = StepStats()
        st = lib().qed_read_stats(self._h, C.byref(s))
        if st not in (QED_OK, QED_ERR_CAPACITY, QED_ERR_TIMEOUT):   # step outcomes
            self._check(st)
        return stats_dict(s)
