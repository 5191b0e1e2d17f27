"""The C ABI library builds, loads without a GPU and exports every function
that include/qed.h declares; the ctypes mirrors match the C struct sizes."""
import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qed.h")


def _declared():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qed_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libqed():
    from paper_2008_10468_gb300 import qed
    if not os.path.exists(qed.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        import __graft_entry__
        __graft_entry__.build()
    return C.CDLL(qed.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("qed_init", "qed_destroy", "qed_synchrotron_F1F2", "qed_event_step",
                 "qed_plan", "qed_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libqed):
    missing = [n for n in _declared() if not hasattr(libqed, n)]
    assert not missing, missing


def test_struct_mirrors_match(libqed):
    from paper_2008_10468_gb300 import qed
    libqed.qed_abi_struct_size.restype = C.c_size_t
    libqed.qed_abi_struct_size.argtypes = [C.c_char_p]
    sizes = {n: libqed.qed_abi_struct_size(n.encode()) for n in
             ("qed_config", "qed_particles", "qed_host_particles", "qed_step_stats",
              "qed_event_record")}
    assert sizes["qed_config"] == C.sizeof(qed.Config)
    assert sizes["qed_particles"] == C.sizeof(qed.Particles)
    assert sizes["qed_host_particles"] == C.sizeof(qed.HostParticles)
    assert sizes["qed_step_stats"] == C.sizeof(qed.StepStats)
    assert sizes["qed_event_record"] == qed.EVENT_DTYPE.itemsize
    assert libqed.qed_abi_struct_size(b"nope") == 0


def test_config_defaults_without_gpu(libqed):
    from paper_2008_10468_gb300 import qed
    cfg = qed.Config()
    libqed.qed_config_default(C.byref(cfg))
    assert cfg.p_max == pytest.approx(0.01) and cfg.dt_periods == 0.1
    assert cfg.process_mask == 3 and cfg.cascade_in_step == 1
