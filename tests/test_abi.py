"""The C-ABI library builds, loads and exports every function include/fmm.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2302_07567_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    names = _declared()
    assert "fmm_field" in names and "fmm_field_adjoint" in names and len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fmm_\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert getattr(lib, n) is not None


def test_host_side_argument_checks(libpath):
    """Plan creation validates its arguments without touching a GPU."""
    lib = ctypes.CDLL(libpath)
    lib.fmm_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_uint]
    lib.fmm_strerror.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    bad = [(0, 4, 64, 0.5, 1), (100, 0, 64, 0.5, 1), (100, 13, 64, 0.5, 1), (100, 4, 1, 0.5, 1),
           (100, 4, 64, 0.0, 1), (100, 4, 64, float("nan"), 1), (100, 4, 64, 0.5, 7), (100, 4, 5000, 0.5, 1)]
    for N, n, leaf, eta, prec in bad:
        assert lib.fmm_plan_create(ctypes.byref(h), N, n, leaf, eta, prec, 0) == 1
    assert lib.fmm_plan_create(ctypes.byref(h), 100, 4, 64, 0.5, 1, 0x100) == 1  # unknown flag bit
    assert lib.fmm_plan_create(ctypes.byref(h), 100, 4, 64, 0.5, 1, 128) == 1  # unknown flag bit
    assert lib.fmm_plan_create(ctypes.byref(h), 100, 4, 64, 0.5, 1, 16) == 1  # the test kernel is FP64 only
    lib.fmm_plan_destroy.argtypes = [ctypes.c_void_p]
    for flags in (32, 32 | 8 | 2 | 1, 64 | 4):  # gbar term, with size-aware lists, bounds checks, recompute; serial
        assert lib.fmm_plan_create(ctypes.byref(h), 100, 4, 64, 0.5, 1, flags) == 0
        lib.fmm_plan_destroy(h)
    assert lib.fmm_plan_create(ctypes.byref(h), 4096, 4, 64, 0.5, 1, 0) == 0
    lib.fmm_plan_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    nb = ctypes.c_size_t()
    assert lib.fmm_plan_workspace_bytes(h, ctypes.byref(nb)) == 0 and nb.value > 4096 * 100
    # FMM_RECOMPUTE: the adjoint's W and Lambda share the forward's L and M
    # buffers, (C+1) (6 + 4) m floats less (C = 127 clusters, m = 125 here)
    h2 = ctypes.c_void_p()
    assert lib.fmm_plan_create(ctypes.byref(h2), 4096, 4, 64, 0.5, 1, 1) == 0
    nb2 = ctypes.c_size_t()
    assert lib.fmm_plan_workspace_bytes(h2, ctypes.byref(nb2)) == 0
    assert nb.value - nb2.value >= 128 * 10 * 125 * 4
    lib.fmm_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.fmm_plan_destroy(h2)
    lib.fmm_field.argtypes = [ctypes.c_void_p] * 7
    one = ctypes.c_void_p(256)
    assert lib.fmm_field(h, one, one, one, one, one, None) == 2  # no workspace attached
    # the recorded step: nothing recorded yet, NULL arguments, no workspace
    lib.fmm_step_graph_create.argtypes = [ctypes.c_void_p] * 12
    lib.fmm_step_graph_launch.argtypes = [ctypes.c_void_p] * 2
    lib.fmm_step_graph_destroy.argtypes = [ctypes.c_void_p]
    assert lib.fmm_step_graph_launch(h, one) == 5
    assert lib.fmm_step_graph_launch(None, one) == 1
    assert lib.fmm_step_graph_create(h, None, one, one, None, None, one, one, None, None, None, one) == 1
    assert lib.fmm_step_graph_create(h, one, one, one, one, None, one, one, one, one, one, one) == 1  # wE without wB
    assert lib.fmm_step_graph_create(h, one, one, one, None, None, one, one, None, None, None, one) == 2
    assert lib.fmm_step_graph_destroy(h) == 0
    lib.fmm_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.fmm_copy(None, one, 16, None) == 1
    assert lib.fmm_copy(one, ctypes.c_void_p(264), 16, None) == 1  # misaligned source
    assert lib.fmm_copy(one, one, 24, None) == 1  # not a multiple of 16 bytes
    assert lib.fmm_copy(one, one, 0, None) == 0  # nothing to copy
    lib.fmm_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.fmm_plan_destroy(h)
    assert lib.fmm_strerror(3) == b"interaction-list capacity exceeded"


def test_stats_layout_matches_the_binding(libpath):
    """The binding's ctypes fmm_stats has the size of the library's struct,
    and one stage name per stage slot."""
    from paper_2302_07567_gb300 import fmm
    lib = ctypes.CDLL(libpath)
    lib.fmm_stats_bytes.restype = ctypes.c_size_t
    assert lib.fmm_stats_bytes() == ctypes.sizeof(fmm.Stats)
    slots = dict(fmm.Stats._fields_)["stage_ms"]._length_
    assert slots == len(fmm.STAGES) == 18
