"""The allocation-free gbar entry point against the plan's gbar (GPU).

fmm_gamma_bar_noalloc serves callers that cannot allocate device memory
(for instance while a stream is being captured into a graph): its partial
sums live in a fixed scratch array inside the library.  It must return the
same gbar as fmm_field computes, on consecutive calls that reuse that
scratch, and refuse sizes beyond its fixed limit.  This file sorts last so a
run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2302_07567_gb300 import fmm
from paper_2302_07567_gb300.workloads import make_beam

pytestmark = pytest.mark.gpu
MAX_N = 16777216


def _noalloc(p: torch.Tensor, N: int) -> float:
    out = torch.full((1,), -1.0, dtype=torch.float64, device=p.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
    rc = fmm.lib().fmm_gamma_bar_noalloc(ctypes.c_void_p(p.data_ptr()), N, ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == fmm.FMM_OK
    torch.cuda.synchronize()
    return float(out.item())


def _plan_gbar(x, p, q) -> float:
    N = x.shape[0]
    plan = fmm.Plan(N, 2, 64, 0.5, precision="fp64")
    plan.field(x, p, q)
    torch.cuda.synchronize()
    return float(plan.export("gbar")[0])


def test_noalloc_gamma_bar_matches_the_plan_on_consecutive_calls():
    dev = torch.device("cuda:0")
    beams = [make_beam("chirp1m", N=300_001), make_beam("cylinder64k", N=5_000)]
    got = []
    for x, p, q in beams:  # two calls in a row; the second reuses the scratch of the first
        X, Pm, Q = (torch.as_tensor(a, device=dev) for a in (x, p, q))
        got.append((_noalloc(Pm, x.shape[0]), X, Pm, Q))
    for g, X, Pm, Q in got:
        ref = _plan_gbar(X, Pm, Q)
        assert g == ref, (g, ref)
        assert 1.0 < g < 200.0
    assert got[0][0] != got[1][0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = torch.zeros((4, 3), dtype=torch.float64, device="cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    f = fmm.lib().fmm_gamma_bar_noalloc
    assert f(ctypes.c_void_p(p.data_ptr()), MAX_N + 1, ctypes.c_void_p(out.data_ptr()), None) == fmm.FMM_EINVAL
    assert f(ctypes.c_void_p(p.data_ptr()), 0, ctypes.c_void_p(out.data_ptr()), None) == fmm.FMM_EINVAL
    assert np.isclose(_noalloc(p, 4), 1.0)
