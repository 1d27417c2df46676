"""Recorded steps: the forward and adjoint replayed as CUDA graphs (GPU).

A replay runs the recorded calls' kernels in the same order, so on the same
input it must equal the eager calls bit for bit, and after the inputs are
updated in place it must equal the eager calls on the new input.  A replay
whose lists no longer fit the capacities reports the overflow and writes
nothing.
"""
import numpy as np
import pytest
import torch

from paper_2302_07567_gb300 import fmm
from paper_2302_07567_gb300.workloads import make_beam, make_weights

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(*arrs, dtype=None):
    return [torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype) for a in arrs]


def eager(N, n, leaf, eta, prec, flags, X, P, Q, WE=None, WB=None):
    plan = fmm.Plan(N, n, leaf, eta, precision=prec, flags=flags)
    E, B = plan.field(X, P, Q)
    out = [E, B]
    if WE is not None:
        out += list(plan.adjoint(X, P, Q, WE, WB))
    torch.cuda.synchronize()
    return [t.cpu() for t in out]


CASES = [("cylinder64k", 8192, 6, 128, "fp32", 0), ("cylinder64k", 8192, 6, 128, "fp32", fmm.FMM_RECOMPUTE),
         ("gauss4k", 4096, 4, 64, "fp64", 0), ("gauss4k", 4096, 4, 64, "fp32", fmm.FMM_SERIAL)]


@pytest.mark.parametrize("work,N,n,leaf,prec,flags", CASES)
def test_replay_equals_the_eager_step(work, N, n, leaf, prec, flags):
    x, p, q = make_beam(work, N=N)
    wE, wB = make_weights(N)
    odt = torch.float32 if prec == "fp32" else torch.float64
    X, P, Q = dev(x, p, q)
    WE, WB = dev(wE, wB, dtype=odt)
    ref = eager(N, n, leaf, 0.5, prec, flags, X, P, Q, WE, WB)
    plan = fmm.Plan(N, n, leaf, 0.5, precision=prec, flags=flags)
    outs = plan.record_step(X, P, Q, WE, WB)
    for a, b in zip(outs, ref):  # the recording's own eager step
        assert torch.equal(a.cpu(), b)
    for o in outs:
        o.zero_()
    k0 = fmm.kernel_launches()
    for _ in range(2):
        plan.replay()
        for a, b in zip(outs, ref):
            assert torch.equal(a.cpu(), b)
    assert fmm.kernel_launches() - k0 >= 2 * 20  # a replay counts the kernels it runs
    # the adjoint's state after a replay lets the eager adjoint follow as usual
    g = plan.adjoint(X, P, Q, WE, WB)
    for a, b in zip(g, ref[2:]):
        assert torch.equal(a.cpu(), b)


def test_replay_follows_inputs_updated_in_place():
    N, n, leaf = 8192, 6, 128
    x, p, q = make_beam("cylinder64k", N=N)
    wE, wB = make_weights(N)
    X, P, Q = dev(x, p, q)
    WE, WB = dev(wE, wB, dtype=torch.float32)
    plan = fmm.Plan(N, n, leaf, 0.5, precision="fp32")
    outs = plan.record_step(X, P, Q, WE, WB)
    rng = np.random.default_rng(3)
    for step in range(3):  # a drifting beam, new weights and charges every step
        X.add_(torch.as_tensor(rng.standard_normal((N, 3)) * 2e-6, device=DEV))
        P.mul_(1.0 + 1e-3 * step)
        Q.mul_(1.01)
        WE.copy_(torch.as_tensor(rng.standard_normal((N, 3)), device=DEV, dtype=torch.float32))
        plan.replay()
        ref = eager(N, n, leaf, 0.5, "fp32", 0, X, P, Q, WE, WB)
        for a, b in zip(outs, ref):
            assert torch.equal(a.cpu(), b)


def test_forward_only_recording():
    N = 4096
    x, p, q = make_beam("gauss4k", N=N)
    X, P, Q = dev(x, p, q)
    plan = fmm.Plan(N, 4, 64, 0.5, precision="fp32")
    E, B = plan.record_step(X, P, Q)
    ref = eager(N, 4, 64, 0.5, "fp32", 0, X, P, Q)
    E.zero_()
    plan.replay()
    assert torch.equal(E.cpu(), ref[0]) and torch.equal(B.cpu(), ref[1])


def test_replay_without_a_recording_is_a_state_error():
    plan = fmm.Plan(4096, 4, 64, 0.5, precision="fp32")
    with pytest.raises(fmm.FMMError) as e:
        plan.replay()
    assert e.value.status == fmm.FMM_ESTATE


def test_recording_refuses_host_timing():
    N = 4096
    x, p, q = make_beam("gauss4k", N=N)
    plan = fmm.Plan(N, 4, 64, 0.5, precision="fp32", flags=fmm.FMM_TIMING)
    with pytest.raises(fmm.FMMError) as e:
        plan.record_step(*dev(x, p, q))
    assert e.value.status == fmm.FMM_EINVAL


def test_replay_reports_an_overflow_and_writes_nothing():
    N, n, leaf = 4096, 4, 64
    xa, pa, qa = make_beam("gauss4k", N=N)
    # a second input whose P2P list is longer than the first's
    xb = xa.copy()
    xb[:, 2] *= 0.02  # a flattened bunch: many more near neighbours per leaf
    probe = fmm.Plan(N, n, leaf, 0.5, precision="fp32")
    probe.field(*dev(xa, pa, qa))
    ca = probe.stats()["p2p_pairs"]
    probe.field(*dev(xb, pa, qa))
    cb = probe.stats()["p2p_pairs"]
    assert cb > ca
    plan = fmm.Plan(N, n, leaf, 0.5, precision="fp32", capacity=(ca, 0, 0))
    X, P, Q = dev(xa, pa, qa)
    E, B = plan.record_step(X, P, Q)
    assert plan.stats()["cap_p2p"] == ca  # it fitted: no growth, the graph holds this workspace
    e0 = E.clone()
    X.copy_(torch.as_tensor(xb, device=DEV))
    with pytest.raises(fmm.FMMError) as e:
        plan.replay()
    assert e.value.status == fmm.FMM_EOVERFLOW
    assert torch.equal(E, e0)  # nothing written
    E2, B2 = plan.record_step(X, P, Q)  # grows the lists and records anew
    ref = eager(N, n, leaf, 0.5, "fp32", 0, X, P, Q)
    assert torch.equal(E2.cpu(), ref[0]) and torch.equal(B2.cpu(), ref[1])
