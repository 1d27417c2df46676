"""The work model of Section 5 at a transition N_t = 2^kappa N0 (oracle).

Section 5 explains the jumps of the P2P and M2L times against N: at
N = N_t the balanced tree has depth kappa and full leaves of N0 particles;
one particle more gives depth kappa + 1 and leaves of about N0 / 2.  With a
bounded number of partners per cluster, the P2P work (particle pairs) then
drops (the model: to one half) and grows again until the next transition,
while the M2L work (cluster pairs) jumps (the model: doubles) and then stays
flat until 2 N_t.  These checks run on the oracle's tree and lists for the
uniform cube of the paper's experiments.  At these small sizes the number
of partners per leaf still grows with depth (boundary leaves), so the
bounds are the model's directions with margins, not its exact ratios.
"""
import pytest

from oracle import bldtt
from paper_2302_07567_gb300.workloads import make_beam


def _work(N, N0, eta=0.5):
    x, p, _ = make_beam("cube", N=N)
    plan = bldtt.build_plan(x, p, 2, N0, eta)
    mem = plan.tree.members
    w_p2p = sum(len(mem[a]) * len(mem[b]) for a, b in plan.p2p)
    return plan.tree.kappa, w_p2p, len(plan.m2l)


@pytest.mark.parametrize("N0,kappa", [(27, 6), (64, 6)])
def test_transition_jumps(N0, kappa):
    Nt = (1 << kappa) * N0
    k0, p0, m0 = _work(Nt, N0)
    k1, p1, m1 = _work(Nt + 1, N0)
    k2, p2, m2 = _work(2 * Nt, N0)
    # the depth rule: N_t fills 2^kappa leaves; one particle more needs a level
    assert (k0, k1, k2) == (kappa, kappa + 1, kappa + 1)
    # P2P work drops just above N_t and grows past it by 2 N_t
    assert p1 < 0.85 * p0
    assert p2 > 2.0 * p1
    # M2L work jumps just above N_t, then stays flat up to 2 N_t
    assert m1 > 1.5 * m0
    assert abs(m2 - m1) <= 0.15 * m1
