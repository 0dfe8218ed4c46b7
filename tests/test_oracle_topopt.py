"""Pins of the oracle's optimisation loop (paper Section 2.5)."""
import numpy as np

from oracle import topopt
from synth import problems


def test_loop_decreases_compliance_and_keeps_volume():
    prob = problems.cantilever(24, 8, 2, load="edge", volfrac=0.3, rmin=1.5)
    x, hist = topopt.top3d(prob, iters=8, solver="direct")
    c = [h.compliance for h in hist]
    # compliance falls monotonically over the first iterations of the
    # cantilever from a uniform start
    assert all(b < a for a, b in zip(c, c[1:]))
    for h in hist:
        assert abs(h.volume - prob.volfrac) < 2e-3
    assert np.all((x >= 0) & (x <= 1))


def test_direct_and_pcg_solvers_give_same_trajectory():
    prob = problems.cantilever(12, 4, 3, load="edge", volfrac=0.3, rmin=1.5)
    _, h1 = topopt.top3d(prob, iters=3, solver="direct")
    _, h2 = topopt.top3d(prob, iters=3, solver="pcg", rtol=1e-12)
    for a, b in zip(h1, h2):
        assert abs(a.compliance - b.compliance) <= 1e-8 * a.compliance
        assert b.pcg_iters > 0


def test_passive_void_stays_empty():
    nelx, nely, nelz = 16, 8, 2
    pas = problems.void_cylinder_z(nelx, nely, nelz, 8.0, 4.0, 2.5)
    prob = problems.cantilever(nelx, nely, nelz, volfrac=0.3, passive=pas)
    x, hist = topopt.top3d(prob, iters=3)
    assert np.all(x[pas == 1] == 0.0)
    assert abs(hist[-1].volume - 0.3) < 2e-3
