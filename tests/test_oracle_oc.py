"""Pins of the oracle's OC update (paper Section 2.3)."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import oc
from synth import problems


def _inputs(n=500, seed=21):
    x = problems.random_density(n, seed, 0.0, 1.0)
    x[::17] = 0.0
    x[::23] = 1.0
    dc = -problems.random_density(n, seed + 1, 1e-3, 10.0)
    pas = np.zeros(n, np.uint8)
    pas[5::31] = 1
    pas[9::37] = 2
    return x, dc, pas


def test_candidate_respects_move_limits_and_bounds():
    x, dc, _ = _inputs()
    for lam in (1e-6, 1e-2, 1.0, 1e3):
        xn = oc.oc_candidate(x, dc, lam, 0.2)
        assert np.all(xn >= np.maximum(0.0, x - 0.2) - 1e-15)
        assert np.all(xn <= np.minimum(1.0, x + 0.2) + 1e-15)
        # unconstrained elements take the OC fixed-point value x sqrt(-dc/lambda)
        B = x * np.sqrt(-dc / lam)
        free = (B > np.maximum(0, x - 0.2)) & (B < np.minimum(1, x + 0.2))
        assert np.allclose(xn[free], B[free], rtol=1e-15)


def test_volume_monotone_in_lambda():
    x, dc, pas = _inputs()
    lams = np.logspace(-6, 6, 200)
    V = [oc.oc_candidate(x, dc, l, 0.2)[pas == 0].sum() for l in lams]
    assert np.all(np.diff(V) <= 1e-12)


@pytest.mark.parametrize("tol", [1e-3, 1e-12])
def test_bisection_brackets_exact_root(tol):
    x, dc, pas = _inputs()
    volfrac = 0.4
    xn, lam, nh, vol = oc.oc_update(x, dc, volfrac, pas, 0.2, tol)
    target = volfrac * np.count_nonzero(pas == 0)
    # pinned passive elements
    assert np.all(xn[pas == 1] == 0.0) and np.all(xn[pas == 2] == 1.0)
    # independent root of the (continuous, monotone) volume function
    g = lambda l: oc.oc_candidate(x, dc, l, 0.2)[pas == 0].sum() - target
    root = brentq(g, 1e-12, 1e9, xtol=1e-300, rtol=1e-15)
    assert abs(lam - root) <= 2 * tol * root
    # the bracket halves each step: about log2(1e9 / (2 tol root)) steps
    assert abs(nh - np.log2(1e9 / (2 * tol * root))) < 2
    if tol <= 1e-12:
        assert abs(vol / target - 1) <= 1e-6


def test_bisection_volume_error_small():
    prob = problems.config_small()
    x = prob.initial_density()
    dc = -problems.random_density(prob.nel, 3, 0.1, 5.0)
    xn, lam, nh, vol = oc.oc_update(x, dc, prob.volfrac, None, 0.2, 1e-3)
    assert abs(vol / (prob.volfrac * prob.nel) - 1) < 2e-3
    assert 30 <= nh <= 45
