"""Pins of the oracle's optimisation loop (paper Section 2.5)."""
import numpy as np
import pytest

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


def _density_problem():
    """A tiny cantilever with one void and two solid passive elements inside
    the design domain, and a graded design field."""
    from oracle import filters
    prob = problems.cantilever(5, 3, 2, load="edge", volfrac=0.4, rmin=1.5)
    pas = np.zeros(prob.nel, np.uint8)
    pas[7] = 1
    pas[[8, 22]] = 2
    prob.passive = pas
    x = problems.random_density(prob.nel, 31, 0.2, 0.9)
    x[pas == 1] = 0.0
    x[pas == 2] = 1.0
    H = filters.filter_matrix(prob.nelx, prob.nely, prob.nelz, prob.rmin)
    return prob, x, H, filters.row_sums(H)


def test_density_branch_pins_passive_elements_in_the_filtered_field():
    from oracle import filters
    prob, x, H, Hs = _density_problem()
    xphys = topopt.physical_density(prob, x, H, Hs, "density")
    pas = prob.passive
    assert np.all(xphys[pas == 1] == 0.0) and np.all(xphys[pas == 2] == 1.0)
    # design elements keep the plain filtered value, which the passive
    # neighbours (x = 0 or 1) enter with their pinned x
    Hb = filters.filter_matrix_bruteforce(prob.nelx, prob.nely, prob.nelz, prob.rmin)
    ref = (Hb @ x) / np.asarray(Hb.sum(axis=1)).ravel()
    d = pas == 0
    assert np.allclose(xphys[d], ref[d], rtol=1e-14, atol=0)


def test_density_branch_sensitivity_is_the_derivative_of_the_compliance():
    """The sensitivities the density-filter branch hands to OC equal central
    differences of c(x) = f^T u(xphys(x)), with dense solves and the
    brute-force filter: this catches a missing chain rule, a chain rule
    through the pinned elements, or pinning applied at the wrong point."""
    from oracle import fem, filters
    prob, x, H, Hs = _density_problem()
    KE, _, f = topopt.state_setup(prob)
    xphys = topopt.physical_density(prob, x, H, Hs, "density")
    _, c, dcf, _ = topopt.filtered_sensitivity(prob, x, xphys, H, Hs, KE, f, "density",
                                               solver="dense")
    Hb = filters.filter_matrix_bruteforce(prob.nelx, prob.nely, prob.nelz, prob.rmin)
    hs = np.asarray(Hb.sum(axis=1)).ravel()
    pas = prob.passive

    def compliance(xv):
        xp = (Hb @ xv) / hs
        xp[pas == 1] = 0.0
        xp[pas == 2] = 1.0
        E = fem.simp_modulus(xp, prob.penal, prob.E0, prob.Emin)
        K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
        return float(f @ fem.solve_dense(K, f, prob.fixed))

    assert compliance(x) == pytest.approx(c, rel=1e-12)
    h = 1e-6
    scale = np.abs(dcf).max()
    # every element, passive ones included: their x enters the neighbours'
    # filtered values even though their own filtered value is pinned
    for e in range(prob.nel):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        fd = (compliance(xp) - compliance(xm)) / (2 * h)
        assert abs(fd - dcf[e]) <= 1e-6 * scale, e


def test_density_branch_oc_acts_on_x_and_counts_the_volume_of_x():
    """One density-filter OC iteration: the move limit is taken around x (not
    the filtered field), passive elements keep their pinned x, and the
    recorded volume is the design volume of the new x, on target at a tight
    bisection tolerance."""
    prob, x, H, Hs = _density_problem()
    prob.bisect_tol = 1e-12
    xnew, hist = topopt.top3d(prob, iters=1, solver="dense", filter_kind="density", x_init=x)
    pas = prob.passive
    d = pas == 0
    assert np.all(np.abs(xnew[d] - x[d]) <= prob.move + 1e-15)
    assert np.all(xnew[pas == 1] == 0.0) and np.all(xnew[pas == 2] == 1.0)
    assert hist[0].volume == pytest.approx(xnew[d].mean(), rel=1e-14)
    assert abs(hist[0].volume / prob.volfrac - 1.0) <= 1e-6
