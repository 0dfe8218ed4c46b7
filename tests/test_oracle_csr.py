"""Pins of the oracle's C part (oracle/csr_pcg.c) against the NumPy oracle:
the assembled CSR operator equals apply_bc(assemble(...)), its Jacobi-PCG
reaches the direct solution, and the element steps, the filter and the OC
bisection agree with their NumPy restatements."""
import shutil

import numpy as np
import pytest

from oracle import csr, fem, filters, oc
from synth import problems

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")


def _case(seed=3):
    prob = problems.cantilever(7, 4, 3, load="edge")
    x = problems.random_density(prob.nel, seed, 0.05, 1.0)
    E = fem.simp_modulus(x, prob.penal)
    KE = fem.element_stiffness(prob.nu)
    return prob, x, E, KE


def test_csr_operator_equals_numpy_assembly():
    prob, x, E, KE = _case()
    fx = prob.fixed.copy()
    fx[[5, 40, 77]] = 1
    op = csr.Operator(prob.nelx, prob.nely, prob.nelz, E, KE, fx)
    ref = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), fx)
    assert abs(op.matrix() - ref).max() <= 1e-13 * abs(ref).max()
    op.close()


def test_csr_pcg_reaches_the_direct_solution():
    prob, x, E, KE = _case(4)
    op = csr.Operator(prob.nelx, prob.nely, prob.nelz, E, KE, prob.fixed)
    f = fem.masked_load(prob.load, prob.fixed)
    u, its = op.pcg(f, rtol=1e-12)
    K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
    u_ref = fem.solve_direct(K, f, prob.fixed)
    assert its > 10
    assert np.linalg.norm(u - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    op.close()


def test_csr_element_steps_filter_and_oc_match_numpy():
    prob, x, E, KE = _case(5)
    u = problems.random_vector(prob.ndof, 6)
    c, ce, dc = csr.element_steps(prob.nelx, prob.nely, prob.nelz, KE, u, x, prob.penal)
    ce_ref = fem.element_energies(prob.nelx, prob.nely, prob.nelz, KE, u)
    c_ref, dc_ref = fem.compliance_and_sensitivity(x, ce_ref, prob.penal)
    assert np.allclose(ce, ce_ref, rtol=1e-12, atol=0)
    assert np.allclose(dc, dc_ref, rtol=1e-12, atol=0)
    assert c == pytest.approx(c_ref, rel=1e-12)
    dcf = csr.sensitivity_filter(prob.nelx, prob.nely, prob.nelz, 1.5, x, dc)
    H = filters.filter_matrix(prob.nelx, prob.nely, prob.nelz, 1.5)
    assert np.allclose(dcf, filters.sensitivity_filter(H, filters.row_sums(H), x, dc),
                       rtol=1e-12, atol=0)
    pas = np.zeros(prob.nel, np.uint8)
    pas[3], pas[10] = 1, 2
    xn, h = csr.oc_update(x, dcf, 0.4, pas, 0.2, 1e-3)
    xr, lam, hr, vol = oc.oc_update(x, dcf, 0.4, pas, 0.2, 1e-3)
    assert h == hr
    assert np.allclose(xn, xr, rtol=0, atol=1e-12)
    assert csr.threads() >= 1
