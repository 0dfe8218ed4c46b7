"""The SIMP + OC optimisation loop (FP64, assembled K, direct or PCG solve).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 2.5: FEM analysis -> sensitivities -> sensitivity filter ->
OC design update -> convergence check, repeated.  The paper gives no stopping
tolerance, so the loop runs a fixed number of iterations.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import fem, filters, oc


@dataclasses.dataclass
class IterRecord:
    it: int
    compliance: float
    volume: float          # design volume fraction after the update
    change: float          # max |x_new - x|
    lam: float
    halvings: int
    pcg_iters: int


def state_setup(prob):
    KE = fem.element_stiffness(prob.nu)
    fixed = prob.fixed
    f = fem.masked_load(prob.load, fixed)
    return KE, fixed, f


def analyse(prob, x, KE, f, solver="direct", rtol=1e-12, x0=None):
    """Solve K(x) u = f and return (u, ce, c, dc, pcg_iters)."""
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    its = 0
    if solver in ("direct", "dense"):
        K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
        u = (fem.solve_direct if solver == "direct" else fem.solve_dense)(K, f, prob.fixed)
    elif solver == "pcg":
        K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
        d = K.diagonal()
        u, its, _ = fem.jacobi_pcg(lambda v: K @ v, d, f, rtol=rtol, x0=x0)
    else:
        raise ValueError(solver)
    ce = fem.element_energies(prob.nelx, prob.nely, prob.nelz, KE, u)
    c, dc = fem.compliance_and_sensitivity(x, ce, prob.penal, prob.E0, prob.Emin)
    return u, ce, c, dc, its


def physical_density(prob, x, H, Hs, filter_kind):
    """The field the analysis sees: x itself (sensitivity filter), or the
    filtered field H x / Hs with passive elements pinned (density filter,
    Section 2.4 with the passive regions of Section 2.3)."""
    if filter_kind != "density":
        return x
    passive = prob.passive_or_zeros()
    xphys = filters.density_filter(H, Hs, x)
    xphys[passive == 1] = 0.0
    xphys[passive == 2] = 1.0
    return xphys


def filtered_sensitivity(prob, x, xphys, H, Hs, KE, f, filter_kind, solver="direct",
                         rtol=1e-12, x0=None):
    """Analysis on xphys and the sensitivities the OC update receives:
    returns (u, c, dcf, pcg_iters).  Sensitivity filter: dcf = H(x dc) /
    (Hs max(1e-3, x)).  Density filter: dcf = d c(xphys(x)) / dx by the chain
    rule through the filter; pinned elements carry nothing back."""
    u, ce, c, dc, its = analyse(prob, xphys, KE, f, solver=solver, rtol=rtol, x0=x0)
    if filter_kind == "density":
        dcf = filters.density_filter_chain(H, Hs, dc, prob.passive_or_zeros())
    else:
        dcf = filters.sensitivity_filter(H, Hs, x, dc)
    return u, c, dcf, its


def top3d(prob, iters=None, solver="direct", rtol=1e-12, filter_kind="sensitivity",
          x_init=None):
    """Run the loop; returns (x, history list of IterRecord)."""
    iters = prob.iters if iters is None else iters
    KE, fixed, f = state_setup(prob)
    H = filters.filter_matrix(prob.nelx, prob.nely, prob.nelz, prob.rmin)
    Hs = filters.row_sums(H)
    passive = prob.passive_or_zeros()
    x = prob.initial_density() if x_init is None else x_init.copy()
    hist: List[IterRecord] = []
    u = None
    for it in range(iters):
        # the OC update and its volume act on x (also with the density filter)
        xphys = physical_density(prob, x, H, Hs, filter_kind)
        u, c, dcf, its = filtered_sensitivity(prob, x, xphys, H, Hs, KE, f, filter_kind,
                                              solver=solver, rtol=rtol, x0=u)
        xnew, lam, nh, vol = oc.oc_update(x, dcf, prob.volfrac, passive, prob.move,
                                          prob.bisect_tol)
        ndes = max(1, int(np.count_nonzero(passive == 0)))
        hist.append(IterRecord(it, c, vol / ndes, float(np.max(np.abs(xnew - x))), lam, nh, its))
        x = xnew
    return x, hist
