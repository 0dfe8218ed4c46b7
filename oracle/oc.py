"""Optimality Criteria update with bisection on the volume multiplier (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 2.3: the filtered sensitivities drive the OC update rule; the
Lagrange multiplier of the volume constraint is found by bisection; standard
move limits are applied; the volume constraint accounts for passive
(non-design) regions.  Readings taken where the paper is silent:

* update  x_new = clamp(x sqrt(-dc~ / lambda), max(0, x - move), min(1, x + move))
  (dv = 1; lower bound 0 -- Emin keeps K non-singular);
* lambda bracket [0, 1e9], stop when (l2 - l1) / (l1 + l2) <= tol;
* volume test on design elements only: sum_design x_new > volfrac * n_design
  raises l1 (ties lower l2);
* void elements pinned at 0, solid elements at 1, neither counted.
"""
from __future__ import annotations

import numpy as np


def oc_candidate(x, dc, lam, move):
    """x_new(lambda) for every element (before passive pinning)."""
    B = np.sqrt(np.maximum(0.0, -dc) / lam)
    return np.maximum(0.0, np.maximum(x - move, np.minimum(1.0, np.minimum(x + move, x * B))))


def oc_update(x, dc, volfrac, passive=None, move=0.2, tol=1e-3, l1=0.0, l2=1e9):
    """Scalar bisection, one candidate lambda at a time.

    Returns (x_new, lambda_mid_last, halvings, design volume of x_new).
    """
    if passive is None:
        passive = np.zeros(x.size, dtype=np.uint8)
    design = passive == 0
    target = volfrac * np.count_nonzero(design)
    halvings = 0
    lmid = 0.5 * (l1 + l2)
    xnew = x.copy()
    while (l2 - l1) / (l1 + l2) > tol:
        lmid = 0.5 * (l1 + l2)
        xnew = oc_candidate(x, dc, lmid, move)
        xnew[passive == 1] = 0.0
        xnew[passive == 2] = 1.0
        if np.sum(xnew[design]) > target:
            l1 = lmid
        else:
            l2 = lmid
        halvings += 1
    return xnew, lmid, halvings, float(np.sum(xnew[design]))


def design_volume(xnew, passive=None):
    if passive is None:
        return float(np.sum(xnew))
    return float(np.sum(xnew[passive == 0]))
