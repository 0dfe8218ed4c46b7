"""Geometric multigrid V-cycle with learned parameters (FP64, plain NumPy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper, which solves K U = F with a sparse direct solver
(Section 2.2).  This module defines the library's learned preconditioner for
the same K (Sections 2.2-2.3: K = sum_e E_e KE, E_e from the SIMP law), so
that its GPU application can be checked against a plain restatement:

Hierarchy.  Level 0 is the design grid.  Level l+1 halves every element
count of level l, rounding up (n -> (n + 1) // 2); coarsening stops once the
largest element count is at most 4 or the smallest is below 2.  Coarse node
C sits on fine node 2C (coarse nodes past the fine grid's last node are
allowed).  A coarse dof is clamped when the fine dof at 2C exists and is
clamped.

Coarse operator (rediscretisation).  A coarse element covers the 2 x 2 x 2
fine elements (2i + a, 2j + b, 2k + c); missing ones (past the fine grid)
count as modulus 0.  Its modulus is  s_l * (sum_children E^q_l / 8)^(1/q_l)
and its stiffness that modulus times the same unit KE: the trilinear element
stiffness scales with the element size, so s = 2 reproduces the Galerkin
operator P^T K P for a uniform modulus.

Transfer.  Prolongation P is trilinear interpolation per component, with
weights prod_d (1 - |F_d - 2 C_d| / 2) for |F_d - 2 C_d| <= 1, clamped dofs
of either grid zeroed; restriction is its transpose.

Smoother.  Damped Jacobi, z <- z + om_l D^-1 (b - K z), D = diag(K) per dof
(0 on clamped dofs), nu sweeps (default 1) before and nu after the coarse
correction, the first from z = 0.  On the coarsest level, `sweeps` sweeps from z = 0.
The damping is relative to the level's largest eigenvalue of D^-1 K:
om_l = w_l * 2 / lam_l with lam_l = min(1.2 rq, l1), rq the Rayleigh
quotient z^T K z / z^T D z after POWER_STEPS steps of the power iteration
z <- D^-1 K z / rq from a fixed start vector (hash_start), l1 the bound
max_a sum_b |KE_ab| / KE_aa that no modulus field can exceed (5.36 for
nu = 0.3).  The power iteration approaches lam from below; with the 1.2
margin every smoother with 0 < w < 1 converges (a fixed weight such as 0.5
does not: void-bounded nodes reach lam = 4.5).

The V-cycle is linear in b and symmetric: pre- and post-smoothers are the
same symmetric operator and restriction is the transpose of prolongation.

Learned parameters theta = (w_0..w_L, q_1..q_L, s_1..s_L); the training loss
of a snapshot (r, e = K^-1 r) is the energy norm of the error left by one
application, ||e - V r||_K^2 / ||e||_K^2 = (z^T K z - 2 z^T r + r^T e) / (r^T e).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import fem


@dataclasses.dataclass
class Level:
    dims: tuple            # (nelx, nely, nelz)
    fixed: np.ndarray      # bool [3N]
    ed: np.ndarray         # element dofs [nel, 24]
    E: np.ndarray = None   # moduli [nel]
    dinv: np.ndarray = None
    lam: float = 1.0       # estimate of the largest eigenvalue of D^-1 K


def hierarchy(nelx, nely, nelz, fixed, max_levels=10) -> List[Level]:
    """The level list (level 0 first) with the injected clamps."""
    lv = [Level((nelx, nely, nelz), np.asarray(fixed) != 0, fem.element_dofs(nelx, nely, nelz))]
    while (max(lv[-1].dims) > 4 and min(lv[-1].dims) >= 2 and len(lv) <= max_levels):
        d = lv[-1].dims
        dc = tuple((n + 1) // 2 for n in d)
        nx, ny, nz = (n + 1 for n in d)
        cx, cy, cz = (n + 1 for n in dc)
        ff = lv[-1].fixed.reshape(nz, ny, nx, 3)
        fc = np.zeros((cz, cy, cx, 3), bool)
        kk, jj, ii = 2 * np.arange(cz), 2 * np.arange(cy), 2 * np.arange(cx)
        ok_k, ok_j, ok_i = kk < nz, jj < ny, ii < nx
        fc[np.ix_(ok_k, ok_j, ok_i)] = ff[np.ix_(kk[ok_k], jj[ok_j], ii[ok_i])]
        lv.append(Level(dc, fc.reshape(-1), fem.element_dofs(*dc)))
    return lv


def coarse_moduli(E, dims, q, s):
    """s (sum over the 8 child slots of E^q / 8)^(1/q); missing children 0."""
    nelx, nely, nelz = dims
    cx, cy, cz = ((n + 1) // 2 for n in dims)
    Ep = np.zeros((2 * cz, 2 * cy, 2 * cx))
    Ep[:nelz, :nely, :nelx] = np.asarray(E).reshape(nelz, nely, nelx)
    m = (Ep.reshape(cz, 2, cy, 2, cx, 2) ** q).sum(axis=(1, 3, 5)) / 8.0
    return (s * m ** (1.0 / q)).reshape(-1)


def prolongation_1d(nf, nc):
    """Dense 1D trilinear weights [nf fine nodes, nc coarse nodes]."""
    P = np.zeros((nf, nc))
    for C in range(nc):
        for dlt in (-1, 0, 1):
            F = 2 * C + dlt
            if 0 <= F < nf:
                P[F, C] = 1.0 - abs(dlt) / 2.0
    return P


def prolong(fine: Level, coarse: Level, zc):
    Px, Py, Pz = (prolongation_1d(nf + 1, nc + 1) for nf, nc in zip(fine.dims, coarse.dims))
    cx, cy, cz = (n + 1 for n in coarse.dims)
    Z = np.where(coarse.fixed, 0.0, zc).reshape(cz, cy, cx, 3)
    out = np.einsum("kc,jb,ia,cbad->kjid", Pz, Py, Px, Z).reshape(-1)
    return np.where(fine.fixed, 0.0, out)


def restrict(fine: Level, coarse: Level, rf):
    Px, Py, Pz = (prolongation_1d(nf + 1, nc + 1) for nf, nc in zip(fine.dims, coarse.dims))
    nx, ny, nz = (n + 1 for n in fine.dims)
    R = np.where(fine.fixed, 0.0, rf).reshape(nz, ny, nx, 3)
    out = np.einsum("kc,jb,ia,kjid->cbad", Pz, Py, Px, R).reshape(-1)
    return np.where(coarse.fixed, 0.0, out)


def operator(L: Level, KE, v):
    """K v on a level (element sum; clamped rows and columns removed, the
    clamped entries of the result set to 0 as the smoother needs)."""
    q = np.where(L.fixed, 0.0, v)
    ye = (q[L.ed] @ KE) * L.E[:, None]
    y = np.bincount(L.ed.ravel(), weights=ye.ravel(), minlength=v.size)
    return np.where(L.fixed, 0.0, y)


POWER_STEPS = 16
POWER_MARGIN = 1.2


def l1_bound(KE):
    """max_a sum_b |KE_ab| / KE_aa: a bound on lam_max(D^-1 K) for any moduli."""
    return float(np.max(np.abs(KE).sum(axis=1) / np.diag(KE)))


def hash_start(n):
    """Start vector of the power iteration: entry i is the fractional part of
    i * 2654435761 / 2^32 (Knuth's multiplicative hash) minus 1/2."""
    i = np.arange(n, dtype=np.uint64)
    return ((i * np.uint64(2654435761)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5


def rayleigh_power(L: Level, KE, steps=POWER_STEPS):
    """Rayleigh quotient of D^-1 K after `steps` power steps from hash_start."""
    z = np.where(L.fixed | (L.dinv == 0), 0.0, hash_start(L.fixed.size))
    lam = 1.0
    for _ in range(steps):
        t = operator(L, KE, z)
        dz = np.where(L.dinv > 0, z / np.where(L.dinv > 0, L.dinv, 1.0), 0.0)
        lam = float(z @ t) / float(z @ dz)
        z = L.dinv * t / lam
    return lam


def lambda_max(L: Level, KE, steps=POWER_STEPS):
    """The eigenvalue bound the smoother uses: min(1.2 rq, l1)."""
    return min(POWER_MARGIN * rayleigh_power(L, KE, steps), l1_bound(KE))


def setup(lv: List[Level], E0, KE, q, s):
    """Moduli, inverse diagonals and eigenvalue estimates of every level for
    fine moduli E0."""
    lv[0].E = np.asarray(E0, dtype=np.float64)
    for l in range(1, len(lv)):
        lv[l].E = coarse_moduli(lv[l - 1].E, lv[l - 1].dims, q[l], s[l])
    for L in lv:
        d = np.bincount(L.ed.ravel(), weights=(L.E[:, None] * np.diag(KE)[None, :]).ravel(),
                        minlength=L.fixed.size)
        L.dinv = np.where(L.fixed | (d <= 0), 0.0, 1.0 / np.where(d > 0, d, 1.0))
        L.lam = lambda_max(L, KE)


def damping(L: Level, w):
    """om = w * 2 / lam: below the stability limit for w < 1."""
    return w * 2.0 / L.lam


def vcycle(lv: List[Level], KE, b, w, sweeps, l=0, nu=1):
    """z = V b on level l (recursive); nu damped-Jacobi sweeps before and
    after each coarse correction."""
    L = lv[l]
    om = damping(L, w[l])
    z = om * L.dinv * b
    if l == len(lv) - 1:
        for _ in range(sweeps - 1):
            z = z + om * L.dinv * (b - operator(L, KE, z))
        return z
    for _ in range(nu - 1):
        z = z + om * L.dinv * (b - operator(L, KE, z))
    bc = restrict(L, lv[l + 1], b - operator(L, KE, z))
    z = z + prolong(L, lv[l + 1], vcycle(lv, KE, bc, w, sweeps, l + 1, nu))
    for _ in range(nu):
        z = z + om * L.dinv * (b - operator(L, KE, z))
    return z


def energy_loss(K, r, e, z):
    """||e - z||_K^2 / ||e||_K^2 for e = K^-1 r, as (z^T K z - 2 z^T r + r^T e) / r^T e."""
    rte = float(r @ e)
    return (float(z @ (K @ z)) - 2.0 * float(z @ r) + rte) / rte


def default_theta(nlev):
    """Initial parameters: w = 2/3 on every level (damping 4 / (3 lam)),
    q = 1 (arithmetic mean), s = 2 (the size scaling of the rediscretised
    stiffness)."""
    return np.concatenate([np.full(nlev, 2.0 / 3.0), np.ones(nlev - 1), np.full(nlev - 1, 2.0)])


def split_theta(theta, nlev):
    """(w[0..L], q[0..L], s[0..L]); q[0], s[0] unused (set to 1)."""
    theta = np.asarray(theta, dtype=np.float64)
    w = theta[:nlev]
    q = np.concatenate([[1.0], theta[nlev:2 * nlev - 1]])
    s = np.concatenate([[1.0], theta[2 * nlev - 1:3 * nlev - 2]])
    return w, q, s
