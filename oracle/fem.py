"""Finite element analysis on a structured grid of unit hex8 elements (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 2.2: 8-node hexahedral elements, element stiffness matrices
pre-computed once, global stiffness K assembled from them (COO -> CSR), the
system K U = F solved directly, clamped dofs imposed by modifying the system
(not by penalty).  Section 2.3: SIMP modulus E_e = Emin + rho_e^p (E0 - Emin);
compliance sensitivities.

Conventions (this project's own; the paper gives none):
  element local node a + 2b + 4c sits at corner offset (a, b, c) in {0,1}^3;
  strain vector (xx, yy, zz, gamma_xy, gamma_yz, gamma_zx);
  unit element size (the paper measures rmin in elements, Section 4.2).

Clamped dofs: the operator restricted to the free dofs, with identity rows
and columns on the clamped ones ("modify the system matrix and load vector",
Section 2.2, with prescribed value 0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------- element


def _corners():
    return np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)],
                    dtype=np.float64)   # row n = a + 2b + 4c


def shape_gradients(x: float, y: float, z: float) -> np.ndarray:
    """Gradients [8, 3] of the trilinear shape functions on [0,1]^3 at (x,y,z).

    N_n = (a ? x : 1-x) * (b ? y : 1-y) * (c ? z : 1-z).
    """
    g = np.zeros((8, 3))
    for n, (a, b, c) in enumerate(_corners()):
        fx = x if a else 1 - x
        fy = y if b else 1 - y
        fz = z if c else 1 - z
        dx = 1.0 if a else -1.0
        dy = 1.0 if b else -1.0
        dz = 1.0 if c else -1.0
        g[n] = [dx * fy * fz, fx * dy * fz, fx * fy * dz]
    return g


def elasticity_matrix(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Isotropic 6x6 constitutive matrix (engineering shear strains)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def strain_matrix(g: np.ndarray) -> np.ndarray:
    """B [6, 24] from shape gradients g [8, 3]; dof 3n + c."""
    B = np.zeros((6, 24))
    for n in range(8):
        dx, dy, dz = g[n]
        B[0, 3 * n + 0] = dx
        B[1, 3 * n + 1] = dy
        B[2, 3 * n + 2] = dz
        B[3, 3 * n + 0] = dy
        B[3, 3 * n + 1] = dx
        B[4, 3 * n + 1] = dz
        B[4, 3 * n + 2] = dy
        B[5, 3 * n + 0] = dz
        B[5, 3 * n + 2] = dx
    return B


def element_stiffness(nu: float = 0.3, E: float = 1.0) -> np.ndarray:
    """KE = integral over the unit cube of B^T C B (Section 2.2, "element
    stiffness matrices are pre-computed").

    2x2x2 Gauss-Legendre quadrature is exact here: the integrand is at most
    quadratic in each coordinate.
    """
    C = elasticity_matrix(E, nu)
    gp = [0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)]
    KE = np.zeros((24, 24))
    for x in gp:
        for y in gp:
            for z in gp:
                B = strain_matrix(shape_gradients(x, y, z))
                KE += 0.125 * B.T @ C @ B
    return KE


# ---------------------------------------------------------------- mesh


def element_dofs(nelx: int, nely: int, nelz: int) -> np.ndarray:
    """edofMat [nel, 24]: global dof of each element's local dof 3n + c."""
    i, j, k = np.meshgrid(np.arange(nelx), np.arange(nely), np.arange(nelz), indexing="ij")
    # order elements as e = i + nelx (j + nely k)
    i = i.transpose(2, 1, 0).ravel()
    j = j.transpose(2, 1, 0).ravel()
    k = k.transpose(2, 1, 0).ravel()
    nx, ny = nelx + 1, nely + 1
    ed = np.zeros((i.size, 24), dtype=np.int64)
    for n, (a, b, c) in enumerate(_corners().astype(int)):
        node = (i + a) + nx * ((j + b) + ny * (k + c))
        for comp in range(3):
            ed[:, 3 * n + comp] = 3 * node + comp
    return ed


def simp_modulus(x: np.ndarray, penal: float, E0: float = 1.0, Emin: float = 1e-9) -> np.ndarray:
    """E_e = Emin + x_e^p (E0 - Emin)  (Section 2.3)."""
    return Emin + x ** penal * (E0 - Emin)


def assemble(nelx: int, nely: int, nelz: int, E: np.ndarray, KE: np.ndarray) -> sp.csr_matrix:
    """K = sum_e E_e P_e^T KE P_e as CSR (Section 2.2: COO, then CSR)."""
    ed = element_dofs(nelx, nely, nelz)
    n = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    iK = np.repeat(ed, 24, axis=1).ravel()
    jK = np.tile(ed, (1, 24)).ravel()
    sK = (E[:, None] * KE.ravel()[None, :]).ravel()
    return sp.coo_matrix((sK, (iK, jK)), shape=(n, n)).tocsr()


def apply_bc(K: sp.csr_matrix, fixed: np.ndarray) -> sp.csr_matrix:
    """Clamped dofs: zero their rows and columns, unit diagonal."""
    free = (fixed == 0).astype(np.float64)
    D = sp.diags(free)
    return (D @ K @ D + sp.diags(1.0 - free)).tocsr()


def matvec_elementwise(nelx, nely, nelz, E, KE, p, fixed) -> np.ndarray:
    """y = Kbar p with Kbar the clamped operator, by the element sum.

    y = sum_e E_e P_e^T KE P_e (p with clamped entries zeroed); then
    y_d = p_d on clamped dofs.  Same operator as ``apply_bc(assemble(...))``.
    """
    ed = element_dofs(nelx, nely, nelz)
    q = np.where(fixed != 0, 0.0, p)
    ye = (q[ed] @ KE) * E[:, None]           # KE symmetric
    y = np.bincount(ed.ravel(), weights=ye.ravel(), minlength=p.size)
    return np.where(fixed != 0, p, y)


def matvec_rows(nelx, nely, nelz, E, KE, p, fixed, rows, absolute=False):
    """Selected entries y[rows] of y = Kbar p (``matvec_elementwise``), each
    summed over the (at most 8) elements around its node; with `absolute`,
    the same sums of |E_e KE_ij p_j| (the size of the terms being summed).
    For grids too large to assemble."""
    nx, ny = nelx + 1, nely + 1
    out = np.zeros(len(rows))
    for t, d in enumerate(rows):
        if fixed[d]:
            out[t] = abs(p[d]) if absolute else p[d]
            continue
        node, comp = divmod(int(d), 3)
        i, j, k = node % nx, (node // nx) % ny, node // (nx * ny)
        acc = 0.0
        for c in (0, 1):
            for b in (0, 1):
                for a in (0, 1):
                    ei, ej, ek = i - a, j - b, k - c
                    if not (0 <= ei < nelx and 0 <= ej < nely and 0 <= ek < nelz):
                        continue
                    e = ei + nelx * (ej + nely * ek)
                    row = KE[3 * (a + 2 * b + 4 * c) + comp]
                    for m, (aa, bb, cc) in enumerate(_corners().astype(int)):
                        nd = (ei + aa) + nx * ((ej + bb) + ny * (ek + cc))
                        for cm in range(3):
                            dof = 3 * nd + cm
                            v = 0.0 if fixed[dof] else p[dof]
                            term = E[e] * row[3 * m + cm] * v
                            acc += abs(term) if absolute else term
        out[t] = acc
    return out


def masked_load(f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    return np.where(fixed != 0, 0.0, f)


def solve_direct(Kbar: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """Sparse direct solve of the clamped system (Section 2.2)."""
    free = np.flatnonzero(fixed == 0)
    u = np.zeros_like(f)
    Kff = Kbar[free][:, free].tocsc()
    u[free] = spla.spsolve(Kff, f[free])
    return u


def solve_dense(Kbar: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """Brute force for tiny meshes: dense LU of the free block."""
    free = np.flatnonzero(fixed == 0)
    u = np.zeros_like(f)
    A = Kbar.toarray()[np.ix_(free, free)]
    u[free] = np.linalg.solve(A, f[free])
    return u


def jacobi_pcg(matvec, diag: np.ndarray, f: np.ndarray, rtol: float = 1e-8,
               maxit: int = 100000, x0=None, true_residual=True):
    """Preconditioned conjugate gradients with M = diag(K) (textbook form).

    Stops when ||f - K u||_2 <= rtol ||f||_2.  The recurrence residual decides
    the loop; with ``true_residual`` the exit is confirmed with f - K u and
    the iteration continues if the true residual is still above rtol.
    Returns (u, iterations, final true relative residual).
    """
    u = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - matvec(u)
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return np.zeros_like(f), 0, 0.0
    dinv = 1.0 / diag
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        if np.linalg.norm(r) <= rtol * fn:
            if not true_residual:
                break
            rt = f - matvec(u)
            if np.linalg.norm(rt) <= rtol * fn:
                break
            r = rt
            z = dinv * r
            p = z.copy()
            rz = r @ z
        q = matvec(p)
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    res = np.linalg.norm(f - matvec(u)) / fn
    return u, it, res


def jacobi_diagonal(nelx, nely, nelz, E, KE, fixed) -> np.ndarray:
    """diag(Kbar): sum over elements of E_e KE_dd, 1 on clamped dofs."""
    ed = element_dofs(nelx, nely, nelz)
    d = np.bincount(ed.ravel(), weights=(E[:, None] * np.diag(KE)[None, :]).ravel(),
                    minlength=3 * (nelx + 1) * (nely + 1) * (nelz + 1))
    return np.where(fixed != 0, 1.0, d)


def element_energies(nelx, nely, nelz, KE, u) -> np.ndarray:
    """ce_e = u_e^T KE u_e (Section 2.3 sensitivities, unit modulus)."""
    ed = element_dofs(nelx, nely, nelz)
    ue = u[ed]
    return np.einsum("ei,ij,ej->e", ue, KE, ue)


def compliance_and_sensitivity(x, ce, penal, E0=1.0, Emin=1e-9):
    """c = sum_e E_e ce_e;  dc_e = -p x_e^(p-1) (E0 - Emin) ce_e  (Section 2.3)."""
    c = float(np.sum(simp_modulus(x, penal, E0, Emin) * ce))
    dc = -penal * x ** (penal - 1.0) * (E0 - Emin) * ce
    return c, dc
