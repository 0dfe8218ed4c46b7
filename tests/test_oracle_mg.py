"""Pins of the oracle's multigrid preconditioner (oracle/mg.py): transfer
operators against interpolation of linear fields and their adjoint identity,
coarse moduli by hand, the rediscretised coarse operator against the
Galerkin product P^T K P, and the V-cycle's symmetry, positivity and its
one-level closed form."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, mg
from synth import problems


@pytest.mark.parametrize("nel", [4, 5, 7, 8])
def test_prolongation_interpolates_linear_fields_exactly(nel):
    nc = (nel + 1) // 2 + 1
    P = mg.prolongation_1d(nel + 1, nc)
    a, b = 0.3, -1.7
    coarse = a + b * 2.0 * np.arange(nc)          # coarse node C sits on fine node 2C
    assert np.allclose(P @ coarse, a + b * np.arange(nel + 1), rtol=0, atol=1e-14)


def test_restriction_is_the_transpose_of_prolongation():
    prob = problems.cantilever(11, 6, 5)
    fixed = prob.fixed.copy()
    rng = np.random.default_rng(3)
    fixed[rng.choice(fixed.size, 40, replace=False)] = 1
    lv = mg.hierarchy(11, 6, 5, fixed)
    assert len(lv) >= 2 and lv[1].dims == (6, 3, 3)
    zc = rng.standard_normal(lv[1].fixed.size)
    rf = rng.standard_normal(lv[0].fixed.size)
    lhs = mg.prolong(lv[0], lv[1], zc) @ rf
    rhs = zc @ mg.restrict(lv[0], lv[1], rf)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_coarse_moduli_by_hand():
    E = np.full(4 * 4 * 2, 0.7)
    for q in (1.0, 2.0, 0.5):
        assert np.allclose(mg.coarse_moduli(E, (4, 4, 2), q, 2.0), 1.4, rtol=1e-14)
    # arithmetic mean of one 2x2x2 block
    E = np.arange(1.0, 9.0)
    assert mg.coarse_moduli(E, (2, 2, 2), 1.0, 1.0)[0] == pytest.approx(4.5, rel=1e-15)
    assert mg.coarse_moduli(E, (2, 2, 2), 2.0, 1.0)[0] == pytest.approx(
        np.sqrt(np.mean(E ** 2)), rel=1e-15)
    # odd element counts: the last coarse layer has half its children
    E = np.ones(3 * 2 * 2)
    c = mg.coarse_moduli(E, (3, 2, 2), 1.0, 2.0)
    assert np.allclose(c, [2.0, 1.0], rtol=1e-15)


def test_rediscretised_operator_equals_galerkin_for_uniform_modulus():
    """Nested trilinear spaces: with a uniform modulus the coarse operator
    of modulus 2E (s = 2, any q) is exactly P^T K P."""
    nelx, nely, nelz = 6, 4, 4
    KE = fem.element_stiffness(0.3)
    K = fem.assemble(nelx, nely, nelz, np.full(nelx * nely * nelz, 0.8), KE)
    Px, Py, Pz = (mg.prolongation_1d(n + 1, n // 2 + 1) for n in (nelx, nely, nelz))
    P = sp.kron(sp.kron(sp.csr_matrix(Pz), sp.csr_matrix(Py)), sp.csr_matrix(Px))
    P = sp.kron(P, sp.identity(3)).tocsr()
    G = (P.T @ K @ P).toarray()
    Ec = mg.coarse_moduli(np.full(nelx * nely * nelz, 0.8), (nelx, nely, nelz), 1.0, 2.0)
    Kc = fem.assemble(nelx // 2, nely // 2, nelz // 2, Ec, KE).toarray()
    assert np.abs(G - Kc).max() <= 1e-12 * np.abs(Kc).max()


def _small_levels(seed=5):
    prob = problems.cantilever(12, 6, 6, load="edge")
    fixed = prob.fixed.copy()
    rng = np.random.default_rng(seed)
    fixed[rng.choice(fixed.size, 30, replace=False)] = 1
    x = problems.random_density(prob.nel, seed, 1e-3, 1.0)
    E = fem.simp_modulus(x, 3.0)
    KE = fem.element_stiffness(0.3)
    lv = mg.hierarchy(12, 6, 6, fixed)
    w, q, s = mg.split_theta(mg.default_theta(len(lv)), len(lv))
    q = q.copy()
    q[1:] = 0.7
    mg.setup(lv, E, KE, q, s)
    return lv, KE, w, fixed, E


def test_vcycle_is_symmetric_and_positive():
    lv, KE, w, fixed, _ = _small_levels()
    assert len(lv) == 3
    rng = np.random.default_rng(9)
    u = np.where(fixed, 0, rng.standard_normal(fixed.size))
    v = np.where(fixed, 0, rng.standard_normal(fixed.size))
    Vu, Vv = mg.vcycle(lv, KE, u, w, 12), mg.vcycle(lv, KE, v, w, 12)
    assert u @ Vv == pytest.approx(v @ Vu, rel=1e-12)
    assert u @ Vu > 0 and v @ Vv > 0


def test_one_level_vcycle_is_damped_jacobi():
    """A grid too small to coarsen: V = sum_{k<m} (I - w D^-1 K)^k w D^-1."""
    prob = problems.cantilever(4, 3, 2)
    lv = mg.hierarchy(4, 3, 2, prob.fixed)
    assert len(lv) == 1
    KE = fem.element_stiffness(0.3)
    E = fem.simp_modulus(problems.random_density(prob.nel, 2, 0.1, 1.0), 3.0)
    mg.setup(lv, E, KE, [1.0], [1.0])
    free = ~lv[0].fixed
    K = fem.assemble(4, 3, 2, E, KE).toarray() * np.outer(free, free)
    Dw = np.diag(mg.damping(lv[0], 0.45) * lv[0].dinv)
    T = np.eye(K.shape[0]) - Dw @ K
    V = sum(np.linalg.matrix_power(T, k) for k in range(7)) @ Dw
    b = np.where(lv[0].fixed, 0, np.random.default_rng(1).standard_normal(K.shape[0]))
    assert np.allclose(mg.vcycle(lv, KE, b, [0.45], 7), V @ b, rtol=1e-12, atol=1e-14)


def test_energy_loss_is_the_energy_norm_error():
    lv, KE, w, fixed, E = _small_levels()
    K = fem.apply_bc(fem.assemble(12, 6, 6, E, KE), fixed)
    rng = np.random.default_rng(4)
    r = np.where(fixed, 0, rng.standard_normal(fixed.size))
    e = fem.solve_direct(K, r, fixed.astype(np.uint8))
    z = mg.vcycle(lv, KE, r, w, 12)
    direct = ((e - z) @ (K @ (e - z))) / (e @ (K @ e))
    assert mg.energy_loss(K, r, e, z) == pytest.approx(direct, rel=1e-9)


def test_vcycle_preconditioner_beats_jacobi_on_a_cantilever():
    prob = problems.cantilever(24, 8, 8, load="centre", volfrac=0.2, rmin=1.5)
    x = problems.random_density(prob.nel, 8, 0.05, 1.0)
    E = fem.simp_modulus(x, 3.0)
    KE = fem.element_stiffness(0.3)
    K = fem.apply_bc(fem.assemble(24, 8, 8, E, KE), prob.fixed)
    f = fem.masked_load(prob.load, prob.fixed)
    lv = mg.hierarchy(24, 8, 8, prob.fixed)
    w, q, s = mg.split_theta(mg.default_theta(len(lv)), len(lv))
    mg.setup(lv, E, KE, q, s)

    def pcg(prec):
        u = np.zeros_like(f)
        r = f.copy()
        z = prec(r)
        p = z.copy()
        rz = r @ z
        for it in range(1, 5000):
            qv = K @ p
            a = rz / (p @ qv)
            u += a * p
            r -= a * qv
            if np.linalg.norm(r) <= 1e-8 * np.linalg.norm(f):
                return it
            z = prec(r)
            rzn = r @ z
            p = z + rzn / rz * p
            rz = rzn
        return 5000

    d = K.diagonal()
    it_j = pcg(lambda r: r / d)
    it_mg = pcg(lambda r: mg.vcycle(lv, KE, r, w, 20))
    assert it_mg * 3 < it_j, (it_mg, it_j)


def test_eigenvalue_estimate_bounds_the_smoother():
    """The eigenvalue bound the smoother uses is at least the exact
    lam_max(D^-1 K) (so the damping 2 w / lam keeps every sweep convergent)
    and not far above it, on a graded design with void elements next to
    solid ones; the l1 bound holds for any moduli."""
    prob = problems.cantilever(6, 4, 4, load="edge")
    x = problems.random_density(prob.nel, 12, 0.0, 1.0)
    x[::3] = 0.0
    E = fem.simp_modulus(x, 3.0)
    KE = fem.element_stiffness(0.3)
    lv = mg.hierarchy(6, 4, 4, prob.fixed)
    mg.setup(lv, E, KE, [1.0] * len(lv), [1.0] * len(lv))
    L = lv[0]
    free = ~L.fixed
    K = fem.assemble(6, 4, 4, E, KE).toarray()[np.ix_(free, free)]
    d = np.diag(K)
    lam = np.linalg.eigvalsh(K / np.sqrt(np.outer(d, d)))[-1]
    assert lam <= L.lam <= 1.2 * lam
    assert 0.85 * lam <= mg.rayleigh_power(L, KE) <= lam * (1 + 1e-12)
    assert lam <= mg.l1_bound(KE) and mg.l1_bound(KE) == pytest.approx(59.0 / 11.0, rel=1e-12)
