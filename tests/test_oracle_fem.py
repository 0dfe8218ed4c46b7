"""Pins of the CPU oracle's finite element part against mathematics.

Nothing here compares the oracle with itself: each check is a closed form of
linear elasticity, an invariant of the discretisation, or brute force.
"""
import numpy as np
import pytest

from oracle import fem
from synth import problems

NU = 0.3
LAM = NU / ((1 + NU) * (1 - 2 * NU))     # 15/26 for nu = 0.3
MU = 1 / (2 * (1 + NU))                  # 5/13


def corner_xyz():
    return np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], float)


def nodal(field):
    """Element dof vector (3n + c) sampled from a displacement field."""
    X = corner_xyz()
    return np.concatenate([field(*X[n]) for n in range(8)])


def test_ke_integer_structure_and_spectrum():
    # For E = 1, nu = 0.3 the hex8 stiffness is (5/1872) times an integer
    # matrix with diagonal 88 and spectrum {0^6, 24^2, 44^3, 72^3, 96, 144^8, 468}.
    KE = fem.element_stiffness(NU)
    Kint = KE * 1872 / 5
    assert np.allclose(Kint, np.round(Kint), atol=1e-10)
    Kint = np.round(Kint)
    assert np.array_equal(Kint, Kint.T)
    assert np.all(np.diag(Kint) == 88)
    assert np.all(Kint.sum(axis=1) == 0)
    ev = np.sort(np.linalg.eigvalsh(Kint))
    expect = np.array([0] * 6 + [24] * 2 + [44] * 3 + [72] * 3 + [96] + [144] * 8 + [468], float)
    assert np.allclose(ev, expect, atol=1e-9)
    assert np.isclose(np.trace(Kint), 2112)


def test_ke_rigid_body_null_space():
    KE = fem.element_stiffness(NU)
    modes = [lambda x, y, z: np.array([1.0, 0, 0]),
             lambda x, y, z: np.array([0, 1.0, 0]),
             lambda x, y, z: np.array([0, 0, 1.0]),
             lambda x, y, z: np.array([-y, x, 0.0]),
             lambda x, y, z: np.array([0.0, -z, y]),
             lambda x, y, z: np.array([z, 0.0, -x])]
    R = np.stack([nodal(m) for m in modes], axis=1)
    assert np.linalg.matrix_rank(R) == 6
    assert np.abs(KE @ R).max() < 1e-14


@pytest.mark.parametrize("field,energy", [
    (lambda x, y, z: np.array([x, 0, 0]), LAM + 2 * MU),          # eps_xx = 1
    (lambda x, y, z: np.array([y, 0, 0]), MU),                     # gamma_xy = 1
    (lambda x, y, z: np.array([0, z, 0]), MU),                     # gamma_yz = 1
    (lambda x, y, z: np.array([y, x, 0]), 4 * MU),                 # gamma_xy = 2
    (lambda x, y, z: np.array([x, y, z]), 9 * LAM + 6 * MU),       # eps = I
    (lambda x, y, z: np.array([x, -y, 0]), 4 * MU),                # eps_xx = 1, eps_yy = -1
])
def test_ke_uniform_strain_energies(field, energy):
    # For a uniform strain, u^T KE u = int eps : C : eps dV over the unit cube
    # = lam (tr eps)^2 + 2 mu eps:eps (tensor strains).
    KE = fem.element_stiffness(NU)
    u = nodal(field)
    assert np.isclose(u @ KE @ u, energy, rtol=1e-14)


def test_ke_lame_split_is_integer():
    # KE = (lam/72) A_lam + (mu/72) A_mu with integer A_lam (|.| <= 8) and A_mu (|.| <= 32).
    K1 = fem.element_stiffness(0.0, E=1.0)           # nu = 0: lam = 0, mu = 1/2
    A_mu = K1 / (0.5 / 72)
    assert np.allclose(A_mu, np.round(A_mu), atol=1e-10)
    assert np.abs(A_mu).max() == pytest.approx(32)
    KE = fem.element_stiffness(NU)
    A_lam = (KE - MU / 72 * A_mu) / (LAM / 72)
    assert np.allclose(A_lam, np.round(A_lam), atol=1e-10)
    assert np.abs(A_lam).max() == pytest.approx(8)


def test_assembly_symmetric_and_rigid_modes():
    nelx, nely, nelz = 3, 2, 2
    KE = fem.element_stiffness(NU)
    E = problems.random_density(nelx * nely * nelz, 1)
    K = fem.assemble(nelx, nely, nelz, E, KE)
    assert abs(K - K.T).max() < 1e-14
    N = (nelx + 1) * (nely + 1) * (nelz + 1)
    k, j, i = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(float)
    for rot in ([1, 0, 0], [0, 1, 0], [0, 0, 1]):
        u = np.cross(np.array(rot, float)[None, :], X).ravel()
        assert np.abs(K @ u).max() < 1e-13
    assert np.abs(K @ np.tile([1.0, 2.0, 3.0], N)).max() < 1e-13


def test_elementwise_matvec_equals_assembled_operator():
    nelx, nely, nelz = 4, 3, 2
    prob = problems.cantilever(nelx, nely, nelz)
    KE = fem.element_stiffness(NU)
    E = fem.simp_modulus(problems.random_density(prob.nel, 2), 3.0)
    K = fem.apply_bc(fem.assemble(nelx, nely, nelz, E, KE), prob.fixed)
    p = problems.random_vector(prob.ndof, 3)
    y1 = K @ p
    y2 = fem.matvec_elementwise(nelx, nely, nelz, E, KE, p, prob.fixed)
    assert np.abs(y1 - y2).max() <= 1e-14 * np.abs(y1).max()
    # clamped rows are identity rows
    fx = prob.fixed != 0
    assert np.array_equal(y2[fx], p[fx])


def test_patch_test_linear_field_reproduced():
    # Impose a general linear displacement on the boundary of a 3x3x3 mesh of
    # homogeneous material; the interior nodes must reproduce it exactly.
    n = 3
    KE = fem.element_stiffness(NU)
    E = np.full(n ** 3, 0.8)
    K = fem.assemble(n, n, n, E, KE).tocsr()
    k, j, i = np.meshgrid(*(np.arange(n + 1),) * 3, indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(float)
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.25]])
    b = np.array([0.1, -0.2, 0.3])
    u_exact = (X @ A.T + b).ravel()
    interior = ((X > 0) & (X < n)).all(1)
    idof = np.flatnonzero(np.repeat(interior, 3))
    bdof = np.flatnonzero(~np.repeat(interior, 3))
    Kii = K[idof][:, idof].toarray()
    Kib = K[idof][:, bdof].toarray()
    ui = np.linalg.solve(Kii, -Kib @ u_exact[bdof])
    assert np.abs(ui - u_exact[idof]).max() < 1e-12


def test_uniaxial_bar_closed_form():
    # Bar on symmetry planes (u_x = 0 on x = 0, u_y = 0 on y = 0, u_z = 0 on
    # z = 0), unit tension on x = L with consistent nodal forces.  Exact
    # solution: u = (x, -nu y, -nu z) / E.  Exercises the clamped-dof mask and
    # load vector conventions of the C interface.
    nelx, nely, nelz = 5, 2, 3
    N = (nelx + 1) * (nely + 1) * (nelz + 1)
    k, j, i = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    fixed = np.zeros(3 * N, np.uint8)
    fixed[3 * np.flatnonzero(i == 0) + 0] = 1
    fixed[3 * np.flatnonzero(j == 0) + 1] = 1
    fixed[3 * np.flatnonzero(k == 0) + 2] = 1
    f = np.zeros(3 * N)
    wy = np.where((j == 0) | (j == nely), 0.5, 1.0)
    wz = np.where((k == 0) | (k == nelz), 0.5, 1.0)
    face = i == nelx
    f[3 * np.flatnonzero(face)] = (wy * wz)[face]
    Eval = 0.7
    E = np.full(nelx * nely * nelz, Eval)
    KE = fem.element_stiffness(NU)
    K = fem.apply_bc(fem.assemble(nelx, nely, nelz, E, KE), fixed)
    u = fem.solve_direct(K, f, fixed)
    exact = np.stack([i, -NU * j, -NU * k], 1).ravel() / Eval
    assert np.abs(u - exact).max() < 1e-12


def test_dense_direct_pcg_agree_and_energy_identity():
    prob = problems.cantilever(4, 3, 2, load="edge")
    KE = fem.element_stiffness(NU)
    x = problems.random_density(prob.nel, 5, 0.1, 1.0)
    E = fem.simp_modulus(x, 3.0)
    K = fem.apply_bc(fem.assemble(4, 3, 2, E, KE), prob.fixed)
    f = fem.masked_load(prob.load, prob.fixed)
    u_dense = fem.solve_dense(K, f, prob.fixed)
    u_direct = fem.solve_direct(K, f, prob.fixed)
    u_pcg, its, res = fem.jacobi_pcg(lambda v: K @ v, K.diagonal(), f, rtol=1e-13)
    scale = np.abs(u_dense).max()
    assert np.abs(u_direct - u_dense).max() < 1e-11 * scale
    assert np.abs(u_pcg - u_dense).max() < 1e-9 * scale
    assert res <= 1e-13 and its > 0
    ce = fem.element_energies(4, 3, 2, KE, u_dense)
    c, _ = fem.compliance_and_sensitivity(x, ce, 3.0)
    assert np.isclose(f @ u_dense, c, rtol=1e-12)


def test_jacobi_diagonal_matches_operator():
    prob = problems.cantilever(3, 2, 2)
    KE = fem.element_stiffness(NU)
    E = fem.simp_modulus(problems.random_density(prob.nel, 6), 3.0)
    K = fem.apply_bc(fem.assemble(3, 2, 2, E, KE), prob.fixed)
    d = fem.jacobi_diagonal(3, 2, 2, E, KE, prob.fixed)
    assert np.allclose(d, K.diagonal(), rtol=1e-15, atol=0)
    # every KE diagonal entry equals 88 * 5 / 1872
    assert np.allclose(np.diag(KE), 88 * 5 / 1872, rtol=1e-14)


def test_uniform_density_scaling():
    prob = problems.cantilever(4, 2, 2)
    KE = fem.element_stiffness(NU)
    f = fem.masked_load(prob.load, prob.fixed)
    us = []
    for x0 in (1.0, 0.3):
        E = fem.simp_modulus(np.full(prob.nel, x0), 3.0)
        K = fem.apply_bc(fem.assemble(4, 2, 2, E, KE), prob.fixed)
        us.append(fem.solve_direct(K, f, prob.fixed) * E[0])
    assert np.abs(us[0] - us[1]).max() < 1e-11 * np.abs(us[0]).max()


def test_sensitivity_matches_finite_difference():
    prob = problems.cantilever(4, 2, 2)
    KE = fem.element_stiffness(NU)
    f = fem.masked_load(prob.load, prob.fixed)
    x = problems.random_density(prob.nel, 7, 0.3, 0.9)

    def comp(xv):
        E = fem.simp_modulus(xv, 3.0)
        K = fem.apply_bc(fem.assemble(4, 2, 2, E, KE), prob.fixed)
        u = fem.solve_direct(K, f, prob.fixed)
        ce = fem.element_energies(4, 2, 2, KE, u)
        return fem.compliance_and_sensitivity(xv, ce, 3.0)

    _, dc = comp(x)
    h = 1e-6
    for e in (0, 5, prob.nel - 1):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        fd = (comp(xp)[0] - comp(xm)[0]) / (2 * h)
        assert np.isclose(fd, dc[e], rtol=1e-6)


def test_matvec_rows_equal_the_element_sum():
    """The row-by-row form (used at sizes too large to assemble) agrees with
    the vectorised element sum and the assembled operator."""
    from synth import problems
    nelx, nely, nelz = 5, 4, 3
    prob = problems.cantilever(nelx, nely, nelz)
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.uniform(0.01, 1.0, prob.nel)
    p = rng.standard_normal(prob.ndof)
    KE = fem.element_stiffness(0.3)
    E = fem.simp_modulus(x, 3.0)
    y = fem.matvec_elementwise(nelx, nely, nelz, E, KE, p, prob.fixed)
    Kb = fem.apply_bc(fem.assemble(nelx, nely, nelz, E, KE), prob.fixed)
    rows = rng.choice(prob.ndof, 60, replace=False)
    yr = fem.matvec_rows(nelx, nely, nelz, E, KE, p, prob.fixed, rows)
    assert np.allclose(yr, y[rows], rtol=1e-12, atol=1e-12)
    assert np.allclose(yr, (Kb @ p)[rows], rtol=1e-12, atol=1e-12)
    ab = fem.matvec_rows(nelx, nely, nelz, E, KE, p, prob.fixed, rows, absolute=True)
    assert np.all(ab >= np.abs(yr) - 1e-12)
