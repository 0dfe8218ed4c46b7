"""FP64-accurate K p on the tensor cores by exact integer slicing (the
operator of Section 2.2) against the oracle's assembled FP64 operator, the
CUDA-core FP64 kernel, and in whole solves."""
import numpy as np
import pytest

from oracle import fem
from synth import problems
from tests.gpu_helpers import lib_ctx, random_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _reference(prob, x, p):
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
    Kabs = abs(fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, np.abs(KE)),
                            prob.fixed))
    return K @ p, Kabs @ np.abs(p)


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 2, 2), (16, 8, 8), (31, 9, 8), (33, 5, 3),
                                  (20, 6, 45), (60, 20, 4)])
def test_sliced_matvec_matches_assembled_operator(dims):
    prob = random_problem(*dims, seed=7 + sum(dims))
    x = problems.random_density(prob.nel, 1, 1e-3, 1.0)
    p = problems.random_vector(prob.ndof, 2)
    ref, ab = _reference(prob, x, p)
    ctx = lib_ctx(prob, fp64_tc=1)
    y = ctx.matvec(x, p)
    err = np.abs(y - ref)
    assert np.all(err <= 1e-13 * ab + 1e-300), (err / np.maximum(ab, 1e-300)).max()
    ctx64 = lib_ctx(prob, fp64_tc=0)
    y64 = ctx64.matvec(x, p)
    # as accurate as the CUDA-core FP64 kernel: both within a few units of
    # FP64 rounding of the sum of |terms|
    assert np.all(np.abs(y - y64) <= 1e-14 * ab + 1e-300)
    print(dims, "max |y - ref| / sum|terms|:", (err / np.maximum(ab, 1e-300)).max(),
          "CUDA-core kernel:", (np.abs(y64 - ref) / np.maximum(ab, 1e-300)).max())
    ctx.close()
    ctx64.close()


def test_sliced_matvec_over_a_wide_dynamic_range():
    """Entries from 1e-200 to 1e12, exact zeros and subnormal numbers in one
    vector: each element is scaled by its own largest entry."""
    prob = random_problem(14, 7, 5, seed=11)
    x = problems.random_density(prob.nel, 3, 1e-3, 1.0)
    rng = np.random.Generator(np.random.PCG64(12))
    p = rng.standard_normal(prob.ndof) * 10.0 ** rng.uniform(-200, 12, prob.ndof)
    p[rng.choice(prob.ndof, 40, replace=False)] = 0.0
    p[rng.choice(prob.ndof, 10, replace=False)] = 5e-320
    ref, ab = _reference(prob, x, p)
    ctx = lib_ctx(prob, fp64_tc=1)
    y = ctx.matvec(x, p)
    assert np.all(np.abs(y - ref) <= 1e-13 * ab + 1e-300)
    ctx.close()


@pytest.mark.parametrize("precision,precond", [(0, 0), (1, 0), (1, 2), (0, 2)])
def test_solves_with_the_sliced_matvec(precision, precond):
    """FP64 Jacobi-PCG, the defect correction's FP64 residuals and flexible
    CG with the sliced operator: the direct solution, and the FP64 form's
    iteration count within 2 % of the CUDA-core kernel's."""
    prob = problems.cantilever(40, 12, 10, load="centre", volfrac=0.3)
    x = problems.random_density(prob.nel, 11, 1e-3, 1.0)
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal)
    K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
    u_ref = fem.solve_direct(K, fem.masked_load(prob.load, prob.fixed), prob.fixed)
    its = {}
    for tc in (1, 0):
        ctx = lib_ctx(prob, precision=precision, precond=precond, fp64_tc=tc, inner_rtol=0.01)
        u, info = ctx.solve(x)
        assert info["status"] == 0 and info["relres"] <= 1.5e-8
        assert np.linalg.norm(u - u_ref) <= 1e-5 * np.linalg.norm(u_ref)
        its[tc] = info["iters"]
        ctx.close()
    if precision == 0 and precond == 0:
        assert abs(its[1] - its[0]) <= 0.02 * its[0] + 2, its
