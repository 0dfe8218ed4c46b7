"""Parity at the benchmark's full size, 480x160x80, in the launch
configuration the benchmark times: sampled outputs that the oracle computes
one by one, and properties that hold at any size."""
import numpy as np
import pytest

from oracle import fem
from synth import problems
from tests.gpu_helpers import lib_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def big():
    return problems.config_large()


def sampled_rows(prob, n, seed):
    """Random dofs plus the ones at the edges of the kernels' tiles and of
    the domain: the corners, the clamped face, the load node, node columns
    15/16 and rows 7/8 (tile seams), the top layer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = prob.nelx + 1, prob.nely + 1, prob.nelz + 1
    nodes = list(rng.choice(prob.nnode, n, replace=False))
    for (i, j, k) in [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny // 2, nz // 2),
                      (nx - 1, ny // 2, nz // 2), (15, 7, 3), (16, 8, 4), (30, 14, nz - 1),
                      (nx - 1, 0, 0), (0, ny - 1, nz - 1), (465, 154, 40)]:
        nodes.append(i + nx * (j + ny * k))
    return np.array([3 * nd + c for nd in nodes for c in range(3)])


def test_full_size_matvecs_on_sampled_rows(big):
    prob = big
    x = problems.random_density(prob.nel, 61, 1e-3, 1.0)
    p = problems.random_vector(prob.ndof, 62)
    p32 = p.astype(np.float32)
    ctx = lib_ctx(prob)
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    rows = sampled_rows(prob, 120, 63)
    args = (prob.nelx, prob.nely, prob.nelz, E, KE)
    y64 = ctx.matvec(x, p)
    ref = fem.matvec_rows(*args, p, prob.fixed, rows)
    ab = fem.matvec_rows(*args, p, prob.fixed, rows, absolute=True)
    assert np.all(np.abs(y64[rows] - ref) <= 1e-13 * ab + 1e-300)
    p64 = p32.astype(np.float64)
    ref32 = fem.matvec_rows(*args, p64, prob.fixed, rows)
    ab32 = fem.matvec_rows(*args, p64, prob.fixed, rows, absolute=True)
    for prec, tol in [(1, 2.0 ** -8), (2, 2.0 ** -16)]:
        y = ctx.matvec_lowp(x, p32, prec).astype(np.float64)
        assert np.all(np.abs(y[rows] - ref32) <= tol * ab32 + 1e-30), prec
    ctx.close()


@pytest.mark.parametrize("form", ["jacobi", "lmg"])
def test_full_size_oc_iteration_properties(big, form):
    """One OC iteration from x0 in the BF16 defect-correction form with the
    Jacobi preconditioner and in the benchmark's form (learned multigrid,
    kept inner direction, inner tolerance 0.05, FP64 residuals on the sliced
    tensor-core K u): true FP64 residual at most 1e-8 (the library's own and
    the oracle's recomputation), volume on target to the bisection
    tolerance, the energy identity f^T u = sum E_e ce_e, and
    ce_e = u_e^T KE u_e on sampled elements of the library's own
    displacement."""
    from paper_2504_05604_gb300 import BF16_DC, LMG
    prob = big
    if form == "lmg":
        ctx = lib_ctx(prob, precision=BF16_DC, precond=LMG, inner_rtol=0.05, mg_keep_dir=1, fp64_tc=1)
    else:
        ctx = lib_ctx(prob, precision=BF16_DC)
    rec = ctx.step()
    assert rec["status"] == 0 and rec["relres"] <= 1e-8
    assert abs(rec["volume"] / prob.volfrac - 1.0) <= 1e-3
    u = ctx.displacement()
    f = fem.masked_load(prob.load, prob.fixed)
    x0 = prob.initial_density()
    fu = float(f @ u)
    # the true residual recomputed with the oracle's operator (element sum,
    # FP64): the two evaluations of f - K u differ only by rounding
    KE = fem.element_stiffness(prob.nu)
    E0 = fem.simp_modulus(x0, prob.penal, prob.E0, prob.Emin)
    Ku = fem.matvec_elementwise(prob.nelx, prob.nely, prob.nelz, E0, KE, u, prob.fixed)
    relres = np.linalg.norm(f - Ku) / np.linalg.norm(f)
    assert relres <= 1.01e-8, relres
    del Ku
    ce, dc, c = ctx.sensitivity(x0, u)
    assert c == pytest.approx(fu, rel=1e-6)
    assert rec["compliance"] == pytest.approx(c, rel=1e-12)
    rng = np.random.Generator(np.random.PCG64(64))
    els = np.concatenate([rng.choice(prob.nel, 200, replace=False), [0, prob.nel - 1]])
    nx, ny = prob.nelx + 1, prob.nely + 1
    i, j, k = els % prob.nelx, (els // prob.nelx) % prob.nely, els // (prob.nelx * prob.nely)
    corner = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]   # local node a + 2b + 4c
    ed = np.stack([3 * ((i + a) + nx * ((j + b) + ny * (k + c))) + comp
                   for (a, b, c) in corner for comp in range(3)], axis=1)
    ce_ref = np.einsum("ei,ij,ej->e", u[ed], KE, u[ed])
    # the physical u is smooth: u_e^T KE u_e cancels heavily (rigid parts),
    # so rounding is bounded by the sum of |terms|, not by ce itself
    ab = np.einsum("ei,ij,ej->e", np.abs(u[ed]), np.abs(KE), np.abs(u[ed]))
    assert np.all(np.abs(ce[els] - ce_ref) <= 1e-13 * ab + 1e-300)
    ctx.close()
