"""The learned multigrid preconditioner on the GPU against the oracle's
V-cycle (oracle/mg.py), and the solves and OC iterations it serves."""
import numpy as np
import pytest

from oracle import fem, mg, topopt
from synth import problems
from tests.gpu_helpers import lib_ctx, random_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def per_level(theta, nlev):
    """The library's 10 parameters (w_0..w_3, q_1..q_3, s_1..s_3, index
    min(level, 3)) as the oracle's per-level arrays."""
    g = [min(l, 3) for l in range(nlev)]
    w = np.array([theta[i] for i in g])
    q = np.array([1.0] + [theta[4 + i - 1] for i in g[1:]])
    s = np.array([1.0] + [theta[7 + i - 1] for i in g[1:]])
    return w, q, s


def oracle_cycle(prob, x, r, theta, sweeps=6, nu=1):
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    lv = mg.hierarchy(prob.nelx, prob.nely, prob.nelz, prob.fixed)
    w, q, s = per_level(theta, len(lv))
    mg.setup(lv, E, KE, q, s)
    return mg.vcycle(lv, KE, np.where(prob.fixed != 0, 0.0, r), w, sweeps, nu=nu), len(lv)


# the larger grids keep their finest levels on the tensor-core kernels and
# run the rest in the one-CTA bottom cycle; the small ones run wholly in it
@pytest.mark.parametrize("dims,prec,tol", [((20, 8, 6), 2, 2e-4), ((20, 8, 6), 1, 3e-2),
                                           ((33, 9, 7), 2, 2e-4), ((5, 3, 2), 2, 2e-4),
                                           ((64, 24, 16), 2, 2e-4), ((64, 24, 16), 1, 3e-2),
                                           ((96, 20, 12), 2, 2e-4)])
def test_cycle_matches_oracle(dims, prec, tol):
    from paper_2504_05604_gb300 import LMG
    prob = random_problem(*dims, seed=sum(dims))
    x = problems.random_density(prob.nel, 3, 1e-3, 1.0)
    r = problems.random_vector(prob.ndof, 4)
    ctx = lib_ctx(prob, precision=prec, precond=LMG)
    theta = ctx.mg_params()
    assert np.allclose(theta, [2.0 / 3.0] * 4 + [1.0] * 3 + [2.0] * 3)
    z = ctx.mg_apply(x, r)
    zr, nlev = oracle_cycle(prob, x, r, theta)
    assert ctx.mg_levels() == nlev
    err = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    assert err <= tol, err
    assert np.all(z[prob.fixed != 0] == 0.0)
    # non-default parameters reach every level
    th2 = np.array([0.4, 0.45, 0.55, 0.6, 0.6, 1.5, 0.8, 1.7, 2.2, 2.6])
    ctx.set_mg_params(th2)
    z2 = ctx.mg_apply(x, r)
    zr2, _ = oracle_cycle(prob, x, r, th2)
    err2 = np.linalg.norm(z2 - zr2) / np.linalg.norm(zr2)
    assert err2 <= tol, err2
    ctx.close()


def test_cycle_with_two_smoothing_sweeps_matches_oracle():
    from paper_2504_05604_gb300 import LMG
    prob = random_problem(20, 8, 6, seed=34)
    x = problems.random_density(prob.nel, 3, 1e-3, 1.0)
    r = problems.random_vector(prob.ndof, 4)
    ctx = lib_ctx(prob, precision=2, precond=LMG, mg_nu=2, mg_sweeps=9)
    z = ctx.mg_apply(x, r)
    zr, _ = oracle_cycle(prob, x, r, ctx.mg_params(), sweeps=9, nu=2)
    assert np.linalg.norm(z - zr) <= 2e-4 * np.linalg.norm(zr)
    ctx.close()


def test_parameters_out_of_range_are_refused():
    from paper_2504_05604_gb300 import LMG, To3dError
    prob = problems.cantilever(8, 4, 4)
    ctx = lib_ctx(prob, precond=LMG)
    for bad in ([1.0] + [0.5] * 3 + [1.0] * 3 + [2.0] * 3,
                [0.5] * 4 + [0.01] + [1.0] * 2 + [2.0] * 3,
                [0.5] * 4 + [1.0] * 3 + [0.0, 2.0, 2.0]):
        with pytest.raises(To3dError):
            ctx.set_mg_params(bad)
    with pytest.raises(To3dError):
        ctx.set_mg_params([0.5] * 9)
    ctx.close()


def _direct(prob, x):
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    K = fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)
    f = fem.masked_load(prob.load, prob.fixed)
    return fem.solve_direct(K, f, prob.fixed)


@pytest.mark.parametrize("prec,tol", [(0, 1e-6), (1, 1e-5), (2, 1e-5)])
def test_solve_with_multigrid_matches_direct(prec, tol):
    from paper_2504_05604_gb300 import LMG
    prob = problems.cantilever(40, 12, 10, load="centre", volfrac=0.3)
    x = problems.random_density(prob.nel, 11, 1e-3, 1.0)
    u_ref = _direct(prob, x)
    ctx = lib_ctx(prob, precision=prec, precond=LMG, inner_rtol=0.01)
    u, info = ctx.solve(x)
    assert info["status"] == 0 and info["relres"] <= 1.5e-8
    assert np.linalg.norm(u - u_ref) <= tol * np.linalg.norm(u_ref)
    jac = lib_ctx(prob, precision=0)
    _, ij = jac.solve(x)
    print(f"precision {prec}: multigrid {info['iters']} iterations, Jacobi-PCG {ij['iters']}")
    assert info["iters"] * 4 < ij["iters"]
    ctx.close()
    jac.close()


@pytest.mark.parametrize("prec,kw", [(0, {}), (1, {}),
                                     (1, dict(inner_rtol=0.05, mg_keep_dir=1, fp64_tc=1))])
def test_oc_trajectory_with_multigrid_matches_oracle(prec, kw):
    """The last case is the benchmark's form: kept inner direction, inner
    tolerance 0.05, FP64 residuals on the sliced tensor-core K u."""
    from paper_2504_05604_gb300 import LMG
    prob = problems.cantilever(30, 10, 4, load="edge", volfrac=0.3, rmin=1.5)
    iters = 6
    x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct")
    ctx = lib_ctx(prob, precision=prec, precond=LMG, **{"inner_rtol": 0.01, **kw})
    recs = ctx.run(iters)
    for r, h in zip(recs, hist):
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
        assert r["halvings"] == h.halvings
    assert np.abs(ctx.density() - x_ref).max() <= 1e-4
    ctx.close()


def test_training_lowers_the_loss_and_the_iterations_on_a_new_design():
    """Learned on residuals of one design, applied to another of the same
    family: the mean energy loss falls, and the solve on the held-out design
    needs no more iterations than with the initial parameters (and far fewer
    than Jacobi-PCG)."""
    from paper_2504_05604_gb300 import LMG
    prob = problems.cantilever(48, 16, 8, load="centre", volfrac=0.2, rmin=2.5)
    ctx = lib_ctx(prob, precision=0, precond=LMG)
    for _ in range(4):
        ctx.step()
    ctx.mg_train(nsnap=4, steps=0, lr=0.1, seed=1)
    for _ in range(2):
        ctx.step()
    first, last = ctx.mg_train(nsnap=4, steps=15, lr=0.1, seed=1, append=True)
    print(f"training loss {first:.4f} -> {last:.4f}; theta {np.round(ctx.mg_params(), 3)}")
    assert last < first
    theta = ctx.mg_params()
    for _ in range(6):
        ctx.step()
    x_new = ctx.density()
    ctx.close()
    its = {}
    for name, th in (("init", None), ("trained", theta)):
        c = lib_ctx(prob, precision=0, precond=LMG)
        if th is not None:
            c.set_mg_params(th)
        u, info = c.solve(x_new)
        assert info["status"] == 0 and info["relres"] <= 1.5e-8
        its[name] = info["iters"]
        c.close()
    jac = lib_ctx(prob, precision=0)
    _, ij = jac.solve(x_new)
    jac.close()
    print(f"held-out design: init {its['init']}, trained {its['trained']}, Jacobi {ij['iters']}")
    assert its["trained"] <= its["init"]
    assert its["trained"] * 3 < ij["iters"]
