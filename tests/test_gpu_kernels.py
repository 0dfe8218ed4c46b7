"""GPU parity of each step of the path against the CPU oracle (C interface).

Tolerances: FP64 kernels 1e-13 relative (matvec; only summation order
differs), 1e-12 (energies, filter); the low-precision matvec is compared
with an FP64 emulation of its operand rounding to 1e-5 of sum|K||p| (FP32
accumulation), and with the exact operator to the 16-bit format's unit
roundoff; solves to 1e-6 (FP64) and 1e-5 (defect correction) relative.
"""
import numpy as np
import pytest

from oracle import fem, filters, oc
from synth import problems
from tests.gpu_helpers import emulate_lowp, lib_ctx, random_problem

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (3, 2, 2), (16, 8, 8), (31, 9, 8), (33, 5, 3), (60, 20, 4), (20, 6, 45)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def oracle_operator(prob, x):
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    return fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz, E, KE), prob.fixed)


@pytest.mark.parametrize("dims", SIZES)
def test_matvec64_matches_assembled_operator(dims):
    prob = random_problem(*dims, seed=sum(dims))
    x = problems.random_density(prob.nel, 1, 0.0, 1.0)
    p = problems.random_vector(prob.ndof, 2)
    K = oracle_operator(prob, x)
    y_ref = K @ p
    ctx = lib_ctx(prob)
    y = ctx.matvec(x, p)
    scale = np.abs(K) @ np.abs(p)
    assert np.all(np.abs(y - y_ref) <= 1e-13 * scale + 1e-300)
    fx = prob.fixed != 0
    assert np.array_equal(y[fx], p[fx])


def test_matvec64_device_pointers():
    import torch
    prob = random_problem(20, 7, 5, seed=3)
    x = problems.random_density(prob.nel, 4)
    p = problems.random_vector(prob.ndof, 5)
    ctx = lib_ctx(prob)
    xd = torch.tensor(x, device="cuda")
    pd = torch.tensor(p, device="cuda")
    yd = torch.empty_like(pd)
    ctx.matvec(xd, pd, yd)
    torch.cuda.synchronize()
    y = ctx.matvec(x, p)
    assert np.array_equal(yd.cpu().numpy(), y)


@pytest.mark.parametrize("nu", [0.3, 0.33])
@pytest.mark.parametrize("prec,tol_exact", [(1, 2.0 ** -8), (2, 2.0 ** -16), (3, 2.0 ** -10),
                                             (4, 2.0 ** -20)])
@pytest.mark.parametrize("dims", SIZES)
def test_matvec_tensor_core(dims, prec, tol_exact, nu):
    # nu = 0.3 uses one combined integer B (3 A_lam + 2 A_mu); nu = 0.33 has
    # no small rational lam/mu and exercises the split B = [A_lam; A_mu]
    prob = random_problem(*dims, seed=7 + sum(dims))
    prob.nu = nu
    x = problems.random_density(prob.nel, 8, 0.0, 1.0)
    p32 = problems.random_vector(prob.ndof, 9).astype(np.float32)
    ctx = lib_ctx(prob, nu=nu)
    y = ctx.matvec_lowp(x, p32, prec).astype(np.float64)
    y_emul, bound = emulate_lowp(prob, x, p32, prec)
    free = prob.fixed == 0
    err = np.abs(y - y_emul)[free]
    assert np.all(err <= 1e-5 * bound[free] + 1e-30), err.max()
    K = oracle_operator(prob, x)
    y_exact = K @ p32.astype(np.float64)
    assert np.all(np.abs(y - y_exact)[free] <= tol_exact * bound[free] + 1e-30)
    fx = ~free
    assert np.array_equal(y[fx].astype(np.float32), p32[fx])


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4])
def test_solve_matches_direct(precision):
    prob = random_problem(24, 8, 4, seed=11, partial_clamp=False)
    x = problems.random_density(prob.nel, 12, 0.1, 1.0)
    x[prob.passive == 1] = 0.0
    x[prob.passive == 2] = 1.0
    K = oracle_operator(prob, x)
    f = fem.masked_load(prob.load, prob.fixed)
    u_ref = fem.solve_direct(K, f, prob.fixed)
    ctx = lib_ctx(prob, precision=precision, warm_start=0)
    u, info = ctx.solve(x)
    assert info["status"] == 0 and info["relres"] <= 1e-8
    res = np.linalg.norm(f - K @ u) / np.linalg.norm(f)
    assert res <= 1.5e-8
    tol = 1e-6 if precision == 0 else 1e-5
    assert np.abs(u - u_ref).max() <= tol * np.abs(u_ref).max()


@pytest.mark.parametrize("fp64_tc", [0, 1])
@pytest.mark.parametrize("dims", SIZES)
def test_sensitivity(dims, fp64_tc):
    """FP64 CUDA-core energies, and (fp64_tc) energies on the tensor cores by
    exact slicing of u_e."""
    prob = random_problem(*dims, seed=21 + sum(dims))
    x = problems.random_density(prob.nel, 22, 0.0, 1.0)
    u = problems.random_vector(prob.ndof, 23)
    KE = fem.element_stiffness(prob.nu)
    ce_ref = fem.element_energies(prob.nelx, prob.nely, prob.nelz, KE, u)
    c_ref, dc_ref = fem.compliance_and_sensitivity(x, ce_ref, prob.penal)
    ctx = lib_ctx(prob, fp64_tc=fp64_tc)
    ce, dc, c = ctx.sensitivity(x, u)
    assert np.allclose(ce, ce_ref, rtol=1e-12, atol=1e-12 * np.abs(ce_ref).max())
    assert np.allclose(dc, dc_ref, rtol=1e-12, atol=1e-12 * np.abs(dc_ref).max())
    assert c == pytest.approx(c_ref, rel=1e-12)


@pytest.mark.parametrize("rmin", [1.5, 2.5, 4.0])
@pytest.mark.parametrize("dims", [(1, 1, 1), (7, 5, 3), (33, 9, 8), (60, 20, 4)])
def test_filter(dims, rmin):
    prob = random_problem(*dims, seed=31, rmin=rmin)
    x = problems.random_density(prob.nel, 32, 0.0, 1.0)
    dc = -problems.random_density(prob.nel, 33, 0.0, 5.0)
    H = filters.filter_matrix(*dims, rmin)
    Hs = filters.row_sums(H)
    ctx = lib_ctx(prob)
    got = ctx.filter(dc, x=x)
    ref = filters.sensitivity_filter(H, Hs, x, dc)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    got = ctx.filter(x, kind=1)
    assert np.allclose(got, filters.density_filter(H, Hs, x), rtol=1e-12)
    got = ctx.filter(dc, kind=1, transpose=True)
    assert np.allclose(got, filters.density_filter_chain(H, Hs, dc), rtol=1e-12,
                       atol=1e-12 * np.abs(dc).max())


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("tol", [1e-3, 1e-9])
def test_oc_update(levels, tol):
    prob = random_problem(40, 12, 6, seed=41, partial_clamp=False)
    x = problems.random_density(prob.nel, 42, 0.0, 1.0)
    x[prob.passive == 1] = 0.0
    x[prob.passive == 2] = 1.0
    dc = -problems.random_density(prob.nel, 43, 1e-3, 10.0)
    ctx = lib_ctx(prob, oc_levels=levels, bisect_tol=tol)
    xn, lam, vol, nh = ctx.oc_update(x, dc)
    xr, lam_r, nh_r, vol_r = oc.oc_update(x, dc, prob.volfrac, prob.passive, prob.move, tol)
    assert nh == nh_r
    assert lam == pytest.approx(lam_r, rel=1e-14)
    assert np.abs(xn - xr).max() <= 1e-14
    assert vol == pytest.approx(vol_r, rel=1e-13)
    assert np.all(xn[prob.passive == 1] == 0) and np.all(xn[prob.passive == 2] == 1)


@pytest.mark.parametrize("precision", [1, 3])
def test_single_slice_forms_converge_on_void_riddled_problems(precision):
    """The single-slice operands on the small uneven cantilevers with
    spherical voids: every solve reaches the FP64 tolerance (escalating to
    two slices where the single slice stalls), and the first OC iteration's
    compliance matches the FP64 form's."""
    probs = problems.config_batched(64)[:12]
    for pr in probs:
        ref = lib_ctx(pr).step()
        r = lib_ctx(pr, precision=precision).step()
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert r["compliance"] == pytest.approx(ref["compliance"], rel=1e-6)
