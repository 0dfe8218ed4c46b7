"""Learned preconditioner on the GPU against the oracle (C interface).

Tolerances.  A convolution multiplies BF16 operands exactly and accumulates
K = 27 C_in products in FP32: its error is a few units of 2^-24 times
sqrt(K) times sum |w||x|; 3e-5 of that sum bounds it with a wide margin.
The data gradient rounds the upstream gradient to BF16 first (the oracle
does the same).  The whole network stores every activation in BF16
(relative rounding 2^-9 per layer, 15 layers).  Against an FP64 emulation
of exactly those rounding points (the oracle's pieces plus BF16 rounding)
the output agrees to relative L2 <= 1e-2.  Gradients decorrelate from any
emulation once one rounding flips upstream (every later rounding then sees
a different operand), so they are compared with the plain FP64 oracle: the
BF16 rounding alone moves the deep layers' gradients by up to ~13 % (an
FP64 emulation of the rounding points shows cosine ~0.993 on the CPU), and
the bound is a cosine >= 0.98 and relative L2 <= 0.25.  Pass-through
networks carry the residual through exactly up to the BF16 rounding of the
network input (2^-8 relative, allowing for the FP32 step before it).
"""
import numpy as np
import pytest

from oracle import cnn, fem
from synth import problems
from tests.gpu_helpers import bf16_network, lib_ctx, random_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


# ---------------------------------------------------------------- helpers


def gpu_shape(name, co, ci):
    return (16 if name == "out" else co), (16 if name == "e0a" else ci)


def to_flat(params):
    """Oracle parameters -> the library's flat FP32 vector (per layer
    weights [27][C_out][C_in], tap = 9 dz + 3 dy + dx, then bias)."""
    out = []
    for name, co, ci in cnn.layer_shapes():
        cog, cig = gpu_shape(name, co, ci)
        w = np.zeros((27, cog, cig), np.float32)
        w[:, :co, :ci] = params[name + ".w"].transpose(2, 3, 4, 0, 1).reshape(27, co, ci)
        b = np.zeros(cog, np.float32)
        b[:co] = params[name + ".b"]
        out += [w.ravel(), b]
    return np.concatenate(out)


def from_flat(flat):
    params, off = {}, 0
    for name, co, ci in cnn.layer_shapes():
        cog, cig = gpu_shape(name, co, ci)
        w = flat[off:off + 27 * cog * cig].reshape(27, cog, cig)[:, :co, :ci]
        off += 27 * cog * cig
        params[name + ".w"] = w.reshape(3, 3, 3, co, ci).transpose(3, 4, 0, 1, 2).astype(np.float64)
        params[name + ".b"] = flat[off:off + co].astype(np.float64)
        off += cog
    assert off == flat.size
    return params


def bf16_params(params):
    """The oracle parameters rounded to what the GPU multiplies with (BF16
    weights, FP32 biases)."""
    import torch
    return {k: (torch.tensor(v).bfloat16().double().numpy() if k.endswith(".w")
                else v.astype(np.float32).astype(np.float64)) for k, v in params.items()}


def random_params(seed):
    p = cnn.init_params(seed)
    r = np.random.Generator(np.random.PCG64(seed + 1))
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * r.standard_normal(p[k].shape)
    return p


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cosine(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


def cl_to_cf(t):
    """channels-last torch tensor [Z,Y,X,C] -> FP64 numpy [C,Z,Y,X]."""
    return t.float().cpu().numpy().astype(np.float64).transpose(3, 0, 1, 2)


def w_to_oracle(W):
    """[27, Cout, Cin] torch -> [Cout, Cin, 3, 3, 3] FP64 numpy."""
    w = W.float().cpu().numpy().astype(np.float64)
    return w.reshape(3, 3, 3, w.shape[1], w.shape[2]).transpose(3, 4, 0, 1, 2)


# ---------------------------------------------------------- convolutions


@pytest.mark.parametrize("Z,Y,X,C1,C2,Cout,relu", [
    (5, 6, 7, 16, 0, 16, False),      # 210 voxels: ragged last warp tile
    (4, 4, 9, 16, 16, 48, True),      # concatenated input
    (3, 5, 4, 32, 0, 8, False),
    (2, 3, 5, 64, 64, 128, True),
    (1, 1, 1, 16, 0, 16, False),      # single voxel: only the centre tap
])
def test_conv_forward_matches_oracle(Z, Y, X, C1, C2, Cout, relu):
    import torch
    from paper_2504_05604_gb300 import conv3d_forward
    g = torch.Generator(device="cuda").manual_seed(Z * 100 + Cout)
    in1 = torch.randn(Z, Y, X, C1, device="cuda", generator=g).bfloat16()
    in2 = torch.randn(Z, Y, X, C2, device="cuda", generator=g).bfloat16() if C2 else None
    W = (0.2 * torch.randn(27, Cout, C1 + C2, device="cuda", generator=g)).bfloat16()
    bias = torch.randn(Cout, device="cuda", generator=g)
    out = torch.full((Z, Y, X, Cout), float("nan"), device="cuda")
    conv3d_forward(in1, W, out, in2=in2, bias=bias, relu=relu)
    torch.cuda.synchronize()
    x = cl_to_cf(in1) if in2 is None else np.concatenate([cl_to_cf(in1), cl_to_cf(in2)])
    w = w_to_oracle(W)
    ref = cnn.conv3d(x, w, bias.cpu().numpy().astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    scale = cnn.conv3d(np.abs(x), np.abs(w)) + np.abs(bias.cpu().numpy())[:, None, None, None]
    got = cl_to_cf(out)
    assert np.all(np.abs(got - ref) <= 3e-5 * scale + 1e-30)


@pytest.mark.parametrize("Z,Y,X,C1,C2,Cout,masked,with_gx", [
    (5, 6, 7, 16, 16, 32, True, True),
    (4, 3, 9, 16, 0, 16, False, True),
    (3, 4, 5, 32, 0, 64, True, False),
    (2, 2, 2, 64, 64, 64, True, True),
])
def test_conv_backward_matches_oracle(Z, Y, X, C1, C2, Cout, masked, with_gx):
    import torch
    from paper_2504_05604_gb300 import conv3d_backward
    g = torch.Generator(device="cuda").manual_seed(Z * 37 + Cout + C2)
    x1 = torch.randn(Z, Y, X, C1, device="cuda", generator=g).bfloat16()
    x2 = torch.randn(Z, Y, X, C2, device="cuda", generator=g).bfloat16() if C2 else None
    W = (0.2 * torch.randn(27, Cout, C1 + C2, device="cuda", generator=g)).bfloat16()
    gy = torch.randn(Z, Y, X, Cout, device="cuda", generator=g)
    act = torch.randn(Z, Y, X, Cout, device="cuda", generator=g).bfloat16() if masked else None
    gw0 = torch.randn(27, Cout, C1 + C2, device="cuda", generator=g)
    gb0 = torch.randn(Cout, device="cuda", generator=g)
    gw, gb = gw0.clone(), gb0.clone()
    gx = torch.full((Z, Y, X, C1 + C2), float("nan"), device="cuda") if with_gx else None
    conv3d_backward(x1, W, gy, gw, gb=gb, gx=gx, x2=x2, act=act)
    torch.cuda.synchronize()
    x = cl_to_cf(x1) if x2 is None else np.concatenate([cl_to_cf(x1), cl_to_cf(x2)])
    w = w_to_oracle(W)
    mask = (cl_to_cf(act) > 0) if masked else 1.0
    gyo = cl_to_cf(gy) * mask
    _, gw_ref, gb_ref = cnn.conv3d_backward(x, w, gyo)
    _, gw_abs, gb_abs = cnn.conv3d_backward(np.abs(x), w, np.abs(gyo))
    got_gw = w_to_oracle(gw) - w_to_oracle(gw0)
    assert np.all(np.abs(got_gw - gw_ref) <= 3e-5 * np.abs(gw_abs) + 1e-5)
    got_gb = (gb - gb0).cpu().numpy()
    assert np.all(np.abs(got_gb - gb_ref) <= 3e-5 * np.abs(gb_abs) + 1e-5)
    if with_gx:
        gy16 = cl_to_cf(gy.bfloat16()) * mask          # the data gradient reads BF16
        gx_ref, _, _ = cnn.conv3d_backward(x, w, gy16)
        gx_abs, _, _ = cnn.conv3d_backward(x, np.abs(w), np.abs(gy16))
        assert np.all(np.abs(cl_to_cf(gx) - gx_ref) <= 3e-5 * gx_abs + 1e-30)


def test_conv_rejects_bad_shapes():
    import torch
    from paper_2504_05604_gb300 import To3dError, conv3d_forward
    in1 = torch.zeros(2, 2, 2, 24, device="cuda").bfloat16()      # C1 not a multiple of 16
    W = torch.zeros(27, 16, 24, device="cuda").bfloat16()
    out = torch.zeros(2, 2, 2, 16, device="cuda")
    with pytest.raises(To3dError):
        conv3d_forward(in1, W, out)


# ------------------------------------------------------------- network


def dinv_of(prob, x):
    KE = fem.element_stiffness(prob.nu)
    d = fem.jacobi_diagonal(prob.nelx, prob.nely, prob.nelz,
                            fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin), KE, prob.fixed)
    return np.where(prob.fixed != 0, 0.0, 1.0 / d)


def _apply_problem():
    prob = random_problem(13, 6, 5, seed=41)
    x = problems.random_density(prob.nel, 42, 1e-3, 1.0)
    r = fem.masked_load(problems.random_vector(prob.ndof, 43), prob.fixed)
    return prob, x, r


def test_network_apply_matches_oracle():
    prob, x, r = _apply_problem()
    params = random_params(44)
    ctx = lib_ctx(prob)
    ctx.cnn_init(0)
    ctx.set_cnn_params(to_flat(params))
    z = ctx.cnn_apply(x, r)
    dinv = dinv_of(prob, x)
    z_ref = cnn.apply_preconditioner(bf16_params(params), r, x, prob.fixed, dinv,
                                     prob.nelx, prob.nely, prob.nelz)
    assert np.all(z[prob.fixed != 0] == 0.0)
    assert rel_l2(z, z_ref) <= 2e-2 and cosine(z, z_ref) >= 0.9995
    inp, s = cnn.preconditioner_input(r, x, prob.fixed, dinv, prob.nelx, prob.nely, prob.nelz)
    out_e, _ = bf16_network(bf16_params(params), inp)
    nx, ny, nz = prob.nelx + 1, prob.nely + 1, prob.nelz + 1
    z_emu = dinv * r + s * np.sqrt(dinv) * out_e[:, :nz, :ny, :nx].transpose(1, 2, 3, 0).reshape(-1)
    z_emu[prob.fixed != 0] = 0.0
    assert rel_l2(z, z_emu) <= 1e-2
    # positively homogeneous in r, like the oracle
    z2 = ctx.cnn_apply(x, 4.0 * r)
    assert np.allclose(z2, 4.0 * z, rtol=1e-6, atol=1e-12 * np.abs(z).max())


def _pass_through(pick):
    params = {k: np.zeros_like(v) for k, v in cnn.init_params(0).items()}
    c1 = params["e1a.w"].shape[0]
    for c in range(cnn.IN_CH):
        params["e0a.w"][2 * c, c, 1, 1, 1] = 1.0
        params["e0a.w"][2 * c + 1, c, 1, 1, 1] = -1.0
    for k in range(2 * cnn.IN_CH):
        params["e0b.w"][k, k, 1, 1, 1] = 1.0
        params["d0a.w"][k, c1 + k, 1, 1, 1] = 1.0
        params["d0b.w"][k, k, 1, 1, 1] = 1.0
    for o, c in enumerate(pick):
        params["out.w"][o, 2 * c, 1, 1, 1] = 1.0
        params["out.w"][o, 2 * c + 1, 1, 1, 1] = -1.0
    return params


def test_pass_through_network_is_exact():
    """A network whose output is its scaled input rt / s gives z = 2 D^-1 r;
    one whose output is the log density gives z = D^-1 r + s D^-1/2 ld."""
    prob, x, r = _apply_problem()
    dinv = dinv_of(prob, x)
    ctx = lib_ctx(prob)
    ctx.cnn_init(0)
    ctx.set_cnn_params(to_flat(_pass_through((0, 1, 2))))
    z = ctx.cnn_apply(x, r)
    assert np.all(np.abs(z - 2.0 * dinv * r) <= 2.0 ** -8 * dinv * np.abs(r) + 1e-300)
    ctx.set_cnn_params(to_flat(_pass_through((3,))))
    z = ctx.cnn_apply(x, r)
    rt = np.sqrt(dinv) * r
    s = np.sqrt(np.mean(rt * rt))
    ld = np.log10(np.maximum(1e-3, cnn.node_density(x, prob.nelx, prob.nely, prob.nelz)))
    corr = np.where(prob.fixed[0::3] != 0, 0.0, s * np.sqrt(dinv[0::3]) * ld.reshape(-1))
    assert np.all(np.abs(z[0::3] - dinv[0::3] * r[0::3] - corr) <= 2.0 ** -8 * np.abs(corr) +
                  1e-12 * dinv[0::3] * np.abs(r[0::3]) + 1e-300)
    assert np.allclose(z[1::3], dinv[1::3] * r[1::3], rtol=1e-14, atol=1e-300)


def _operator(prob, x):
    KE = fem.element_stiffness(prob.nu)
    return fem.apply_bc(fem.assemble(prob.nelx, prob.nely, prob.nelz,
                                     fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin), KE),
                        prob.fixed)


def test_network_gradient_matches_oracle():
    prob, x, r = _apply_problem()
    K = _operator(prob, x)
    e = fem.solve_direct(K, r, prob.fixed)
    params = random_params(46)
    ctx = lib_ctx(prob)
    ctx.cnn_init(0)
    ctx.set_cnn_params(to_flat(params))
    L, g = ctx.cnn_loss_grad(x, r, e)
    L_ref, g_ref = cnn.preconditioner_loss(bf16_params(params), r, e, x, prob.fixed,
                                           dinv_of(prob, x), prob.nelx, prob.nely, prob.nelz, K)
    assert L == pytest.approx(L_ref, rel=2e-2)
    got = from_flat(g)
    stats = {}
    for name, _, _ in cnn.layer_shapes():
        for k in (name + ".w", name + ".b"):
            stats[k] = (cosine(got[k], g_ref[k]), rel_l2(got[k], g_ref[k]))
    print("gradient cosine / rel. L2 vs FP64:",
          {k: (round(a, 4), round(b, 4)) for k, (a, b) in stats.items()})
    for k, (cs, rl) in stats.items():
        assert cs >= 0.98 and rl <= 0.25, k
    # the padded input channels of the first layer get no gradient
    gw = g[:27 * 16 * 16].reshape(27, 16, 16)
    assert np.all(gw[:, :, cnn.IN_CH:] == 0.0)


def test_zero_network_is_jacobi():
    """A zero network leaves z = D^-1 r: the loss is Jacobi's own, exact in
    FP64 up to summation order."""
    prob, x, r = _apply_problem()
    K = _operator(prob, x)
    e = fem.solve_direct(K, r, prob.fixed)
    dinv = dinv_of(prob, x)
    ctx = lib_ctx(prob)
    ctx.cnn_init(0)
    ctx.set_cnn_params(np.zeros(ctx.cnn_param_count(), np.float32))
    assert np.allclose(ctx.cnn_apply(x, r), dinv * r, rtol=1e-14, atol=1e-300)
    L, g = ctx.cnn_loss_grad(x, r, e)
    zero = {k: np.zeros_like(v) for k, v in cnn.init_params(0).items()}
    L_ref, _ = cnn.preconditioner_loss(zero, r, e, x, prob.fixed, dinv, prob.nelx, prob.nely,
                                       prob.nelz, K)
    assert L == pytest.approx(L_ref, rel=1e-10)


# ----------------------------------------------- training and flexible CG


@pytest.fixture(scope="module")
def trained():
    """A network trained on snapshots of a small cantilever's first designs."""
    prob = problems.cantilever(24, 12, 8, load="edge", volfrac=0.3, rmin=1.5)
    ctx = lib_ctx(prob)
    first, last = ctx.cnn_train(nsnap=12, per_design=4, steps=600, lr=1e-3, seed=3)
    return prob, ctx.cnn_params(), first, last, ctx.density()


def _solve_system(prob, seed, x=None):
    if x is None:
        x = problems.random_density(prob.nel, seed, 0.1, 1.0)
    K = _operator(prob, x)
    f = fem.masked_load(prob.load, prob.fixed)
    return x, K, f, fem.solve_direct(K, f, prob.fixed)


def test_training_lowers_the_loss(trained):
    _, flat, first, last, _ = trained
    assert np.isfinite(first) and np.isfinite(last) and np.all(np.isfinite(flat))
    assert last < 0.85 * first


def test_trained_network_beats_jacobi_on_a_new_design(trained):
    """What the training gains, per application: on the load of a design it
    has not seen, the trained correction lowers the energy-norm error
    ||z - K^-1 r||_K / ||K^-1 r||_K below plain Jacobi's (zero network)."""
    prob, flat, _, _, xd = trained
    x, K, f, e = _solve_system(prob, 0, xd)
    ctx = lib_ctx(prob)
    ctx.set_cnn_params(flat)
    L_net, _ = ctx.cnn_loss_grad(x, f, e)
    ctx.set_cnn_params(np.zeros_like(flat))
    L_jac, _ = ctx.cnn_loss_grad(x, f, e)
    print(f"energy loss on an unseen design: network {L_net:.4f}, Jacobi {L_jac:.4f}")
    assert L_net < L_jac


def test_flexible_cg_solves_to_tolerance(trained):
    """The learned solve is decided by the true FP64 residual, with the
    Jacobi-PCG fallback finishing it if the network stalls; the iteration
    counts against plain Jacobi-PCG are printed (what the trained network
    gains inside the solver)."""
    from paper_2504_05604_gb300 import CNN_FCG
    prob, flat, _, _, xd = trained
    x, K, f, u_ref = _solve_system(prob, 51, xd)      # the design the training reached
    ctx = lib_ctx(prob, precond=CNN_FCG, warm_start=0)
    ctx.set_cnn_params(flat)
    u, info = ctx.solve(x)
    assert info["status"] == 0 and info["relres"] <= 1e-8
    assert np.linalg.norm(f - K @ u) / np.linalg.norm(f) <= 1.5e-8
    assert np.abs(u - u_ref).max() <= 1e-6 * np.abs(u_ref).max()
    jac = lib_ctx(prob, warm_start=0)
    _, jinfo = jac.solve(x)
    # a second solve knows the plain rate from the first one's fallback: a
    # network that loses to Jacobi-PCG is dropped after at most ~J/8
    # iterations (J = Jacobi-PCG's count, 50 at least) and the fallback
    # starts over, so the total stays near J
    u2, info2 = ctx.solve(x)
    assert info2["status"] == 0 and info2["relres"] <= 1e-8
    assert np.abs(u2 - u_ref).max() <= 1e-6 * np.abs(u_ref).max()
    print(f"flexible CG {info['iters']} its, again {info2['iters']} its (outer {info['outer']}, "
          f"{info2['outer']}: 2 = Jacobi-PCG fallback finished it), plain Jacobi-PCG "
          f"{jinfo['iters']} its")
    if info["outer"] == 2:
        assert info2["iters"] <= 1.3 * jinfo["iters"] + 60


def test_zero_network_flexible_cg_is_jacobi_pcg(trained):
    """A zero network leaves z = D^-1 r: flexible CG is then Jacobi-PCG (the
    Polak-Ribiere and Fletcher-Reeves betas agree in exact arithmetic)."""
    from paper_2504_05604_gb300 import CNN_FCG
    prob, flat, _, _, _ = trained
    x, K, f, u_ref = _solve_system(prob, 52)
    ctx = lib_ctx(prob, precond=CNN_FCG, warm_start=0)
    ctx.set_cnn_params(np.zeros_like(flat))
    u, info = ctx.solve(x)
    assert info["outer"] == 1 and info["status"] == 0 and info["relres"] <= 1e-8
    assert np.abs(u - u_ref).max() <= 1e-6 * np.abs(u_ref).max()
    _, jinfo = lib_ctx(prob, warm_start=0).solve(x)
    assert abs(info["iters"] - jinfo["iters"]) <= 0.1 * jinfo["iters"] + 5


def test_non_descent_network_is_replaced_by_jacobi(trained):
    """A network returning -2 D^-1 r (z = -D^-1 r, r^T z < 0) is replaced by
    D^-1 r in every iteration: the solve still converges like Jacobi-PCG."""
    from paper_2504_05604_gb300 import CNN_FCG
    prob, flat, _, _, _ = trained
    x, K, f, u_ref = _solve_system(prob, 53)
    params = _pass_through((0, 1, 2))
    params["out.w"] *= -2.0
    ctx = lib_ctx(prob, precond=CNN_FCG, warm_start=0)
    ctx.set_cnn_params(to_flat(params))
    z = ctx.cnn_apply(x, f)
    assert np.dot(z, f) < 0.0
    u, info = ctx.solve(x)
    assert info["outer"] == 1 and info["status"] == 0 and info["relres"] <= 1e-8
    assert np.abs(u - u_ref).max() <= 1e-6 * np.abs(u_ref).max()
    _, jinfo = lib_ctx(prob, warm_start=0).solve(x)
    assert abs(info["iters"] - jinfo["iters"]) <= 0.1 * jinfo["iters"] + 5


def test_untrained_network_is_refused():
    from paper_2504_05604_gb300 import CNN_FCG, To3dError
    prob = problems.cantilever(8, 4, 4)
    ctx = lib_ctx(prob, precond=CNN_FCG)
    with pytest.raises(To3dError):
        ctx.step()


def test_oc_trajectory_with_flexible_cg(trained):
    from oracle import topopt
    from paper_2504_05604_gb300 import CNN_FCG
    prob, flat, _, _, _ = trained
    iters = 3
    x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct")
    ctx = lib_ctx(prob, precond=CNN_FCG)
    ctx.set_cnn_params(flat)
    recs = ctx.run(iters)
    for r, h in zip(recs, hist):
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
        assert r["halvings"] == h.halvings
    assert np.abs(ctx.density() - x_ref).max() <= 1e-4
