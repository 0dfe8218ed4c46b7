"""Pins of the oracle's convolutions and preconditioner network."""
import numpy as np
import pytest

from oracle import cnn, fem


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3d_equals_direct_loops():
    r = rng(1)
    x = r.standard_normal((3, 4, 3, 5))
    w = r.standard_normal((2, 3, 3, 3, 3))
    b = r.standard_normal(2)
    y = cnn.conv3d(x, w, b)
    C, Z, Y, X = x.shape
    for o in range(2):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    s = b[o]
                    for i in range(C):
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    zz, y2, x2 = z + dz - 1, yy + dy - 1, xx + dx - 1
                                    if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                                        s += w[o, i, dz, dy, dx] * x[i, zz, y2, x2]
                    assert y[o, z, yy, xx] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_identity_and_shift_kernels():
    x = rng(2).standard_normal((3, 5, 4, 6))
    w = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1, 1] = 1.0
    assert np.array_equal(cnn.conv3d(x, w), x)
    w = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1, 2] = 1.0          # reads x + 1: shift left, zero at the end
    y = cnn.conv3d(x, w)
    assert np.array_equal(y[..., :-1], x[..., 1:]) and np.all(y[..., -1] == 0)


def test_pool_and_upsample_adjoints():
    r = rng(3)
    a = r.standard_normal((2, 4, 6, 8))
    b = r.standard_normal((2, 2, 3, 4))
    assert np.sum(cnn.avgpool2(a) * b) == pytest.approx(np.sum(a * cnn.avgpool2_backward(b)))
    assert np.sum(cnn.up2(b) * a) == pytest.approx(np.sum(b * cnn.up2_backward(a)))
    assert np.allclose(cnn.avgpool2(cnn.up2(b)), b)


def test_conv3d_backward_finite_differences():
    r = rng(4)
    x = r.standard_normal((2, 3, 4, 3))
    w = r.standard_normal((3, 2, 3, 3, 3))
    b = r.standard_normal(3)
    gy = r.standard_normal((3, 3, 4, 3))
    f = lambda x_, w_, b_: float(np.sum(cnn.conv3d(x_, w_, b_) * gy))
    gx, gw, gb = cnn.conv3d_backward(x, w, gy)
    h = 1e-6
    for idx in [(0, 1, 2, 1), (1, 0, 0, 2), (1, 2, 3, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert (f(xp, w, b) - f(xm, w, b)) / (2 * h) == pytest.approx(gx[idx], rel=1e-6)
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 1, 2, 2, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert (f(x, wp, b) - f(x, wm, b)) / (2 * h) == pytest.approx(gw[idx], rel=1e-6)
    assert gb == pytest.approx(gy.sum(axis=(1, 2, 3)))


def test_network_gradient_finite_differences():
    ch = (2, 3, 3, 2)
    params = cnn.init_params(5, ch=ch)
    r = rng(6)
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * r.standard_normal(params[k].shape)
    x = r.standard_normal((cnn.IN_CH, 8, 8, 8))
    target = r.standard_normal((cnn.OUT_CH, 8, 8, 8))

    def loss(p):
        out, _ = cnn.forward(p, x)
        return cnn.relative_loss(out, target)[0]

    out, cache = cnn.forward(params, x)
    L, gout = cnn.relative_loss(out, target)
    grads, _ = cnn.backward(params, cache, gout)
    h = 1e-6
    for key, idx in [("e0a.w", (1, 2, 0, 1, 2)), ("e2b.w", (0, 1, 1, 1, 1)),
                     ("e3a.w", (1, 0, 2, 0, 1)), ("d2a.w", (2, 4, 1, 2, 0)),
                     ("d0a.w", (0, 3, 1, 1, 1)), ("out.w", (2, 1, 0, 0, 0)),
                     ("d1b.b", (1,)), ("out.b", (0,))]:
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[key][idx] += h
        pm[key][idx] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert fd == pytest.approx(grads[key][idx], rel=1e-5, abs=1e-9), key


def _zero_params(ch=cnn.CHANNELS):
    return {k: np.zeros_like(v) for k, v in cnn.init_params(0, ch=ch).items()}


def _pass_through(params, pick):
    """Hand-built network whose output channel c is input channel pick[c].

    ReLU layers carry a signed value v as the pair (relu(v), relu(-v)): the
    first layer writes +v and -v, the level-0 layers copy the pairs (through
    the skip connection, the deeper levels stay zero) and the output layer
    forms relu(v) - relu(-v) = v.
    """
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


def _dinv(nelx, nely, nelz, x, fixed):
    KE = fem.element_stiffness(0.3)
    d = fem.jacobi_diagonal(nelx, nely, nelz, fem.simp_modulus(x, 3.0), KE, fixed)
    return np.where(fixed != 0, 0.0, 1.0 / d)


def _small_problem(seed, nelx=5, nely=3, nelz=2):
    r = rng(seed)
    n = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    fixed = np.zeros(n, np.uint8)
    face = (nelx + 1) * np.arange((nely + 1) * (nelz + 1))       # nodes with i = 0
    for c in range(3):
        fixed[3 * face + c] = 1            # clamped x = 0 face
    fixed[3 * 7 + 1] = 1                   # one more dof
    x = r.uniform(1e-4, 1.0, nelx * nely * nelz)
    return nelx, nely, nelz, x, r.standard_normal(n), fixed


def test_node_density_brute_force():
    nelx, nely, nelz = 3, 2, 2
    x = rng(7).uniform(0, 1, nelx * nely * nelz)
    d = cnn.node_density(x, nelx, nely, nelz)
    for k in range(nelz + 1):
        for j in range(nely + 1):
            for i in range(nelx + 1):
                vals = [x[ei + nelx * (ej + nely * ek)]
                        for ek in (k - 1, k) for ej in (j - 1, j) for ei in (i - 1, i)
                        if 0 <= ei < nelx and 0 <= ej < nely and 0 <= ek < nelz]
                assert d[k, j, i] == pytest.approx(sum(vals) / len(vals), rel=1e-14)


def test_pass_through_network_returns_residual():
    """Output = the scaled input rt / s: z = D^-1 r + D^-1/2 rt = 2 D^-1 r."""
    nelx, nely, nelz, x, res, fixed = _small_problem(8)
    dinv = _dinv(nelx, nely, nelz, x, fixed)
    params = _pass_through(_zero_params(), pick=(0, 1, 2))
    z = cnn.apply_preconditioner(params, res, x, fixed, dinv, nelx, nely, nelz)
    assert np.allclose(z, np.where(fixed != 0, 0.0, 2.0 * dinv * res), rtol=1e-13, atol=1e-300)
    z0 = cnn.apply_preconditioner(_zero_params(), res, x, fixed, dinv, nelx, nely, nelz)
    assert np.allclose(z0, np.where(fixed != 0, 0.0, dinv * res), rtol=1e-14, atol=1e-300)


def test_pass_through_network_returns_log_density():
    nelx, nely, nelz, x, res, fixed = _small_problem(9)
    dinv = _dinv(nelx, nely, nelz, x, fixed)
    params = _pass_through(_zero_params(), pick=(3,))
    z = cnn.apply_preconditioner(params, res, x, fixed, dinv, nelx, nely, nelz)
    rt = np.where(fixed != 0, 0.0, np.sqrt(dinv) * res)
    s = np.sqrt(np.mean(rt * rt))
    ld = np.log10(np.maximum(1e-3, cnn.node_density(x, nelx, nely, nelz))).reshape(-1)
    ref = dinv * res + s * np.sqrt(dinv) * np.repeat(ld, 3) * np.tile([1.0, 0.0, 0.0], ld.size)
    assert np.allclose(z, np.where(fixed != 0, 0.0, ref), rtol=1e-13, atol=1e-300)
    # output channels 1 and 2 have no weights: a bias comes out times s D^-1/2
    params["out.b"][:] = [1.0, 2.0, 3.0]
    z = cnn.apply_preconditioner(params, res, x, fixed, dinv, nelx, nely, nelz)
    ref = dinv[1::3] * res[1::3] + s * np.sqrt(dinv[1::3]) * 2.0
    assert np.allclose(z[1::3], np.where(fixed[1::3] != 0, 0.0, ref), rtol=1e-13)


def test_preconditioner_is_positively_homogeneous():
    nelx, nely, nelz, x, res, fixed = _small_problem(10)
    dinv = _dinv(nelx, nely, nelz, x, fixed)
    params = cnn.init_params(11, ch=(4, 4, 4, 4))
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.05 * rng(12).standard_normal(params[k].shape)
    z1 = cnn.apply_preconditioner(params, res, x, fixed, dinv, nelx, nely, nelz)
    z2 = cnn.apply_preconditioner(params, 3.7 * res, x, fixed, dinv, nelx, nely, nelz)
    assert np.allclose(z2, 3.7 * z1, rtol=1e-12, atol=1e-300)
    assert np.all(z1[fixed != 0] == 0.0) and np.any(z1 != 0.0)


def _operator(nelx, nely, nelz, x, fixed):
    KE = fem.element_stiffness(0.3)
    return fem.apply_bc(fem.assemble(nelx, nely, nelz, fem.simp_modulus(x, 3.0), KE), fixed)


def test_energy_loss_against_cholesky():
    """L = ||z - e||_K^2 / ||e||_K^2 through a dense Cholesky factor of the
    free block (K_ff = C C^T, ||v||_K = ||C^T v||), for a zero network
    (plain Jacobi), a pass-through network and a random one."""
    nelx, nely, nelz, x, res, fixed = _small_problem(16)
    K = _operator(nelx, nely, nelz, x, fixed)
    dinv = _dinv(nelx, nely, nelz, x, fixed)
    free = np.flatnonzero(fixed == 0)
    Ch = np.linalg.cholesky(K.toarray()[np.ix_(free, free)])
    r = np.where(fixed != 0, 0.0, res)
    e = fem.solve_dense(K, r, fixed)
    knorm2 = lambda v: float(np.sum((Ch.T @ v[free]) ** 2))
    for params in (_zero_params(), _pass_through(_zero_params(), pick=(0, 1, 2)),
                   cnn.init_params(17)):
        z = cnn.apply_preconditioner(params, r, x, fixed, dinv, nelx, nely, nelz)
        L, _ = cnn.preconditioner_loss(params, r, e, x, fixed, dinv, nelx, nely, nelz, K)
        assert L == pytest.approx(knorm2(z - e) / knorm2(e), rel=1e-9)


def test_preconditioner_loss_gradient_finite_differences():
    nelx, nely, nelz, x, res, fixed = _small_problem(13)
    K = _operator(nelx, nely, nelz, x, fixed)
    dinv = _dinv(nelx, nely, nelz, x, fixed)
    r = np.where(fixed != 0, 0.0, res)
    e = fem.solve_dense(K, r, fixed)
    params = cnn.init_params(14, ch=(2, 3, 3, 2))
    L, grads = cnn.preconditioner_loss(params, r, e, x, fixed, dinv, nelx, nely, nelz, K)
    h = 1e-6
    for key, idx in [("e0a.w", (1, 3, 1, 1, 0)), ("d0a.w", (1, 4, 2, 1, 1)), ("out.b", (2,)),
                     ("e2b.w", (1, 2, 0, 1, 2))]:
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[key][idx] += h
        pm[key][idx] -= h
        fd = (cnn.preconditioner_loss(pp, r, e, x, fixed, dinv, nelx, nely, nelz, K)[0] -
              cnn.preconditioner_loss(pm, r, e, x, fixed, dinv, nelx, nely, nelz, K)[0]) / (2 * h)
        assert fd == pytest.approx(grads[key][idx], rel=1e-5, abs=1e-10), key
