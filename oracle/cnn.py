"""Naive FP64 3D convolutions and the preconditioner network (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The learned preconditioner is a small U-Net on the node grid: four levels
with 16/32/64/64 channels, 3x3x3 convolutions with zero "same" padding,
2x2x2 average pooling down, nearest-neighbour x2 up with skip
concatenation, ReLU.  Input: the three components of the Jacobi-scaled
residual D^-1/2 r divided by their RMS, and log10 of the node density;
output: three components of a correction added to Jacobi, z = D^-1 r +
RMS * D^-1/2 Net(...).  Tensors are channels-first [C, Z, Y, X]
here; weights are [C_out, C_in, 3, 3, 3].

Parity: pinned by tests/test_oracle_cnn.py (direct-loop convolution,
identity and shift kernels, finite-difference gradients of every layer
and of the whole network, brute-force node densities, and hand-built
pass-through networks that return the residual and the log density
exactly, which pins the input scaling, channel order, padding and output
mapping; the energy-norm loss against a dense Cholesky factor).

The preconditioner is not part of the paper (whose solver is plain PCG,
Section 2.3); this file defines what the library's learned preconditioner
computes so that its kernels can be checked.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (16, 32, 64, 64)
IN_CH, OUT_CH = 4, 3


def pad1(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))


def conv3d(x, w, b=None):
    """y[o, z, y, x] = b[o] + sum_{i, dz, dy, dx} w[o, i, dz, dy, dx] x[i, z+dz-1, y+dy-1, x+dx-1]."""
    C, Z, Y, X = x.shape
    xp = pad1(x)
    y = np.zeros((w.shape[0], Z, Y, X))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                y += np.einsum("oi,izyx->ozyx", w[:, :, dz, dy, dx], patch)
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv3d_backward(x, w, gy):
    """Gradients of conv3d: (gx, gw, gb) for upstream gradient gy."""
    C, Z, Y, X = x.shape
    xp = pad1(x)
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", gy, patch)
                gxp[:, dz:dz + Z, dy:dy + Y, dx:dx + X] += np.einsum("oi,ozyx->izyx",
                                                                      w[:, :, dz, dy, dx], gy)
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gy.sum(axis=(1, 2, 3))


def avgpool2(x):
    C, Z, Y, X = x.shape
    return x.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(gy):
    C, Z, Y, X = gy.shape
    return gy.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def layer_shapes(ch=CHANNELS, cin=IN_CH, cout=OUT_CH):
    """(name, C_out, C_in) of every convolution, in forward order."""
    c0, c1, c2, c3 = ch
    return [("e0a", c0, cin), ("e0b", c0, c0),
            ("e1a", c1, c0), ("e1b", c1, c1),
            ("e2a", c2, c1), ("e2b", c2, c2),
            ("e3a", c3, c2), ("e3b", c3, c3),
            ("d2a", c2, c3 + c2), ("d2b", c2, c2),
            ("d1a", c1, c2 + c1), ("d1b", c1, c1),
            ("d0a", c0, c1 + c0), ("d0b", c0, c0),
            ("out", cout, c0)]


def init_params(seed=0, ch=CHANNELS):
    rng = np.random.Generator(np.random.PCG64(seed))
    params = {}
    for name, co, ci in layer_shapes(ch):
        std = np.sqrt(2.0 / (27 * ci))
        params[name + ".w"] = rng.standard_normal((co, ci, 3, 3, 3)) * std
        params[name + ".b"] = np.zeros(co)
    return params


def forward(params, x):
    """U-Net forward; returns (output, cache for backward).  Spatial sizes
    must be divisible by 8."""
    cache = {}

    def conv(name, inp, act=True):
        y = conv3d(inp, params[name + ".w"], params[name + ".b"])
        cache[name] = (inp, y)
        return relu(y) if act else y

    e0 = conv("e0b", conv("e0a", x))
    e1 = conv("e1b", conv("e1a", avgpool2(e0)))
    e2 = conv("e2b", conv("e2a", avgpool2(e1)))
    e3 = conv("e3b", conv("e3a", avgpool2(e2)))
    d2 = conv("d2b", conv("d2a", np.concatenate([up2(e3), e2])))
    d1 = conv("d1b", conv("d1a", np.concatenate([up2(d2), e1])))
    d0 = conv("d0b", conv("d0a", np.concatenate([up2(d1), e0])))
    out = conv("out", d0, act=False)
    cache["e0"], cache["e1"], cache["e2"] = e0, e1, e2
    return out, cache


def backward(params, cache, gout):
    """Gradients of all parameters for upstream gradient gout of the output."""
    grads = {}

    def bconv(name, gy, act=True):
        inp, y = cache[name]
        if act:
            gy = gy * (y > 0)
        gx, gw, gb = conv3d_backward(inp, params[name + ".w"], gy)
        grads[name + ".w"], grads[name + ".b"] = gw, gb
        return gx

    c0, c1, c2, c3 = (params["e0a.w"].shape[0], params["e1a.w"].shape[0],
                      params["e2a.w"].shape[0], params["e3a.w"].shape[0])
    g = bconv("out", gout, act=False)
    g = bconv("d0a", bconv("d0b", g))
    g_up1, g_e0 = g[:c1], g[c1:]
    g = bconv("d1a", bconv("d1b", up2_backward(g_up1)))
    g_up2, g_e1 = g[:c2], g[c2:]
    g = bconv("d2a", bconv("d2b", up2_backward(g_up2)))
    g_up3, g_e2 = g[:c3], g[c3:]
    g = bconv("e3a", bconv("e3b", up2_backward(g_up3)))
    g_e2 = g_e2 + avgpool2_backward(g)
    g = bconv("e2a", bconv("e2b", g_e2))
    g_e1 = g_e1 + avgpool2_backward(g)
    g = bconv("e1a", bconv("e1b", g_e1))
    g_e0 = g_e0 + avgpool2_backward(g)
    gx = bconv("e0a", bconv("e0b", g_e0))
    return grads, gx


def relative_loss(out, target):
    """L = |out - target|^2 / |target|^2 and dL/dout."""
    d = out - target
    t2 = float(np.sum(target * target))
    return float(np.sum(d * d)) / t2, 2.0 * d / t2


# ------------------------------------------------- the network as preconditioner


def node_density(x, nelx, nely, nelz):
    """Mean density of the elements sharing each node, node grid [nz, ny, nx].

    Elements are numbered e = i + nelx (j + nely k), nodes on the
    (nelx+1) x (nely+1) x (nelz+1) grid.
    """
    xe = np.asarray(x, dtype=np.float64).reshape(nelz, nely, nelx)
    s = np.zeros((nelz + 1, nely + 1, nelx + 1))
    cnt = np.zeros_like(s)
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                s[c:c + nelz, b:b + nely, a:a + nelx] += xe
                cnt[c:c + nelz, b:b + nely, a:a + nelx] += 1.0
    return s / cnt


def padded_node_shape(nelx, nely, nelz):
    """Node grid rounded up to multiples of 8 (three pooling levels)."""
    return tuple((n + 1 + 7) // 8 * 8 for n in (nelz, nely, nelx))


def preconditioner_input(r, x, fixed, dinv, nelx, nely, nelz):
    """Network input [4, Zp, Yp, Xp] and the scale s.

    The residual enters Jacobi-scaled, rt = D^-1/2 r (dinv = 1/diag(K) per
    dof, clamped entries zero), which takes the 1e9 stiffness contrast of
    SIMP out of what the network sees; s = RMS(rt) over all 3N dofs.
    Channels 0..2: the x, y, z components of rt / s; channel 3:
    log10(max(1e-3, node density)).  Zero outside the node grid.
    """
    nx, ny, nz = nelx + 1, nely + 1, nelz + 1
    free = np.asarray(fixed) == 0
    rt = np.where(free, np.sqrt(dinv) * np.asarray(r, dtype=np.float64), 0.0)
    s = float(np.sqrt(np.sum(rt * rt) / rt.size))
    Zp, Yp, Xp = padded_node_shape(nelx, nely, nelz)
    inp = np.zeros((IN_CH, Zp, Yp, Xp))
    rn = (rt / s if s > 0 else rt).reshape(nz, ny, nx, 3)
    for c in range(3):
        inp[c, :nz, :ny, :nx] = rn[..., c]
    inp[3, :nz, :ny, :nx] = np.log10(np.maximum(1e-3, node_density(x, nelx, nely, nelz)))
    return inp, s


def _network_to_dofs(out, nelx, nely, nelz):
    nx, ny, nz = nelx + 1, nely + 1, nelz + 1
    return np.stack([out[c, :nz, :ny, :nx] for c in range(OUT_CH)], axis=-1).reshape(-1)


def apply_preconditioner(params, r, x, fixed, dinv, nelx, nely, nelz):
    """z = D^-1 r + s D^-1/2 Net(input): Jacobi plus a learned correction in
    the Jacobi-scaled variables; zero on clamped dofs (dof d = 3n + c).  A
    zero network gives plain Jacobi."""
    inp, s = preconditioner_input(r, x, fixed, dinv, nelx, nely, nelz)
    out, _ = forward(params, inp)
    free = np.asarray(fixed) == 0
    z = dinv * np.asarray(r, dtype=np.float64) + s * np.sqrt(dinv) * _network_to_dofs(
        out, nelx, nely, nelz)
    return np.where(free, z, 0.0)


def preconditioner_loss(params, r, e, x, fixed, dinv, nelx, nely, nelz, K):
    """Training loss of one sample in the energy norm, and its gradients.

    With z = M(r) (``apply_preconditioner``) and e = K^-1 r the exact
    correction, L = ||z - e||_K^2 / ||e||_K^2 = (z^T K z - 2 z^T r + r^T e) /
    (r^T e), K the clamped operator.  L < 1 implies r^T z > z^T K z / 2 > 0:
    a preconditioner that beats z = 0 on a residual is a descent direction
    for it.  Returns (L, grads) with dL/dz = 2 (K z - r) / (r^T e) carried
    back through the output scaling (s D^-1/2) and the network.
    """
    inp, s = preconditioner_input(r, x, fixed, dinv, nelx, nely, nelz)
    nx, ny, nz = nelx + 1, nely + 1, nelz + 1
    free = np.asarray(fixed) == 0
    r = np.where(free, np.asarray(r, dtype=np.float64), 0.0)
    out, cache = forward(params, inp)
    z = np.where(free, dinv * r + s * np.sqrt(dinv) * _network_to_dofs(out, nelx, nely, nelz),
                 0.0)
    q = K @ z
    rte = float(np.dot(r, e))
    L = (float(np.dot(z, q)) - 2.0 * float(np.dot(z, r)) + rte) / rte
    gz = np.where(free, 2.0 * (q - r) / rte, 0.0)
    gout = np.zeros_like(out)
    gout[:, :nz, :ny, :nx] = (s * np.sqrt(dinv) * gz).reshape(nz, ny, nx, 3).transpose(3, 0, 1, 2)
    grads, _ = backward(params, cache, gout)
    return L, grads
