"""Helpers shared by the GPU parity tests: problem builders and an emulation
of the tensor-core operand rounding written on top of the oracle's pieces."""
import numpy as np

from oracle import fem
from synth import problems


def lib_ctx(prob, **kw):
    from paper_2504_05604_gb300 import Context
    return Context.from_problem(prob, **kw)


def random_problem(nelx, nely, nelz, seed, passive=True, partial_clamp=True, rmin=1.5):
    prob = problems.cantilever(nelx, nely, nelz, load="edge", rmin=rmin)
    rng = np.random.Generator(np.random.PCG64(seed))
    if passive and prob.nel > 4:
        pas = np.zeros(prob.nel, np.uint8)
        pas[rng.choice(prob.nel, max(1, prob.nel // 20), replace=False)] = 1
        pas[rng.choice(prob.nel, max(1, prob.nel // 30), replace=False)] = 2
        pas[0] = 0
        prob.passive = pas
    if partial_clamp:
        fx = prob.fixed.copy()
        nodes = rng.choice(prob.nnode, max(1, prob.nnode // 15), replace=False)
        fx[3 * nodes + rng.integers(0, 3, nodes.size)] = 1
        prob.fixed = fx
    return prob


def bf16_round(a32):
    b = np.ascontiguousarray(a32, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def emulate_lowp(prob, x, p32, prec):
    """y = Kbar p with the operand rounding of the tensor-core forms, in FP64:
    element vectors taken relative to their local node 0, then rounded as
    the form prescribes."""
    nelx, nely, nelz = prob.nelx, prob.nely, prob.nelz
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    ed = fem.element_dofs(nelx, nely, nelz)
    fixed = prob.fixed != 0
    q = np.where(fixed, np.float32(0), p32.astype(np.float32))
    pe = q[ed]                                       # float32 [nel, 24]
    # the kernel takes each element vector relative to its local node 0
    # (KE annihilates translations), in FP32, before any rounding
    pe = (pe - np.tile(pe[:, 0:3], (1, 8))).astype(np.float32)
    if prec == 1:
        pe = bf16_round(pe).astype(np.float64)
    elif prec == 2:
        hi = bf16_round(pe)
        lo = bf16_round((pe - hi).astype(np.float32))
        pe = hi.astype(np.float64) + lo.astype(np.float64)
    elif prec in (3, 4):
        m = np.abs(pe).max(axis=1)
        _, ex = np.frexp(np.where(m > 0, m, 1.0))
        s = np.ldexp(1.0, 11 - ex)[:, None].astype(np.float32)
        v = (pe * s).astype(np.float32)
        hi = v.astype(np.float16).astype(np.float32)
        if prec == 4:
            lo = (v - hi).astype(np.float16).astype(np.float32)
            pe = (hi.astype(np.float64) + lo.astype(np.float64)) / s
        else:
            pe = hi.astype(np.float64) / s
    ye = (pe @ KE) * E[:, None]
    y = np.bincount(ed.ravel(), weights=ye.ravel(), minlength=p32.size)
    absb = (np.abs(q[ed].astype(np.float64)) @ np.abs(KE)) * E[:, None]
    bound = np.bincount(ed.ravel(), weights=absb.ravel(), minlength=p32.size)
    return np.where(fixed, p32, y), bound


# ------------------------------------------- BF16 emulation of the network


def _round_bf16(a):
    return bf16_round(np.asarray(a, np.float64).astype(np.float32)).astype(np.float64)


def bf16_network(params, x):
    """Forward and backward of the oracle's U-Net with the GPU's rounding
    points: the network input and every ReLU / pooling output rounded to
    BF16, the data gradient formed from the upstream gradient rounded to
    BF16 (the weight gradient from the unrounded one).  Everything else in
    FP64 on top of the oracle's convolution, pooling and loss pieces.
    Returns (out, backward) with backward(gout) -> grads."""
    from oracle import cnn
    q = _round_bf16
    cache = {}

    def conv(name, inp, act=True):
        y = cnn.conv3d(inp, params[name + ".w"], params[name + ".b"])
        cache[name] = (inp, y)
        return q(cnn.relu(y)) if act else y

    e0 = conv("e0b", conv("e0a", q(x)))
    e1 = conv("e1b", conv("e1a", q(cnn.avgpool2(e0))))
    e2 = conv("e2b", conv("e2a", q(cnn.avgpool2(e1))))
    e3 = conv("e3b", conv("e3a", q(cnn.avgpool2(e2))))
    d2 = conv("d2b", conv("d2a", np.concatenate([cnn.up2(e3), e2])))
    d1 = conv("d1b", conv("d1a", np.concatenate([cnn.up2(d2), e1])))
    d0 = conv("d0b", conv("d0a", np.concatenate([cnn.up2(d1), e0])))
    out = conv("out", d0, act=False)
    c1, c2, c3 = (params["e1a.w"].shape[0], params["e2a.w"].shape[0], params["e3a.w"].shape[0])

    def backward(gout):
        grads = {}

        def bconv(name, gy, act=True):
            inp, y = cache[name]
            if act:
                gy = gy * (y > 0)
            _, gw, gb = cnn.conv3d_backward(inp, params[name + ".w"], gy)
            gx, _, _ = cnn.conv3d_backward(inp, params[name + ".w"], q(gy))
            grads[name + ".w"], grads[name + ".b"] = gw, gb
            return gx

        g = bconv("out", gout, act=False)
        g = bconv("d0a", bconv("d0b", g))
        g_up1, g_e0 = g[:c1], g[c1:]
        g = bconv("d1a", bconv("d1b", cnn.up2_backward(g_up1)))
        g_up2, g_e1 = g[:c2], g[c2:]
        g = bconv("d2a", bconv("d2b", cnn.up2_backward(g_up2)))
        g_up3, g_e2 = g[:c3], g[c3:]
        g = bconv("e3a", bconv("e3b", cnn.up2_backward(g_up3)))
        g = bconv("e2a", bconv("e2b", g_e2 + cnn.avgpool2_backward(g)))
        g = bconv("e1a", bconv("e1b", g_e1 + cnn.avgpool2_backward(g)))
        bconv("e0a", bconv("e0b", g_e0 + cnn.avgpool2_backward(g)))
        return grads

    return out, backward
