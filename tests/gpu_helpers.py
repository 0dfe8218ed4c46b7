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
    """y = Kbar p with the operand rounding of the tensor-core forms, in FP64."""
    nelx, nely, nelz = prob.nelx, prob.nely, prob.nelz
    KE = fem.element_stiffness(prob.nu)
    E = fem.simp_modulus(x, prob.penal, prob.E0, prob.Emin)
    ed = fem.element_dofs(nelx, nely, nelz)
    fixed = prob.fixed != 0
    q = np.where(fixed, np.float32(0), p32.astype(np.float32))
    pe = q[ed]                                       # float32 [nel, 24]
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
