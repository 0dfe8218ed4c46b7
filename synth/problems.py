"""Seeded cantilever workloads on a structured hex8 voxel grid.

Numbering used everywhere in this project:

* element (i, j, k), 0 <= i < nelx, ...   ->  e = i + nelx * (j + nely * k)
* node    (i, j, k), 0 <= i <= nelx, ...  ->  n = i + (nelx+1) * (j + (nely+1) * k)
* degree of freedom                        ->  d = 3 * n + c, c in {x=0, y=1, z=2}

The paper's usage example and benchmark (Section 3 and Section 4.2) are
cantilevers: the x = 0 face is clamped and a vertical point load acts on the
free end.  Passive elements model its non-design obstacles (Section 2.3):
0 = design, 1 = void (pinned at density 0), 2 = solid (pinned at density 1).

Nothing in this module computes any part of the optimisation method; it only
produces masks, loads and random numbers.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

DESIGN, VOID, SOLID = 0, 1, 2


def node_count(nelx: int, nely: int, nelz: int) -> int:
    return (nelx + 1) * (nely + 1) * (nelz + 1)


def element_count(nelx: int, nely: int, nelz: int) -> int:
    return nelx * nely * nelz


@dataclasses.dataclass
class Problem:
    """One SIMP/OC problem instance (inputs only)."""
    name: str
    nelx: int
    nely: int
    nelz: int
    volfrac: float
    penal: float
    rmin: float
    fixed: np.ndarray            # uint8 [3N], 1 = clamped dof
    load: np.ndarray             # float64 [3N]
    passive: Optional[np.ndarray] = None   # uint8 [nel] or None
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    move: float = 0.2
    bisect_tol: float = 1e-3
    iters: int = 50

    @property
    def nel(self) -> int:
        return element_count(self.nelx, self.nely, self.nelz)

    @property
    def nnode(self) -> int:
        return node_count(self.nelx, self.nely, self.nelz)

    @property
    def ndof(self) -> int:
        return 3 * self.nnode

    def passive_or_zeros(self) -> np.ndarray:
        if self.passive is None:
            return np.zeros(self.nel, dtype=np.uint8)
        return self.passive

    def initial_density(self) -> np.ndarray:
        """x0 = volfrac on design elements, 0 on void, 1 on solid."""
        x = np.full(self.nel, self.volfrac, dtype=np.float64)
        pas = self.passive_or_zeros()
        x[pas == VOID] = 0.0
        x[pas == SOLID] = 1.0
        return x


def _node(nelx, nely, i, j, k):
    return i + (nelx + 1) * (j + (nely + 1) * k)


def clamp_face_x0(nelx: int, nely: int, nelz: int) -> np.ndarray:
    fixed = np.zeros(3 * node_count(nelx, nely, nelz), dtype=np.uint8)
    j, k = np.meshgrid(np.arange(nely + 1), np.arange(nelz + 1), indexing="ij")
    nodes = _node(nelx, nely, 0, j.ravel(), k.ravel())
    for c in range(3):
        fixed[3 * nodes + c] = 1
    return fixed


def cantilever(nelx: int, nely: int, nelz: int, *, load: str = "edge",
               load_node: Optional[Tuple[int, int, int]] = None,
               volfrac: float = 0.3, penal: float = 3.0, rmin: float = 1.5,
               passive: Optional[np.ndarray] = None, iters: int = 50,
               name: str = "cantilever", **kw) -> Problem:
    """Cantilever clamped on x = 0 with unit -y loads.

    load = "edge":   F_y = -1 on every node of the edge x = nelx, y = 0.
    load = "centre": F_y = -1 on node (nelx, nely/2, nelz/2).
    load = "node":   F_y = -1 on ``load_node``.
    """
    N = node_count(nelx, nely, nelz)
    f = np.zeros(3 * N, dtype=np.float64)
    if load == "edge":
        ks = np.arange(nelz + 1)
        f[3 * _node(nelx, nely, nelx, 0, ks) + 1] = -1.0
    elif load == "centre":
        f[3 * _node(nelx, nely, nelx, nely // 2, nelz // 2) + 1] = -1.0
    elif load == "node":
        i, j, k = load_node
        f[3 * _node(nelx, nely, i, j, k) + 1] = -1.0
    else:
        raise ValueError(load)
    return Problem(name=name, nelx=nelx, nely=nely, nelz=nelz, volfrac=volfrac,
                   penal=penal, rmin=rmin, fixed=clamp_face_x0(nelx, nely, nelz),
                   load=f, passive=passive, iters=iters, **kw)


def void_cylinder_z(nelx: int, nely: int, nelz: int, cx: float, cy: float,
                    radius: float) -> np.ndarray:
    """Element (i, j, .) is void iff (i+1/2-cx)^2 + (j+1/2-cy)^2 < radius^2."""
    i = np.arange(nelx) + 0.5
    j = np.arange(nely) + 0.5
    inside = ((i[None, :] - cx) ** 2 + (j[:, None] - cy) ** 2) < radius ** 2   # [nely, nelx]
    pas = np.zeros((nelz, nely, nelx), dtype=np.uint8)
    pas[:, inside] = VOID
    return pas.reshape(-1)


def config_small(iters: int = 50) -> Problem:
    """60x20x4 cantilever, edge load, volfrac 0.3, rmin 1.5."""
    return cantilever(60, 20, 4, load="edge", volfrac=0.3, rmin=1.5, iters=iters,
                      name="cantilever 60x20x4 edge load")


def config_void_cylinder(iters: int = 100) -> Problem:
    """240x80x40 cantilever, edge load, void cylinder r=15 about (120, 40)."""
    pas = void_cylinder_z(240, 80, 40, 120.0, 40.0, 15.0)
    return cantilever(240, 80, 40, load="edge", volfrac=0.3, rmin=1.5,
                      passive=pas, iters=iters,
                      name="cantilever 240x80x40 void cylinder")


def config_large(iters: int = 100, nelx: int = 480, nely: int = 160, nelz: int = 80) -> Problem:
    """480x160x80 cantilever, load at the centre of the x = nelx face,
    volfrac 0.2, rmin 2.5.  Smaller grids of the same shape are available
    through the size arguments."""
    return cantilever(nelx, nely, nelz, load="centre", volfrac=0.2, rmin=2.5,
                      iters=iters, name=f"cantilever {nelx}x{nely}x{nelz} centre load")


def config_paper_benchmark(iters: int = 200) -> Problem:
    """The paper's benchmark size (Section 4.2): 32x16x16, volfrac 0.2,
    penal 3, rmin 4; point load at the centre of the free end's bottom edge."""
    return cantilever(32, 16, 16, load="node", load_node=(32, 0, 8), volfrac=0.2,
                      rmin=4.0, iters=iters, name="cantilever 32x16x16 (paper benchmark)")


def config_paper_usage(iters: int = 200) -> Problem:
    """The paper's usage example (Section 3): the 32x16x16 benchmark
    cantilever with a cylindrical non-design obstacle.  The paper does not
    give the obstacle's geometry; here: a void cylinder along z through the
    whole depth, axis at (x, y) = (16, 8) (mid-span, mid-height), radius 3.5
    elements."""
    pas = void_cylinder_z(32, 16, 16, 16.0, 8.0, 3.5)
    return cantilever(32, 16, 16, load="node", load_node=(32, 0, 8), volfrac=0.2,
                      rmin=4.0, iters=iters, passive=pas,
                      name="cantilever 32x16x16 with a cylindrical obstacle (paper usage example)")


def config_batched(nprob: int = 64, seed: int = 20250407) -> List[Problem]:
    """Independent cantilevers of uneven sizes with 0-3 spherical voids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(nprob):
        nelx = int(rng.integers(32, 129))
        nely = int(rng.integers(16, 65))
        nelz = int(rng.integers(8, 33))
        volfrac = float(rng.uniform(0.1, 0.4))
        lj = int(rng.integers(0, nely + 1))
        lk = int(rng.integers(0, nelz + 1))
        nsph = int(rng.integers(0, 4))
        ci = np.arange(nelx) + 0.5
        cj = np.arange(nely) + 0.5
        ck = np.arange(nelz) + 0.5
        K, J, I = np.meshgrid(ck, cj, ci, indexing="ij")
        pas = np.zeros((nelz, nely, nelx), dtype=np.uint8)
        # elements touching the load node, and the clamped x = 0 layer
        guard = np.zeros_like(pas, dtype=bool)
        guard[max(lk - 1, 0):lk + 1, max(lj - 1, 0):lj + 1, nelx - 1] = True
        guard[:, :, 0] = True
        placed, tries = 0, 0
        while placed < nsph and tries < 100:
            tries += 1
            r = float(rng.uniform(3.0, 10.0))
            c = rng.uniform([0, 0, 0], [nelx, nely, nelz])
            inside = (I - c[0]) ** 2 + (J - c[1]) ** 2 + (K - c[2]) ** 2 < r * r
            if np.any(inside & guard):
                continue
            pas[inside] = VOID
            placed += 1
        out.append(cantilever(nelx, nely, nelz, load="node", load_node=(nelx, lj, lk),
                              volfrac=volfrac, rmin=1.5, passive=pas.reshape(-1),
                              name=f"batched[{p}] {nelx}x{nely}x{nelz}"))
    return out


def random_density(nel: int, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Smooth-ish random densities in [lo, hi] (uniform draw)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=nel)


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(n)
