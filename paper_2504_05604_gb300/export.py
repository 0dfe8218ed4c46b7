"""Post-processing of an optimised design (host side, after the GPU loop).

The paper's workflow ends with the voxels of pseudo-density above 0.5
(Section 3, Fig. 1b) and an STL export of the optimised geometry (Sections
2.5 and 3).  This module writes both, headless:

* ``voxels(x, dims, level)``      boolean voxel grid [nelz, nely, nelx];
* ``write_voxels(path, ...)``     that grid as a .npy file;
* ``isosurface(x, dims, level)``  a closed triangle surface of the density
  field at ``level`` by marching tetrahedra;
* ``write_stl(path, tris)``       binary STL.

Surface extraction.  The element densities are the samples of a scalar
field at the element centres, surrounded by one layer of zeros so that the
surface closes at the domain boundary.  Every cell of 2 x 2 x 2 neighbouring
samples is cut into six tetrahedra around its main diagonal; in a
tetrahedron with one (or three) samples inside (>= level) the surface is the
triangle through the three edges that leave the lone sample, with two
inside it is the quadrilateral through the four edges that join the inside
pair to the outside pair (two triangles).  Crossing points are linearly
interpolated along the edges.  Each triangle is oriented so that its normal
points from the inside samples to the outside ones.  Because neighbouring
tetrahedra share their faces (the six-tetrahedron split is the same in every
cell), the pieces join into a closed, consistently oriented surface.
Coordinates are in element lengths with the grid's corner at the origin.
"""
from __future__ import annotations

import struct

import numpy as np

# the six tetrahedra of a cell around its diagonal from corner 0 to corner 7
# (corner index a + 2b + 4c at offset (a, b, c)): each path 0 -> 7 along the
# three axes in some order
_TETS = np.array([[0, 1, 3, 7], [0, 1, 5, 7], [0, 2, 3, 7], [0, 2, 6, 7], [0, 4, 5, 7],
                  [0, 4, 6, 7]])
_CORNER = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.float64)


def voxels(x, dims, level=0.5):
    """Boolean voxels [nelz, nely, nelx] of elements with x > level."""
    nelx, nely, nelz = dims
    return np.asarray(x).reshape(nelz, nely, nelx) > level


def write_voxels(path, x, dims, level=0.5):
    np.save(path, voxels(x, dims, level))


def isosurface(x, dims, level=0.5):
    """Triangles [T, 3, 3] (vertex coordinates) of the level surface."""
    nelx, nely, nelz = dims
    f = np.zeros((nelz + 2, nely + 2, nelx + 2))
    f[1:-1, 1:-1, 1:-1] = np.asarray(x, dtype=np.float64).reshape(nelz, nely, nelx)
    # sample (i, j, k) of f sits at the centre of element (i-1, j-1, k-1)
    kk, jj, ii = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1),
                             indexing="ij")
    base = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)          # cell origins
    cval = np.stack([f[base[:, 2] + c, base[:, 1] + b, base[:, 0] + a]
                     for a, b, c in _CORNER.astype(int)], axis=1)           # [cells, 8]
    # keep cells the surface crosses
    ins = cval >= level
    cross = ins.any(axis=1) & ~ins.all(axis=1)
    base, cval = base[cross], cval[cross]
    tris = []
    for tet in _TETS:
        v = cval[:, tet]                                   # [n, 4]
        p = base[:, None, :] + _CORNER[tet][None, :, :] - 0.5  # sample positions [n, 4, 3]
        inside = v >= level
        cnt = inside.sum(axis=1)
        for n_in in (1, 2, 3):
            sel = cnt == n_in
            if not np.any(sel):
                continue
            vs, ps, ins_s = v[sel], p[sel], inside[sel]
            # order the four vertices: inside ones first (stable)
            order = np.argsort(~ins_s, axis=1, kind="stable")
            vs = np.take_along_axis(vs, order, axis=1)
            ps = np.take_along_axis(ps, order[:, :, None], axis=1)

            def cut(a, b):
                t = (level - vs[:, a]) / (vs[:, b] - vs[:, a])
                return ps[:, a] + t[:, None] * (ps[:, b] - ps[:, a])

            if n_in == 1:
                pieces = [(cut(0, 1), cut(0, 2), cut(0, 3))]
            elif n_in == 3:
                pieces = [(cut(0, 3), cut(1, 3), cut(2, 3))]
            else:
                q0, q1, q2, q3 = cut(0, 2), cut(0, 3), cut(1, 3), cut(1, 2)
                pieces = [(q0, q1, q2), (q0, q2, q3)]
            inner = ps[:, :n_in].mean(axis=1)
            outer = ps[:, n_in:].mean(axis=1)
            for a, b, c in pieces:
                t = np.stack([a, b, c], axis=1)
                nrm = np.cross(b - a, c - a)
                flip = np.einsum("ij,ij->i", nrm, outer - inner) < 0
                t[flip] = t[flip][:, [0, 2, 1]]
                tris.append(t)
    if not tris:
        return np.zeros((0, 3, 3))
    out = np.concatenate(tris, axis=0)
    area = np.linalg.norm(np.cross(out[:, 1] - out[:, 0], out[:, 2] - out[:, 0]), axis=1)
    return out[area > 0]


def write_stl(path, tris, name=b"to3d design"):
    """Binary STL: 80-byte header, triangle count, per triangle the unit
    normal, three vertices (float32) and a zero attribute word."""
    tris = np.asarray(tris, dtype=np.float64)
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    ln = np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm = np.where(ln > 0, nrm / np.where(ln > 0, ln, 1.0), 0.0)
    rec = np.zeros(len(tris), dtype=[("n", "<f4", 3), ("v", "<f4", (3, 3)), ("a", "<u2")])
    rec["n"] = nrm
    rec["v"] = tris
    with open(path, "wb") as fh:
        fh.write(name[:80].ljust(80, b" "))
        fh.write(struct.pack("<I", len(tris)))
        fh.write(rec.tobytes())


def read_stl(path):
    """Triangles of a binary STL written by ``write_stl``."""
    with open(path, "rb") as fh:
        fh.read(80)
        (n,) = struct.unpack("<I", fh.read(4))
        rec = np.frombuffer(fh.read(), dtype=[("n", "<f4", 3), ("v", "<f4", (3, 3)), ("a", "<u2")],
                            count=n)
    return rec["v"].astype(np.float64)


def enclosed_volume(tris):
    """Volume inside a closed, outward-oriented surface (divergence theorem)."""
    t = np.asarray(tris, dtype=np.float64)
    return float(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0)
