"""Post-processing: voxel dump and the marching-tetrahedra STL export of a
density field (CPU, no GPU)."""
import numpy as np
import pytest

from paper_2504_05604_gb300 import export


def _edges_closed(tris):
    """Every edge of a closed, consistently oriented surface appears once in
    each direction."""
    from collections import Counter
    key = lambda p: tuple(np.round(p, 9))
    fwd = Counter()
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            fwd[(key(t[a]), key(t[b]))] += 1
    return all(fwd.get((b, a), 0) == n for (a, b), n in fwd.items())


def test_single_voxel_gives_a_closed_outward_surface():
    x = np.zeros(27)
    x[13] = 1.0                                   # centre of a 3x3x3 grid
    tris = export.isosurface(x, (3, 3, 3))
    assert len(tris) > 0
    assert _edges_closed(tris)
    v = export.enclosed_volume(tris)
    assert v > 0                                  # outward normals
    # the 0.5 level surface of one full sample lies halfway to the zero
    # neighbours: an octahedron-like body of volume 1/6 * (1)^3 * ... > 0
    assert v < 1.0


def test_ball_volume_and_closedness():
    n = 20
    k, j, i = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((i - 10) ** 2 + (j - 10) ** 2 + (k - 10) ** 2)
    x = np.clip(6.5 - r, 0.0, 1.0).ravel()        # smooth ramp: level 0.5 at r = 6
    tris = export.isosurface(x, (n, n, n))
    assert _edges_closed(tris)
    assert export.enclosed_volume(tris) == pytest.approx(4.0 / 3.0 * np.pi * 6.0 ** 3, rel=0.03)


def test_stl_round_trip_and_voxels(tmp_path):
    x = np.zeros(4 * 3 * 2)
    x[[1, 2, 5]] = 0.9
    tris = export.isosurface(x, (4, 3, 2))
    path = tmp_path / "d.stl"
    export.write_stl(path, tris)
    back = export.read_stl(path)
    assert back.shape == tris.shape
    assert np.allclose(back, tris, atol=1e-5)
    assert path.stat().st_size == 84 + 50 * len(tris)
    vp = tmp_path / "v.npy"
    export.write_voxels(vp, x, (4, 3, 2))
    vox = np.load(vp)
    assert vox.shape == (2, 3, 4) and vox.sum() == 3
