"""The seeded synthetic workloads match the recipe they are documented with
(clamps, loads, obstacles, ranges, determinism).  No method arithmetic."""
import numpy as np

from synth import problems


def node(nelx, nely, i, j, k):
    return i + (nelx + 1) * (j + (nely + 1) * k)


def test_cantilever_clamps_and_edge_load():
    nelx, nely, nelz = 7, 3, 2
    p = problems.cantilever(nelx, nely, nelz, load="edge")
    fixed = p.fixed.reshape(-1, 3)
    for k in range(nelz + 1):
        for j in range(nely + 1):
            for i in range(nelx + 1):
                assert np.all(fixed[node(nelx, nely, i, j, k)] == (1 if i == 0 else 0))
    f = p.load.reshape(-1, 3)
    edge = [node(nelx, nely, nelx, 0, k) for k in range(nelz + 1)]
    assert np.all(f[edge, 1] == -1.0)
    assert np.count_nonzero(f) == nelz + 1


def test_centre_and_node_loads():
    p = problems.config_large(nelx=8, nely=4, nelz=6)
    f = p.load.reshape(-1, 3)
    assert np.flatnonzero(f[:, 1]).tolist() == [node(8, 4, 8, 2, 3)]
    q = problems.config_paper_benchmark()
    f = q.load.reshape(-1, 3)
    assert (q.nelx, q.nely, q.nelz, q.volfrac, q.rmin, q.iters) == (32, 16, 16, 0.2, 4.0, 200)
    assert np.flatnonzero(f[:, 1]).tolist() == [node(32, 16, 32, 0, 8)]


def test_void_cylinder_counts():
    pas = problems.void_cylinder_z(240, 80, 40, 120.0, 40.0, 15.0).reshape(40, 80, 240)
    layer = pas[0]
    assert np.all(pas == layer[None])
    # lattice points (i + 1/2, j + 1/2) strictly inside a circle of radius 15
    assert int(np.count_nonzero(layer)) == sum(
        1 for i in range(240) for j in range(80)
        if (i + 0.5 - 120) ** 2 + (j + 0.5 - 40) ** 2 < 225)


def test_batched_recipe_and_determinism():
    a = problems.config_batched(16)
    b = problems.config_batched(16)
    for p, q in zip(a, b):
        assert (p.nelx, p.nely, p.nelz, p.volfrac) == (q.nelx, q.nely, q.nelz, q.volfrac)
        assert np.array_equal(p.passive, q.passive) and np.array_equal(p.load, q.load)
    for p in problems.config_batched(64):
        assert 32 <= p.nelx <= 128 and 16 <= p.nely <= 64 and 8 <= p.nelz <= 32
        assert 0.1 <= p.volfrac <= 0.4 and p.rmin == 1.5
        f = p.load.reshape(-1, 3)
        (n,) = np.flatnonzero(f[:, 1])
        i = n % (p.nelx + 1)
        j = (n // (p.nelx + 1)) % (p.nely + 1)
        k = n // ((p.nelx + 1) * (p.nely + 1))
        assert i == p.nelx
        pas = p.passive.reshape(p.nelz, p.nely, p.nelx)
        assert set(np.unique(pas)) <= {0, 1}
        assert not np.any(pas[:, :, 0])                       # clamped layer stays solid-able
        touch = pas[max(k - 1, 0):k + 1, max(j - 1, 0):j + 1, p.nelx - 1]
        assert not np.any(touch)                              # nothing void at the load


def test_initial_density_respects_passive():
    pas = problems.void_cylinder_z(10, 6, 2, 5.0, 3.0, 2.0)
    pas[0] = problems.SOLID
    p = problems.cantilever(10, 6, 2, passive=pas, volfrac=0.25)
    x = p.initial_density()
    assert np.all(x[pas == problems.VOID] == 0.0)
    assert np.all(x[pas == problems.SOLID] == 1.0)
    assert np.all(x[pas == problems.DESIGN] == 0.25)
