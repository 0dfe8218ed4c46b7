"""Whole OC iterations on the GPU against the oracle's loop."""
import numpy as np
import pytest

from oracle import topopt
from synth import problems
from tests.gpu_helpers import lib_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_trajectory_matches_oracle(precision):
    prob = problems.cantilever(30, 10, 4, load="edge", volfrac=0.3, rmin=1.5)
    iters = 12
    x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct")
    ctx = lib_ctx(prob, precision=precision)
    recs = ctx.run(iters)
    for r, h in zip(recs, hist):
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
        assert r["volume"] == pytest.approx(h.volume, abs=1e-6)
        assert r["halvings"] == h.halvings
    x = ctx.density()
    assert np.abs(x - x_ref).max() <= 1e-4


def test_passive_void_cylinder_step():
    nelx, nely, nelz = 40, 16, 6
    pas = problems.void_cylinder_z(nelx, nely, nelz, 20.0, 8.0, 4.0)
    prob = problems.cantilever(nelx, nely, nelz, volfrac=0.3, passive=pas)
    x_ref, hist = topopt.top3d(prob, iters=3, solver="direct")
    ctx = lib_ctx(prob, precision=1)
    recs = ctx.run(3)
    for r, h in zip(recs, hist):
        assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
    x = ctx.density()
    assert np.all(x[pas == 1] == 0.0) and np.all(x[pas == 2] == 1.0)
    assert np.abs(x - x_ref).max() <= 1e-4


def test_smoke_entry():
    import __graft_entry__ as g
    g.smoke()


@pytest.mark.parametrize("precision", [0, 1])
def test_density_filter_trajectory_matches_oracle(precision):
    """Density-filter OC (Section 2.4): analysis on H x / Hs, chain rule
    H^T (dc / Hs) over the unpinned elements, OC on x; with passive void and
    solid regions."""
    from paper_2504_05604_gb300 import FILTER_DENS
    nelx, nely, nelz = 30, 10, 4
    pas = problems.void_cylinder_z(nelx, nely, nelz, 15.0, 5.0, 2.5)
    # a solid passive block under the loaded edge: its pinned filtered
    # densities carry no sensitivity back through the filter
    k, j, i = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    pas[((i >= nelx - 3) & (j <= 1)).ravel()] = 2
    prob = problems.cantilever(nelx, nely, nelz, load="edge", volfrac=0.3, rmin=1.5,
                               passive=pas)
    iters = 8
    x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct", filter_kind="density")
    ctx = lib_ctx(prob, precision=precision, filter=FILTER_DENS)
    recs = ctx.run(iters)
    for r, h in zip(recs, hist):
        assert r["status"] == 0 and r["relres"] <= 1e-8
        assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
        assert r["halvings"] == h.halvings
    x = ctx.density()
    assert np.all(x[pas == 1] == 0.0) and np.all(x[pas == 2] == 1.0)
    assert np.abs(x - x_ref).max() <= 1e-4
