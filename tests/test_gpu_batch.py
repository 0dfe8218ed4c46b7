"""Batched independent problems (one graph per problem and OC iteration)
against the oracle loop, and the 64-problem synthetic batch by properties."""
import numpy as np
import pytest

from oracle import topopt
from synth import problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _sphere_void(nelx, nely, nelz, c, r):
    k, j, i = np.meshgrid(np.arange(nelz) + 0.5, np.arange(nely) + 0.5, np.arange(nelx) + 0.5,
                          indexing="ij")
    inside = (i - c[0]) ** 2 + (j - c[1]) ** 2 + (k - c[2]) ** 2 < r * r
    return np.where(inside, 1, 0).astype(np.uint8).ravel()


def small_batch():
    return [
        problems.cantilever(20, 8, 4, load="edge", volfrac=0.3),
        problems.cantilever(24, 10, 6, load="node", load_node=(24, 5, 3), volfrac=0.25,
                            passive=_sphere_void(24, 10, 6, (12, 5, 3), 2.5)),
        problems.cantilever(16, 6, 6, load="centre", volfrac=0.35, rmin=2.5),
    ]


@pytest.mark.parametrize("precision", [2, 4])
def test_batch_matches_oracle_loop(precision):
    from paper_2504_05604_gb300 import Batch
    probs = small_batch()
    iters = 4
    batch = Batch(probs, precision=precision)
    recs = [batch.step() for _ in range(iters)]
    for i, prob in enumerate(probs):
        x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct")
        for it in range(iters):
            r, h = recs[it][i], hist[it]
            assert r["status"] == 0 and r["relres"] <= 1e-8
            assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
            assert r["volume"] == pytest.approx(h.volume, abs=1e-6)
            assert r["halvings"] == h.halvings
        assert np.abs(batch.density(i) - x_ref).max() <= 1e-4
        if prob.passive is not None:
            assert np.all(batch.density(i)[prob.passive == 1] == 0.0)
    batch.close()


def test_batch_rejects_fp64_form():
    from paper_2504_05604_gb300 import Batch, To3dError
    with pytest.raises(To3dError):
        Batch(small_batch()[:1], precision=0)


def test_full_synthetic_batch_properties():
    # 64 cantilevers of uneven sizes with 0-3 spherical voids (seeded)
    from paper_2504_05604_gb300 import Batch
    probs = problems.config_batched(64)
    batch = Batch(probs)
    r1 = batch.step()
    r2 = batch.step()
    for i, prob in enumerate(probs):
        for r in (r1[i], r2[i]):
            assert r["status"] == 0 and r["relres"] <= 1e-8
            assert abs(r["volume"] - prob.volfrac) < 2e-3
        assert r2[i]["compliance"] < r1[i]["compliance"]
        x = batch.density(i)
        assert np.all((x >= 0) & (x <= 1))
        if prob.passive is not None:
            assert np.all(x[prob.passive == 1] == 0.0)
    batch.close()


def test_batch_density_filter_matches_oracle_loop():
    from paper_2504_05604_gb300 import FILTER_DENS, Batch
    probs = small_batch()[:2]
    # a solid passive slab under the load of the first problem
    pas = np.zeros(probs[0].nel, np.uint8)
    k, j, i = np.meshgrid(np.arange(4), np.arange(8), np.arange(20), indexing="ij")
    pas[((i >= 17) & (j == 0)).ravel()] = 2
    probs[0].passive = pas
    iters = 3
    batch = Batch(probs, precision=2, filter=FILTER_DENS)
    recs = [batch.step() for _ in range(iters)]
    for i, prob in enumerate(probs):
        x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct", filter_kind="density")
        for it in range(iters):
            r, h = recs[it][i], hist[it]
            assert r["status"] == 0 and r["relres"] <= 1e-8
            assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
            assert r["halvings"] == h.halvings
        assert np.abs(batch.density(i) - x_ref).max() <= 1e-4
    batch.close()


def test_batch_with_learned_multigrid_matches_oracle_loop():
    """The learned-multigrid defect correction inside the per-problem graphs
    (set-up, V-cycles and MG-PCG captured with the device-side loops), with
    non-default parameters set after creation."""
    from paper_2504_05604_gb300 import LMG, Batch
    probs = small_batch()
    iters = 4
    batch = Batch(probs, precision=1, precond=LMG, inner_rtol=0.01)
    batch.set_mg_params([0.8, 0.8, 0.8, 0.8, 0.7, 0.9, 0.7, 1.8, 1.8, 1.6])
    recs = [batch.step() for _ in range(iters)]
    for i, prob in enumerate(probs):
        x_ref, hist = topopt.top3d(prob, iters=iters, solver="direct")
        for it in range(iters):
            r, h = recs[it][i], hist[it]
            assert r["status"] == 0 and r["relres"] <= 1e-8
            assert r["compliance"] == pytest.approx(h.compliance, rel=1e-5)
            assert r["halvings"] == h.halvings
        assert np.abs(batch.density(i) - x_ref).max() <= 1e-4
    batch.close()


def test_full_synthetic_batch_with_learned_multigrid():
    from paper_2504_05604_gb300 import LMG, Batch
    probs = problems.config_batched(64)
    batch = Batch(probs, precision=1, precond=LMG, inner_rtol=0.01)
    for _ in range(2):
        recs = batch.step()
    for i, prob in enumerate(probs):
        assert recs[i]["status"] == 0 and recs[i]["relres"] <= 1e-8
        assert abs(recs[i]["volume"] - prob.volfrac) < 2e-3
    batch.close()
