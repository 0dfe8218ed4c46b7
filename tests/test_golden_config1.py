"""The 60x20x4 cantilever's stored oracle trajectory (tests/golden).

CPU: the oracle reproduces the stored values (regression pin of the stored
file against its generator) and the stored volumes are on target to 1e-6.
GPU: the library's loop, FP64 and the tensor-core forms (single-slice BF16,
the benchmark's form; BF16 hi+lo; scaled FP16), against the stored
trajectory: first ten compliances to 1e-5, final compliance to 1e-3 (the
final-design bar), volume on target to 1e-6 in every iteration.
"""
import json
import os

import numpy as np
import pytest

from synth import problems

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config1_oracle.json")


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def problem(g):
    prob = problems.config_small(iters=g["problem"]["iters"])
    prob.bisect_tol = g["problem"]["bisect_tol"]
    return prob


def test_oracle_reproduces_stored_trajectory():
    from oracle import topopt
    g = golden()
    _, hist = topopt.top3d(problem(g), iters=3, solver="direct")
    for h, c, nh in zip(hist, g["compliance"], g["halvings"]):
        assert h.compliance == pytest.approx(c, rel=1e-10)
        assert h.halvings == nh


def test_stored_volumes_on_target():
    g = golden()
    v = np.array(g["volume"])
    assert np.all(np.abs(v / g["problem"]["volfrac"] - 1.0) <= 1e-6)
    c = np.array(g["compliance"])
    assert np.all(np.diff(c[:10]) < 0)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,lmg", [(0, False), (1, False), (2, False), (3, False), (1, True)])
def test_gpu_loop_matches_stored_trajectory(precision, lmg):
    """Every precision with Jacobi, and the benchmark's form (BF16 defect
    correction, learned multigrid with its default parameters, kept inner
    direction, inner tolerance 0.05, FP64 residuals on the sliced
    tensor-core K u)."""
    import __graft_entry__ as ge
    ge.build()
    from tests.gpu_helpers import lib_ctx
    from paper_2504_05604_gb300 import LMG
    g = golden()
    prob = problem(g)
    kw = dict(precond=LMG, inner_rtol=0.05, mg_keep_dir=1, fp64_tc=1) if lmg else {}
    ctx = lib_ctx(prob, precision=precision, **kw)
    recs = ctx.run(g["problem"]["iters"])
    comp = np.array([r["compliance"] for r in recs])
    vol = np.array([r["volume"] for r in recs])
    assert all(r["status"] == 0 and r["relres"] <= 1e-8 for r in recs)
    assert np.all(np.abs(vol / prob.volfrac - 1.0) <= 1e-6)
    ref = np.array(g["compliance"])
    assert np.all(np.abs(comp[:10] / ref[:10] - 1.0) <= 1e-5)
    assert abs(comp[-1] / ref[-1] - 1.0) <= 1e-3
    print(f"precision {precision}: final compliance {comp[-1]:.6f} vs stored {ref[-1]:.6f}, "
          f"max rel. deviation over the run {np.max(np.abs(comp / ref - 1.0)):.2e}")
