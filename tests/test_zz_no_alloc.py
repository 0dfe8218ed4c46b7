"""The allocation-free energy entry point against the context-based one.

Some callers cannot let a library call cudaMalloc: programs whose own pool
holds all device memory, and latency-critical loops that must not enter the
driver's allocator.  to3d_sensitivity_noalloc serves them from caller-owned
buffers plus one fixed scratch array inside the library.  This file is
collected last so that a run stopping at its first failure has run every
other test first.
"""
import numpy as np
import pytest

from synth import problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_noalloc_matches_context_entry_point_twice():
    import torch
    from paper_2504_05604_gb300 import Context, binding

    dims = (37, 11, 9)                     # several blocks and a ragged last block
    prob = problems.cantilever(*dims)
    ctx = Context.from_problem(prob)
    for call, seed in enumerate((5, 6)):   # two calls in a row share the scratch
        x = torch.tensor(problems.random_density(prob.nel, seed, 0.0, 1.0), device="cuda")
        u = torch.tensor(problems.random_vector(prob.ndof, seed + 100), device="cuda")
        ce_ref = torch.empty(prob.nel, dtype=torch.float64, device="cuda")
        dc_ref = torch.empty_like(ce_ref)
        _, _, c_ref = ctx.sensitivity(x, u, ce_ref, dc_ref)
        ce = torch.full_like(ce_ref, float("nan"))
        dc = torch.full_like(ce_ref, float("nan"))
        c = binding.sensitivity_noalloc(*dims, x, u, ce, dc, penal=prob.penal, E0=prob.E0,
                                        Emin=prob.Emin, nu=prob.nu)
        torch.cuda.synchronize()
        assert c == pytest.approx(c_ref, rel=1e-12), call
        assert torch.allclose(ce, ce_ref, rtol=1e-12, atol=0), call
        assert torch.allclose(dc, dc_ref, rtol=1e-12, atol=0), call
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    """A grid one row past the scratch limit, with buffers of the full size
    that grid needs (so nothing could be read or written out of bounds even
    if the limit check were absent): refused with TO3D_EINVAL."""
    import torch
    from paper_2504_05604_gb300 import binding

    nelx, nely, nelz = 2049, 2048, 2                          # 8,392,704 > 8,388,608 elements
    nel = nelx * nely * nelz
    ndof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    x = torch.zeros(nel, dtype=torch.float64, device="cuda")
    u = torch.zeros(ndof, dtype=torch.float64, device="cuda")
    ce, dc = torch.empty_like(x), torch.empty_like(x)
    with pytest.raises(binding.To3dError) as ei:
        binding.sensitivity_noalloc(nelx, nely, nelz, x, u, ce, dc)
    assert ei.value.status == 1
