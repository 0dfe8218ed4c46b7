"""Pins of the oracle's linear-decay filter (paper Section 2.4)."""
import numpy as np
import pytest

from oracle import filters
from synth import problems

SQ2, SQ3, SQ5, SQ6 = np.sqrt(2), np.sqrt(3), np.sqrt(5), np.sqrt(6)

# Interior row sums sum_d max(0, rmin - |d|) over integer offsets, written out
# by hand from the shells |d|^2 = 0, 1, 2, 3, 4, 5, 6 (multiplicities 1, 6,
# 12, 8, 6, 24, 24).
HS_INTERIOR = {
    1.5: 1.5 + 6 * 0.5 + 12 * (1.5 - SQ2),
    2.5: 2.5 + 6 * 1.5 + 12 * (2.5 - SQ2) + 8 * (2.5 - SQ3) + 6 * 0.5
    + 24 * (2.5 - SQ5) + 24 * (2.5 - SQ6),
}
STENCIL_SIZE = {1.5: 19, 2.5: 81, 4.0: 251}


@pytest.mark.parametrize("rmin", [1.5, 2.5])
def test_interior_row_sum_closed_form(rmin):
    H = filters.filter_matrix(7, 7, 7, rmin)
    Hs = filters.row_sums(H)
    centre = 3 + 7 * (3 + 7 * 3)
    assert Hs[centre] == pytest.approx(HS_INTERIOR[rmin], rel=1e-14)
    assert H[centre].nnz == STENCIL_SIZE[rmin]


def test_interior_row_sum_rmin4():
    # 251 offsets with |d| < 4 (distance exactly 4 has weight 0)
    assert len(filters.stencil_offsets(4.0)) == 251
    assert sum(w for *_, w in filters.stencil_offsets(4.0)) == pytest.approx(269.4392630972, rel=1e-10)


@pytest.mark.parametrize("rmin", [1.5, 2.5, 3.0])
def test_offset_loop_equals_bruteforce(rmin):
    Hb = filters.filter_matrix_bruteforce(5, 4, 3, rmin)
    Ho = filters.filter_matrix(5, 4, 3, rmin)
    assert abs(Hb - Ho).max() < 1e-15
    assert abs(Ho - Ho.T).max() == 0


@pytest.mark.parametrize("rmin", [1.5, 2.5])
def test_normalised_rows_and_constant_fixed_point(rmin):
    nelx, nely, nelz = 6, 5, 4
    H = filters.filter_matrix(nelx, nely, nelz, rmin)
    Hs = filters.row_sums(H)
    assert np.allclose(np.asarray((H / Hs[:, None]).sum(1)).ravel(), 1.0, rtol=0, atol=1e-15)
    n = nelx * nely * nelz
    x = np.full(n, 0.37)
    dc = np.full(n, -2.5)
    assert np.allclose(filters.sensitivity_filter(H, Hs, x, dc), dc, rtol=1e-14)
    assert np.allclose(filters.density_filter(H, Hs, x), x, rtol=1e-14)


@pytest.mark.parametrize("rmin", [1.5, 2.5])
def test_stencil_form_equals_matrix_form(rmin):
    nelx, nely, nelz = 7, 5, 4
    n = nelx * nely * nelz
    H = filters.filter_matrix(nelx, nely, nelz, rmin)
    Hs = filters.row_sums(H)
    x = problems.random_density(n, 11)
    dc = -problems.random_density(n, 12)
    a = filters.sensitivity_filter(H, Hs, x, dc)
    b = filters.sensitivity_filter_stencil(nelx, nely, nelz, rmin, x, dc)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()
    assert np.allclose(filters.row_sums_stencil(nelx, nely, nelz, rmin), Hs, rtol=1e-15)


def test_sensitivity_filter_small_by_hand():
    # 3x1x1 row, rmin 1.5: weights 1.5 (self) and 0.5 (face neighbours).
    H = filters.filter_matrix(3, 1, 1, 1.5)
    Hs = filters.row_sums(H)
    assert np.allclose(Hs, [2.0, 2.5, 2.0])
    x = np.array([0.5, 0.2, 1e-4])
    dc = np.array([-1.0, -2.0, -3.0])
    expect0 = (1.5 * 0.5 * -1.0 + 0.5 * 0.2 * -2.0) / (2.0 * 0.5)
    expect2 = (0.5 * 0.2 * -2.0 + 1.5 * 1e-4 * -3.0) / (2.0 * 1e-3)
    got = filters.sensitivity_filter(H, Hs, x, dc)
    assert got[0] == pytest.approx(expect0, rel=1e-15)
    assert got[2] == pytest.approx(expect2, rel=1e-15)


def test_density_filter_chain_rule_matches_finite_difference():
    nelx, nely, nelz = 4, 3, 3
    n = nelx * nely * nelz
    H = filters.filter_matrix(nelx, nely, nelz, 1.5)
    Hs = filters.row_sums(H)
    w = problems.random_vector(n, 13)
    x = problems.random_density(n, 14)

    def g(xv):               # a smooth scalar of the filtered field
        xt = filters.density_filter(H, Hs, xv)
        return float(np.sum(w * xt ** 2))

    xt = filters.density_filter(H, Hs, x)
    grad = filters.density_filter_chain(H, Hs, 2 * w * xt)
    h = 1e-6
    for e in (0, 17, n - 1):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        assert (g(xp) - g(xm)) / (2 * h) == pytest.approx(grad[e], rel=1e-7)
