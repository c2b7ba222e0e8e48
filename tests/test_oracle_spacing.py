"""Pins of the grid step for non-square images (Sec. 3.5.1).

Sec. 3.5.1 builds the lattice Xi in [-Y, Y] x [-X, X] "without loss of
generality X >= Y", derives one step Delta from the larger dimension, bounds
it by 1/4 < Delta <= 1, and remarks that psi(Delta omega) on Omega gives the
same spectra.  The oracle's default ("common") takes one Delta for both axes;
the alternative ("per_axis") stretches each axis to [-X, X].  The tests below
check which statements each reading meets, the frame invariants of both, and
pin the common reading's values to the square grid's (a non-square grid is
a window of the square one).
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o

NONSQUARE = [(64, 256), (48, 80), (128, 256), (30, 64), (80, 48), (63, 100)]


def _steps(rows, cols, spacing, max_scale="max"):
    j0 = o.default_scales(rows, cols)
    X = o.grid_extent(j0, max_scale)
    gm, gn = o.grid_denominators(rows, cols, spacing)
    return X / gm, X / gn, X


def test_common_step_meets_delta_bounds_per_axis_does_not():
    # Sec. 3.5.1: 1/4 < Delta <= 1 for the default extent X = 2^{2 j0 - 1}
    bad_per_axis = 0
    for rows in range(4, 260, 3):
        for cols in (4, 15, 16, 63, 64, 100, 255, 256, 511, 1024):
            dr, dc, _ = _steps(rows, cols, "common")
            assert dr == dc
            assert 0.25 < dr <= 1.0, (rows, cols, dr)
            pr, pc, _ = _steps(rows, cols, "per_axis")
            if not (0.25 < pr <= 1.0 and 0.25 < pc <= 1.0):
                bad_per_axis += 1
    assert bad_per_axis > 0
    # e.g. 128 x 256: j0 = 4, X = 128; per axis the rows step by 128/64 = 2
    pr, pc, _ = _steps(128, 256, "per_axis")
    assert (pr, pc) == (2.0, 1.0)
    assert _steps(128, 256, "common")[:2] == (1.0, 1.0)


def test_common_grid_is_delta_times_omega_with_y_at_most_x():
    # Sec. 3.5.1: Xi = Delta * Omega with one Delta (psi(Delta omega) on Omega),
    # rows inside [-Y, Y] and columns inside [-X, X] with X >= Y
    for rows, cols in NONSQUARE:
        j0 = o.default_scales(rows, cols)
        o1, o2, xi1, xi2 = o.grid(rows, cols, j0, spacing="common")
        d = _steps(rows, cols, "common")[0]
        np.testing.assert_array_equal(xi1, o1 * d)
        np.testing.assert_array_equal(xi2, o2 * d)
        X = o.grid_extent(j0)
        Y = d * (min(rows, cols) // 2)
        big, small = (xi1, xi2) if cols >= rows else (xi2, xi1)
        assert np.abs(big).max() == X
        assert np.abs(small).max() == Y <= X
        # the per-axis grid has two different steps and Y = X
        _, _, p1, p2 = o.grid(rows, cols, j0, spacing="per_axis")
        assert np.abs(p1).max() == np.abs(p2).max() == X
        with np.errstate(invalid="ignore", divide="ignore"):
            r1 = np.unique(np.round(p1[o1 != 0] / o1[o1 != 0], 12))
            r2 = np.unique(np.round(p2[o2 != 0] / o2[o2 != 0], 12))
        assert r1.size == r2.size == 1 and r1[0] != r2[0]


@pytest.mark.parametrize("spacing", ["common", "per_axis"])
@pytest.mark.parametrize("shape", NONSQUARE)
def test_tightness_parseval_reconstruction(spacing, shape):
    # Sec. 3.2 theorem / Sec. 3.6: sum_i psi_i^2 = 1, ||c|| = ||f||, inv(fwd(f)) = f
    s = o.frame_sum(*shape, spacing=spacing)
    assert np.abs(s - 1.0).max() <= 1e-14
    f = np.random.default_rng(7).standard_normal(shape)
    c = o.forward(f, spacing=spacing)
    assert abs(np.sum(c * c) / np.sum(f * f) - 1.0) <= 1e-12
    assert np.abs(o.inverse(c, spacing=spacing) - f).max() <= 1e-12
    # the coefficients are real (Sec. 3.8.1 fix, applied to every plane)
    assert np.abs(np.imag(o.forward_complex(f, spacing=spacing))).max() <= 1e-13


@pytest.mark.parametrize("shape", NONSQUARE)
def test_common_spectra_are_a_window_of_the_square_grid(shape):
    # One Delta for both axes: the M x N lattice is the part |o| <= floor(L/2)
    # of the max x max lattice, so the unfixed spectra are the square grid's
    # values there (same j0, same X, same Delta; identical arithmetic)
    rows, cols = shape
    n = max(rows, cols)
    j0 = o.default_scales(rows, cols)
    assert o.default_scales(n, n) == j0
    r_idx = o.freq_index(rows) % n
    c_idx = o.freq_index(cols) % n
    for i in range(o.num_planes(j0)):
        sq = o.spectrum_raw(n, n, j0, i)
        ns = o.spectrum_raw(rows, cols, j0, i, spacing="common")
        np.testing.assert_array_equal(ns, sq[np.ix_(r_idx, c_idx)])
    # the per-axis reading is not a window of the square grid
    i = o.plane_table(j0).index(("h", j0 - 1, 1))
    sq = o.spectrum_raw(n, n, j0, i)[np.ix_(r_idx, c_idx)]
    assert np.abs(o.spectrum_raw(rows, cols, j0, i, spacing="per_axis") - sq).max() > 0.1


def test_readings_agree_on_square_images():
    for n in (16, 64, 63):
        for i in range(o.num_planes(o.default_scales(n, n))):
            j0 = o.default_scales(n, n)
            np.testing.assert_array_equal(o.spectrum(n, n, j0, i, spacing="common"),
                                          o.spectrum(n, n, j0, i, spacing="per_axis"))


def test_unknown_spacing_rejected():
    with pytest.raises(ValueError):
        o.grid_denominators(64, 128, "isotropic")
