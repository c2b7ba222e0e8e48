"""Pins of the oracle's smooth-shearlet variant (Sec. 3.4, eqs. newPsi1, smoothPsi).

The paper fixes: the tensor scaling function Phi_hat = varphi x varphi
(Sec. 2.4 eq. Phi), Psi1_hat = sqrt(Phi_hat(w/4)^2 - Phi_hat(w)^2) supported in
[-4, 4]^2 minus [-1/2, 1/2]^2, the telescoping identity
Phi_hat^2 + sum_j Psi1_hat^2(4^-j w) = 1 (so the frame stays Parseval), and
that the glued seam shearlets become smooth across the seam lines, where the
construction of Sec. 3.1 has a kink.
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o


def test_psi1_support_and_symmetry():
    rng = np.random.default_rng(1)
    w = rng.uniform(-0.5, 0.5, size=(2, 1000))
    assert np.all(o.Psi1_hat(*w) == 0.0)  # inside [-1/2, 1/2]^2
    w = rng.uniform(4.0, 9.0, size=(2, 1000)) * rng.choice([-1, 1], size=(2, 1000))
    assert np.all(o.Psi1_hat(w[0], rng.uniform(-9, 9, 1000)) == 0.0)  # |w1| >= 4
    assert np.all(o.Psi1_hat(rng.uniform(-9, 9, 1000), w[1]) == 0.0)  # |w2| >= 4
    w = rng.uniform(-5, 5, size=(2, 1000))
    p = o.Psi1_hat(w[0], w[1])
    np.testing.assert_array_equal(p, o.Psi1_hat(w[1], w[0]))
    np.testing.assert_array_equal(p, o.Psi1_hat(-w[0], w[1]))
    # on the plateau (1 <= max|w_i|, max|w_i| / 4 <= 1/2) it is 1
    assert o.Psi1_hat(1.5, 0.3) == pytest.approx(1.0, abs=1e-15)
    assert o.Psi1_hat(-0.2, 2.0) == pytest.approx(1.0, abs=1e-15)


def test_tensor_scaling_function():
    assert o.Phi_hat(0.3, -0.5) == 1.0
    assert o.Phi_hat(1.0, 0.0) == 0.0 and o.Phi_hat(0.2, -1.3) == 0.0
    w = np.linspace(0.51, 0.99, 7)
    np.testing.assert_allclose(o.Phi_hat(w, 0.1), o.varphi(w), atol=0)
    np.testing.assert_allclose(o.Phi_hat(w, w), o.varphi(w) ** 2, atol=1e-15)


def test_telescoping_partition():
    # Phi_hat^2(w) + sum_{j>=0} Psi1_hat^2(4^-j w) = 1 on all of R^2 (Sec. 3.4)
    rng = np.random.default_rng(2)
    w = rng.uniform(-300, 300, size=(2, 4000)) * rng.choice([1e-3, 1e-1, 1.0], size=(1, 4000))
    acc = o.Phi_hat(*w) ** 2
    for j in range(8):  # 4^-7 * 300 < 1/2: every later term vanishes
        acc = acc + o.Psi1_hat(*(w * 4.0**-j)) ** 2
    np.testing.assert_allclose(acc, 1.0, atol=1e-14)


@pytest.mark.parametrize("rows,cols,scales", [(64, 64, 3), (128, 128, 3), (256, 256, 4), (96, 128, 3), (480, 640, 4)])
def test_smooth_frame_is_tight(rows, cols, scales):
    # the Parseval property of Sec. 3.4 on the discrete grid, to rounding
    assert np.abs(o.frame_sum(rows, cols, scales, smooth=True) - 1.0).max() <= 1e-14


def test_smooth_transform_invariants():
    rng = np.random.default_rng(3)
    f = rng.normal(size=(64, 64))
    c = o.forward(f, 3, smooth=True)
    assert abs((c**2).sum() - (f**2).sum()) <= 1e-12 * (f**2).sum()  # Parseval
    np.testing.assert_allclose(o.inverse(c, 3, smooth=True), f, atol=1e-12)  # perfect reconstruction
    assert np.abs(o.forward_complex(f, 3).imag).max() <= 1e-13
    cx = np.stack([np.fft.ifft2(o.spectrum(64, 64, 3, i, smooth=True) * np.fft.fft2(f)) for i in range(29)])
    assert np.abs(cx.imag).max() <= 1e-13  # real coefficients after the Nyquist fix (Sec. 3.8.1)
    # the smooth and the classic constructions differ (only the radial factor and the low-pass)
    assert np.abs(c - o.forward(f, 3)).max() > 1e-3


def test_smooth_matches_brute_force_dft():
    # c_i = Re ifft2(psi_i fft2 f) against explicit DFT matrices at 16x16
    rng = np.random.default_rng(4)
    f = rng.normal(size=(16, 16))
    n = np.arange(16)
    Fm = np.exp(-2j * np.pi * np.outer(n, n) / 16)
    c = o.forward(f, 2, smooth=True)
    for i in range(o.num_planes(2)):
        s = o.spectrum(16, 16, 2, i, smooth=True)
        ref = np.real(np.conj(Fm) @ (s * (Fm @ f @ Fm)) @ np.conj(Fm)) / 256.0
        np.testing.assert_allclose(c[i], ref, atol=1e-13)


def _seam(x1, x2, j, smooth):
    # continuous glued seam shearlet k = -2^j of scale j: h formula where |x2| <= |x1|, v formula elsewhere
    J, a = 2.0**j, 4.0**-j
    if smooth:
        rh = rv = o.Psi1_hat(a * x1, a * x2)
    else:
        rh, rv = o.psi1_hat(a * x1), o.psi1_hat(a * x2)
    h = rh * o.psi2_hat(J * x2 / x1 - J)
    v = rv * o.psi2_hat(J * x1 / x2 - J)
    return np.where(abs(x2) <= abs(x1), h, v)


@pytest.mark.parametrize("c", [11.0, 13.0, 40.0, 50.0])
def test_seam_shearlet_smooth_across_the_diagonal(c):
    # one-sided derivatives along xi1 at the seam xi1 = xi2 (scale 2, where the
    # radial factor is in a transition band): a jump for Sec. 3.1's
    # construction, none for Sec. 3.4's
    h = 1e-5
    jump = {}
    for smooth in (False, True):
        right = (_seam(c + 2 * h, c, 2, smooth) - _seam(c + h, c, 2, smooth)) / h
        left = (_seam(c - h, c, 2, smooth) - _seam(c - 2 * h, c, 2, smooth)) / h
        jump[smooth] = abs(float(right - left))
    assert jump[False] > 1e-3
    assert jump[True] < 1e-4


# ---------------------------------------------------------------------------
# variants of the auxiliary function v (Sec. 2.1 and Sec. 3.4 remark construction_v)
# ---------------------------------------------------------------------------

VFUNS = ["meyer", "quadratic", ("poly", 1), ("poly", 5), "cinf"]


def test_v_poly_k3_is_the_paper_polynomial():
    # v'(x) = c x^3 (x-1)^3 with v(1) = 1 gives c = -140 and eq. (v)
    np.testing.assert_allclose(o._v_poly_coeffs(3), [0, 0, 0, 0, 35, -84, 70, -20], atol=1e-12)
    x = np.linspace(-0.2, 1.2, 57)
    np.testing.assert_allclose(o.v(x, ("poly", 3)), o.v(x), atol=2e-15)


def test_v_quadratic_closed_form():
    # the piecewise quadratic quoted in Sec. 2.1
    np.testing.assert_allclose(o.v([0.25, 0.5, 0.75], "quadratic"), [0.125, 0.5, 0.875], atol=0)


@pytest.mark.parametrize("vfun", VFUNS)
def test_v_variant_shape(vfun):
    x = np.linspace(0.0, 1.0, 201)
    y = o.v(x, vfun)
    assert y[0] == 0.0 and y[-1] == 1.0
    assert np.all(np.diff(y) >= -1e-15)  # nondecreasing
    np.testing.assert_allclose(y + o.v(1.0 - x, vfun), 1.0, atol=1e-14)  # symmetry around (1/2, 1/2)
    assert np.all(o.v(np.array([-1.0, -1e-9]), vfun) == 0.0) and np.all(o.v(np.array([1 + 1e-9, 3.0]), vfun) == 1.0)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_v_poly_flatness_order(k):
    # v^{(n)}(0) = 0 for 1 <= n <= k (C^k shearlets, Sec. 3.4): v(h) = O(h^{k+1}) and the
    # Taylor coefficient of order k+1 is c/(k+1) with c = (-1)^k (2k+1)!/(k!)^2
    from math import factorial

    c = (-1) ** k * factorial(2 * k + 1) / factorial(k) ** 2
    for h in (1e-2, 5e-3):
        assert o.v(h, ("poly", k)) == pytest.approx(abs(c) / (k + 1) * h ** (k + 1), rel=0.1)


def test_v_cinf_flat_at_the_ends():
    # every derivative vanishes at 0 and 1: v(h) decays faster than any power
    for h in (0.05, 0.02):
        assert o.v(h, "cinf") < h**8
        assert 1.0 - o.v(1.0 - h, "cinf") < h**8


@pytest.mark.parametrize("vfun", VFUNS)
@pytest.mark.parametrize("smooth", [False, True])
def test_v_variant_frames_are_tight(vfun, smooth):
    # any v with v(x) + v(1-x) = 1 keeps both partitions of unity, hence a Parseval frame
    assert np.abs(o.frame_sum(64, 64, 3, smooth=smooth, vfun=vfun) - 1.0).max() <= 1e-14
    assert np.abs(o.frame_sum(128, 96, 3, smooth=smooth, vfun=vfun) - 1.0).max() <= 1e-14


def test_v_variants_change_the_spectra():
    base = o.spectra(32, 32, 2)
    for vfun in VFUNS[1:]:
        assert np.abs(o.spectra(32, 32, 2, vfun=vfun) - base).max() > 1e-3
