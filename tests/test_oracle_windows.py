"""Pins of the oracle's window functions (Sec. 2.1, 2.4, 3.4) against the paper.

Each test checks a fact the paper states or proves, evaluated on dense
samples; none re-types the oracle's own formula.
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o

XS = np.linspace(-3.0, 4.0, 70001)


def test_v_boundary_values():
    # eq. (v): 0 left of 0, 1 right of 1, continuous at both ends
    assert o.v(-1e-9) == 0.0 and o.v(0.0) == 0.0
    assert o.v(1.0) == pytest.approx(1.0, abs=1e-15)
    assert o.v(1.0 + 1e-9) == 1.0
    assert o.v(0.5) == pytest.approx(0.5, abs=1e-15)


def test_v_point_symmetry():
    # Lemma (Sec. 2.1): v(x) + v(1 - x) = 1 for all real x
    # the polynomial rounds to within ~40 eps of the exact value near x = 1
    np.testing.assert_allclose(o.v(XS) + o.v(1.0 - XS), 1.0, rtol=0, atol=1e-14)


def test_v_derivative_closed_form():
    # Remark (Sec. 3.4): v'(x) = -140 x^3 (x - 1)^3 on [0, 1]; a central
    # difference of the oracle's v must match it (pins all four coefficients)
    x = np.linspace(0.01, 0.99, 981)
    h = 1e-5
    fd = (o.v(x + h) - o.v(x - h)) / (2 * h)
    np.testing.assert_allclose(fd, -140.0 * x**3 * (x - 1.0) ** 3, rtol=0, atol=1e-8)


def test_b_support_and_peak():
    # eq. (b): supp b = [-4,-1] u [1,4], b(+-2) = 1, symmetric
    assert o.b(2.0) == pytest.approx(1.0, abs=1e-15)
    assert o.b(-2.0) == pytest.approx(1.0, abs=1e-15)
    w = XS[np.abs(XS) < 1.0]
    assert np.all(o.b(w) == 0.0)
    assert np.all(o.b(np.array([4.0 + 1e-9, 5.0, -4.5])) == 0.0)
    np.testing.assert_array_equal(o.b(XS), o.b(-XS))


def test_b_dyadic_partition():
    # Lemma propertySumbj: sum_{j>=-1} b^2(2^-j w) = 1 for |w| >= 1 and
    # sin^2(pi/2 v(2w-1)) on 1/2 < |w| < 1, 0 for |w| <= 1/2
    w = np.linspace(0.0, 300.0, 30001)
    s = sum(o.b(2.0 ** (-j) * w) ** 2 for j in range(-1, 12))
    big = w >= 1.0
    np.testing.assert_allclose(s[big], 1.0, rtol=0, atol=4e-15)
    mid = (w > 0.5) & (w < 1.0)
    np.testing.assert_allclose(s[mid], np.sin(0.5 * np.pi * o.v(2 * w[mid] - 1)) ** 2, atol=4e-15)
    assert np.all(s[w <= 0.5] == 0.0)


def test_psi1_closed_form():
    # Sec. 3.4: sqrt(b^2(2w) + b^2(w)) equals the piecewise closed form
    w = np.abs(XS * 1.3)
    closed = np.where(
        w <= 0.5, 0.0,
        np.where(w < 1.0, np.sin(0.5 * np.pi * o.v(2 * w - 1)),
                 np.where(w <= 2.0, 1.0,
                          np.where(w < 4.0, np.cos(0.5 * np.pi * o.v(0.5 * w - 1)), 0.0))))
    # near |w| = 4 the rounded v exceeds 1 by ulps, so the closed form's cos is
    # a tiny negative number where sqrt(b^2) is its absolute value
    np.testing.assert_allclose(o.psi1_hat(XS * 1.3), np.abs(closed), rtol=0, atol=3e-15)


def test_psi1_support():
    # Thm PropertyPsi1: supp psi1 = [-4,-1/2] u [1/2,4]; psi1 = 1 on [1,2] (Sec. 3.5.1)
    assert np.all(o.psi1_hat(np.linspace(-0.5, 0.5, 1001)) == 0.0)
    assert np.all(o.psi1_hat(np.array([4.0 + 1e-12, 4.5, -4.5, 10.0])) == 0.0)
    # at the support edge |w| = 4 the value is cos(pi/2) in floating point
    assert np.all(o.psi1_hat(np.array([4.0, -4.0])) < 1e-16)
    np.testing.assert_allclose(o.psi1_hat(np.linspace(1.0, 2.0, 1001)), 1.0, atol=1e-15)
    assert o.psi1_hat(0.75) > 0 and o.psi1_hat(3.0) > 0


def test_psi1_scale_partition():
    # Thm PropertyPsi1: sum_{j>=0} |psi1(2^{-2j} w)|^2 = 1 for |w| > 1
    w = np.linspace(1.0 + 1e-12, 2.0**15, 200001)
    s = sum(o.psi1_hat(4.0 ** (-j) * w) ** 2 for j in range(0, 10))
    np.testing.assert_allclose(s, 1.0, rtol=0, atol=4e-15)


def test_finite_scale_sum():
    # eq. (sum_over_finite_scales): with j0 scales the sum is 1 on
    # 1 <= |w| <= 2^{2 j0 - 1} and decays to 0 at 2^{2 j0}
    for j0 in (1, 2, 3, 5):
        X = 2.0 ** (2 * j0 - 1)
        w = np.linspace(0.0, 4 * X, 40001)
        s = sum(o.psi1_hat(4.0 ** (-j) * w) ** 2 for j in range(j0))
        inside = (w >= 1.0) & (w <= X)
        np.testing.assert_allclose(s[inside], 1.0, atol=4e-15)
        assert np.all(s[w > 2 * X] == 0.0)
        assert np.all(s[w >= 2 * X] < 1e-30)  # cos(pi/2)^2 at the edge
        assert np.all(s[w <= 0.5] == 0.0)
        tail = (w > X) & (w < 2 * X)
        assert np.all(s[tail] <= 1.0)
        assert np.all(s[(w >= 1.1 * X) & (w < 2 * X)] < 1.0)  # strictly decaying


def test_psi2_values_and_support():
    # eq. (Psi2): psi2(0) = 1, psi2(+-1) = 0, supp = [-1, 1], even
    assert o.psi2_hat(0.0) == 1.0
    assert o.psi2_hat(1.0) == 0.0 and o.psi2_hat(-1.0) == 0.0
    assert np.all(o.psi2_hat(np.array([1.5, -1.01, 3.0])) == 0.0)
    np.testing.assert_allclose(o.psi2_hat(XS), o.psi2_hat(-XS), atol=0)


def test_psi2_three_term_lemma():
    # Lemma PropertyPsi2: psi2^2(w-1) + psi2^2(w) + psi2^2(w+1) = 1 for |w| <= 1
    w = np.linspace(-1.0, 1.0, 20001)
    s = o.psi2_hat(w - 1) ** 2 + o.psi2_hat(w) ** 2 + o.psi2_hat(w + 1) ** 2
    np.testing.assert_allclose(s, 1.0, atol=3e-15)


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4, 5])
def test_psi2_shear_partition(j):
    # Thm PropertyPsi2: sum_{k=-2^j}^{2^j} |psi2(k + 2^j w)|^2 = 1 for |w| <= 1
    w = np.linspace(-1.0, 1.0, 8001)
    J = 2**j
    s = sum(o.psi2_hat(k + J * w) ** 2 for k in range(-J, J + 1))
    np.testing.assert_allclose(s, 1.0, atol=3e-15)


def test_scaling_overlap():
    # eq. (overlapPsi1Phi): psi1^2 + varphi^2 = 1 on [1/2, 1]; varphi = 1 on
    # [-1/2, 1/2] and 0 from 1 on
    w = np.linspace(0.5, 1.0, 5001)
    np.testing.assert_allclose(o.psi1_hat(w) ** 2 + o.varphi(w) ** 2, 1.0, atol=3e-15)
    assert np.all(o.varphi(np.linspace(-0.5, 0.5, 101)) == 1.0)
    assert np.all(o.varphi(np.array([1.0, 1.5, -2.0])) == 0.0)


def test_phi_hat_cone_form():
    # eq. (phi): phi_hat = 1 on [-1/2,1/2]^2, and follows varphi of the
    # larger coordinate (second form of eq. (phi))
    g = np.linspace(-0.5, 0.5, 41)
    X1, X2 = np.meshgrid(g, g)
    assert np.all(o.phi_hat(X1, X2) == 1.0)
    rng = np.random.default_rng(3)
    a = rng.uniform(-1.5, 1.5, 2000)
    c = rng.uniform(-1.5, 1.5, 2000)
    m = np.maximum(np.abs(a), np.abs(c))
    expect = np.where(m <= 0.5, 1.0, np.where(m < 1.0, np.cos(0.5 * np.pi * o.v(2 * m - 1)), 0.0))
    np.testing.assert_allclose(o.phi_hat(a, c), expect, atol=1e-15)
