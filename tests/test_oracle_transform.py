"""Pins of the oracle's forward / inverse / adjoint (Sec. 3.1 - 3.3, 3.6, 3.8)."""

import os

import numpy as np
import pytest

from oracle import ffst_oracle as o


def _dft(L):
    p = np.arange(L)
    return np.exp(-2j * np.pi * np.outer(p, p) / L)


@pytest.mark.parametrize("n", [8, 16])
def test_forward_equals_brute_force_dft(n):
    # eq. (shearletTransform) with explicit DFT matrices instead of numpy.fft
    rng = np.random.default_rng(10 + n)
    f = rng.standard_normal((n, n))
    W = _dft(n)
    Winv = np.conj(W) / n
    Fhat = W @ f @ W.T
    S = o.spectra(n, n)
    expect = np.stack([np.real(Winv @ (S[i] * Fhat) @ Winv.T) for i in range(S.shape[0])])
    np.testing.assert_allclose(o.forward(f), expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (12, 16)])
def test_forward_equals_time_domain_correlation(shape):
    # Sec. 3.1: c(i, m) = <f, psi_{i}(. - t_m)> with the time-domain shearlet
    # psi_i = ifft2(psi_hat_i); evaluated as an explicit circular correlation
    M, N = shape
    rng = np.random.default_rng(1)
    f = rng.standard_normal((M, N))
    S = o.spectra(M, N)
    c = o.forward(f)
    for i in range(S.shape[0]):
        psi = np.fft.ifft2(S[i])
        assert np.abs(psi.imag).max() < 1e-15  # real shearlets after the fix
        psi = psi.real
        direct = np.empty((M, N))
        for m1 in range(M):
            for m2 in range(N):
                direct[m1, m2] = np.sum(f * np.roll(psi, (m1, m2), axis=(0, 1)))
        np.testing.assert_allclose(c[i], direct, rtol=0, atol=1e-13)


def test_parseval_frame_matrix_8x8():
    # Sec. 3.2 theorem: the system is a Parseval frame, i.e. U^T U = I for the
    # matrix U whose rows are all translated shearlets (brute force, 8x8)
    n = 8
    S = o.spectra(n, n)
    rows = []
    for i in range(S.shape[0]):
        psi = np.real(np.fft.ifft2(S[i]))
        for m1 in range(n):
            for m2 in range(n):
                rows.append(np.roll(psi, (m1, m2), axis=(0, 1)).ravel())
    U = np.array(rows)
    assert U.shape == (S.shape[0] * n * n, n * n)
    np.testing.assert_allclose(U.T @ U, np.eye(n * n), rtol=0, atol=1e-14)
    # and the oracle's forward is that matrix
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n, n))
    np.testing.assert_allclose(o.forward(f).ravel(), U @ f.ravel(), atol=1e-14)


@pytest.mark.parametrize("shape", [(64, 64), (48, 80), (63, 65), (128, 96), (32, 7)])
def test_parseval_and_reconstruction(shape, golden_dir):
    # Parseval: sum_i ||c_i||^2 = ||f||^2; reconstruction error about 2e-15
    # for a random image (Sec. 3.6)
    with open(os.path.join(golden_dir, "accuracy.txt")) as fh:
        acc = dict(l.split() for l in fh if l.strip() and not l.startswith("#"))
    rng = np.random.default_rng(7)
    f = rng.uniform(0.0, 1.0, shape)
    c = o.forward(f)
    assert abs(np.sum(c**2) / np.sum(f**2) - 1.0) <= 1e-13
    rec = o.inverse(c)
    assert np.abs(rec - f).max() <= 10 * float(acc["reconstruction_max_abs"])
    assert np.abs(o.adjoint(c) - f).max() <= 1e-13


def test_inverse_vs_adjoint_differ_by_rounding():
    rng = np.random.default_rng(8)
    c = rng.standard_normal((29, 64, 64))
    assert np.abs(o.inverse(c) - o.adjoint(c)).max() <= 1e-13


@pytest.mark.parametrize("shape", [(64, 64), (48, 80)])
def test_adjoint_dot_product(shape):
    # <T x, c> = <x, T* c>
    rng = np.random.default_rng(9)
    x = rng.standard_normal(shape)
    c = rng.standard_normal((o.num_planes(o.default_scales(*shape)),) + shape)
    lhs = np.sum(o.forward(x) * c)
    rhs = np.sum(x * o.adjoint(c))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("shape", [(64, 64), (48, 80), (16, 32)])
def test_real_coefficients_only_with_fix(shape):
    # Sec. 3.8.1: without the fix the finest-scale non-axis planes get an
    # imaginary part for even sizes; with it the imaginary part is rounding
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 1.0, shape)
    fixed = o.forward_complex(f)
    assert np.abs(fixed.imag).max() <= 1e-14 * max(1.0, np.abs(fixed.real).max())
    raw = o.forward_complex(f, real_fix=False)
    table = o.plane_table(o.default_scales(*shape))
    jmax = max(j for _, j, _ in table)
    imag = np.abs(raw.imag).mean(axis=(1, 2))
    for i, (kap, j, k) in enumerate(table):
        if j == jmax and k != 0:
            assert imag[i] > 1e-6, (i, kap, j, k)
        if kap == "lowpass" or (kap in ("h", "v") and k == 0):
            assert imag[i] <= 1e-15


def test_shift_equivariance():
    # translation invariance (Sec. 1 / Sec. 3.7 remark (ii)): the transform of a
    # circularly shifted image is the shifted transform
    rng = np.random.default_rng(12)
    f = rng.standard_normal((48, 64))
    c = o.forward(f)
    cs = o.forward(np.roll(f, (5, -9), axis=(0, 1)))
    np.testing.assert_allclose(cs, np.roll(c, (5, -9), axis=(1, 2)), atol=1e-13)


def test_transpose_equivariance():
    # square image: forward(f^T) swaps h(j,k) <-> v(j,k) planes, transposed
    rng = np.random.default_rng(13)
    f = rng.standard_normal((32, 32))
    table = o.plane_table(2)
    c = o.forward(f)
    ct = o.forward(f.T)
    for i, (kap, j, k) in enumerate(table):
        p = table.index(("v" if kap == "h" else "h", j, k)) if kap in ("h", "v") else i
        np.testing.assert_allclose(ct[i], c[p].T, atol=1e-13)


def test_mean_abs_vector():
    # eq. (shearlet_meanvalue) on a constant image: only the low-pass plane
    # carries energy, d(0) = |value|
    f = np.full((32, 32), 0.75)
    d = o.mean_abs(o.forward(f))
    assert d[0] == pytest.approx(0.75, abs=1e-14)
    assert np.all(d[1:] <= 1e-14)


def test_shrink_closed_forms():
    # textbook soft / hard thresholding, per plane thresholds broadcast over the plane
    c = np.array([[[3.0, -0.5], [1.0, -2.5]], [[0.2, -0.2], [4.0, 0.0]]])
    tau = np.array([1.0, 0.5])
    np.testing.assert_array_equal(o.shrink(c, tau, "soft"), [[[2.0, 0.0], [0.0, -1.5]], [[0.0, 0.0], [3.5, 0.0]]])
    np.testing.assert_array_equal(o.shrink(c, tau, "hard"), [[[3.0, 0.0], [0.0, -2.5]], [[0.0, 0.0], [4.0, 0.0]]])
    np.testing.assert_array_equal(o.shrink(c, 0.0, "soft"), c)  # zero threshold: identity
    np.testing.assert_array_equal(o.shrink(c, 0.0, "hard"), np.where(c != 0, c, 0.0))
    with pytest.raises(ValueError):
        o.shrink(c, 1.0, "median")


def test_shrink_invariants():
    rng = np.random.default_rng(4)
    c = rng.normal(size=(3, 16, 16))
    a, b = 0.3, 0.45
    s = o.shrink(c, a, "soft")
    assert np.all(np.abs(s) <= np.abs(c)) and np.all(s * c >= 0)  # shrinks toward 0, keeps signs
    np.testing.assert_allclose(o.shrink(s, b, "soft"), o.shrink(c, a + b, "soft"), atol=1e-15)  # semigroup
    h = o.shrink(c, a, "hard")
    np.testing.assert_array_equal(o.shrink(h, a, "hard"), h)  # idempotent
    # soft = hard minus tau*sign on the kept entries
    np.testing.assert_allclose(s, np.where(h != 0, h - a * np.sign(h), 0.0), atol=1e-15)
    # the low-pass plane of a constant image is the value itself: shrinking it is a scalar map
    d = o.forward(np.full((32, 32), 0.75))
    np.testing.assert_allclose(o.shrink(d, 0.25, "soft")[0], 0.5, atol=1e-13)


def test_precomputed_spectra_forms_agree():
    # forward_with / adjoint_with (spectra computed once, Sec. 3.5) give the
    # same stack and image as the per-call forms
    rng = np.random.default_rng(40)
    f = rng.standard_normal((32, 48))
    psi = o.spectra(32, 48)
    np.testing.assert_allclose(o.forward_with(psi, f), o.forward(f), rtol=0, atol=1e-14)
    c = rng.standard_normal(psi.shape)
    np.testing.assert_allclose(o.adjoint_with(psi, c), o.adjoint(c), rtol=0, atol=1e-13)
