"""Pins of the oracle's one-sided (complex) shearlets, Sec. 3.8.2.

The paper states that one-sided spectra give complex shearlets with the
frame properties of the real case; the reading (which side, the grid's
self-paired lines) is documented in ``half_plane``.  What is fixed by the
mathematics: exactly one of each pair {omega, -omega} is kept, the spectra
of z_i vanish on the other side, Re z_i = c_i / sqrt(2), the image comes
back from Re z, and the imaginary part is the real transform with the
multiplier -i sign(omega) psi_hat (a Hilbert pair).
"""

import numpy as np
import pytest

from oracle import ffst_oracle as o


def _neg(a):
    # a(-omega) on the FFT grid
    return np.roll(a[::-1, ::-1], 1, axis=(0, 1))


@pytest.mark.parametrize("rows,cols,scales", [(32, 32, 2), (64, 64, 3), (48, 64, 3)])
def test_half_plane_pairs(rows, cols, scales):
    for i in range(o.num_planes(scales)):
        h = o.half_plane(rows, cols, scales, i)
        np.testing.assert_array_equal(h + _neg(h), 1.0)  # exactly one of each pair
        assert set(np.unique(h)) <= {0.0, 0.5, 1.0}
        if i:  # 1/2 only at the self-conjugate grid points (omega = -omega mod the grid)
            o1, o2, _, _ = o.grid(rows, cols, scales)
            selfc = (np.mod(2 * o1, cols) == 0) & (np.mod(2 * o2, rows) == 0)
            np.testing.assert_array_equal(h == 0.5, selfc)


@pytest.mark.parametrize("rows,cols,scales", [(64, 64, 3), (48, 64, 3)])
def test_onesided_coefficients(rows, cols, scales):
    rng = np.random.default_rng(5)
    f = rng.normal(size=(rows, cols))
    z = o.forward_onesided(f, scales)
    c = o.forward(f, scales)
    np.testing.assert_allclose(z[0].real, c[0], atol=1e-13)
    assert np.abs(z[0].imag).max() <= 1e-13
    np.testing.assert_allclose(np.sqrt(2.0) * z[1:].real, c[1:], atol=1e-13)  # Re z_i = c_i / sqrt(2)
    np.testing.assert_allclose(o.inverse_onesided(z, scales), f, atol=1e-12)  # reconstruction
    # one-sided: the spectrum of z_i vanishes wherever h_i = 0
    for i in range(1, z.shape[0]):
        h = o.half_plane(rows, cols, scales, i)
        assert np.abs(np.fft.fft2(z[i])[h == 0]).max() <= 1e-10 * max(1.0, np.abs(np.fft.fft2(f)).max())
    # Hilbert pair: Im z_i sqrt(2) is the real transform with multiplier -i sign(omega) psi_hat
    F = np.fft.fft2(f)
    for i in range(1, z.shape[0]):
        psi = o.spectrum(rows, cols, scales, i)
        sgn = 2.0 * o.half_plane(rows, cols, scales, i) - 1.0
        d = np.fft.ifft2(-1j * sgn * psi * F)
        assert np.abs(d.imag).max() <= 1e-12
        np.testing.assert_allclose(np.sqrt(2.0) * z[i].imag, d.real, atol=1e-12)


def test_onesided_energy():
    # |z_i|^2 sums to |c_i|^2 up to the self-conjugate grid points
    rng = np.random.default_rng(6)
    f = rng.normal(size=(64, 64))
    z = o.forward_onesided(f, 3)
    c = o.forward(f, 3)
    assert abs((np.abs(z) ** 2).sum() - (c**2).sum()) <= 1e-2 * (c**2).sum()
    # a plane without energy at the self-conjugate points keeps it exactly
    o1, o2, _, _ = o.grid(64, 64, 3)
    selfc = (np.mod(2 * o1, 64) == 0) & (np.mod(2 * o2, 64) == 0)
    for i in range(1, z.shape[0]):
        if np.all(o.spectrum(64, 64, 3, i)[selfc] == 0):
            assert (np.abs(z[i]) ** 2).sum() == pytest.approx((c[i] ** 2).sum(), rel=1e-12)
