"""FP64 reference of the shearlet-regularised deconvolution (test infrastructure only).

The same objective, step size and FISTA momentum as the GPU application,
written with NumPy and the FFST oracle's forward/adjoint:

    J(x) = 1/2 ||A x - y||^2 + lam * sum_{i>=1} sum_m sqrt(c_i(m)^2 + eps^2),  c = T x,
    grad J = A^T (A x - y) + lam * T^T (c / sqrt(c^2 + eps^2))  (plane 0 zeroed),
    step 1/(1 + lam/eps), t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2.

The spectra are computed once per call (``psi``) and used for every forward
and adjoint of the iteration, as the paper precomputes them (Sec. 3.5).
"""

import numpy as np

from . import ffst_oracle as o


def blur(x, psf):
    return np.real(np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(psf)))


def objective(x, y, psf, lam, eps, psi):
    c = o.forward_with(psi, x)
    return 0.5 * np.sum((blur(x, psf) - y) ** 2) + lam * np.sum(np.sqrt(c[1:] ** 2 + eps * eps))


def gradient(x, y, psf, lam, eps, psi):
    c = o.forward_with(psi, x)
    r = c / np.sqrt(c * c + eps * eps)
    r[0] = 0.0
    return blur(blur(x, psf) - y, psf) + lam * o.adjoint_with(psi, r)


def deconvolve(y, psf, lam=5e-3, eps=1e-3, steps=200, scales=None):
    M, N = y.shape
    psi = o.spectra(M, N, scales)
    step = 1.0 / (1.0 + lam / eps)
    x = y.copy()
    z = y.copy()
    tk = 1.0
    hist = []
    for _ in range(steps):
        hist.append(objective(z, y, psf, lam, eps, psi))
        x_new = z - step * gradient(z, y, psf, lam, eps, psi)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        z = x_new + ((tk - 1.0) / t_new) * (x_new - x)
        x, tk = x_new, t_new
    return x, hist
