"""Shearlet-regularised deconvolution through the differentiable transform.

Recovers an image x from a blurred, noisy observation y = A x + n by
minimising

    J(x) = 1/2 ||A x - y||^2 + lam * sum_{i >= 1} sum_m sqrt(c_i(m)^2 + eps^2),
    c = T x  (the shearlet coefficients, plane 0 = low-pass unpenalised),

with accelerated gradient steps (FISTA momentum).  The shearlet term goes
through ``shearlet_transform`` (forward: ffst_forward, backward: the
hand-written ffst_adjoint); the blur A is the application's periodic
Gaussian operator, applied with torch.fft.  A Gaussian blur with unit sum
has ||A|| <= 1 and the shearlet frame is Parseval (||T|| = 1), so the
gradient is (1 + lam/eps)-Lipschitz and the step is 1 / (1 + lam/eps).
"""

from __future__ import annotations

import math

import numpy as np

from . import shearlet_transform


def gaussian_psf(rows: int, cols: int, sigma: float = 2.0, radius: int = 8) -> np.ndarray:
    """Periodic sampled Gaussian (support |dy|, |dx| <= radius), unit sum, centred at (0, 0)."""
    psf = np.zeros((rows, cols))
    ax = np.arange(-radius, radius + 1)
    g = np.exp(-(ax[:, None] ** 2 + ax[None, :] ** 2) / (2.0 * sigma**2))
    g /= g.sum()
    for a, dy in enumerate(ax):
        for b, dx in enumerate(ax):
            psf[dy % rows, dx % cols] += g[a, b]
    return psf


class Blur:
    """Periodic convolution with a PSF (its transfer function is real and even)."""

    def __init__(self, psf: np.ndarray, device):
        import torch

        self.H = torch.fft.rfft2(torch.from_numpy(psf).to(device=device, dtype=torch.float32))
        self.shape = psf.shape

    def __call__(self, x):
        import torch

        return torch.fft.irfft2(torch.fft.rfft2(x) * self.H, s=self.shape)

    adjoint = __call__  # the Gaussian PSF is symmetric, so A^T = A


def objective(x, y, blur, plan, lam: float, eps: float):
    """J(x) as a differentiable torch scalar."""
    c = shearlet_transform(x, plan)
    fid = 0.5 * ((blur(x) - y) ** 2).sum()
    reg = lam * (c[1:] ** 2 + eps * eps).sqrt().sum()
    return fid + reg


def deconvolve(y, plan, blur: Blur, lam: float = 5e-3, eps: float = 1e-3, steps: int = 200, callback=None):
    """FISTA-accelerated gradient descent on J from x0 = y; returns (x, [J per step])."""
    import torch

    step = 1.0 / (1.0 + lam / eps)
    x = y.clone()
    z = y.clone()
    tk = 1.0
    history = []
    for it in range(steps):
        z = z.detach().requires_grad_(True)
        J = objective(z, y, blur, plan, lam, eps)
        (g,) = torch.autograd.grad(J, z)
        history.append(float(J.detach()))
        with torch.no_grad():
            x_new = z - step * g
            t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * tk * tk))
            z = x_new + ((tk - 1.0) / t_new) * (x_new - x)
            x, tk = x_new, t_new
        if callback:
            callback(it, x, J)
    return x.detach(), history
