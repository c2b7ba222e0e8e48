"""Plain FP64 CPU oracle of the Fast Finite Shearlet Transform (FFST).

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the
CUDA library: only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  The product path never does, and
it shares no code, tables or constants with the CUDA sources.

Everything here is the paper's definition written out directly, in float64,
with NumPy's FFT as the only library step (Haeuser & Steidl, "Fast Finite
Shearlet Transform: a tutorial", arXiv:1202.1773):

* windows ``v``, ``b``, ``psi1_hat``, ``psi2_hat``, ``varphi``, ``phi_hat``:
  Sec. 2.1 eqs. (v), (b), (Psi1), (Psi2) and Sec. 2.4 eq. (phi);
* smooth shearlets (``smooth=True``): ``Phi_hat`` Sec. 2.4 eq. (Phi) and
  ``Psi1_hat`` Sec. 3.4 eqs. (newPsi1), (smoothPsi);
* cones C^h, C^v, C^x: Sec. 2.3;
* discretisation j0, a_j, s_{j,k}, the index set Omega: Sec. 3.1;
* frequency grid Xi (X = 2^{2 j0 - 1}): Sec. 3.5.1;
* plane index i <-> (kappa, j, k), eta = 2^{j0+2} - 3: Sec. 3.5.2;
* forward transform: Sec. 3.1 eq. (shearletTransform);
* inverse transform: Sec. 3.3 eq. (inverseShearletTransform);
* real-coefficient mirroring of the Nyquist row/column: Sec. 3.8.1;
* per-plane mean |c| d(i): Sec. 3.5.2 eq. (shearlet_meanvalue); soft and
  hard shrinkage of the coefficients (denoising, named in Sec. 1; textbook
  definitions, the paper gives none).

Readings of passages where the paper is silent or ambiguous (each is listed
in the project's design notes):

* axis: omega_1 runs along columns (x), omega_2 along rows (y); the
  coefficient stack is stored as ``[eta, M, N]`` (plane-major);
* grid: one step Delta = X / floor(max(M, N)/2) for both axes, xi = Delta *
  omega (the paper's odd-size symmetric linspace of the larger dimension,
  padded by one sample for even sizes and the last sample dropped, written
  as a product), so the lattice lies in [-Y, Y] x [-X, X] with Y <= X; the
  option ``spacing="per_axis"`` stretches each axis to [-X, X] instead;
* cone membership is decided exactly on the integer frequency indices;
* the Nyquist fix replaces psi(w1, -M/2) by sqrt((psi(w1)^2 + psi(-w1)^2)/2)
  (same for the column -N/2), which reproduces the paper's mirroring example
  and keeps sum_i psi_i^2 = 1.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, the paper's lemmas/theorems, printed tables and worked
examples, brute-force DFTs and invariants.  Square spectra are pinned by
transpose symmetry and the window pins; non-square spectra of the default
grid are pinned to the square ones (with one step Delta the M x N lattice is
a window of the max x max lattice), and the Sec. 3.5.1 statements that
single out that grid (one Delta, 1/4 < Delta <= 1, X >= Y) are tested.
"""

from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Sec. 2.1: auxiliary functions
# ---------------------------------------------------------------------------


def _v_poly_coeffs(k: int):
    """Coefficients a_n of v(x) = sum_n a_n x^n on [0, 1] for v'(x) = c x^k (x-1)^k, v(1) = 1
    (Sec. 3.4 remark construction_v): the binomial expansion of x^k (x-1)^k integrated
    term by term, c = (-1)^k (2k+1)! / (k!)^2 (a Beta integral)."""
    from math import comb, factorial

    c = (-1) ** k * factorial(2 * k + 1) / factorial(k) ** 2
    a = np.zeros(2 * k + 2)
    for m in range(k + 1):
        a[k + m + 1] = c * comb(k, m) * (-1) ** (k - m) / (k + m + 1)
    return a


def v(x, vfun="meyer"):
    """Auxiliary function v, Sec. 2.1 eq. (v) and its variants (Sec. 2.1, Sec. 3.4
    remark construction_v); 0 for x < 0 and 1 for x > 1 in every variant.

    * "meyer": 35x^4 - 84x^5 + 70x^6 - 20x^7 on [0, 1] (the paper's choice);
    * "quadratic": 2x^2 on [0, 1/2], 1 - 2(1 - x)^2 on [1/2, 1] (Sec. 2.1, the
      simpler choice the paper quotes);
    * ("poly", k): v'(x) = c x^k (x - 1)^k, v(1) = 1 (C^k shearlets; k = 3 is "meyer");
    * "cinf": s(x-1) / (s(x-1) + s(x)), s(x) = exp(-(1/(1+x)^2 + 1/(1-x)^2)) (C^infinity).
    """
    x = np.asarray(x, dtype=np.float64)
    if vfun == "meyer":
        # the polynomial in nested (Horner) form, which rounds less near x = 1
        poly = x**4 * (35.0 + x * (-84.0 + x * (70.0 - 20.0 * x)))
    elif vfun == "quadratic":
        poly = np.where(x <= 0.5, 2.0 * x * x, 1.0 - 2.0 * (1.0 - x) ** 2)
    elif isinstance(vfun, tuple) and vfun[0] == "poly":
        # Horner on [0, 1/2] and the symmetry v(x) = 1 - v(1 - x) above it,
        # which keeps the high-degree cancellation near x = 1 out
        a = _v_poly_coeffs(int(vfun[1]))

        def horner(y):
            out = np.zeros_like(y)
            for coef in a[::-1]:
                out = out * y + coef
            return out

        poly = np.where(x <= 0.5, horner(x), 1.0 - horner(1.0 - x))
    elif vfun == "cinf":
        with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
            s0 = np.exp(-(1.0 / x**2 + 1.0 / (2.0 - x) ** 2))          # s(x - 1)
            s1 = np.exp(-(1.0 / (1.0 + x) ** 2 + 1.0 / (1.0 - x) ** 2))  # s(x)
            poly = s0 / (s0 + s1)
        poly = np.where(x <= 0.0, 0.0, np.where(x >= 1.0, 1.0, poly))
    else:
        raise ValueError(f"unknown v variant {vfun!r}")
    return np.where(x < 0.0, 0.0, np.where(x > 1.0, 1.0, poly))


def b(omega, vfun="meyer"):
    """Bump b(omega), Sec. 2.1 eq. (b): supported on 1 <= |omega| <= 4."""
    w = np.abs(np.asarray(omega, dtype=np.float64))
    rise = np.sin(0.5 * np.pi * v(w - 1.0, vfun))
    fall = np.cos(0.5 * np.pi * v(0.5 * w - 1.0, vfun))
    return np.where((w >= 1.0) & (w <= 2.0), rise,
                    np.where((w > 2.0) & (w <= 4.0), fall, 0.0))


def psi1_hat(omega, vfun="meyer"):
    """Radial (scale) window, Sec. 2.1 eq. (Psi1): sqrt(b(2w)^2 + b(w)^2)."""
    return np.sqrt(b(2.0 * np.asarray(omega, dtype=np.float64), vfun) ** 2 + b(omega, vfun) ** 2)


def psi2_hat(omega, vfun="meyer"):
    """Directional window, Sec. 2.1 eq. (Psi2).

    sqrt(v(1 + w)) for w <= 0 and sqrt(v(1 - w)) for w > 0.
    """
    w = np.asarray(omega, dtype=np.float64)
    return np.where(w <= 0.0, np.sqrt(v(1.0 + w, vfun)), np.sqrt(v(1.0 - w, vfun)))


def varphi(omega, vfun="meyer"):
    """1-D scaling window of Sec. 2.4 (the function written varphi there)."""
    w = np.abs(np.asarray(omega, dtype=np.float64))
    mid = np.cos(0.5 * np.pi * v(2.0 * w - 1.0, vfun))
    return np.where(w <= 0.5, 1.0, np.where(w < 1.0, mid, 0.0))


def Phi_hat(w1, w2, vfun="meyer"):
    """Tensor-product scaling function varphi(w1) varphi(w2), Sec. 2.4 eq. (Phi)."""
    return varphi(w1, vfun) * varphi(w2, vfun)


def Psi1_hat(w1, w2, vfun="meyer"):
    """2-D radial window of the smooth shearlets, Sec. 3.4 eq. (newPsi1):
    sqrt(Phi_hat(w/4)^2 - Phi_hat(w)^2); supported in [-4, 4]^2 minus
    [-1/2, 1/2]^2."""
    w1 = np.asarray(w1, dtype=np.float64)
    w2 = np.asarray(w2, dtype=np.float64)
    d = Phi_hat(0.25 * w1, 0.25 * w2, vfun) ** 2 - Phi_hat(w1, w2, vfun) ** 2
    return np.sqrt(np.maximum(d, 0.0))


def phi_hat(xi1, xi2, vfun="meyer"):
    """Cone-adapted scaling function, Sec. 2.4 eq. (phi).

    varphi(xi1) where |xi2| <= |xi1|, varphi(xi2) where |xi1| < |xi2|.
    """
    xi1 = np.asarray(xi1, dtype=np.float64)
    xi2 = np.asarray(xi2, dtype=np.float64)
    return np.where(np.abs(xi2) <= np.abs(xi1), varphi(xi1, vfun), varphi(xi2, vfun))


# ---------------------------------------------------------------------------
# Sec. 3.1 / 3.5: discretisation, grid and indexing
# ---------------------------------------------------------------------------


def default_scales(rows: int, cols: int) -> int:
    """j0 = floor(1/2 log2 max(M, N)), Sec. 3.1 (table in Sec. 3.5.1).

    Integer arithmetic: floor(log2 n) is n.bit_length() - 1.
    """
    n = max(int(rows), int(cols))
    if n < 1:
        raise ValueError("empty image")
    return (n.bit_length() - 1) // 2


def num_planes(scales: int) -> int:
    """eta = 1 + sum_{j<j0} 2^{j+2} = 2^{j0+2} - 3, Sec. 3.5.2."""
    return 1 + sum(2 ** (j + 2) for j in range(scales))


def plane_table(scales: int):
    """Index i -> (kappa, j, k), Sec. 3.5.2.

    kappa is one of 'lowpass', 'h', 'v', 'seam'.  Plane 0 is the low-pass;
    then per scale j (J = 2^j), rotating counter-clockwise: h with k = 0,
    h with k = -1 .. -(J-1), the seam shearlet with k = -J, v with
    k = -(J-1) .. J-1, the seam shearlet with k = +J, and h with
    k = J-1 .. 1 (the paper's "k = 2^j, ..., 1" starts at the seam already
    listed, so the h run starts at J-1).
    """
    table = [("lowpass", -1, 0)]
    for j in range(scales):
        J = 2**j
        table.append(("h", j, 0))
        for k in range(-1, -J, -1):
            table.append(("h", j, k))
        table.append(("seam", j, -J))
        for k in range(-J + 1, J):
            table.append(("v", j, k))
        table.append(("seam", j, J))
        for k in range(J - 1, 0, -1):
            table.append(("h", j, k))
    assert len(table) == num_planes(scales)
    return table


def freq_index(L: int) -> np.ndarray:
    """Integer frequencies of Omega (Sec. 3.1) in FFT storage order.

    Omega covers -floor(L/2) .. ceil(L/2)-1; storage position p holds
    p for p < ceil(L/2) and p - L otherwise (numpy.fft order).
    """
    p = np.arange(L, dtype=np.int64)
    half = (L + 1) // 2
    return np.where(p < half, p, p - L)


def grid_extent(scales: int, max_scale: str = "max") -> float:
    """Largest grid value X, Sec. 3.5.1: X = 2^{2 j0 - 1} (the paper's choice X_3,
    the largest finest scale, its option maxScale = 'max') or X = 2^{2 j0 - 2}
    (X_2, the smallest reasonable finest scale, maxScale = 'min'); Sec. 3.5.1
    allows any X between the two."""
    if max_scale not in ("max", "min"):
        raise ValueError(f"max_scale must be 'max' or 'min', not {max_scale!r}")
    return 2.0 ** (2 * scales - (1 if max_scale == "max" else 2))


def grid_spacing(L: int, scales: int, max_scale: str = "max") -> float:
    """Grid step Delta for a dimension of length L spanning [-X, X], Sec. 3.5.1:
    X / floor(L/2).

    For odd L the paper's grid is linspace(-X, X, L), step 2X/(L-1) =
    X/floor(L/2); for even L it pads to L+1 and drops the last sample,
    which keeps the same step.
    """
    X = grid_extent(scales, max_scale)
    h = L // 2
    if h == 0:
        return 0.0
    return X / h


SPACINGS = ("common", "per_axis")


def grid_denominators(rows: int, cols: int, spacing: str = "common"):
    """Integer denominators (g_m, g_n) of the grid: xi2 = o2 X / g_m, xi1 = o1 X / g_n.

    "common" (default): Sec. 3.5.1 derives one step Delta from the larger
    dimension, N = max(M, N) ("without loss of generality"): both axes use
    Delta = X / floor(max(M, N)/2), so the lattice is Xi in [-Y, Y] x [-X, X]
    with Y = Delta floor(min(M, N)/2) <= X, the paper's "X >= Y", and Xi =
    Delta * Omega, the paper's remark that psi(Delta omega) on Omega gives the
    same spectra.  "per_axis": each axis spans [-X, X] with its own step
    X / floor(L/2) (Y = X).  Both are Parseval frames; they coincide for
    square images.
    """
    if spacing == "common":
        g = max(rows, cols) // 2
        return g, g
    if spacing == "per_axis":
        return rows // 2, cols // 2
    raise ValueError(f"spacing must be one of {SPACINGS}, not {spacing!r}")


def grid(rows: int, cols: int, scales: int, max_scale: str = "max", spacing: str = "common"):
    """Integer indices (o1, o2) and grid points (xi1, xi2), shape (M, N).

    xi1 (omega_1) varies along columns, xi2 (omega_2) along rows.
    """
    gm, gn = grid_denominators(rows, cols, spacing)
    X = grid_extent(scales, max_scale)
    o1 = freq_index(cols)[None, :] * np.ones((rows, 1), dtype=np.int64)
    o2 = freq_index(rows)[:, None] * np.ones((1, cols), dtype=np.int64)
    xi1 = o1 * (X / gn)
    xi2 = o2 * (X / gm)
    return o1, o2, xi1, xi2


def cones(rows: int, cols: int, o1, o2, spacing: str = "common"):
    """Masks of C^h, C^v and the seam lines C^x on the grid, Sec. 2.3.

    |xi2| < |xi1|  <=>  |o2| g_n < |o1| g_m (see ``grid_denominators``),
    decided in integers.  The origin belongs to none of them.
    """
    gm, gn = grid_denominators(rows, cols, spacing)
    lhs = np.abs(o2) * gn
    rhs = np.abs(o1) * gm
    nonzero = (o1 != 0) | (o2 != 0)
    ch = (lhs < rhs) & nonzero
    cv = (lhs > rhs) & nonzero
    cx = (lhs == rhs) & nonzero
    return ch, cv, cx


# ---------------------------------------------------------------------------
# Sec. 3.1 / 3.4.1 / 3.8.1: spectra
# ---------------------------------------------------------------------------


def _ratio(num, den, mask):
    out = np.zeros(num.shape, dtype=np.float64)
    np.divide(num, den, out=out, where=mask)
    return out


def spectrum_raw(rows: int, cols: int, scales: int, i: int, smooth: bool = False, vfun="meyer",
                 max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """Spectrum of plane i on Xi without the Nyquist fix, FFT storage order.

    Sec. 3.1 eq. (shearletTransform):
      low-pass:  phi_hat(xi)                                      (Sec. 2.4)
      h, |k|<J:  psi1(4^-j xi1) psi2(2^j xi2/xi1 + k) on C^h      (eq. horizontalShearlet)
      v, |k|<J:  psi1(4^-j xi2) psi2(2^j xi1/xi2 + k) on C^v      (eq. verticalShearlet)
      seam |k|=J: the glued sum psi^h + psi^v + psi^x: the h formula on
                  C^h and on the seam lines, the v formula on C^v.
    smooth=True gives the smooth shearlets of Sec. 3.4 eq. (smoothPsi): the
    radial factor of both cones is Psi1_hat(4^-j xi) (eq. newPsi1) and the
    low-pass is the tensor product Phi_hat(xi) (Sec. 2.4 eq. Phi).  vfun
    selects the auxiliary function v of every window (see ``v``), max_scale
    the grid extent X (see ``grid_extent``), spacing the grid step of a
    non-square image (see ``grid_denominators``).
    """
    kappa, j, k = plane_table(scales)[i]
    o1, o2, xi1, xi2 = grid(rows, cols, scales, max_scale, spacing)
    if kappa == "lowpass":
        return Phi_hat(xi1, xi2, vfun) if smooth else phi_hat(xi1, xi2, vfun)
    ch, cv, cx = cones(rows, cols, o1, o2, spacing)
    a = 4.0 ** (-j)
    J = 2.0**j
    if smooth:
        r = Psi1_hat(a * xi1, a * xi2, vfun)
        h_part = r * psi2_hat(J * _ratio(xi2, xi1, xi1 != 0) + k, vfun)
        v_part = r * psi2_hat(J * _ratio(xi1, xi2, xi2 != 0) + k, vfun)
    else:
        h_part = psi1_hat(a * xi1, vfun) * psi2_hat(J * _ratio(xi2, xi1, xi1 != 0) + k, vfun)
        v_part = psi1_hat(a * xi2, vfun) * psi2_hat(J * _ratio(xi1, xi2, xi2 != 0) + k, vfun)
    if kappa == "h":
        return np.where(ch, h_part, 0.0)
    if kappa == "v":
        return np.where(cv, v_part, 0.0)
    return np.where(ch | cx, h_part, 0.0) + np.where(cv, v_part, 0.0)


def nyquist_mirror(psi: np.ndarray) -> np.ndarray:
    """Real-coefficient fix of Sec. 3.8.1 on one spectrum (FFT order).

    For even M the row omega_2 = -M/2 has no conjugate partner inside the
    grid; its values are mirrored around the omega_1 = 0 axis and scaled by
    1/sqrt(2):  psi'(w1) = sqrt((psi(w1)^2 + psi(-w1)^2) / 2).  The same is
    done for the column omega_1 = -N/2 when N is even.  Where psi(w1) and
    psi(-w1) have disjoint supports this is the paper's mirrored-and-scaled
    row; where they are equal (axis shearlets) it leaves the row unchanged.
    """
    out = psi.copy()
    M, N = psi.shape
    if M % 2 == 0:
        r = M // 2
        row = psi[r, :]
        mirror = row[(-np.arange(N)) % N]
        out[r, :] = np.sqrt(0.5 * (row**2 + mirror**2))
    if N % 2 == 0:
        c = N // 2
        col = psi[:, c]
        mirror = col[(-np.arange(M)) % M]
        out[:, c] = np.sqrt(0.5 * (col**2 + mirror**2))
    return out


def spectrum(rows: int, cols: int, scales: int, i: int, real_fix: bool = True, smooth: bool = False,
             vfun="meyer", max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """Spectrum psi_hat_i of plane i (FFT storage order), fix applied by default.

    The fix is on by default, as the paper's ``realReal`` option (Sec. 3.5.3).
    """
    raw = spectrum_raw(rows, cols, scales, i, smooth, vfun, max_scale, spacing)
    return nyquist_mirror(raw) if real_fix else raw


def spectra(rows: int, cols: int, scales: int | None = None, real_fix: bool = True,
            smooth: bool = False, vfun="meyer", max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """Stack of all eta spectra, shape (eta, M, N), Sec. 3.5.2."""
    if scales is None:
        scales = default_scales(rows, cols)
    return np.stack([spectrum(rows, cols, scales, i, real_fix, smooth, vfun, max_scale, spacing)
                     for i in range(num_planes(scales))])


def frame_sum(rows: int, cols: int, scales: int | None = None, real_fix: bool = True,
              smooth: bool = False, vfun="meyer", max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """sum_i psi_hat_i^2 on the grid (Sec. 3.6, frame tightness)."""
    if scales is None:
        scales = default_scales(rows, cols)
    acc = np.zeros((rows, cols))
    for i in range(num_planes(scales)):
        acc += spectrum(rows, cols, scales, i, real_fix, smooth, vfun, max_scale, spacing) ** 2
    return acc


# ---------------------------------------------------------------------------
# Sec. 3.1 / 3.3: transforms
# ---------------------------------------------------------------------------


def forward_complex(f: np.ndarray, scales: int | None = None, real_fix: bool = True,
                    spacing: str = "common") -> np.ndarray:
    """c_i = ifft2(psi_hat_i * fft2(f)) as complex numbers, Sec. 3.1 eq. (shearletTransform)."""
    f = np.asarray(f, dtype=np.float64)
    M, N = f.shape
    if scales is None:
        scales = default_scales(M, N)
    F = np.fft.fft2(f)
    return np.stack([np.fft.ifft2(spectrum(M, N, scales, i, real_fix, spacing=spacing) * F)
                     for i in range(num_planes(scales))])


def forward_plane(F: np.ndarray, scales: int, i: int, smooth: bool = False, vfun="meyer",
                  max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """One real coefficient plane from a precomputed F = fft2(f)."""
    M, N = F.shape
    return np.real(np.fft.ifft2(spectrum(M, N, scales, i, smooth=smooth, vfun=vfun, max_scale=max_scale,
                                         spacing=spacing) * F))


def forward(f: np.ndarray, scales: int | None = None, smooth: bool = False, vfun="meyer",
            max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """Real coefficient stack (eta, M, N): the real part of ``forward_complex``.

    With the Nyquist fix the imaginary part is rounding noise (Sec. 3.8.1).
    """
    f = np.asarray(f, dtype=np.float64)
    M, N = f.shape
    if scales is None:
        scales = default_scales(M, N)
    F = np.fft.fft2(f)
    return np.stack([forward_plane(F, scales, i, smooth, vfun, max_scale, spacing)
                     for i in range(num_planes(scales))])


def adjoint(c: np.ndarray, scales: int | None = None, smooth: bool = False, vfun="meyer",
            max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """T* c = Re ifft2( sum_i psi_hat_i * fft2(c_i) ), Sec. 3.3.

    For a Parseval frame T* = T^-1 (Sec. 3.2, eq. shearlet_transform_as_matrix).
    """
    c = np.asarray(c, dtype=np.float64)
    _, M, N = c.shape
    if scales is None:
        scales = default_scales(M, N)
    acc = np.zeros((M, N), dtype=np.complex128)
    for i in range(num_planes(scales)):
        acc += spectrum(M, N, scales, i, smooth=smooth, vfun=vfun, max_scale=max_scale,
                        spacing=spacing) * np.fft.fft2(c[i])
    return np.real(np.fft.ifft2(acc))


def inverse(c: np.ndarray, scales: int | None = None, smooth: bool = False, vfun="meyer",
            max_scale: str = "max", spacing: str = "common") -> np.ndarray:
    """Re ifft2( sum_i psi_hat_i * fft2(c_i) / sum_i psi_hat_i^2 ), Sec. 3.3.

    Sec. 3.3 eq. (inverseShearletTransform) sums the products; the division
    by sum_i psi_hat_i^2 (identically 1 for the Parseval frame of Sec. 3.2,
    up to rounding) is kept as an explicit normalisation.
    """
    c = np.asarray(c, dtype=np.float64)
    _, M, N = c.shape
    if scales is None:
        scales = default_scales(M, N)
    acc = np.zeros((M, N), dtype=np.complex128)
    den = np.zeros((M, N))
    for i in range(num_planes(scales)):
        s = spectrum(M, N, scales, i, smooth=smooth, vfun=vfun, max_scale=max_scale, spacing=spacing)
        acc += s * np.fft.fft2(c[i])
        den += s * s
    return np.real(np.fft.ifft2(acc / den))


def forward_with(psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Real coefficient stack from precomputed spectra psi = spectra(M, N, ...):
    c_i = Re ifft2(psi_i * fft2(f)), Sec. 3.1 eq. (shearletTransform).  Sec. 3.5
    precomputes the spectra once and uses them for both directions; this is
    that form, for loops that transform many images of one size."""
    F = np.fft.fft2(np.asarray(f, dtype=np.float64))
    return np.stack([np.real(np.fft.ifft2(psi[i] * F)) for i in range(psi.shape[0])])


def adjoint_with(psi: np.ndarray, c: np.ndarray) -> np.ndarray:
    """T* c = Re ifft2(sum_i psi_i * fft2(c_i)) from precomputed spectra (Sec. 3.3)."""
    acc = np.zeros(psi.shape[1:], dtype=np.complex128)
    for i in range(psi.shape[0]):
        acc += psi[i] * np.fft.fft2(np.asarray(c[i], dtype=np.float64))
    return np.real(np.fft.ifft2(acc))


def mean_abs(c: np.ndarray) -> np.ndarray:
    """d(i) = 1/(MN) sum |c(., ., i)|, Sec. 3.5.2 eq. (shearlet_meanvalue)."""
    c = np.asarray(c)
    return np.abs(c).reshape(c.shape[0], -1).mean(axis=1)


def shrink(c: np.ndarray, tau, mode: str) -> np.ndarray:
    """Per-plane coefficient shrinkage for denoising (an application the
    paper names in Sec. 1; it defines no operator).  The textbook forms, with
    tau[i] the threshold of plane i (a scalar applies to every plane):

    * soft: sign(c) * max(|c| - tau, 0)
    * hard: c where |c| > tau, else 0
    """
    c = np.asarray(c, dtype=np.float64)
    t = np.broadcast_to(np.asarray(tau, dtype=np.float64).reshape(-1, *([1] * (c.ndim - 1))), c.shape) \
        if np.ndim(tau) else np.full(c.shape, float(tau))
    if mode == "soft":
        return np.sign(c) * np.maximum(np.abs(c) - t, 0.0)
    if mode == "hard":
        return np.where(np.abs(c) > t, c, 0.0)
    raise ValueError(f"unknown shrinkage mode {mode!r}")


# ---------------------------------------------------------------------------
# Sec. 3.8.2: complex (one-sided) shearlets
# ---------------------------------------------------------------------------


def half_plane(rows: int, cols: int, scales: int, i: int, spacing: str = "common") -> np.ndarray:
    """Selector h_i(omega) of the one-sided shearlet of plane i (FFT order).

    Sec. 3.8.2 builds complex shearlets by keeping one side of each spectrum;
    the paper does not say which side or what happens on the grid's
    self-paired lines.  The reading used here: on C^h and the seam lines the
    side omega_1 > 0, on C^v the side omega_2 > 0; on the Nyquist column
    (omega_1 = -N/2) the side omega_2 > 0 and on the Nyquist row
    (omega_2 = -M/2) the side omega_1 > 0, so that of every pair
    {omega, -omega} exactly one point is kept (h + h(-.) = 1); the
    self-conjugate points (omega = -omega on the grid) get 1/2; the low-pass
    stays two-sided (h = 1/2 everywhere, so its complex coefficient is the
    real one).
    """
    kappa, _, _ = plane_table(scales)[i]
    if kappa == "lowpass":
        return np.full((rows, cols), 0.5)
    o1, o2, _, _ = grid(rows, cols, scales, spacing=spacing)
    ch, cv, cx = cones(rows, cols, o1, o2, spacing)
    ny_c = (cols % 2 == 0) & (o1 == -(cols // 2))
    ny_r = (rows % 2 == 0) & (o2 == -(rows // 2))
    s_h = np.where(ny_c, np.sign(np.where(ny_r, 0, o2)), np.sign(o1))
    s_v = np.where(ny_r, np.sign(np.where(ny_c, 0, o1)), np.sign(o2))
    s = np.where(ch | cx, s_h, np.where(cv, s_v, 0))
    return 0.5 * (1.0 + s)


def forward_onesided(f: np.ndarray, scales: int | None = None, **opts) -> np.ndarray:
    """Complex coefficients z_i = sqrt(2) ifft2(psi_hat_i h_i fft2(f)), i >= 1, and
    z_0 = ifft2(psi_hat_0 fft2(f)) (Sec. 3.8.2), shape (eta, M, N), complex.

    With h_i + h_i(-.) = 1, Re z_i = c_i / sqrt(2) for i >= 1 and z_0 = c_0
    for a real image (the frame property of the real transform carries over).
    """
    f = np.asarray(f, dtype=np.float64)
    M, N = f.shape
    if scales is None:
        scales = default_scales(M, N)
    F = np.fft.fft2(f)
    out = []
    for i in range(num_planes(scales)):
        psi = spectrum(M, N, scales, i, **opts)
        w = np.sqrt(2.0) * half_plane(M, N, scales, i, opts.get("spacing", "common")) if i else 1.0
        out.append(np.fft.ifft2(psi * w * F))
    return np.stack(out)


def inverse_onesided(z: np.ndarray, scales: int | None = None, **opts) -> np.ndarray:
    """Image from one-sided coefficients: the real transform's inverse of
    c_0 = Re z_0, c_i = sqrt(2) Re z_i (Sec. 3.8.2 with Sec. 3.3)."""
    z = np.asarray(z)
    c = np.sqrt(2.0) * np.real(z)
    c[0] = np.real(z[0])
    return inverse(c, scales, **opts)
