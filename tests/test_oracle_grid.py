"""Pins of the oracle's discretisation, indexing and spectra (Sec. 3.1, 3.5, 3.6, 3.8)."""

import os

import numpy as np
import pytest

from oracle import ffst_oracle as o


def _read(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_scales_table(golden_dir):
    # Sec. 3.5.1 table: N -> j0
    for lo, hi, j0 in _read(golden_dir, "scales_table.txt"):
        for n in range(int(lo), int(hi) + 1):
            assert o.default_scales(n, n) == int(j0)
            assert o.default_scales(3, n) == int(j0)  # larger dimension decides


def test_eta_and_per_scale_counts(golden_dir):
    # Sec. 3.5.2 tables: eta(j0) and planes per scale
    rows = _read(golden_dir, "eta_table.txt")
    for tag, a, b in rows:
        if tag == "eta":
            assert o.num_planes(int(a)) == int(b)
            assert len(o.plane_table(int(a))) == int(b)
            assert 2 ** (int(a) + 2) - 3 == int(b)
    table = o.plane_table(4)
    counts = {}
    for kappa, j, k in table:
        counts[j] = counts.get(j, 0) + 1
    for tag, a, b in rows:
        if tag == "per_scale":
            assert counts[int(a)] == int(b)


def test_index_order_text():
    # Sec. 3.5.2: per scale, h k=0, h k=-1..-(J-1), seam k=-J, v k=-(J-1)..J-1,
    # seam k=+J, then h with decreasing positive shear
    t = o.plane_table(3)
    assert t[0] == ("lowpass", -1, 0)
    assert t[1:5] == [("h", 0, 0), ("seam", 0, -1), ("v", 0, 0), ("seam", 0, 1)]
    assert t[5:13] == [("h", 1, 0), ("h", 1, -1), ("seam", 1, -2), ("v", 1, -1),
                       ("v", 1, 0), ("v", 1, 1), ("seam", 1, 2), ("h", 1, 1)]
    s2 = t[13:29]
    assert s2[0] == ("h", 2, 0) and s2[4] == ("seam", 2, -4) and s2[12] == ("seam", 2, 4)
    assert [k for _, _, k in s2[5:12]] == list(range(-3, 4))
    assert [k for _, _, k in s2[13:]] == [3, 2, 1]


def test_grid_spacing_statements():
    # Sec. 3.5.1: Delta = 2^{2 j0}/(N-1) for odd N; Delta = 1 iff N = 2^{2j0}+1;
    # 1/4 < Delta <= 1 over the sizes of the j0 table
    for j0 in range(1, 6):
        assert o.grid_spacing(2 ** (2 * j0) + 1, j0) == 1.0
    for n in range(4, 1025):
        j0 = o.default_scales(n, n)
        d = o.grid_spacing(n if n % 2 else n + 1, j0)
        assert 0.25 < d <= 1.0
        if n % 2:
            assert d == pytest.approx(2.0 ** (2 * j0) / (n - 1), rel=1e-15)


def test_grid_matches_padded_linspace():
    # Sec. 3.5.1: for even N pad to N+1, take linspace(-X, X, N+1), drop the
    # last sample; in fftshift order that is the oracle's grid
    for n, j0 in [(8, 1), (16, 2), (64, 3), (15, 1), (33, 2), (100, 3)]:
        X = 2.0 ** (2 * j0 - 1)
        odd = n if n % 2 else n + 1
        lin = np.linspace(-X, X, odd)[:n]
        ours = np.fft.fftshift(o.freq_index(n) * o.grid_spacing(n, j0))
        np.testing.assert_allclose(ours, lin, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (64, 64), (48, 80), (63, 65), (128, 96), (30, 4)])
def test_frame_tightness(golden_dir, shape):
    # Sec. 3.6: max |sum_i psi_i^2 - 1| about 8e-15 (40 times machine precision)
    paper = float(dict(_read(golden_dir, "accuracy.txt"))["frame_tightness_max_abs"])
    s = o.frame_sum(*shape)
    assert np.abs(s - 1.0).max() <= 1.25 * paper  # <= 1e-14


def test_frame_tightness_512():
    s = o.frame_sum(512, 512)
    assert np.abs(s - 1.0).max() <= 1e-14


def test_fp64_divisor_rounds_to_one_in_fp32():
    # the inverse's normalisation sum_i psi_i^2 is exactly 1.0f in float32
    for shape in [(64, 64), (48, 80), (256, 256)]:
        s = o.frame_sum(*shape)
        assert np.all(s.astype(np.float32) == np.float32(1.0))


def test_mirror_toy_example(golden_dir):
    # Sec. 3.8.1 Figure mirroring: the first row [8 6 4 2 0 0 0 0 0] becomes
    # (1/sqrt 2)[8 6 4 2 0 2 4 6 8].  Embed it as the Nyquist column of an
    # even-width spectrum: the column omega_1 = -N/2 is mirrored in omega_2.
    rows = dict((r[0], [float(x) for x in r[1:]]) for r in _read(golden_dir, "mirror_toy.txt"))
    before = np.array(rows["before"])
    after = np.array(rows["after_times_sqrt2"]) / np.sqrt(2.0)
    M = before.size  # 9 (odd): omega_2 = -4..4
    psi = np.zeros((M, 10))
    psi[:, 5] = np.fft.ifftshift(before)  # column omega_1 = -5 (Nyquist)
    out = o.nyquist_mirror(psi)
    np.testing.assert_allclose(np.fft.fftshift(out[:, 5]), after, atol=1e-15)
    # every other column untouched (M odd: no Nyquist row)
    np.testing.assert_array_equal(np.delete(out, 5, axis=1), np.delete(psi, 5, axis=1))
    # an axis-symmetric row is kept unchanged ("h and v kept")
    sym = np.zeros((10, 9))
    sym[5, :] = np.fft.ifftshift([1, 2, 3, 4, 5, 4, 3, 2, 1])
    np.testing.assert_allclose(o.nyquist_mirror(sym)[5], sym[5], atol=1e-15)


def _centroid_angle(rows, cols, scales, i):
    # angle (mod pi) of the psi^2-weighted doubled-angle centroid of plane i
    _, _, xi1, xi2 = o.grid(rows, cols, scales)
    w = o.spectrum(rows, cols, scales, i) ** 2
    z = np.sum(w * np.exp(2j * np.arctan2(xi2, xi1)))
    return (np.angle(z) / 2.0) % np.pi


def test_orientation_and_counter_clockwise_order():
    # Sec. 3.1: psi2(2^j xi2/xi1 + k) peaks where xi2/xi1 = -k 2^-j, and
    # Sec. 3.5.2: indices rotate counter-clockwise from the horizontal h k=0
    M = N = 64
    j0 = 3  # X = 32, Delta = 1: xi equals the integer frequency
    table = o.plane_table(j0)
    # h, j=1, k=-1: value 1 at xi = (4, 2) (ratio 1/2, |4^-1 xi1| = 1)
    i = table.index(("h", 1, -1))
    P = o.spectrum(M, N, j0, i)
    assert P[2, 4] == pytest.approx(1.0, abs=1e-15)
    assert P[-2, 4] == 0.0  # mirrored ratio -1/2 is another shear's wedge
    assert P[4, 2] == 0.0   # transposed point lies in the vertical cone
    # v, j=1, k=1: xi1/xi2 = -1/2 at (xi1, xi2) = (-2, 4)
    i = table.index(("v", 1, 1))
    P = o.spectrum(M, N, j0, i)
    assert P[4, -2] == pytest.approx(1.0, abs=1e-15)
    assert P[4, 2] == 0.0
    # counter-clockwise: centroid angle grows monotonically within a scale
    for j in range(j0):
        idx = [n for n, (kap, jj, k) in enumerate(table) if jj == j]
        ang = np.array([_centroid_angle(M, N, j0, n) for n in idx])
        ang[0] = 0.0 if ang[0] > np.pi / 2 else ang[0]  # h k=0 sits at 0 == pi
        assert np.all(np.diff(ang) > 0), (j, ang)
        # seams at 45 and 135 degrees, v k=0 at 90 degrees
        J = 2**j
        assert ang[J] == pytest.approx(np.pi / 4, abs=1e-6)
        assert ang[2 * J] == pytest.approx(np.pi / 2, abs=1e-6)
        assert ang[3 * J] == pytest.approx(3 * np.pi / 4, abs=1e-6)


def test_lowpass_and_support_bands():
    # Sec. 2.4 / 3.5.1: low-pass = 1 on |xi|_inf <= 1/2; scale j lives on
    # 2^{2j-1} <= |xi|_inf <= 2^{2j+2}
    M = N = 64
    j0 = 3
    _, _, xi1, xi2 = o.grid(M, N, j0)
    m = np.maximum(np.abs(xi1), np.abs(xi2))
    low = o.spectrum(M, N, j0, 0)
    assert np.all(low[m <= 0.5] == 1.0) and np.all(low[m >= 1.0] == 0.0)
    for i, (kap, j, k) in enumerate(o.plane_table(j0)):
        if kap == "lowpass":
            continue
        P = o.spectrum(M, N, j0, i)
        outside = (m < 2.0 ** (2 * j - 1)) | (m > 2.0 ** (2 * j + 2))
        assert np.all(P[outside] == 0.0)


def test_spectra_symmetric_after_fix():
    # Sec. 3.8.1: after the fix psi(-w) = psi(w) on the periodic grid, so the
    # products with a real image's spectrum are Hermitian
    for shape in [(16, 16), (64, 48), (63, 64), (64, 63)]:
        S = o.spectra(*shape)
        flipped = np.roll(S[:, ::-1, ::-1], shift=(1, 1), axis=(1, 2))
        np.testing.assert_allclose(S, flipped, atol=1e-15)
        raw = o.spectra(*shape, real_fix=False)
        if shape[0] % 2 == 0 and shape[1] % 2 == 0:
            flipped = np.roll(raw[:, ::-1, ::-1], shift=(1, 1), axis=(1, 2))
            assert np.abs(raw - flipped).max() > 0.1  # the unfixed spectra are not


def test_transpose_symmetry_square():
    # square grids: transposing swaps the cones, h(j,k) <-> v(j,k); seam and
    # low-pass planes map to themselves
    n, j0 = 64, 3
    table = o.plane_table(j0)
    S = o.spectra(n, n)
    for i, (kap, j, k) in enumerate(table):
        if kap == "h":
            partner = table.index(("v", j, k))
        elif kap == "v":
            partner = table.index(("h", j, k))
        else:
            partner = i
        np.testing.assert_allclose(S[i].T, S[partner], atol=1e-15)


def test_max_scale_min_grid():
    # maxScale = 'min' (Sec. 3.5.3 option, Sec. 3.5.1 choice X_2 = 2^{2 j0 - 2}): half the
    # extent of the default X_3 = 2^{2 j0 - 1}; both keep the frame tight
    for n, j0 in ((64, 3), (256, 4)):
        assert o.grid_spacing(n, j0, "min") * 2 == o.grid_spacing(n, j0)
        _, _, xi1, _ = o.grid(n, n, j0, "min")
        assert np.abs(xi1).max() == 2.0 ** (2 * j0 - 2)
    for smooth in (False, True):
        assert np.abs(o.frame_sum(64, 64, 3, smooth=smooth, max_scale="min") - 1).max() <= 1e-14
        assert np.abs(o.frame_sum(96, 128, 3, smooth=smooth, max_scale="min") - 1).max() <= 1e-14
    # on the smaller grid the finest scale covers less: the finest planes carry
    # less of the spectrum than with the default extent
    fine = [i for i, (kap, j, k) in enumerate(o.plane_table(3)) if j == 2]
    e_max = sum((o.spectrum(64, 64, 3, i) ** 2).sum() for i in fine)
    e_min = sum((o.spectrum(64, 64, 3, i, max_scale="min") ** 2).sum() for i in fine)
    assert e_min < e_max
    with pytest.raises(ValueError):
        o.grid_spacing(64, 3, "mid")
