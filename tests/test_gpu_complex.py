"""One-sided (complex) shearlet coefficients (Sec. 3.8.2) against the FP64 oracle.

The planar stack [eta, 2, M, N] holds Re z_i and Im z_i; both parts are
compared with the oracle's forward_onesided to 1e-5 relative L2 (the real
part is the real transform over sqrt(2), the imaginary part its Hilbert
partner), and ffst_inverse_complex must give the image back.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffst():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1202_1773_gb300 as m

    return m


@pytest.mark.parametrize("rows,cols,scales", [(64, 64, 3), (256, 256, 4), (128, 256, 4), (480, 640, 4)])
def test_complex_matches_oracle(ffst, rows, cols, scales):
    from oracle import ffst_oracle as o
    from paper_1202_1773_gb300 import inputs

    f = inputs.scaled_cartoon(rows, cols, seed=41)
    p = ffst.Plan(rows, cols, scales)
    x = torch.from_numpy(f).cuda()
    z = p.forward_complex(x)
    ref = o.forward_onesided(f.astype(np.float64), scales)
    got = z.cpu().numpy().astype(np.float64)
    for part, want in ((0, ref.real), (1, ref.imag)):
        err = np.linalg.norm(got[:, part] - want) / np.linalg.norm(ref)
        assert err <= 1e-5, (part, err)
    # the real parts are the real transform over sqrt(2) (plane 0 unscaled, no imaginary part)
    c = p.forward(x)
    np.testing.assert_allclose(got[1:, 0] * np.sqrt(2.0), c[1:].cpu().numpy(), atol=1e-5 * float(c.abs().max()))
    assert np.abs(got[0, 1]).max() <= 1e-6 * float(c.abs().max())
    r = p.inverse_complex(z)
    assert float(torch.linalg.norm(r - x) / torch.linalg.norm(x)) <= 1e-5
    p.close()


def test_complex_amplitude_is_shift_stable(ffst):
    # the point of complex shearlets (Sec. 3.8.2): |z| of a shifted image is the shifted |z|
    from paper_1202_1773_gb300 import inputs

    f = inputs.scaled_cartoon(128, 128, seed=42)
    p = ffst.Plan(128, 128)
    x = torch.from_numpy(f).cuda()
    z = p.forward_complex(x)
    zs = p.forward_complex(torch.roll(x, shifts=(5, 9), dims=(0, 1)).contiguous())
    amp = torch.sqrt(z[:, 0] ** 2 + z[:, 1] ** 2)
    amps = torch.sqrt(zs[:, 0] ** 2 + zs[:, 1] ** 2)
    err = float(torch.linalg.norm(torch.roll(amp, shifts=(5, 9), dims=(1, 2)) - amps) / torch.linalg.norm(amp))
    assert err <= 1e-5
    p.close()


def test_complex_argument_checks(ffst):
    p = ffst.Plan(64, 64)
    x = torch.zeros(64, 64, device="cuda")
    with pytest.raises(ValueError):
        p.forward_complex(x, out=torch.empty(p.num_planes, 64, 64, device="cuda"))
    with pytest.raises(ValueError):
        p.inverse_complex(torch.empty(p.num_planes, 64, 64, device="cuda"))
    p.close()
