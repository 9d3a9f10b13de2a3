"""Gaussian convolution / statistical averaging on the GPU against the oracle
(needs a GPU).  Both sides sum the same FP64 terms (the kernel drops those
beyond 8 standard deviations, relative weight e^-32), in different orders:
agreement to 1e-12 of the series' scale."""
import numpy as np
import pytest

from oracle import rmatrix as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1403_5524_gb300 import rm as _rm
    _rm.load_library()
    return _rm


@pytest.mark.parametrize("fwhm", [0.0, 1e-7, 2.9e-4, 9.1e-3])
def test_convolve_against_oracle(rm, fwhm):
    rng = np.random.default_rng(5)
    E = np.sort(rng.uniform(0.0, 0.5, 3001))  # non-uniform mesh, with near-duplicate points
    sig = np.vstack([1 + np.sin(40 * E) ** 2 + 0.3 * rng.random(E.size), np.exp(-E) + rng.random(E.size)])
    w = [2 / 3, 1 / 3]
    ref = orc.convolve_average(E, sig, w, fwhm)
    out = rm.convolve(E, sig, fwhm, weights=w)  # host pointers
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    dev = torch.device("cuda:0")
    dout = rm.convolve(torch.from_numpy(E).to(dev), torch.from_numpy(sig).to(dev), fwhm, weights=w)
    torch.cuda.synchronize()
    assert np.array_equal(dout.cpu().numpy(), out)


def test_convolve_single_series_and_tiny_mesh(rm):
    E = np.array([0.3])
    out = rm.convolve(E, np.array([2.0]), 0.01)
    assert out[0] == 2.0
    E = np.linspace(0, 1, 7)
    s = np.arange(7.0)
    out = rm.convolve(E, s, 0.2)  # default weight 1 for one series
    assert np.abs(out - orc.convolve_average(E, s[None, :], [1.0], 0.2)).max() <= 1e-13 * 6
