"""GPU gamma index (psl_gamma) against the oracle's on synthetic dose pairs:
smooth fields with noise, shifts and scalings, anisotropic voxels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import readout  # noqa: E402
from paper_1302_1861_b300 import capi  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("case", range(4))
def test_gamma_matches_oracle(case):
    rng = np.random.default_rng(case)
    nz, ny, nx = (20, 24, 28) if case % 2 else (16, 16, 16)
    voxel = (0.25, 0.25, 0.25) if case < 2 else (0.2, 0.3, 0.25)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ref = np.exp(-((x - nx / 2) ** 2 + (y - ny / 2) ** 2) / 30.0) * np.exp(-z / 40.0)
    ev = np.roll(ref, case, axis=2) * (1 + 0.02 * case) * (1 + 0.03 * rng.normal(size=ref.shape))
    r_o, n_o = readout.gamma_pass_rate(ref, ev, voxel)
    r_g, n_g = capi.gamma(torch.from_numpy(ref).cuda(), torch.from_numpy(ev).cuda(), voxel)
    assert n_g == n_o
    assert abs(r_g - r_o) <= 2.0 / n_o, (r_g, r_o)
    # identical doses pass everywhere
    r_s, _ = capi.gamma(torch.from_numpy(ref).cuda(), torch.from_numpy(ref).cuda(), voxel)
    assert r_s == 1.0
