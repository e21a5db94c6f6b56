"""GPU parity of the tensor-core 3D convolution against the float64 oracle.

Both sides take the same BF16-rounded inputs and taps.  Bar: the FP32
output within 2e-5 x (sum over k of |a_k b_k|) + 1e-6 of the oracle (FP32
accumulation of up to 27 x 128 products); the BF16 output within one BF16
rounding (2^-8 relative) of that.  Shapes cover every C_out (16, 32, 64,
128), the 8-channel input layer, several pipeline stages, volumes whose
voxel count is not a multiple of the 128-voxel tile, and rows of 128 and 256
voxels (the halo form), each in every form of the kernel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import denoise as dn  # noqa: E402
from paper_1302_1861_b300 import capi  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def _run(x, w, b, relu, mirror=False):
    D, H, W = x.shape[:3]
    ci, co = w.shape[1], w.shape[2]
    xin = _bf16(x).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    cin, cout = (co, ci) if mirror else (ci, co)
    assert x.shape[3] == cin
    wpk = capi.conv3d_pack(wt, ci, co, mirror)
    bias = None if b is None else torch.from_numpy(np.ascontiguousarray(b, np.float32)).cuda()
    out = torch.empty(D * H * W * cout, dtype=torch.bfloat16, device="cuda")
    of = torch.empty(D * H * W * cout, dtype=torch.float32, device="cuda")
    capi.conv3d(xin.view(torch.int16), cin, wpk, bias, cout, W, H, D, relu, out.view(torch.int16), of)
    torch.cuda.synchronize()
    return (out.float().cpu().numpy().reshape(D, H, W, cout), of.cpu().numpy().reshape(D, H, W, cout),
            xin.float().cpu().numpy().astype(np.float64))


@pytest.fixture(params=[0, 1, 2], ids=["default", "gather", "per-tap-tma"])
def form(request):
    capi.conv3d_form(request.param)
    yield request.param
    capi.conv3d_form(0)


@pytest.mark.parametrize("shape,ci,co", [((5, 7, 9), 8, 16), ((8, 8, 8), 16, 16), ((6, 5, 11), 16, 32),
                                         ((4, 9, 6), 32, 64), ((4, 4, 4), 64, 128), ((3, 5, 4), 128, 64),
                                         ((2, 3, 23), 128, 128), ((16, 16, 16), 32, 32), ((3, 5, 64), 16, 16),
                                         ((6, 4, 32), 64, 32), ((2, 2, 200), 16, 64), ((9, 3, 16), 128, 128),
                                         ((4, 8, 8), 8, 16),
                                         # rows of 128 voxels: the halo form (form 0) where C_in % 16 == 0
                                         ((3, 5, 128), 16, 16), ((2, 3, 128), 128, 128), ((3, 3, 256), 32, 64),
                                         ((2, 5, 128), 64, 32), ((2, 2, 128), 16, 128), ((2, 3, 128), 8, 16)])
def test_conv_forward_matches_oracle(shape, ci, co, form):
    rng = np.random.default_rng(ci * 1000 + co)
    x = rng.normal(size=shape + (ci,)).astype(np.float32)
    w = rng.normal(0, 0.2, size=(27, ci, co)).astype(np.float32)
    b = rng.normal(0, 0.1, size=co).astype(np.float32)
    wq = _bf16(w).float().numpy().astype(np.float64)
    for relu in (False, True):
        ob, of, xq = _run(x, w, b, relu)
        ref = dn.conv3d(xq, wq, b.astype(np.float64))
        mag = dn.conv3d(np.abs(xq), np.abs(wq)) + np.abs(b)
        if relu:
            ref = np.maximum(ref, 0.0)
        assert np.all(np.abs(of - ref) <= 2e-5 * mag + 1e-6), np.abs(of - ref).max()
        assert np.all(np.abs(ob - of) <= 2.0 ** -8 * np.abs(of) + 1e-30)


@pytest.mark.parametrize("ci,co,vol", [(16, 16, (5, 6, 8)), (16, 32, (5, 6, 8)), (32, 64, (5, 6, 8)),
                                       (64, 128, (5, 6, 8)), (128, 64, (5, 6, 8)), (32, 64, (2, 3, 128)),
                                       (128, 16, (2, 2, 128))])
def test_mirrored_taps_give_the_input_gradient(ci, co, vol, form):
    """psl_conv3d with the mirrored packing of w, applied to an output
    gradient, is the oracle's input gradient."""
    rng = np.random.default_rng(7 + ci + co)
    gy = rng.normal(size=vol + (co,)).astype(np.float32)
    w = rng.normal(0, 0.2, size=(27, ci, co)).astype(np.float32)
    wq = _bf16(w).float().numpy().astype(np.float64)
    ob, of, gq = _run(gy, w, None, False, mirror=True)
    ref = dn.conv3d_dx(gq, wq)
    mag = dn.conv3d_dx(np.abs(gq), np.abs(wq))
    assert np.all(np.abs(of - ref) <= 2e-5 * mag + 1e-6), np.abs(of - ref).max()


@pytest.mark.parametrize("shape,ci,co", [((6, 7, 9), 8, 16), ((8, 8, 8), 16, 16), ((5, 6, 11), 16, 32),
                                         ((4, 9, 6), 32, 64), ((4, 4, 4), 64, 128), ((3, 5, 4), 128, 64),
                                         ((16, 16, 16), 32, 32)])
def test_weight_gradient_matches_oracle(shape, ci, co):
    rng = np.random.default_rng(11 + ci + co)
    x = rng.normal(size=shape + (ci,)).astype(np.float32)
    gy = rng.normal(size=shape + (co,)).astype(np.float32)
    xb, gb = _bf16(x), _bf16(gy)
    dw = torch.zeros(27 * ci * co, dtype=torch.float32, device="cuda")
    D, H, W = shape
    capi.conv3d_wgrad(xb.cuda().view(torch.int16), ci, gb.cuda().view(torch.int16), co, W, H, D, dw)
    torch.cuda.synchronize()
    xq, gq = xb.float().numpy().astype(np.float64), gb.float().numpy().astype(np.float64)
    ref = dn.conv3d_dw(xq, gq)
    mag = dn.conv3d_dw(np.abs(xq), np.abs(gq))
    got = dw.cpu().numpy().reshape(27, ci, co)
    assert np.all(np.abs(got - ref) <= 2e-5 * mag + 1e-6), np.abs(got - ref).max()


def test_conv_rejects_bad_shapes():
    x = torch.zeros(64 * 8, dtype=torch.int16, device="cuda")
    w = torch.zeros(27 * 8 * 24, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.PslError):
        capi.conv3d_pack(w, 8, 24)                    # C_out 24 is not a tile width
    wpk = torch.zeros(int(capi.lib().psl_conv3d_packed_size(12, 16)), dtype=torch.int16, device="cuda")
    out = torch.zeros(64 * 16, dtype=torch.int16, device="cuda")
    with pytest.raises(capi.PslError):
        capi.conv3d(x, 12, wpk, None, 16, 4, 4, 4, False, out)   # C_in not a multiple of 8


@pytest.mark.parametrize("ci,co", [(128, 128), (16, 16)])
def test_full_volume_sampled_against_direct_sums(ci, co):
    """The bench's shape (128^3 voxels, the halo form's full grid) checked on
    sampled output voxels, each against its 27 x C_in-term sum in float64
    (every output channel of 3000 voxels, borders included)."""
    n = 128
    rng = np.random.default_rng(ci + 3 * co)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1000 + ci + co)                       # seeded inputs
    x = torch.randn(n, n, n, ci, device="cuda", generator=gen).to(torch.bfloat16)
    w = (torch.randn(27, ci, co, device="cuda", generator=gen) * 0.05).contiguous()
    b = (torch.randn(co, device="cuda", generator=gen) * 0.1).contiguous()
    wpk = capi.conv3d_pack(w, ci, co)
    of = torch.empty(n ** 3 * co, dtype=torch.float32, device="cuda")
    capi.conv3d(x.view(-1).view(torch.int16), ci, wpk, b, co, n, n, n, False, None, of)
    torch.cuda.synchronize()
    pts = rng.integers(0, n, size=(3000, 3))
    pts[:200, 0] = rng.choice([0, n - 1], 200)           # faces of the volume (the padding)
    pts[200:400, 2] = rng.choice([0, n - 1], 200)
    P = torch.from_numpy(pts).cuda()
    got = of.view(n, n, n, co)[P[:, 0], P[:, 1], P[:, 2]].cpu().numpy().astype(np.float64)
    # the 27 neighbours of each sampled voxel (zero outside the volume)
    xf = x.float()
    nb = []
    for t in range(27):
        d = torch.tensor([t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1], device="cuda")
        q = P + d
        inside = ((q >= 0) & (q < n)).all(1)
        qc = q.clamp(0, n - 1)
        nb.append(xf[qc[:, 0], qc[:, 1], qc[:, 2]] * inside[:, None])
    xn = torch.stack(nb, 1).cpu().numpy().astype(np.float64)          # [points, 27, ci]
    wq = w.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    bq = b.cpu().numpy().astype(np.float64)
    ref = bq + np.einsum("pti,tio->po", xn, wq)
    mag = np.abs(bq) + np.einsum("pti,tio->po", np.abs(xn), np.abs(wq))
    assert np.all(np.abs(got - ref) <= 2e-5 * mag + 1e-6), np.abs(got - ref).max()
