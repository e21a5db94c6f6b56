"""GPU parity of the denoiser network against the oracle, element by element.

The network stores activations and activation gradients in BF16 (8
significant bits) with FP32 accumulation; the oracle follows the same
definition (oracle.denoise with bf16=True rounds at the same storage
points) in float64 otherwise.  What is left between the two: the order of
the FP32 sums (relative 1e-6) and, where that moves a value across a BF16
rounding boundary, a one-ulp (2^-8 relative) flip that later layers carry.
Bars, element by element (ulp = 2^-8):
* forward output: every voxel within 2^-6 of the output's largest
  magnitude, and 99.9 % within 4 ulps of its own value (+ 2^-10 of that
  largest magnitude);
* every parameter gradient: 99 % of the elements within 4 ulps of their own
  value + 2^-8 of the group's largest magnitude, every element within 2^-4
  of it;
* the loss within 0.5 %, and one Adam step equal, to FP32 rounding, to the
  oracle's update computed from the GPU's own gradients.
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


def _flatten(p):
    parts = []
    for name, ci, co in dn.LAYERS:
        parts += [p[name + ".w"].reshape(-1), p[name + ".b"].reshape(-1)]
    parts += [p["out.w"].reshape(-1), p["out.b"].reshape(-1)]
    return np.concatenate(parts)


def _unflatten(flat):
    out, o = {}, 0
    for name, ci, co in dn.LAYERS:
        n = 27 * ci * co
        out[name + ".w"] = flat[o:o + n].reshape(27, ci, co); o += n
        out[name + ".b"] = flat[o:o + co]; o += co
    out["out.w"] = flat[o:o + 16]; o += 16
    out["out.b"] = flat[o:o + 1]; o += 1
    return out


def _case(seed, n=16):
    rng = np.random.default_rng(seed)
    p = dn.init_params(seed)
    p["out.w"] = rng.normal(0, 0.3, 16)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, p[k].shape)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    dose = np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (0.1 * n * n)) * (1 + 0.2 * rng.normal(size=(n,) * 3))
    rho = 1.0 + 0.5 * (z > n // 2) + 0.05 * rng.random((n,) * 3)
    target = np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (0.1 * n * n))
    return p, dose.astype(np.float32), rho.astype(np.float32), target.astype(np.float32)


def _oracle_input(dose, rho, scale):
    # the GPU feeds BF16 inputs: round them the same way for the oracle
    x = np.zeros(dose.shape + (8,))
    x[..., 0] = torch.from_numpy(dose / np.float32(scale)).to(torch.bfloat16).float().numpy()
    x[..., 1] = torch.from_numpy(rho).to(torch.bfloat16).float().numpy()
    return x


def test_network_forward_backward_and_adam_match_the_oracle():
    n, scale = 16, 1.3
    p, dose, rho, target = _case(3, n)
    d = capi.Denoiser.create(1)
    npar = capi.Denoiser.param_count()
    flat = torch.from_numpy(_flatten(p).astype(np.float32)).cuda()
    assert flat.numel() == npar
    d.params(set=flat)
    # the BF16 taps are what the GPU multiplies with: give the oracle the same
    pq = {k: (torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
              if k.endswith(".w") and k != "out.w" else v.astype(np.float32).astype(np.float64))
          for k, v in p.items()}
    dg, rg, tg = (torch.from_numpy(a).cuda() for a in (dose, rho, target))
    out = torch.empty_like(dg)
    d.forward(dg, rg, n, n, n, scale, out)
    x = _oracle_input(dose, rho, scale)
    y_ref = dn.forward(pq, x, bf16=True) * scale
    y = out.cpu().numpy().astype(np.float64)
    big = np.abs(y_ref).max()
    err = np.abs(y - y_ref)
    assert err.max() <= 2 ** -6 * big, err.max() / big
    assert np.mean(err <= 4 * 2 ** -8 * np.abs(y_ref) + 2 ** -10 * big) >= 0.999
    # gradients of one sample
    loss = d.backward(dg, rg, tg, n, n, n, scale)
    loss_ref, g_ref = dn.loss_and_grads(pq, x, target / scale, bf16=True)
    assert abs(loss - loss_ref) <= 0.005 * loss_ref, (loss, loss_ref)
    grad = torch.empty(npar, dtype=torch.float32, device="cuda")
    d.params(grad=grad)
    g = _unflatten(grad.cpu().numpy().astype(np.float64))
    for k in g_ref:
        a, b = g[k].reshape(-1), g_ref[k].reshape(-1)
        gbig = np.abs(b).max()
        e = np.abs(a - b)
        frac = float(np.mean(e <= 4 * 2 ** -8 * np.abs(b) + 2 ** -8 * gbig))
        assert frac >= 0.99 and e.max() <= 2 ** -4 * gbig, (k, frac, e.max() / gbig)
    # one Adam step = the oracle's update from the GPU's own gradients
    before = torch.empty(npar, dtype=torch.float32, device="cuda")
    d.params(get=before)
    d.step(1e-3)
    after = torch.empty(npar, dtype=torch.float32, device="cuda")
    d.params(get=after)
    pb = _unflatten(before.cpu().numpy().astype(np.float64))
    m, v = {}, {}
    dn.adam_step(pb, g, m, v, 1, 1e-3)
    assert np.allclose(after.cpu().numpy(), _flatten(pb), rtol=1e-5, atol=1e-7)
    d.params(grad=grad)
    assert float(grad.abs().max()) == 0.0                      # cleared by the step
    d.close()


def test_fresh_network_is_the_identity_and_training_reduces_the_loss():
    n = 32
    p, dose, rho, target = _case(5, n)
    d = capi.Denoiser.create(7)
    dg, rg, tg = (torch.from_numpy(a).cuda() for a in (dose, rho, target))
    out = torch.empty_like(dg)
    d.forward(dg, rg, n, n, n, 1.0, out)
    # zero output layer: out = dose, up to the BF16 rounding of the input
    assert np.allclose(out.cpu().numpy(), dose, rtol=2 ** -8, atol=1e-6)
    # training from a non-trivial output layer (from the identity start only
    # the output layer has a gradient and Adam's first steps follow the signs
    # of near-zero values, which depend on the order of FP32 atomics)
    p = torch.empty(capi.Denoiser.param_count(), device="cuda")
    d.params(get=p)
    p[-17:-1] = 0.1
    d.params(set=p)
    losses = []
    for it in range(40):
        losses.append(d.backward(dg, rg, tg, n, n, n, 1.0))
        d.step(2e-3)
    # (measured: 0.33 -> 0.0065 after 10 steps, 0.0064 after 40)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    assert all(np.isfinite(losses))
    d.close()


def test_denoiser_rejects_bad_volumes():
    d = capi.Denoiser.create(0)
    a = torch.zeros(12 * 16 * 16, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.PslError):
        d.forward(a, a, 12, 16, 16, 1.0, a)
    with pytest.raises(capi.PslError):
        d.step(1e-3)                                           # nothing accumulated
    d.close()


def test_kth_smallest_is_exact():
    """psl_kth_smallest (the denoiser's dose scale) against a CPU sort:
    random values with repeats, negatives and zeros, several k, n = 1, a
    dose-like 128^3 volume with +inf, all-equal values."""
    rng = np.random.default_rng(3)
    for n in (1, 1000, 262_145):
        x = rng.normal(0, 1, n).astype(np.float32) * rng.integers(0, 3, n).astype(np.float32)
        x[: n // 7] = np.round(x[: n // 7], 1)
        xs = np.sort(x)
        xt = torch.from_numpy(x).cuda()
        for k in sorted({0, n // 2, max(0, int(0.999 * n) - 1), n - 1}):
            assert capi.kth_smallest(xt, k) == xs[k]
    # a dose-like 128^3 volume (mostly air zeros, an exponential tail, +inf),
    # and values that are all equal
    x = rng.exponential(1.0, 128 ** 3).astype(np.float32)
    x[rng.random(x.size) < 0.6] = 0.0
    x[5] = np.inf
    xs = np.sort(x)
    xt = torch.from_numpy(x).cuda()
    for k in (0, x.size // 2, int(0.999 * x.size) - 1, x.size - 2, x.size - 1):
        assert capi.kth_smallest(xt, k) == xs[k]
    same = torch.full((4097,), 2.5, device="cuda")
    assert capi.kth_smallest(same, 0) == 2.5 and capi.kth_smallest(same, 4096) == 2.5
    with pytest.raises(capi.PslError):
        capi.kth_smallest(torch.zeros(4, device="cuda"), 4)
