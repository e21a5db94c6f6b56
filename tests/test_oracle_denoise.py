"""Pins of the denoiser oracle: brute-force loops on tiny volumes, closed
forms of the convolution (a delta tap is a shift, a constant input sums the
taps), adjointness of the pooling pair, and central finite differences of
the network loss for every parameter group."""
import numpy as np
import pytest

from oracle import denoise as dn


def _brute_conv(x, w, b):
    D, H, W, ci = x.shape
    co = w.shape[2]
    y = np.zeros((D, H, W, co))
    for z in range(D):
        for yy in range(H):
            for xx in range(W):
                acc = np.array(b, np.float64).copy()
                for t, (dz, dy, dx) in enumerate(dn.OFFSETS):
                    zz, y2, x2 = z + dz, yy + dy, xx + dx
                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                        acc += x[zz, y2, x2] @ w[t]
                y[z, yy, xx] = acc
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 3))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    assert np.allclose(dn.conv3d(x, w, b), _brute_conv(x, w, b), atol=1e-12)


def test_conv_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 4, 4, 1))
    # a single tap at offset (+1, 0, -1) reads the input shifted by it
    w = np.zeros((27, 1, 1))
    t = dn.OFFSETS.index((1, 0, -1))
    w[t] = 1.0
    y = dn.conv3d(x, w)[..., 0]
    assert np.allclose(y[:3, :, 1:], x[1:, :, :3, 0]) and np.all(y[3] == 0) and np.all(y[:, :, 0] == 0)
    # a constant input: interior voxels see the sum of all taps
    c = np.ones((5, 5, 5, 2))
    w2 = rng.normal(size=(27, 2, 3))
    y2 = dn.conv3d(c, w2)
    assert np.allclose(y2[2, 2, 2], w2.sum(axis=(0, 1)))
    # a corner sees the 8 taps that stay inside
    inside = [t for t, (dz, dy, dx) in enumerate(dn.OFFSETS) if dz >= 0 and dy >= 0 and dx >= 0]
    assert np.allclose(y2[0, 0, 0], w2[inside].sum(axis=(0, 1)))


def test_conv_gradients_are_the_adjoints():
    """<conv(x), g> = <x, dx(g)> and the weight gradient is the derivative of
    <conv(x; w), g> in w (linear in w)."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 3, 5, 3))
    w = rng.normal(size=(27, 3, 4))
    g = rng.normal(size=(4, 3, 5, 4))
    lhs = (dn.conv3d(x, w) * g).sum()
    assert np.isclose(lhs, (x * dn.conv3d_dx(g, w)).sum())
    assert np.isclose(lhs, (w * dn.conv3d_dw(x, g)).sum())


def test_pooling_pair_adjoint_and_averages():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4, 6, 2, 3))
    g = rng.normal(size=(2, 3, 1, 3))
    assert np.isclose((dn.avgpool2(x) * g).sum(), (x * dn.avgpool2_grad(g)).sum())
    u = rng.normal(size=(2, 3, 1, 3))
    G = rng.normal(size=(4, 6, 2, 3))
    assert np.isclose((dn.upsample2(u) * G).sum(), (u * dn.upsample2_grad(G)).sum())
    assert np.isclose(dn.avgpool2(x)[1, 2, 0, 1], x[2:4, 4:6, 0:2, 1].mean())


@pytest.mark.parametrize("name", ["e0a.w", "e1.b", "b3a.w", "b3b.w", "d2.w", "d0.b", "out.w", "out.b"])
def test_network_gradients_by_finite_differences(name):
    rng = np.random.default_rng(4)
    p = dn.init_params(5)
    p["out.w"] = rng.normal(0, 0.3, 16)                 # non-zero so every layer gets a gradient
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.05, p[k].shape)
    x = np.zeros((8, 8, 8, 8))
    x[..., 0] = rng.random((8, 8, 8))
    x[..., 1] = rng.random((8, 8, 8))
    tgt = rng.random((8, 8, 8))
    loss, g = dn.loss_and_grads(p, x, tgt)
    flat = p[name].reshape(-1)
    for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
        old = flat[idx]
        h = 1e-5
        flat[idx] = old + h
        lp = dn.loss_and_grads(p, x, tgt)[0]
        flat[idx] = old - h
        lm = dn.loss_and_grads(p, x, tgt)[0]
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        an = g[name].reshape(-1)[idx]
        assert abs(fd - an) <= 1e-6 + 1e-4 * abs(fd), (name, idx, fd, an)


def test_adam_first_step_moves_by_lr_against_the_gradient_sign():
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3])}
    m, v = {}, {}
    dn.adam_step(p, g, m, v, 1, 0.01)
    assert np.allclose(p["a"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], atol=1e-6)


def test_round_bf16_hand_values_and_ties():
    """BF16 keeps 8 significant bits: the spacing above 1 is 2^-7; ties go
    to the even neighbour."""
    from oracle import denoise as dn
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -9, -2.0 - 2 ** -6 - 2 ** -8,
                  0.0, 3.5e38])
    # the largest finite BF16 value is (2 - 2^-7) 2^127 = 3.39e38: 3.5e38 rounds to infinity
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, 1.0, -2.0 - 2 ** -6, 0.0, np.inf])
    got = dn.round_bf16(x)
    assert np.array_equal(got, want)
    assert dn.round_bf16(np.array([(2 - 2 ** -7) * 2.0 ** 127]))[0] == (2 - 2 ** -7) * 2.0 ** 127
    r = np.random.default_rng(0).normal(0, 10, 10000)
    q = dn.round_bf16(r)
    assert np.all(np.abs(q - r) <= 2 ** -8 * np.abs(r))       # half a unit in the 8th bit
    assert np.array_equal(dn.round_bf16(q), q)                # idempotent


def test_bf16_network_stays_close_to_the_exact_one():
    """The BF16 storage points move the output by a few units in the 8th
    significant bit, not more (the same parameters, a 16^3 volume)."""
    from oracle import denoise as dn
    rng = np.random.default_rng(1)
    p = dn.init_params(2)
    p["out.w"] = rng.normal(0, 0.3, 16)
    x = np.zeros((16, 16, 16, 8))
    x[..., 0] = rng.random((16, 16, 16))
    x[..., 1] = 1.0
    y, yq = dn.forward(p, x), dn.forward(p, x, bf16=True)
    assert 0 < np.abs(y - yq).max() <= 0.02 * np.abs(y).max()
