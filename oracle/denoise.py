"""CPU oracle of the dose denoiser (TEST INFRASTRUCTURE).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module; it shares no code with the CUDA path.

The paper has no denoiser: this is the learned post-processing step that
maps a low-history dose plus density to a high-history dose, built on the
method's own dose output.  Everything here is the plain definition, in
float64, with numpy array operations as the only primitives:

* conv3d: 3x3x3 taps, zero padding 1, channels last.  Tap t = (dz+1)*9 +
  (dy+1)*3 + (dx+1) for offsets dz, dy, dx in {-1, 0, 1};
  y[z,y,x,o] = b[o] + sum_t sum_i x[z+dz, y+dy, x+dx, i] w[t, i, o].
* its gradients: d x (a convolution with the mirrored taps and transposed
  channels) and d w (a correlation of the input with the output gradient).
* 2x2x2 average pooling, nearest 2x upsampling, ReLU, and their gradients.
* the network: a 4-level encoder-decoder (16/32/64/128 channels) with
  additive skips and a residual output, its mean-squared-error loss and
  backward pass, and the Adam update.

The network is defined with BF16 activations (FP32 accumulation):
forward() and loss_and_grads() take `bf16=True` to round every stored
activation and activation gradient to BF16 (8 significant bits, round to
nearest even) at the points where that definition stores them, in float64
arithmetic otherwise; `bf16=False` is the exact float64 network.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """s[z, y, x] = x[z + dz, y + dy, x + dx], zero outside."""
    D, H, W = x.shape[:3]
    s = np.zeros_like(x)
    zs, zd = (slice(dz, D), slice(0, D - dz)) if dz >= 0 else (slice(0, D + dz), slice(-dz, D))
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    s[zd, yd, xd] = x[zs, ys, xs]
    return s


def conv3d(x: np.ndarray, w: np.ndarray, b=None) -> np.ndarray:
    """x [D,H,W,Ci], w [27,Ci,Co], b [Co] or None -> [D,H,W,Co]."""
    x = np.asarray(x, np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        y += _shift(x, dz, dy, dx) @ np.asarray(w[t], np.float64)
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_dx(gy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient wrt the input: dx[v, i] = sum_t sum_o gy[v - off_t, o] w[t, i, o]."""
    gy = np.asarray(gy, np.float64)
    dx = np.zeros(gy.shape[:3] + (w.shape[1],))
    for t, (dz, dy, dxo) in enumerate(OFFSETS):
        dx += _shift(gy, -dz, -dy, -dxo) @ np.asarray(w[t], np.float64).T
    return dx


def conv3d_dw(x: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """Gradient wrt the taps: dw[t, i, o] = sum_v x[v + off_t, i] gy[v, o]."""
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    ci, co = x.shape[3], gy.shape[3]
    dw = np.zeros((27, ci, co))
    g2 = gy.reshape(-1, co)
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        dw[t] = _shift(x, dz, dy, dx).reshape(-1, ci).T @ g2
    return dw


def avgpool2(x: np.ndarray) -> np.ndarray:
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_grad(g: np.ndarray) -> np.ndarray:
    return upsample2(g) / 8.0


def upsample2(x: np.ndarray) -> np.ndarray:
    return x.repeat(2, 0).repeat(2, 1).repeat(2, 2)


def upsample2_grad(g: np.ndarray) -> np.ndarray:
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even): the value is first
    rounded to float32, whose upper 16 bits BF16 keeps."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(x):
    return x


# ------------------------------------------------------------------ network --
# Layers of the encoder-decoder: (name, C_in, C_out).  The input has two
# channels (dose / scale, density) padded with zeros to 8.
LAYERS = [("e0a", 8, 16), ("e0b", 16, 16), ("e1", 16, 32), ("e2", 32, 64), ("b3a", 64, 128), ("b3b", 128, 64),
          ("d2", 64, 32), ("d1", 32, 16), ("d0", 16, 16)]
IN_CHANNELS = 8


def init_params(seed: int) -> dict:
    """He-normal taps, zero biases; the 1x1 output layer starts at zero so
    the network starts as the identity on the dose (residual output)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in LAYERS:
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), (27, ci, co))
        p[name + ".b"] = np.zeros(co)
    p["out.w"] = np.zeros(16)
    p["out.b"] = np.zeros(1)
    return p


def forward(p: dict, x: np.ndarray, keep: bool = False, bf16: bool = False):
    """x [D,H,W,8] (channel 0 = scaled dose) -> predicted scaled dose [D,H,W]
    (and the activations when keep).  bf16: every stored activation (layer
    outputs after bias and ReLU, pooled and upsampled-plus-skip tensors) is
    rounded to BF16; the output layer stays in full precision."""
    q = round_bf16 if bf16 else _ident
    a = {}
    h = q(relu(conv3d(x, p["e0a.w"], p["e0a.b"]))); a["e0a"] = h
    s0 = q(relu(conv3d(h, p["e0b.w"], p["e0b.b"]))); a["e0b"] = s0
    h = q(avgpool2(s0)); a["p0"] = h
    s1 = q(relu(conv3d(h, p["e1.w"], p["e1.b"]))); a["e1"] = s1
    h = q(avgpool2(s1)); a["p1"] = h
    s2 = q(relu(conv3d(h, p["e2.w"], p["e2.b"]))); a["e2"] = s2
    h = q(avgpool2(s2)); a["p2"] = h
    h = q(relu(conv3d(h, p["b3a.w"], p["b3a.b"]))); a["b3a"] = h
    h = q(relu(conv3d(h, p["b3b.w"], p["b3b.b"]))); a["b3b"] = h
    h = q(upsample2(h) + s2); a["u2"] = h
    h = q(relu(conv3d(h, p["d2.w"], p["d2.b"]))); a["d2"] = h
    h = q(upsample2(h) + s1); a["u1"] = h
    h = q(relu(conv3d(h, p["d1.w"], p["d1.b"]))); a["d1"] = h
    h = q(upsample2(h) + s0); a["u0"] = h
    h = q(relu(conv3d(h, p["d0.w"], p["d0.b"]))); a["d0"] = h
    y = h @ p["out.w"] + p["out.b"][0] + x[..., 0]
    return (y, a) if keep else y


def loss_and_grads(p: dict, x: np.ndarray, target: np.ndarray, bf16: bool = False):
    """Mean squared error over the voxels and its gradient for every
    parameter.  bf16: the forward pass as forward(bf16=True), and every
    stored activation gradient (the output layer's, each layer's input
    gradient, pooled and skip-summed gradients) rounded to BF16; parameter
    gradients are accumulated in full precision."""
    q = round_bf16 if bf16 else _ident
    y, a = forward(p, x, keep=True, bf16=bf16)
    n = y.size
    r = y - target
    loss = float((r * r).mean())
    gy = 2.0 * r / n
    g = {}
    g["out.w"] = (a["d0"].reshape(-1, 16).T @ gy.reshape(-1))
    g["out.b"] = np.array([gy.sum()])
    gh = q(gy[..., None] * p["out.w"] * (a["d0"] > 0))

    def conv_back(name, x_in, gh_out):
        gz = gh_out * (a[name] > 0)
        g[name + ".w"] = conv3d_dw(x_in, gz)
        g[name + ".b"] = gz.reshape(-1, gz.shape[-1]).sum(0)
        return q(conv3d_dx(gz, p[name + ".w"]))

    gu0 = conv_back("d0", a["u0"], gh)
    gs0 = gu0.copy()
    gd1 = q(upsample2_grad(gu0))
    gu1 = conv_back("d1", a["u1"], gd1)
    gs1 = gu1.copy()
    gd2 = q(upsample2_grad(gu1))
    gu2 = conv_back("d2", a["u2"], gd2)
    gs2 = gu2.copy()
    gb3b = q(upsample2_grad(gu2))
    gb3a = conv_back("b3b", a["b3a"], gb3b)
    gp2 = conv_back("b3a", a["p2"], gb3a)
    gs2 = q(gs2 + avgpool2_grad(gp2))
    gp1 = conv_back("e2", a["p1"], gs2)
    gs1 = q(gs1 + avgpool2_grad(gp1))
    gp0 = conv_back("e1", a["p0"], gs1)
    gs0 = q(gs0 + avgpool2_grad(gp0))
    ge0a = conv_back("e0b", a["e0a"], gs0)
    gz = ge0a * (a["e0a"] > 0)
    g["e0a.w"] = conv3d_dw(x, gz)
    g["e0a.b"] = gz.reshape(-1, 16).sum(0)
    return loss, g


def adam_step(p: dict, g: dict, m: dict, v: dict, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) of every parameter, in place."""
    for k in p:
        m[k] = b1 * m.get(k, 0.0) + (1 - b1) * g[k]
        v[k] = b2 * v.get(k, 0.0) + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
