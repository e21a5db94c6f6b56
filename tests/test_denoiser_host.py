"""Host logic of the denoiser's training loop (no GPU): a stalled start is
detected by epoch 3, a falling loss is not."""
import types

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1302_1861_b300 import denoiser as dz  # noqa: E402


class FakeNet:
    """Stands in for capi.Denoiser: a loss that falls by `rate` per step."""

    def __init__(self, rate):
        self.loss, self.rate, self.steps = 1e-3, rate, 0

    def backward(self, lo, rho, hi, nx, ny, nz, scale):
        return self.loss

    def step(self, lr):
        self.steps += 1
        self.loss *= self.rate


def pairs(n=6):
    z = np.zeros((8, 8, 8), np.float32)
    return [types.SimpleNamespace(lo=z, rho=z, hi=z, scale=1.0) for _ in range(n)]


def test_stalled_training_is_detected():
    net = FakeNet(rate=1.0)
    with pytest.raises(dz.TrainingStalled):
        dz.train(net, pairs(), epochs=10, log=None)
    assert net.steps == 4 * 2                      # stopped after epoch 3 (2 steps of 4 pairs per epoch)


def test_falling_loss_trains_to_the_end():
    net = FakeNet(rate=0.8)
    hist = dz.train(net, pairs(), epochs=10, log=None)
    assert len(hist) == 10 and hist[-1] < 0.1 * hist[0]
