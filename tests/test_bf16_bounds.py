"""The per-element BF16 bounds of the network (tests/bf16_bounds.py): they hold with margin for a
numpy emulation of the device's rounding, and they reject plausible mistakes."""
import numpy as np

from oracle import mlp as ref
from tests import bf16_bounds as B

SIZES = [271, 512, 512, 512, 512, 247]


def _case(seed, M=256):
    rng = np.random.default_rng(seed)
    Ws, bs = ref.init_params(SIZES, seed=seed)
    bs = [rng.normal(0, 0.05, b.shape) for b in bs]
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]
    bs = [b.astype(np.float32).astype(np.float64) for b in bs]
    x = rng.normal(0, 1, (M, SIZES[0])).astype(np.float32).astype(np.float64)
    t = rng.normal(0, 1, (M, SIZES[-1])).astype(np.float32).astype(np.float64)
    return Ws, bs, x, t


def test_bounds_hold_with_margin_for_the_emulated_device_arithmetic():
    for seed in (0, 1, 2):
        Ws, bs, x, t = _case(seed)
        r = B.reference(Ws, bs, x, t)
        ye, dWe, dbe = B.emulate(Ws, bs, x, t)
        assert 0.05 < B.worst_ratio(ye, r["y"], r["ey"]) < 0.5, seed
        for l in range(len(Ws)):
            assert B.worst_ratio(dWe[l], r["dW"][l], r["edW"][l]) < 0.75, (seed, l)
            assert B.worst_ratio(dbe[l], r["db"][l], r["edb"][l]) < 0.75, (seed, l)


def test_bounds_reject_plausible_mistakes():
    Ws, bs, x, t = _case(3)
    r = B.reference(Ws, bs, x, t)
    # an output with one hidden layer's bias left out
    bs2 = [b.copy() for b in bs]
    bs2[2][:] = 0.0
    assert B.worst_ratio(ref.forward(Ws, bs2, x)[0], r["y"], r["ey"]) > 1.0
    # one output weight row 10 % off
    Ws2 = [W.copy() for W in Ws]
    Ws2[4][10] *= 1.1
    assert B.worst_ratio(ref.forward(Ws2, bs, x)[0], r["y"], r["ey"]) > 1.0
    # every layer's gradients 10 % off
    for l in range(len(Ws)):
        assert B.worst_ratio(0.9 * r["dW"][l], r["dW"][l], r["edW"][l]) > 1.0, l
        assert B.worst_ratio(0.9 * r["db"][l], r["db"][l], r["edb"][l]) > 1.0, l
    # backpropagation through layer 3 without its GELU' factor
    y, cache = ref.forward(Ws, bs, x)
    G = 2.0 * (y - t) / len(y)
    for l in range(len(Ws) - 1, 0, -1):
        gW = G.T @ cache[l][0]
        G = (G @ Ws[l]) * (ref.gelu_grad(cache[l - 1][1]) if l != 3 else 1.0)
    assert B.worst_ratio(G.T @ cache[0][0], r["dW"][0], r["edW"][0]) > 1.0
