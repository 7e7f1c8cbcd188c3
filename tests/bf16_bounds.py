"""Per-element error bounds of the surrogate network evaluated with BF16 operands and FP32
accumulation (the tensor-core path), against the FP64 oracle of oracle/mlp.py.  Test
infrastructure.

Every GEMM C = A B^T of the device reads BF16 copies of its operands: each copy moves an operand
by at most 2^-9 of its magnitude, so one product moves by at most 2^-8 |a| |b| and the GEMM's
element by at most 2^-8 sum_k |a_ik| |b_jk| (FP32 accumulation adds K 2^-24 of the same sum, far
less).  The bounds below take that per-GEMM quantity, computed in FP64 from the oracle's own
operands of the layer, times a constant c that also covers what the layer's inputs carry in from
the layers before (their own BF16 roundings, which accumulate over the depth of the network):
  - network output y = h W^T + b:        |dy|  <= C_FWD  2^-8 (|h| |W|^T)
  - weight gradient dW = G^T h:          |ddW| <= C_GRAD 2^-8 (|G|^T |h|)
  - bias gradient db = sum over rows G:  |ddb| <= C_GRAD 2^-8 sum |G|
with h the layer's input and G the gradient of the loss with respect to its output.  The
constants are set against a numpy emulation of the device's rounding (to_bf16 / emulate below),
whose largest ratios to 2^-8 (...) are about 0.7 (outputs) and 6 (gradients, after four layers
of backpropagation), and tests/test_bf16_bounds.py checks that the bounds still reject a gradient
off by 10 % or a missing GELU' factor."""
from __future__ import annotations

import numpy as np

from oracle import mlp as ref

EPS8 = 2.0 ** -8
C_FWD = 2.0
C_GRAD = 12.0


def reference(Ws, bs, x, t):
    """FP64 forward, loss and gradients with per-element bounds: a dict with y, ey, loss, dW, db,
    edW, edb (lists over layers)."""
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    y, cache = ref.forward(Ws, bs, x)
    dW, db = ref.backward(Ws, bs, cache, y, t)
    ey = C_FWD * EPS8 * (np.abs(cache[-1][0]) @ np.abs(Ws[-1]).T)
    L = len(Ws)
    M = len(y)
    G = 2.0 * (y - t) / M
    edW, edb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        h = cache[l][0]
        edW[l] = C_GRAD * EPS8 * (np.abs(G).T @ np.abs(h))
        edb[l] = C_GRAD * EPS8 * np.abs(G).sum(0)
        if l > 0:
            G = (G @ Ws[l]) * ref.gelu_grad(cache[l - 1][1])
    return {"y": y, "ey": ey, "loss": ref.mse(y, t), "dW": dW, "db": db, "edW": edW, "edb": edb}


def worst_ratio(got, want, bound) -> float:
    """The largest |got - want| / bound over the elements (<= 1: every element within bound)."""
    got = np.asarray(got, np.float64)
    return float(np.max(np.abs(got - want) / np.maximum(bound, 1e-300)))


def to_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def emulate(Ws, bs, x, t):
    """The device's rounding model in numpy: the input, the weights, the saved z and every stored
    activation and gradient rounded to BF16; products summed in float64 and rounded once to FP32.
    Returns the output and the gradients."""
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    L = len(Ws)
    Wb = [to_bf16(W) for W in Ws]
    h = to_bf16(x)
    hs, zs = [h], []
    for l in range(L):
        z = f32(f32(h @ Wb[l].T) + bs[l])
        if l < L - 1:
            zs.append(to_bf16(z))
            h = to_bf16(ref.gelu(z))
            hs.append(h)
        else:
            y = z
    M = len(y)
    G = to_bf16(f32(2.0 * f32(y - t) / M))
    dW, db = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = f32(G.T @ hs[l])
        db[l] = f32(G.sum(0))
        if l > 0:
            G = to_bf16(f32(f32(G @ Wb[l]) * ref.gelu_grad(zs[l - 1])))
    return y, dW, db
