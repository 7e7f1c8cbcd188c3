"""The surrogate network on the tensor cores (BF16 operands, FP32 accumulation) against the FP64
oracle of oracle/mlp.py: every forward output and every element of every layer's weight and bias
gradients within its per-element BF16 bound (tests/bf16_bounds.py), the loss, Adam's first step,
and training that actually fits."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2411_05799_gb300 import npx
from tests import bf16_bounds as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _own_stream():
    """Each test runs on a torch stream of its own: on the legacy default stream (handle 0) the
    library would create a stream of its own that torch's reads do not wait for."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        yield
    s.synchronize()

SIZES = [271, 512, 512, 512, 512, 247]


def _setup(M=256, seed=0):
    rng = np.random.default_rng(seed)
    Ws, bs = ref.init_params(SIZES, seed=seed)
    bs = [rng.normal(0, 0.05, b.shape) for b in bs]
    x = rng.normal(0, 1, (M, SIZES[0])).astype(np.float32)
    t = rng.normal(0, 1, (M, SIZES[-1])).astype(np.float32)
    net = npx.MLP(SIZES[0], SIZES[-1], max_batch=M, lr=1e-3,
                  stream=torch.cuda.current_stream().cuda_stream)
    net.set_params([W.astype(np.float32) for W in Ws], [b.astype(np.float32) for b in bs])
    Ws = [W.astype(np.float32).astype(np.float64) for W in Ws]     # the values the GPU holds
    bs = [b.astype(np.float32).astype(np.float64) for b in bs]
    return net, Ws, bs, x, t


def test_bounded_wait_gives_up_and_the_context_survives():
    """Every barrier wait of the GEMM is bounded: on a barrier that nothing completes it gives up
    after its two-second limit, or as soon as another warp raises the abort flag, and reports it;
    the context then still runs the network correctly."""
    st = torch.cuda.current_stream().cuda_stream
    gave_up, us = npx.gemm_wait_selftest(False, st)
    assert gave_up == 1 and 1.9e6 <= us <= 6e6, us
    gave_up, us = npx.gemm_wait_selftest(True, st)
    assert gave_up == 1 and 900 <= us <= 5e5, us
    test_forward_matches_fp64_oracle()


def test_params_round_trip():
    net, Ws, bs, x, t = _setup()
    W2, b2 = net.get_params()
    for a, b in zip(W2 + b2, Ws + bs):
        np.testing.assert_array_equal(a, b.astype(np.float32))


def test_forward_matches_fp64_oracle():
    net, Ws, bs, x, t = _setup()
    M = len(x)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(M, SIZES[-1], device="cuda")
    net.forward(xd.data_ptr(), yd.data_ptr(), M)
    torch.cuda.synchronize()
    r = B.reference(Ws, bs, x, np.zeros((M, SIZES[-1])))
    worst = B.worst_ratio(yd.cpu().numpy(), r["y"], r["ey"])
    assert worst <= 1.0, f"an output is {worst:.3g} x its BF16 bound from the FP64 oracle"


def test_gradients_match_fp64_oracle():
    net, Ws, bs, x, t = _setup()
    M = len(x)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, device="cuda")
    net.backward(xd.data_ptr(), td.data_ptr(), M, loss.data_ptr())
    dW, db = net.get_grads()
    r = B.reference(Ws, bs, x, t)
    assert abs(float(loss.item()) - r["loss"]) < 1e-2 * r["loss"]
    for l in range(len(dW)):
        worst = B.worst_ratio(dW[l], r["dW"][l], r["edW"][l])
        assert worst <= 1.0, f"layer {l}: a weight gradient is {worst:.3g} x its BF16 bound"
        worst = B.worst_ratio(db[l], r["db"][l], r["edb"][l])
        assert worst <= 1.0, f"layer {l}: a bias gradient is {worst:.3g} x its BF16 bound"


def test_adam_first_step_moves_each_weight_by_the_learning_rate():
    net, Ws, bs, x, t = _setup()
    M = len(x)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, device="cuda")
    W0, b0 = net.get_params()
    net.backward(xd.data_ptr(), td.data_ptr(), M, loss.data_ptr())
    g, gb = net.get_grads()
    net.adam_step()
    W1, b1 = net.get_params()
    for l in range(len(W0)):
        want = W0[l] - 1e-3 * g[l] / (np.abs(g[l]) + 1e-8)
        np.testing.assert_allclose(W1[l], want, rtol=0, atol=2e-6)


def test_training_fits_a_smooth_map():
    """Fit t = sin(x A) B on random inputs: the loss falls by more than 20x in 300 steps."""
    M = 1024
    rng = np.random.default_rng(7)
    A = rng.normal(0, 0.2, (SIZES[0], 16))
    B = rng.normal(0, 1.0, (16, SIZES[-1]))
    x = rng.normal(0, 1, (M, SIZES[0])).astype(np.float32)
    t = (np.sin(x @ A) @ B).astype(np.float32)
    net = npx.MLP(SIZES[0], SIZES[-1], max_batch=M, lr=1e-3, seed=3,
                  stream=torch.cuda.current_stream().cuda_stream)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = torch.zeros(1, device="cuda")
    losses = []
    for it in range(300):
        net.backward(xd.data_ptr(), td.data_ptr(), M, loss.data_ptr())
        net.adam_step()
        if it % 50 == 0 or it == 299:
            losses.append(float(loss.item()))
    assert losses[-1] < losses[0] / 20, losses
