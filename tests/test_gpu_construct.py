"""Robots built from primitives (the paper's construction calls, simplifyMode) on the CUDA step
against the oracle, per step and over a 200-step window, in every simplify mode."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2411_05799_gb300 import construct, scenes
from paper_2411_05799_gb300.npx import World
from tests.parity import quat_angle, to_gpu
from tests.test_gpu_parity import THREADS, _assert_step_parity

pytestmark = pytest.mark.gpu


def _batch(mode, n):
    rb = construct.cylinder_hexapod(mode)
    z0 = -float(rb.batch(1).p0[:, 2].min()) + 0.01
    rng = np.random.default_rng(40 + mode)
    J = 18 * n
    act = np.stack([rng.uniform(0, 0.5, J), rng.uniform(0.5, 2.0, J), rng.uniform(0, 2 * np.pi, J),
                    np.zeros(J)], 1)
    return rb.batch(n, origin=(0.0, 0.0, z0), act_params=act)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_constructed_hexapod_per_step(mode):
    b = _batch(mode, 64)
    w = World.from_batch(b)
    _assert_step_parity(w, Oracle(b, threads=THREADS), [0, 1, 80, 81, 400, 1201], max_near_frac=0.2)


@pytest.mark.parametrize("mode", [0, 2])
def test_constructed_hexapod_200_step_window(mode):
    b = _batch(mode, 128)
    o = Oracle(b, threads=THREADS)
    o.step(1000, threads=THREADS)
    w = World.from_batch(b)
    to_gpu(w, o)
    o.step(200, threads=THREADS)
    w.step(200)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o.c, axis=1)
    da = quat_angle(r["quat"], o.q)
    assert ((dc <= 1e-3) & (da <= 1e-3)).mean() >= 0.95
    assert (r["status"] == 0).all()


@pytest.mark.parametrize("mode", [1, 3])
def test_four_lanes_per_scene_per_step_and_window(mode):
    """Robots of at most 256 points can run with 4 lanes per scene (8 scenes per warp): per-step
    parity with the oracle, and a 200-step window against 8 lanes per scene."""
    b = _batch(mode, 64)
    w = World.from_batch(b, configure=dict(lanes_per_scene=4, warps_per_block=2))
    assert w.info()["lanes_per_scene"] == 4
    _assert_step_parity(w, Oracle(b, threads=THREADS), [0, 1, 80, 81, 400], max_near_frac=0.2)
    w8 = World.from_batch(b, configure=dict(lanes_per_scene=8, warps_per_block=2))
    w4 = World.from_batch(b, configure=dict(lanes_per_scene=4, warps_per_block=2))
    w8.step(200)
    w4.step(200)
    r8, r4 = w8.read(), w4.read()
    dc = np.linalg.norm(r4["cog"] - r8["cog"], axis=1)
    assert ((dc <= 1e-3) & (quat_angle(r4["quat"], r8["quat"]) <= 1e-3)).mean() >= 0.95
    assert (r4["status"] == 0).all()
