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
