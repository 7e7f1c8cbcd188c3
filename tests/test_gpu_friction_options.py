"""The friction-model options (rows weighted by the normal forces; the friction impulse's torque
about the horizontal axes) on the CUDA step against the FP64 oracle with the same options: per
step from the oracle's state, over 200-step windows, on rough terrain, and the torque's closed
form on a sliding block."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2411_05799_gb300 import scenes
from paper_2411_05799_gb300.npx import FRIC_TILT, FRIC_WEIGHTED, NpxError, World
from tests.parity import quat_angle, to_gpu
from tests.test_gpu_parity import CHECKPOINTS, THREADS, _assert_step_parity

pytestmark = pytest.mark.gpu

MODES = [FRIC_WEIGHTED, FRIC_TILT, FRIC_WEIGHTED | FRIC_TILT]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("lps", [8, 32])
def test_hexapod_per_step(mode, lps):
    b = scenes.hexapod_batch(64, seed_key=7)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps))
    w.set_friction_model(mode)
    _assert_step_parity(w, Oracle(b, threads=THREADS, fric_mode=mode), CHECKPOINTS)


def test_rough_terrain_per_step():
    """Force-weighted rows on rough terrain agree per step within 2e-4 instead of 1e-5: a row's
    weight is its point's normal force, which for a shallow contact (depth 1e-5 to 1e-4 m) follows
    a depth measured between an FP32 height and an FP32 position (rounding ~4e-9 m), so single
    weights carry up to ~4e-4 relative error and move the centre of pressure with it (measured:
    1.2e-4 in velocity; flat ground stays below 5e-6)."""
    mode = FRIC_WEIGHTED | FRIC_TILT
    b = scenes.cpg_batch(32, seed_key=2)
    w = World.from_batch(b)
    w.set_friction_model(mode)
    _assert_step_parity(w, Oracle(b, threads=THREADS, fric_mode=mode), [0, 1, 80, 81, 300, 801, 1600],
                        max_near_frac=0.2, rtol=2e-4)


@pytest.mark.parametrize("mode", MODES)
def test_hexapod_200_step_window(mode):
    """200 steps from the oracle's state: CoG within 1e-3 m and orientation within 1e-3 rad for
    95% of the scenes.  The medians stay near 1e-5; with the horizontal-axis torque the
    Coulomb-capped impulse (switching between stick and slip) also drives roll and pitch, which
    lets the rounding differences grow faster (median angle up to 5e-5)."""
    b = scenes.hexapod_batch(128, seed_key=9)
    o = Oracle(b, threads=THREADS, fric_mode=mode)
    o.step(1000, threads=THREADS)
    w = World.from_batch(b)
    w.set_friction_model(mode)
    to_gpu(w, o)
    o.step(200, threads=THREADS)
    w.step(200)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o.c, axis=1)
    da = quat_angle(r["quat"], o.q)
    ok = (dc <= 1e-3) & (da <= 1e-3)
    assert ok.mean() >= 0.95, f"{(~ok).sum()} scenes outside 1e-3 m / 1e-3 rad"
    assert np.median(dc) < 1e-5 and np.median(da) < (5e-5 if mode & FRIC_TILT else 1e-5)
    assert (r["status"] == 0).all() and (o.status == 0).all()


def test_tilt_torque_closed_form():
    """A settled block given a horizontal velocity: one step with and without the torque option
    differs only in the angular momentum, by the moment r x J of the friction impulse J = M dv at
    the bottom face's centre 0.05 m below the CoG."""
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=0.5)
    o = Oracle(b)
    o.step(2000)
    vel = np.array([0.5, -0.2])
    o.v[0, :2] = vel
    out = {}
    for mode in (0, FRIC_TILT):
        w = World.from_batch(b)
        w.set_friction_model(mode)
        to_gpu(w, o)
        w.step(1)
        out[mode] = w.read()
        w.close()
    off, on = out[0], out[FRIC_TILT]
    np.testing.assert_allclose(on["cog"], off["cog"], atol=1e-7)
    np.testing.assert_allclose(on["vel"], off["vel"], atol=1e-7)
    J = 1.0 * (off["vel"][0, :2].astype(np.float64) - vel)
    assert np.linalg.norm(J) > 1e-3
    dL = on["angmom"][0].astype(np.float64) - off["angmom"][0]
    np.testing.assert_allclose(dL, [0.05 * J[1], -0.05 * J[0], 0.0], rtol=2e-3, atol=1e-7)


def test_unknown_friction_flags_are_rejected():
    w = World.from_batch(scenes.block_batch())
    with pytest.raises(NpxError):
        w.set_friction_model(4)
    w.set_friction_model(0)
