"""Host-side inputs of robot-robot collision: batch concatenation keeps every scene's arrays and
offsets, refuses batches of different worlds, and the arena layout places each arena's robots
where it says, with legs of facing rows within reach of each other."""
import numpy as np
import pytest

from paper_2411_05799_gb300 import construct, scenes


def test_concat_keeps_scenes():
    a = scenes.hexapod_batch(3, seed_key=1)
    r = construct.Robot()
    r.create_box(0.1, 0.2, 0.3, 0.0, 0.0, 0.0, 2.0)
    b = r.batch(2, origin=(0.0, 0.0, 0.5))
    c = scenes.concat([a, b.with_(act_mode=a.act_mode)])
    assert c.n_scenes == 5
    np.testing.assert_array_equal(c.link_off, np.concatenate([a.link_off, a.link_off[-1] + b.link_off[1:]]))
    np.testing.assert_array_equal(c.point_off, np.concatenate([a.point_off, a.point_off[-1] + b.point_off[1:]]))
    for s_c, (src, s) in enumerate([(a, 0), (a, 1), (a, 2), (b, 0), (b, 1)]):
        sub = c.subset([s_c])
        ref = src.subset([s])
        for k in ("p0", "m", "plink", "parent", "anchor", "axis", "lo", "hi", "sensor", "origin", "vel"):
            np.testing.assert_array_equal(getattr(sub, k), getattr(ref, k), err_msg=k)


def test_concat_refuses_different_worlds():
    a = scenes.hexapod_batch(1)
    with pytest.raises(ValueError):
        scenes.concat([a, a.with_(dt=2e-3)])
    with pytest.raises(ValueError):
        scenes.concat([a, scenes.cpg_batch(1)])          # height maps


@pytest.mark.parametrize("size", [2, 4])
def test_arena_layout(size):
    b = scenes.arena_batch(3, size, seed_key=2)
    assert b.n_scenes == 3 * size and b.meta["arena"] == size
    xy = b.origin[:, :2].reshape(3, size, 2)
    np.testing.assert_allclose(xy, np.broadcast_to(np.float32(scenes.ARENA_XY[size]), (3, size, 2)))
    # every robot has its own gait
    J = b.n_joints // b.n_scenes
    assert len({b.act_params[s * J:(s + 1) * J].tobytes() for s in range(b.n_scenes)}) == b.n_scenes
    # the facing rows' legs overlap in y: some points of robot 0 and of the robot across are
    # closer than a few centimetres at rest
    p = [b.p0[b.point_off[s]:b.point_off[s + 1]] + b.origin[s] for s in (0, size // 2)]
    d = np.linalg.norm(p[0][:, None, :] - p[1][None, :, :], axis=2)
    assert d.min() < 0.05
