"""Robot-robot collision (arenas) on the CUDA step against the FP64 oracle: per step from the
oracle's state while legs of neighbouring hexapods collide (flat ground and a shared rough height
map), over 200-step windows, the elastic
collision and the resting stack against their closed forms, robots apart against the plain
kernel, and the call's argument checks."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2411_05799_gb300 import construct, scenes
from paper_2411_05799_gb300.npx import NpxError, World, surrogate_collect
from tests.parity import STEP_RTOL, clone, near_threshold, per_step_compare, quat_angle, rel, to_gpu

pytestmark = pytest.mark.gpu

THREADS = 8
RADIUS = 0.01
# a pair this close to the reach 2 r decides its force (whose damping term jumps there) by
# rounding: FP32 positions of points within a metre of the origin carry ~3e-8 m
NEAR_PAIR = 1e-6


def pairs_in_reach(o: Oracle, size: int, theta=None):
    """Per arena: the point pairs of different robots closer than 2 r, and the smallest
    |distance - 2 r| (how close a pair is to switching), at the oracle's state (with joint
    angles theta if given)."""
    if theta is not None:
        o = clone(o)
        o.theta[:] = theta
    S = o.batch.n_scenes
    x = [o.points_world(s) for s in range(S)]
    n_in = np.zeros(S // size, np.int64)
    gap = np.full(S // size, np.inf)
    for a in range(S // size):
        for i in range(size):
            for j in range(i + 1, size):
                d = np.linalg.norm(x[a * size + i][:, None, :] - x[a * size + j][None, :, :], axis=2)
                n_in[a] += int((d < 2 * RADIUS).sum())
                gap[a] = min(gap[a], float(np.abs(d - 2 * RADIUS).min()))
    return n_in, gap


def _arena_step_parity(w, o, size, checkpoints):
    touched = 0
    n_near = n_tot = 0
    for n in checkpoints:
        o.step(n - o.n, threads=THREADS)
        err, near, o2, _ = per_step_compare(w, o, THREADS)
        n_in, gap = pairs_in_reach(o, size, o2.theta)
        _, gap2 = pairs_in_reach(o2, size)
        near_pair = np.repeat((gap < NEAR_PAIR) | (gap2 < NEAR_PAIR), size)
        touched += int(n_in.sum())
        ok = ~(near | near_pair)
        n_near += int((~ok).sum())
        n_tot += len(ok)
        for k in ("cog", "quat", "vel", "angmom", "theta"):
            worst = err[k][ok].max(initial=0.0)
            assert worst <= STEP_RTOL, f"step {n}: {k} rel err {worst:.3g}"
        assert err["contacts"][ok].max(initial=0) == 0, f"step {n}: contact bits differ"
    assert n_near <= 0.2 * n_tot, f"{n_near}/{n_tot} near-threshold exclusions"
    return touched


@pytest.mark.parametrize("size,lps", [(4, 8), (2, 8), (2, 16)])
def test_arena_hexapods_per_step(size, lps):
    b = scenes.arena_batch(32 // size, size, seed_key=11)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps))
    w.set_arenas(size, RADIUS)
    assert w.info()["lanes_per_scene"] == lps
    o = Oracle(b, threads=THREADS, arena=size, arena_radius=RADIUS)
    touched = _arena_step_parity(w, o, size, [0, 1, 80, 81, 300, 480, 801, 1200, 1600])
    assert touched > 100          # legs were in contact at the checkpoints


def rough_arena_batch(n_arenas, size, seed_key):
    """CPG hexapods on rough terrain in arenas: the members of an arena share the first member's
    height map and stand at the arena layout's places, above its highest cell."""
    b = scenes.cpg_batch(n_arenas * size, seed_key=seed_key)
    S = b.n_scenes
    hmap = (np.arange(S) // size * size).astype(np.int32)
    origin = np.zeros((S, 3), np.float32)
    origin[:, :2] = np.tile(np.asarray(scenes.ARENA_XY[size], np.float32), (n_arenas, 1))
    origin[:, 2] = b.heightmaps[hmap].max(axis=(1, 2)) - scenes.FOOT_Z + 0.01
    return b.with_(hmap=hmap, origin=origin)


@pytest.mark.parametrize("size,lps", [(4, 8), (2, 16)])
def test_arena_rough_terrain_per_step(size, lps):
    """The height-map build of the arena kernel: robots sharing a rough height map collide."""
    b = rough_arena_batch(32 // size, size, seed_key=15)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps))
    w.set_arenas(size, RADIUS)
    o = Oracle(b, threads=THREADS, arena=size, arena_radius=RADIUS)
    touched = _arena_step_parity(w, o, size, [0, 1, 80, 81, 300, 481, 800, 1201])
    assert touched > 20


@pytest.mark.parametrize("size", [2, 4])
def test_arena_200_step_window(size):
    """200 steps from the oracle's state after 0.6 s of walking into each other: CoG within 1e-3 m
    and orientation within 1e-3 rad for 95% of the robots."""
    b = scenes.arena_batch(64 // size, size, seed_key=12)
    o = Oracle(b, threads=THREADS, arena=size, arena_radius=RADIUS)
    o.step(600, threads=THREADS)
    w = World.from_batch(b)
    w.set_arenas(size, RADIUS)
    to_gpu(w, o)
    o.step(200, threads=THREADS)
    w.step(200)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o.c, axis=1)
    da = quat_angle(r["quat"], o.q)
    ok = (dc <= 1e-3) & (da <= 1e-3)
    assert ok.mean() >= 0.95, f"{(~ok).sum()} robots outside; median {np.median(dc):.3g} m {np.median(da):.3g} rad"
    assert np.median(dc) < 1e-4 and np.median(da) < 1e-4, (np.median(dc), np.median(da))
    assert (r["status"] == 0).all()


def _point_robot(m, x, v, dt, zeta):
    r = construct.Robot()
    r.create_point(0.0, 0.0, 0.0, m)
    return r.batch(1, origin=x, dt=dt).with_(vel=np.float32([v]), gravity=(0.0, 0.0, 0.0), contact_zeta=zeta)


def test_elastic_collision_closed_form():
    """Undamped points of 1 and 3 kg meeting at +-1 m/s in free space leave at -2 and 0 m/s, after
    a contact of pi / w_c; the GPU agrees with the textbook result and with the oracle."""
    dt = 1e-5
    b = scenes.concat([_point_robot(1.0, (-0.05, 0.0, 1.0), (1.0, 0.0, 0.0), dt, 0.0),
                       _point_robot(3.0, (0.05, 0.0, 1.0), (-1.0, 0.0, 0.0), dt, 0.0)])
    w = World.from_batch(b)
    w.set_arenas(2, RADIUS)
    w.step(12000)
    v = w.read()["vel"]
    np.testing.assert_allclose(v[:, 0], [-2.0, 0.0], atol=5e-3)
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    o.step(12000)
    np.testing.assert_allclose(v, o.v, atol=1e-4)


def test_box_resting_on_a_box():
    """The top box's corners settle 2 r - M_top g / (4 m_r w_c^2) above the bottom box's."""
    def box(m, z):
        r = construct.Robot()
        r.create_box(0.1, 0.1, 0.05, 0.0, 0.0, 0.0, m)
        return r.batch(1, origin=(0.0, 0.0, z))
    b = scenes.concat([box(2.0, 0.025), box(1.0, 0.095)])
    w = World.from_batch(b)
    w.set_arenas(2, RADIUS)
    w.step(4000)
    xb, xt = w.points(0), w.points(1)
    gap = np.sort(xt[:, 2])[:4].mean() - np.sort(xb[:, 2])[-4:].mean()
    m_r = (1.0 / 8) * (2.0 / 8) / (3.0 / 8)
    assert gap == pytest.approx(2 * RADIUS - abs(b.gravity[2]) / (4 * m_r * 300.0 ** 2), rel=1e-4)


def test_robots_apart_match_the_plain_kernel():
    """Arenas whose robots stay 2 m apart step as the world without arenas (the arena kernel adds
    exact zeros)."""
    b = scenes.arena_batch(16, 2, seed_key=13)
    b = b.with_(origin=b.origin + np.float32([[0, -1, 0], [0, 1, 0]] * 16))
    a = World.from_batch(b, configure=dict(lanes_per_scene=8))
    a.set_arenas(2, RADIUS)
    p = World.from_batch(b, configure=dict(lanes_per_scene=8))
    a.step(100)
    p.step(100)
    ra, rp = a.read(), p.read()
    for k in ("cog", "vel", "angmom", "quat"):
        np.testing.assert_allclose(ra[k], rp[k], rtol=1e-5, atol=1e-6)


def test_non_finite_neighbour_exerts_nothing():
    """A robot written with a velocity that is not a number freezes in its first step; its
    neighbour, legs in reach, feels nothing from it and follows the oracle."""
    b = scenes.arena_batch(1, 2, seed_key=8)
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    o.step(600)
    o.v[1] = np.nan
    w = World.from_batch(b)
    w.set_arenas(2, RADIUS)
    to_gpu(w, o)
    o.step(100)
    w.step(100)
    r = w.read()
    assert r["status"][1] != 0 and o.status[1] != 0 and r["status"][0] == 0
    np.testing.assert_allclose(r["cog"][0], o.c[0], atol=1e-4)
    np.testing.assert_allclose(r["vel"][0], o.v[0], atol=1e-3)


def test_full_size_arenas_sampled():
    """The benchmark's arena workload at full size (4,096 hexapods in arenas of four, autotuned
    launch shape): after 0.6 s of walking into each other, one step from the GPU's own state
    agrees per step with the oracle on sampled arenas (their state copied from the GPU)."""
    size = 4
    b = scenes.arena_batch(1024, size)
    w = World.from_batch(b)
    w.set_arenas(size, RADIUS)
    w.autotune(100)
    w.step(600)
    r0 = w.read()
    kap0 = w.contacts()
    arenas = [0, 301, 702, 1023]
    idx = np.concatenate([np.arange(a * size, (a + 1) * size) for a in arenas])
    sub = b.subset(idx)
    o = Oracle(sub, threads=THREADS, arena=size, arena_radius=RADIUS)
    jo, po = b.joint_off, b.point_off
    o.c[:] = r0["cog"][idx]
    o.q[:] = r0["quat"][idx]
    o.v[:] = r0["vel"][idx]
    o.L[:] = r0["angmom"][idx]
    o.theta[:] = np.concatenate([r0["theta"][jo[s]:jo[s + 1]] for s in idx])
    o.kappa[:] = np.concatenate([kap0[po[s]:po[s + 1]] for s in idx])
    o.n = r0["step"]
    n_in, gap = pairs_in_reach(o, size)
    o2 = clone(o)
    o2.step(1, threads=THREADS)
    _, gap2 = pairs_in_reach(o2, size)
    w.step(1)
    r = w.read()
    near = near_threshold(o, o2, o2.theta) | np.repeat((gap < NEAR_PAIR) | (gap2 < NEAR_PAIR), size)
    ok = ~near
    assert ok.sum() >= len(idx) // 2 and n_in.sum() > 0
    for k, ref in (("cog", o2.c), ("vel", o2.v), ("angmom", o2.L)):
        assert rel(r[k][idx], ref).max(1)[ok].max(initial=0.0) <= STEP_RTOL, k


def test_arena_arguments():
    b = scenes.arena_batch(3, 2, seed_key=14)          # 6 scenes
    w = World.from_batch(b)
    for size, radius in ((3, RADIUS), (4, RADIUS), (2, 0.0), (2, math.inf)):
        with pytest.raises(NpxError):
            w.set_arenas(size, radius)
    w.set_arenas(2, RADIUS)
    with pytest.raises(NpxError):
        w.configure(lanes_per_scene=32)
    with pytest.raises(NpxError, match="arenas"):      # the surrogate describes robots alone
        surrogate_collect(w, 1, None, None)
    w.step(10)
    w.set_arenas(1)                                    # off again: every scene alone
    w.step(10)
    assert (w.read()["status"] == 0).all()


def test_pair_list_overflow_takes_the_full_pass():
    """Robots of an arena stacked almost on top of each other put more point pairs within reach
    than a warp's pair list holds (4,096 entries): the step then takes the full pair pass.  From
    rest the pair forces have no damping term, so they are continuous where pairs leave reach
    (no pair decides its force by rounding), and the first step agrees with the oracle on every
    scene."""
    size = 4
    b = scenes.arena_batch(2, size, seed_key=17)
    org = b.origin.copy()
    for a in range(2):
        for k in range(size):
            org[a * size + k] = org[a * size] + np.float32([0.005 * k, 0.003 * k, 0.0])
    b = b.with_(origin=org, vel=np.zeros_like(b.vel), omega=np.zeros_like(b.omega))
    o = Oracle(b, arena=size, arena_radius=RADIUS, threads=THREADS)
    n_in, _ = pairs_in_reach(o, size)
    assert n_in.min() > 4096, n_in
    w = World.from_batch(b, configure=dict(lanes_per_scene=8))
    w.set_arenas(size, RADIUS)
    err, near, o2, r = per_step_compare(w, o, THREADS)
    assert not near.any()
    for k in ("cog", "quat", "vel", "angmom", "theta"):
        assert err[k].max() <= STEP_RTOL, f"{k} rel err {err[k].max():.3g}"
    assert err["contacts"].max() == 0
    assert np.abs(r["vel"]).max() > 0.1                 # the stack pushes apart


def test_arena_runs_are_deterministic():
    """The pair lists are appended in a fixed order (warp-wide rounds, prefix sums) and summed
    pair after pair, so two runs of the same arenas, through several list rebuilds, joint updates
    and launches, end bit-identical."""
    b = scenes.arena_batch(64, 4, seed_key=19)
    out = []
    for _ in range(2):
        w = World.from_batch(b, configure=dict(lanes_per_scene=8, chunk_steps=250))
        w.set_arenas(4, RADIUS)
        w.step(1000)
        out.append(w.read())
    for k in ("cog", "quat", "vel", "angmom", "theta", "contacts", "status"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_arena_with_friction_options_per_step():
    """Arenas with both friction refinements on (force-weighted rows and the friction impulse's
    horizontal-axis torque; the arena build of the step kernel compiles them in): per step from
    the oracle's state with the same options while legs collide."""
    from paper_2411_05799_gb300.npx import FRIC_TILT, FRIC_WEIGHTED
    mode = FRIC_WEIGHTED | FRIC_TILT
    size = 4
    b = scenes.arena_batch(8, size, seed_key=12)
    w = World.from_batch(b, configure=dict(lanes_per_scene=8))
    w.set_arenas(size, RADIUS)
    w.set_friction_model(mode)
    o = Oracle(b, threads=THREADS, fric_mode=mode, arena=size, arena_radius=RADIUS)
    touched = _arena_step_parity(w, o, size, [0, 1, 80, 81, 300, 480, 801, 1200])
    assert touched > 50
