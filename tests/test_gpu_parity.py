"""CUDA step kernel vs the FP64 oracle, through the C-ABI, on seeded synthetic scenes.

Per step (from the oracle's exact state): every component within 1e-5 relative, contact bits
and sensors exact, except scenes with a point within 1e-5 m of the ground, whose contact bits
rounding decides (counted, and required to be rare).  Over 200-step windows: CoG within 1e-3 m
and orientation within 1e-3 rad for at least 95% of scenes (contacts are chaotic, so the
agreement is checked statistically).  The full-size hexapod workload is checked in the launch
configuration the benchmark uses."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle.oracle import Oracle, quat_matrix
from paper_2411_05799_gb300 import npx, scenes
from paper_2411_05799_gb300.npx import World, NpxError
from tests.parity import (STEP_RTOL, clone, per_step_compare, quat_angle, rel, to_gpu)

pytestmark = pytest.mark.gpu

THREADS = 8


def _assert_step_parity(world, o, checkpoints, max_near_frac=0.1, rtol=STEP_RTOL, worst_out=None):
    n_near = n_tot = 0
    for n in checkpoints:
        o.step(n - o.n, threads=THREADS)
        err, near, _, _ = per_step_compare(world, o, THREADS)
        ok = ~near
        n_near += near.sum()
        n_tot += len(near)
        for k in ("cog", "quat", "vel", "angmom", "theta"):
            worst = err[k][ok].max(initial=0.0)
            if worst_out is not None:
                worst_out[k] = max(worst_out.get(k, 0.0), worst)
            assert worst <= rtol, f"step {n}: {k} rel err {worst:.3g}"
        assert err["contacts"][ok].max(initial=0) == 0, f"step {n}: contact bits differ"
        assert err["sensors"][ok].max(initial=0) == 0, f"step {n}: sensors differ"
    assert n_near <= max_near_frac * n_tot, f"{n_near}/{n_tot} near-threshold exclusions"


CHECKPOINTS = [0, 1, 2, 79, 80, 81, 160, 333, 479, 480, 800, 1201, 1600, 2400]


@pytest.mark.parametrize("lps", [8, 16, 32])
def test_hexapod_per_step(lps):
    b = scenes.hexapod_batch(64, seed_key=7)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps))
    _assert_step_parity(w, Oracle(b, threads=THREADS), CHECKPOINTS)


def test_uneven_per_step():
    b = scenes.uneven_batch(48, seed_key=3)
    w = World.from_batch(b)
    assert w.info()["max_points"] > 512
    _assert_step_parity(w, Oracle(b, threads=THREADS), [0, 1, 80, 81, 400, 999])


def test_single_body_per_step():
    b = scenes.single_body()
    w = World.from_batch(b)
    o = Oracle(b)
    # free flight, first impact, tumbling on the ground, rest
    _assert_step_parity(w, o, [0, 100, 290, 300, 310, 320, 330, 400, 500, 700, 1000, 3000, 9999],
                        max_near_frac=0.3)


def test_rough_terrain_cpg_per_step():
    """Hexapods with per-leg CPG targets on 128 x 128 rough height fields (5 cm cells)."""
    b = scenes.cpg_batch(32, seed_key=2)
    w = World.from_batch(b)
    _assert_step_parity(w, Oracle(b, threads=THREADS), [0, 1, 80, 81, 300, 801, 1600],
                        max_near_frac=0.2)


def test_rough_terrain_200_step_window():
    """The flat hexapods' bar: 95% of the scenes within 1 mm and 1 mrad of the oracle after 200
    steps (on 512 scenes of four such windows all were within 1e-3 and 508 within 1e-5)."""
    dc, da, r, o = _window(scenes.cpg_batch(64, seed_key=3), 500)
    ok = (dc <= 1e-3) & (da <= 1e-3)
    assert ok.mean() >= 0.95, f"{(~ok).sum()} of {len(ok)} scenes outside 1e-3 m / 1e-3 rad"
    assert np.median(dc) < 1e-5


@pytest.mark.parametrize("terrain", ["flat", "rough"])
def test_true_relative_error_of_velocity_and_angular_momentum(terrain):
    """The per-step checks divide by max(|ref|, 1), which for velocities and angular momenta
    (typically 0.2 m/s and 0.04 kg m^2/s) is an absolute bound.  Here the relative error of the
    whole vector, |gpu - oracle| / |oracle|, is bounded by 5e-5 on every scene not decided by
    rounding at the ground (measured worst: 5.3e-6 for v, 7.7e-6 for L).  Vectors shorter than
    1e-3 of their unit are left out (a resting robot's jitter)."""
    b = scenes.hexapod_batch(64, seed_key=7) if terrain == "flat" else scenes.cpg_batch(32, seed_key=2)
    w = World.from_batch(b)
    o = Oracle(b, threads=THREADS)
    worst = {"vel": 0.0, "angmom": 0.0}
    n_checked = 0
    for n in [1, 80, 81, 333, 800, 1600]:
        o.step(n - o.n, threads=THREADS)
        err, near, o2, r = per_step_compare(w, o, THREADS)
        for k, ref in (("vel", o2.v), ("angmom", o2.L)):
            mag = np.linalg.norm(ref, axis=1)
            keep = ~near & (mag >= 1e-3)
            e = np.linalg.norm(np.asarray(r[k], np.float64) - ref, axis=1)[keep] / mag[keep]
            worst[k] = max(worst[k], e.max(initial=0.0))
            n_checked += int(keep.sum())
    assert n_checked > 300
    for k, v in worst.items():
        assert v <= 5e-5, f"{k}: worst relative error {v:.3g}"


def _window(b, n0, horizon=200, lps=0):
    o = Oracle(b, threads=THREADS)
    o.step(n0, threads=THREADS)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps) if lps else None)
    to_gpu(w, o)
    o.step(horizon, threads=THREADS)
    w.step(horizon)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o.c, axis=1)
    da = quat_angle(r["quat"], o.q)
    return dc, da, r, o


@pytest.mark.parametrize("n0", [0, 1000, 4000])
def test_hexapod_200_step_windows(n0):
    dc, da, r, o = _window(scenes.hexapod_batch(128, seed_key=9), n0)
    ok = (dc <= 1e-3) & (da <= 1e-3)
    assert ok.mean() >= 0.95, f"{(~ok).sum()} scenes outside 1e-3 m / 1e-3 rad"
    assert np.median(dc) < 1e-5 and np.median(da) < 1e-5
    assert (r["status"] == 0).all() and (o.status == 0).all()


def test_hexapod_long_horizon_statistics():
    """5 s of walking: per-scene trajectories may part ways, their distributions may not."""
    b = scenes.hexapod_batch(256, seed_key=11)
    o = Oracle(b, threads=THREADS)
    w = World.from_batch(b)
    o.step(5000, threads=THREADS)
    w.step(5000)
    r = w.read()
    for name, g, c in (("height", r["cog"][:, 2], o.c[:, 2]),
                       ("distance", np.linalg.norm(r["cog"][:, :2] - b.origin[:, :2], axis=1),
                        np.linalg.norm(o.c[:, :2] - b.origin[:, :2], axis=1)),
                       ("feet down", [bin(x).count("1") for x in r["contacts"]],
                        [bin(x).count("1") for x in o.sensors])):
        g, c = np.asarray(g, np.float64), np.asarray(c, np.float64)
        se = math.sqrt(g.var() / len(g) + c.var() / len(c)) + 1e-12
        assert abs(g.mean() - c.mean()) <= 3 * se, f"{name}: {g.mean()} vs {c.mean()} (se {se})"
    close = np.linalg.norm(r["cog"] - o.c, axis=1) < 1e-3
    assert close.mean() > 0.5


def test_full_size_hexapod_in_bench_configuration():
    """4,096 hexapods after 1,000 steps (the oracle runs them all): one step from the oracle's
    state in the launch shape the benchmark picks, every scene compared."""
    b = scenes.hexapod_batch(4096)
    w = World.from_batch(b)
    w.autotune(50)
    o = Oracle(b, threads=THREADS)
    o.step(1000, threads=THREADS)
    err, near, o2, r = per_step_compare(w, o, THREADS)
    ok = ~near
    assert near.mean() < 0.1
    for k in ("cog", "quat", "vel", "angmom", "theta"):
        assert err[k][ok].max() <= STEP_RTOL, k
    assert err["contacts"][ok].max() == 0
    # and a 200-step window at full size
    to_gpu(w, o)
    o.step(200, threads=THREADS)
    w.step(200)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o.c, axis=1)
    assert ((dc <= 1e-3) & (quat_angle(r["quat"], o.q) <= 1e-3)).mean() >= 0.95


# ----------------------------------------------------------------------------- closed forms on GPU

def test_gpu_free_fall():
    b = scenes.single_body().with_(origin=np.array([[0.3, -0.2, 2.0]], np.float32))
    w = World.from_batch(b)
    r0 = w.read()
    n, dt, g = 600, b.dt, -b.gravity[2]
    w.step(n)
    r = w.read()
    c0, v0 = r0["cog"][0].astype(np.float64), r0["vel"][0].astype(np.float64)
    assert abs(r["cog"][0, 2] - (c0[2] + n * dt * v0[2] - g * dt * dt * n * (n + 1) / 2)) < 2e-5
    assert abs(r["vel"][0, 2] - (v0[2] - g * n * dt)) < 1e-4
    np.testing.assert_allclose(r["cog"][0, :2], c0[:2] + n * dt * v0[:2], atol=2e-5)
    np.testing.assert_allclose(r["angmom"][0], r0["angmom"][0], rtol=0, atol=0)


def test_gpu_isotropic_rotation():
    wv = np.array([1.3, -2.1, 0.7], np.float32).astype(np.float64)
    b = scenes.block_batch(extent=(0.25, 0.25, 0.25), counts=(3, 3, 3), omega=wv, z_gap=20.0)
    b = b.with_(quat=scenes.random_unit_quat(np.random.default_rng(5), 1))
    w = World.from_batch(b)
    R0 = Rotation.from_quat(np.roll(w.read()["quat"][0].astype(np.float64), -1))
    w.step(500)
    q = w.read()["quat"][0].astype(np.float64)
    want = (Rotation.from_rotvec(500 * b.dt * wv) * R0).as_matrix()
    np.testing.assert_allclose(quat_matrix(q / np.linalg.norm(q)), want, atol=2e-5)


def test_gpu_block_rests_on_plane():
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=0.5)
    w = World.from_batch(b)
    w.step(1000)
    r = w.read()
    m_pt = float(np.float32(1.0 / 18))
    d = 18 * m_pt * -b.gravity[2] / (9 * m_pt * b.contact_omega ** 2)
    assert abs(r["cog"][0, 2] - (0.05 - d)) < 2e-6
    assert np.abs(r["vel"][0]).max() < 1e-5
    w.step(2000)
    r2 = w.read()
    assert np.abs(r2["cog"][0] - r["cog"][0]).max() < 2e-6
    assert r2["contacts"][0] == 1


@pytest.mark.parametrize("theta_deg,mu,sticks", [(20, 0.5, True), (35, 0.5, False), (45, 0.8, False)])
def test_gpu_incline(theta_deg, mu, sticks):
    theta = math.radians(theta_deg)
    b = scenes.tilted_gravity(scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2),
                                                 mass=1.0, mu=mu), theta)
    w = World.from_batch(b)
    vs = []
    for _ in range(300):
        w.step(10)
        vs.append(w.read()["vel"][0, 0])
    vs = np.array(vs, np.float64)
    if sticks:
        assert np.abs(vs[50:]).max() < 1e-5
    else:
        want = b.gravity[0] - float(np.float32(mu)) * -b.gravity[2]
        acc = (vs[-1] - vs[100]) / ((len(vs) - 1 - 100) * 10 * b.dt)
        assert abs(acc - want) < 1e-3 * want


def test_gpu_points_match_oracle_kinematics():
    b = scenes.hexapod_batch(4, seed_key=2)
    rng = np.random.default_rng(4)
    b = b.with_(theta0=rng.uniform(-1, 1, b.n_joints).astype(np.float32),
                quat=scenes.random_unit_quat(rng, 4))
    w = World.from_batch(b)
    o = Oracle(b)
    for s in range(4):
        np.testing.assert_allclose(w.points(s)[:352], o.points_world(s), atol=2e-6)
    r = w.read()
    np.testing.assert_allclose(r["cog"], o.c, atol=2e-6)
    np.testing.assert_allclose(r["angmom"], o.L, rtol=1e-5, atol=1e-8)
    np.testing.assert_allclose(r["omega"], o.omega(), rtol=1e-4, atol=1e-6)


def _window_by_tma(ny, nx):
    """Whether the kernel loads its 16 x 16-cell windows of an ny x nx FP32 map by TMA box copies:
    maps at least the window's size whose rows are a multiple of 16 bytes."""
    return ny >= 16 and nx >= 16 and (4 * nx) % 16 == 0


@pytest.mark.parametrize("ny, nx, spread", [(16, 16, 0.4), (8, 12, 0.4), (40, 48, 1.8), (20, 22, 0.6),
                                            (24, 36, 1.0)])
def test_gpu_heightmap_cells(ny, nx, spread):
    """Random clouds over random height maps: the first step's contact bits agree point for
    point with the oracle's (same single-precision cell and contact decisions).  The maps are the
    size of the kernel's cached window, smaller than it (cells past the map's edge read the
    clamped edge) and larger (points outside the window, windows clamped at the map's edges);
    every cloud also reaches off the map.  Windows load by TMA box copies where the map allows
    (16 x 16, 40 x 48, 24 x 36 cells: windows at every column offset modulo 4, box columns past
    the right edge) and by plain loads elsewhere (8 x 12; 20 x 22, whose rows are not a multiple
    of 16 bytes)."""
    rng = np.random.default_rng(21)
    maps = rng.uniform(-0.05, 0.05, (2, ny, nx)).astype(np.float32)
    S, n = 8, 200
    robots = []
    for _ in range(S):
        pts = scenes.box_uniform(rng, (1.6, 1.6, 0.12), (0, 0, 0), n)
        robots.append(([((1.6, 1.6, 0.12), (0, 0, 0), 1.0, -1, None, None, 0)], [pts]))
    b = scenes._assemble(robots, mu=np.full(S, 0.5), origin=rng.uniform(-spread, spread, (S, 3)) * [1, 1, 0],
                         quat=scenes.random_unit_quat(rng, S), vel=np.zeros((S, 3)),
                         omega=np.zeros((S, 3)), act_params=None, name="lut",
                         hmap=rng.integers(0, 2, S), heightmaps=maps, hm_scale=10.0,
                         hm_origin=(-nx / 20, -ny / 20), act_mode=scenes.ACT_HOLD)
    w = World.from_batch(b)
    assert w.info()["hm_window_tma"] == int(_window_by_tma(ny, nx))
    o = Oracle(b)
    o.step(1)
    w.step(1)
    kap = w.contacts()
    assert kap.sum() > 100
    x = np.concatenate([o.points_world(s) for s in range(S)])
    assert np.count_nonzero(kap != o.kappa) <= 2      # points within rounding of the surface
    assert (kap == o.kappa).mean() > 0.99


@pytest.mark.parametrize("ny, nx", [(40, 48), (40, 46)])
def test_height_map_window_moves_are_exact(ny, nx):
    """The window is a cache of the map: blocks sliding fast across a map (about a metre, two
    window moves for the median block; some windows held at the map's edge, some blocks sliding
    off it) step bit-identically whether every step
    is its own launch (a fresh window each step) or all 400 steps are one launch (windows moved
    inside it); TMA box copies (48 columns) and plain loads (46 columns) alike."""
    rng = np.random.default_rng(33)
    maps = rng.uniform(-0.03, 0.03, (3, ny, nx)).astype(np.float32)
    S = 48
    robots = []
    for _ in range(S):
        pts = scenes.box_uniform(rng, (0.3, 0.3, 0.1), (0, 0, 0), 96)
        robots.append(([((0.3, 0.3, 0.1), (0, 0, 0), 1.0, -1, None, None, 0)], [pts]))
    ang = rng.uniform(0, 2 * np.pi, S)
    vel = np.stack([3.0 * np.cos(ang), 3.0 * np.sin(ang), np.zeros(S)], 1)
    origin = np.concatenate([rng.uniform(-1.2, 1.2, (S, 2)), np.full((S, 1), 0.09)], 1)
    b = scenes._assemble(robots, mu=np.full(S, 0.3), origin=origin, quat=np.tile([1.0, 0, 0, 0], (S, 1)),
                         vel=vel, omega=np.zeros((S, 3)), act_params=None, name="slide",
                         hmap=rng.integers(0, 3, S), heightmaps=maps, hm_scale=10.0,
                         hm_origin=(-nx / 20, -ny / 20), act_mode=scenes.ACT_HOLD)
    one = World.from_batch(b, configure=dict(chunk_steps=1))
    assert one.info()["hm_window_tma"] == int(_window_by_tma(ny, nx))
    one.step(400)
    many = World.from_batch(b, configure=dict(chunk_steps=400))
    many.step(400)
    r1, r2 = one.read(), many.read()
    moved = np.linalg.norm(r2["cog"][:, :2] - origin[:, :2], axis=1)
    assert np.median(moved) > 0.5                    # 5 cells: several window moves per scene
    assert (r2["status"] == 0).all()
    for k in ("cog", "quat", "vel", "angmom", "contacts"):
        assert np.array_equal(r1[k], r2[k]), k


# ----------------------------------------------------------------------------- edge cases

def test_single_point_scene_and_chain_and_max_points():
    rng = np.random.default_rng(1)
    one = ([((0.0, 0.0, 0.0), (0, 0, 0), 0.5, -1, None, None, 0)], [np.zeros((1, 3), np.float32)])
    chain_links = [((0.05, 0.05, 0.05), (0, 0, 0), 0.1, -1, None, None, -1)]
    chain_pts = [scenes.box_lattice((0.05, 0.05, 0.05), (0, 0, 0), (2, 2, 2))]
    for k in range(1, 64):
        ctr = (0.05 * k, 0.0, 0.0)
        chain_links.append(((0.05, 0.05, 0.05), ctr, 0.1, k - 1, (0.05 * k - 0.025, 0, 0),
                            (0.0, 1.0, 0.0), -1))
        chain_pts.append(scenes.box_lattice((0.05, 0.05, 0.05), ctr, (2, 2, 2)))
    big = ([((0.4, 0.4, 0.2), (0, 0, 0), 3.0, -1, None, None, 1)],
           [scenes.box_uniform(rng, (0.4, 0.4, 0.2), (0, 0, 0), 2048)])
    robots = [one, (chain_links, chain_pts), big]
    J = 63
    act = np.zeros((J, 4), np.float32)
    act[:, 0] = 0.2
    act[:, 1] = 1.5
    b = scenes._assemble(robots, mu=[0.7, 0.7, 0.7], origin=[(0, 0, 0.02), (0, 0, 0.05), (0, 0, 0.12)],
                         quat=[(1, 0, 0, 0)] * 3, vel=rng.normal(0, 0.3, (3, 3)),
                         omega=rng.normal(0, 1, (3, 3)), act_params=act, name="edges")
    w = World.from_batch(b)
    info = w.info()
    assert info["max_points"] == 2048 and info["max_links"] == 64 and info["lanes_per_scene"] == 32
    _assert_step_parity(w, Oracle(b), [0, 1, 5, 80, 81, 200, 500], max_near_frac=0.35)


def test_zero_steps_and_chunking_and_graphs_are_bit_exact():
    b = scenes.hexapod_batch(64, seed_key=5)
    ref = World.from_batch(b)
    ref.step(0)
    r0 = ref.read()
    ref.step(1500)
    ra = ref.read()
    w = World.from_batch(b, configure=dict(chunk_steps=250))
    assert np.array_equal(w.read()["cog"], r0["cog"])
    w.use_graphs(False)
    w.step(700)
    w.step(800)
    rb = w.read()
    for k in ("cog", "quat", "vel", "angmom", "theta", "contacts"):
        assert np.array_equal(ra[k], rb[k]), k
    w2 = World.from_batch(b)
    w2.step(1500)
    assert np.array_equal(w2.read()["cog"], ra["cog"])     # deterministic
    assert ra["step"] == rb["step"] == 1500


def test_launch_shapes_agree():
    b = scenes.hexapod_batch(96, seed_key=6)
    outs = []
    for lps, wpb in ((8, 2), (16, 4), (32, 8), (16, 8)):
        w = World.from_batch(b, configure=dict(lanes_per_scene=lps, warps_per_block=wpb))
        w.step(120)
        outs.append(w.read())
    for r in outs[1:]:
        assert rel(r["cog"], outs[0]["cog"]).max() < 1e-5
        assert quat_angle(r["quat"], outs[0]["quat"]).max() < 5e-5


def test_export_import_resumes_exactly():
    b = scenes.hexapod_batch(32, seed_key=8)
    w = World.from_batch(b)
    w.step(333)
    blob = w.export_state()
    w.step(400)
    ra = w.read()
    w2 = World.from_batch(b)
    w2.import_state(blob)
    assert w2.read()["step"] == 333
    w2.step(400)
    rb = w2.read()
    for k in ("cog", "quat", "vel", "angmom", "theta", "contacts", "status"):
        assert np.array_equal(ra[k], rb[k]), k


def test_autotune_keeps_state():
    b = scenes.hexapod_batch(256, seed_key=12)
    w = World.from_batch(b)
    w.step(100)
    before = w.read()
    info = w.autotune(60)
    after = w.read()
    assert info["lanes_per_scene"] in (8, 16, 32)
    for k in ("cog", "quat", "vel", "angmom", "theta", "contacts"):
        assert np.array_equal(before[k], after[k]), k
    assert after["step"] == 100


def test_non_finite_scene_freezes_alone():
    b = scenes.hexapod_batch(8, seed_key=13)
    o = Oracle(b)
    o.step(50)
    w = World.from_batch(b)
    to_gpu(w, o)
    v = o.v.copy()
    v[3, 0] = np.nan
    w.write_state(o.c, o.q, v, o.L, o.theta, o.kappa, o.n)
    w.step(100)
    r = w.read()
    assert r["status"][3] & 1
    assert (np.delete(r["status"], 3) == 0).all()
    np.testing.assert_array_equal(r["cog"][3], o.c[3].astype(np.float32))   # frozen
    wref = World.from_batch(b)
    to_gpu(wref, o)
    wref.step(100)
    rr = wref.read()
    keep = np.arange(8) != 3
    assert np.array_equal(rr["cog"][keep], r["cog"][keep])


def test_runtime_argument_errors():
    b = scenes.hexapod_batch(2)
    w = World.from_batch(b)
    with pytest.raises(NpxError):
        w.step(-1)
    with pytest.raises(NpxError):
        w.configure(lanes_per_scene=12)
    with pytest.raises(NpxError):
        w.add_scenes(b)                   # after finalize
    with pytest.raises(NpxError):
        w.import_state(b"\0" * 16)


def test_ragged_extremes_per_step():
    """One world from a single point up to the largest scene (2,048 points, 64 per lane at 32
    lanes per scene), tumbling onto the ground, step by step against the oracle.  (Two-point rods
    are left out: their inertia about the rod axis is only the point-sphere term, a condition
    number near 1e4, which puts FP32 angular velocities beyond 1e-5 per step; the oracle's rod pin
    covers them.)"""
    counts = [2048, 1, 4, 3, 31, 32, 33, 63, 64, 65, 511, 1024, 1500, 7]
    b = scenes.ragged_bodies(counts, seed_key=5)
    w = World.from_batch(b)
    assert w.info()["max_points"] == 2048 and w.info()["lanes_per_scene"] == 32
    _assert_step_parity(w, Oracle(b, threads=THREADS), [0, 1, 100, 200, 260, 300, 400, 700],
                        max_near_frac=0.3)


def test_size_classes_match_the_oracle():
    """A world that splits into two size classes (small and large scenes, one launch each) gives
    the same 200-step results as the oracle."""
    counts = [8] * 1100 + [600] * 1100
    b = scenes.ragged_bodies(counts, seed_key=6)
    w = World.from_batch(b)
    assert w.info()["size_classes"] == 2
    dc, da, r, o = _window_world(b, w, 200)
    assert ((dc <= 1e-3) & (da <= 1e-3)).mean() >= 0.95
    assert np.median(dc) < 1e-5


@pytest.mark.parametrize("graphs", [True, False])
def test_many_size_classes_run_concurrently(graphs):
    """Six size classes: their launches go round-robin to the world's stream and three side
    streams (forked and joined with events, inside a captured graph or not), each with its own
    work-queue counter; 200 steps agree with the oracle."""
    counts = [c for c in (8, 20, 50, 120, 300, 700) for _ in range(300)]
    b = scenes.ragged_bodies(counts, seed_key=8)
    w = World.from_batch(b)
    w.use_graphs(graphs)
    assert w.info()["size_classes"] == 6
    dc, da, r, o = _window_world(b, w, 200)
    assert (r["status"] == 0).all()
    assert ((dc <= 1e-3) & (da <= 1e-3)).mean() >= 0.95
    assert np.median(dc) < 1e-5


def _window_world(b, w, horizon):
    o = Oracle(b, threads=THREADS)
    to_gpu(w, o)
    o.step(horizon, threads=THREADS)
    w.step(horizon)
    r = w.read()
    return np.linalg.norm(r["cog"] - o.c, axis=1), quat_angle(r["quat"], o.q), r, o


def test_window_copy_wait_gives_up_and_the_context_survives():
    """The height-map window's copy wait is bounded: lanes whose copy never comes give up after
    the one-second limit (the step kernel then freezes the scene with status bit 2), lanes whose
    barrier completed go on, the warp leaves the wait together, and the context still steps a
    rough-terrain world correctly."""
    torch = pytest.importorskip("torch")
    st = torch.cuda.current_stream().cuda_stream
    up, ok, us = npx.window_wait_selftest(st)
    assert (up, ok) == (16, 16)
    assert 0.9e6 <= us <= 5e6, us
    test_rough_terrain_cpg_per_step()
