"""Robot-robot collision in the oracle (the extension named as future work), pinned to mechanics
that does not depend on the oracle: a hand-worked pair force, Newton's third law with central
forces, the textbook elastic collision and the contact time of a spring of the reduced mass,
exact conservation of linear and angular momentum in free flight, the closed-form gap of a box
resting on a box, and no interaction between robots apart or frozen."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, arena_forces
from paper_2411_05799_gb300 import construct, scenes

W_C, RADIUS = 300.0, 0.01


def _point_robot(m, x, v, dt, zeta=1.0):
    r = construct.Robot()
    r.create_point(0.0, 0.0, 0.0, m)
    return r.batch(1, origin=x, dt=dt).with_(vel=np.float32([v]), gravity=(0.0, 0.0, 0.0), contact_zeta=zeta)


def _box_robot(w, h, d, m, x, dt=1e-3):
    r = construct.Robot()
    r.create_box(w, h, d, 0.0, 0.0, 0.0, m)
    return r.batch(1, origin=x, dt=dt)


def test_pair_force_hand_worked():
    """Point a (1 kg) at the origin, its robot's CoG 0.1 m along +y, velocity (1, 0, 0) and
    angular velocity (0, 0, 5); point b (3 kg) at (0.015, 0, 0), its own CoG, velocity (-1, 0, 0).
    Reach 2 r = 0.02 m, so the overlap is 0.005 m; n = (a - b)/|a - b| = (-1, 0, 0); a's velocity
    is v + w x (a - c) = (1, 0, 0) + (0.5, 0, 0); the approach rate is v_n = (1.5 + 1) (-1) = -2.5;
    the reduced mass is 3/4.  f = 0.75 (300^2 0.005 + 2 300 2.5) = 0.75 (450 + 1500) = 1462.5 N,
    on a along -x, on b along +x.  a's torque about its CoG: (0, -0.1, 0) x (-1462.5, 0, 0) =
    (0, 0, -146.25)."""
    f = arena_forces([np.zeros((1, 3)), np.array([[0.015, 0.0, 0.0]])], [np.ones(1), np.full(1, 3.0)],
                     c=[[0.0, 0.1, 0.0], [0.015, 0.0, 0.0]], v=[[1.0, 0, 0], [-1.0, 0, 0]],
                     om=[[0, 0, 5.0], [0, 0, 0]], active=[1, 1], radius=RADIUS, omega_c=W_C, zeta=1.0)
    np.testing.assert_allclose(f[0], [-1462.5, 0, 0, 0, 0, -146.25], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(f[1], [1462.5, 0, 0, 0, 0, 0], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("case", ["separating", "out_of_reach", "coincident", "inactive"])
def test_pair_force_zero_cases(case):
    """No adhesion (a fast separation clamps the force at 0), nothing at or beyond the reach,
    nothing for coincident points (no direction) or an inactive robot."""
    xb = {"separating": 0.015, "out_of_reach": 0.0201, "coincident": 0.0, "inactive": 0.015}[case]
    va = -3.0 if case == "separating" else 1.0
    act = [1, 0] if case == "inactive" else [1, 1]
    f = arena_forces([np.zeros((1, 3)), np.array([[xb, 0.0, 0.0]])], [np.ones(1), np.full(1, 3.0)],
                     c=[[0, 0, 0], [xb, 0, 0]], v=[[va, 0, 0], [-1.0, 0, 0]], om=np.zeros((2, 3)),
                     active=act, radius=RADIUS, omega_c=W_C, zeta=1.0)
    assert (f == 0).all()
    # at exactly the reach the spring term vanishes and the damping needs an approach
    f = arena_forces([np.zeros((1, 3)), np.array([[0.02, 0.0, 0.0]])], [np.ones(1), np.ones(1)],
                     c=np.zeros((2, 3)), v=np.zeros((2, 3)), om=np.zeros((2, 3)), active=[1, 1],
                     radius=RADIUS, omega_c=W_C, zeta=1.0)
    assert (f == 0).all()


def test_third_law_and_central_forces():
    """Three overlapping random clouds with random motion: the forces sum to zero and, being
    central, so do their moments about the origin (sum over robots of c x F + torque)."""
    rng = np.random.default_rng(3)
    x = [rng.uniform(-0.05, 0.05, (n, 3)) + off for n, off in ((40, 0.0), (25, 0.02), (33, -0.01))]
    m = [rng.uniform(0.01, 0.1, len(a)) for a in x]
    c = np.array([a.mean(0) + rng.normal(0, 0.05, 3) for a in x])
    f = arena_forces(x, m, c, rng.normal(0, 1, (3, 3)), rng.normal(0, 3, (3, 3)), [1, 1, 1], RADIUS, W_C, 1.0)
    scale = np.abs(f[:, :3]).sum()
    assert scale > 1.0                       # the clouds do touch
    np.testing.assert_allclose(f[:, :3].sum(0), 0.0, atol=1e-12 * scale)
    moment = (np.cross(c, f[:, :3]) + f[:, 3:]).sum(0)
    np.testing.assert_allclose(moment, 0.0, atol=1e-12 * scale)


def test_elastic_head_on_collision():
    """Undamped (zeta = 0), no gravity, far above the ground: points of 1 and 3 kg meet at +-1 m/s.
    The textbook elastic result is v1' = ((m1 - m2) v1 + 2 m2 v2) / (m1 + m2) = -2 and
    v2' = ((m2 - m1) v2 + 2 m1 v1) / (m1 + m2) = 0; the pair is a spring of the reduced mass with
    natural frequency w_c, so contact lasts half a period, pi / w_c (10.47 ms).  Semi-implicit
    Euler at dt = 1e-5 (w_c dt = 0.003) reaches both within its first-order error."""
    dt = 1e-5
    b = scenes.concat([_point_robot(1.0, (-0.05, 0.0, 1.0), (1.0, 0.0, 0.0), dt, zeta=0.0),
                       _point_robot(3.0, (0.05, 0.0, 1.0), (-1.0, 0.0, 0.0), dt, zeta=0.0)])
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    in_contact = 0
    for _ in range(12000):
        o.step(1)
        in_contact += abs(o.c[0, 0] - o.c[1, 0]) < 2 * RADIUS
    np.testing.assert_allclose(o.v[:, 0], [-2.0, 0.0], atol=5e-3)
    np.testing.assert_allclose(o.v[:, 1:], 0.0, atol=1e-12)
    assert abs(in_contact * dt - math.pi / W_C) <= 3 * dt
    # momentum exactly, energy within the integrator's error
    assert abs(o.v[0, 0] * 1.0 + o.v[1, 0] * 3.0 - (1.0 - 3.0)) < 1e-12
    assert abs(0.5 * o.v[0, 0] ** 2 + 1.5 * o.v[1, 0] ** 2 - 2.0) < 2e-2


def test_damped_collision_dissipates():
    """The same collision with the world's damping (zeta = 1): momentum is kept, kinetic energy
    lost, and the points separate without sticking (no adhesion)."""
    dt = 1e-5
    b = scenes.concat([_point_robot(1.0, (-0.05, 0.0, 1.0), (1.0, 0.0, 0.0), dt),
                       _point_robot(3.0, (0.05, 0.0, 1.0), (-1.0, 0.0, 0.0), dt)])
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    o.step(12000)
    assert abs(o.v[0, 0] + 3.0 * o.v[1, 0] + 2.0) < 1e-12
    assert 0.5 * o.v[0, 0] ** 2 + 1.5 * o.v[1, 0] ** 2 < 0.5 * 2.0
    assert o.v[1, 0] - o.v[0, 0] > 0.0 and abs(o.c[0, 0] - o.c[1, 0]) > 2 * RADIUS


def test_free_flight_momentum_is_conserved():
    """Two walking hexapods thrown at each other with spin, no gravity, 1 m above the ground:
    through the collision the total linear momentum sum M v and the total angular momentum about
    the origin sum (c x M v + L) stay constant to rounding (central, opposite pair forces;
    semi-implicit Euler keeps both exactly), while the robots' paths differ from their paths
    alone."""
    b = scenes.arena_batch(1, 2, seed_key=4).with_(gravity=(0.0, 0.0, 0.0))
    b = b.with_(origin=b.origin + np.float32([0.0, 0.0, 1.0]),
                vel=np.float32([[0.0, 0.3, 0.0], [0.0, -0.3, 0.0]]),
                omega=np.float32([[0.5, 0.0, 1.0], [0.0, -0.4, -0.8]]))
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    alone = Oracle(b)
    M = np.array([o.mass_props(s)[2] for s in range(2)])

    def totals(x):
        P = (M[:, None] * x.v).sum(0)
        H = (np.cross(x.c, M[:, None] * x.v) + x.L).sum(0)
        return P, H

    P0, H0 = totals(o)
    o.step(400)
    alone.step(400)
    P1, H1 = totals(o)
    np.testing.assert_allclose(P1, P0, atol=1e-12)
    np.testing.assert_allclose(H1, H0, atol=1e-12)
    assert np.abs(o.c - alone.c).max() > 1e-3          # they did collide
    assert (o.status == 0).all()


def test_box_resting_on_a_box():
    """A 1 kg box (8 corner points) resting on a 2 kg box of the same footprint on the ground.
    The top box's weight is carried by the 4 vertical corner pairs, springs of stiffness
    m_r w_c^2 with m_r = (1/8)(2/8)/(3/8) = 1/12 kg: the corner gap settles at
    2 r - M_top g / (4 m_r w_c^2) = 0.02 - 9.81 / 30000 m (diagonal pairs are out of reach)."""
    g = 9.81
    bottom = _box_robot(0.1, 0.1, 0.05, 2.0, (0.0, 0.0, 0.025))
    top = _box_robot(0.1, 0.1, 0.05, 1.0, (0.0, 0.0, 0.05 + 0.02 + 0.075 - 0.05))
    b = scenes.concat([bottom, top])
    o = Oracle(b, arena=2, arena_radius=RADIUS)
    o.step(4000)
    xb, xt = o.points_world(0), o.points_world(1)
    gap = np.sort(xt[:, 2])[:4].mean() - np.sort(xb[:, 2])[-4:].mean()
    m_r = (1.0 / 8) * (2.0 / 8) / (3.0 / 8)
    assert gap == pytest.approx(2 * RADIUS - 1.0 * abs(b.gravity[2]) / (4 * m_r * W_C ** 2), rel=1e-6)
    assert abs(b.gravity[2] - (-g)) < 1e-6
    np.testing.assert_allclose(o.v, 0.0, atol=1e-7)


def test_robots_apart_or_frozen_do_not_interact():
    """Hexapods 2 m apart: the arena run is bit-identical to the robots run alone.  A frozen robot
    in reach exerts no force: its neighbour runs exactly as alone."""
    b = scenes.arena_batch(2, 2, seed_key=5)
    far = b.with_(origin=b.origin + np.float32([[0, -1, 0], [0, 1, 0]] * 2))
    o, alone = Oracle(far, arena=2, arena_radius=RADIUS), Oracle(far)
    o.step(500)
    alone.step(500)
    np.testing.assert_array_equal(o.c, alone.c)
    np.testing.assert_array_equal(o.L, alone.L)
    o, alone = Oracle(b, arena=2, arena_radius=RADIUS), Oracle(b)
    o.status[1] = alone.status[1] = 1
    o.step(800)
    alone.step(800)
    np.testing.assert_array_equal(o.c[0], alone.c[0])
    np.testing.assert_array_equal(o.q[0], alone.q[0])


def test_non_finite_neighbour_exerts_nothing():
    """A robot whose velocity is not a number freezes in its first step and its neighbour, in
    reach, steps exactly as alone (its pair forces are not numbers and count as 0)."""
    b = scenes.arena_batch(1, 2, seed_key=8)
    o, alone = Oracle(b, arena=2, arena_radius=RADIUS), Oracle(b)
    o.step(600)
    alone.copy_state_from(o)
    x = [o.points_world(0), o.points_world(1)]
    m = [b.m[:b.point_off[1]], b.m[b.point_off[1]:]]
    assert (np.linalg.norm(x[0][:, None] - x[1][None], axis=2) < 2 * RADIUS).sum() > 0   # legs in reach
    assert np.abs(arena_forces(x, m, o.c, o.v, np.zeros((2, 3)), [1, 1], RADIUS, W_C, 1.0)[0]).max() > 0
    o.v[1] = np.nan
    assert (arena_forces(x, m, o.c, o.v, np.zeros((2, 3)), [1, 1], RADIUS, W_C, 1.0)[0] == 0).all()
    o.step(300)
    alone.status[1] = 1
    alone.step(300)
    assert o.status[1] != 0
    np.testing.assert_array_equal(o.c[0], alone.c[0])


def test_threads_take_whole_arenas():
    """Stepping arenas on several threads gives the single-thread result exactly; a scene count
    that is not a multiple of the arena size is refused."""
    b = scenes.arena_batch(3, 4, seed_key=6)
    a, c = Oracle(b, arena=4, arena_radius=RADIUS), Oracle(b, threads=2, arena=4, arena_radius=RADIUS)
    a.step(300)
    c.step(300)
    np.testing.assert_array_equal(a.c, c.c)
    np.testing.assert_array_equal(a.L, c.L)
    with pytest.raises(ValueError):
        Oracle(b.subset(range(6)), arena=4, arena_radius=RADIUS)
    with pytest.raises(ValueError):
        Oracle(b, arena=4, arena_radius=0.0)
