"""Pins of the FP64 oracle against things other than itself: closed forms of the integrator,
conservation laws, the paper's own normal equations (Eqs. 4-6) solved by a library routine,
textbook rotation conventions (scipy), lattice sums, hand-computed height-map lookups, and the
Coulomb stick/slip law.  Each test is built so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails it."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle.oracle import Oracle, friction_ls, quat_matrix
from paper_2411_05799_gb300 import scenes

G = 9.81


# ----------------------------------------------------------------------------- integrator

def test_free_fall_closed_form():
    b = scenes.single_body()
    b = b.with_(origin=np.array([[0.3, -0.2, 100.0]], np.float32))
    o = Oracle(b)
    c0, v0 = o.c[0].copy(), o.v[0].copy()
    dt, g = b.dt, -b.gravity[2]
    for n in (1, 7, 100, 1000, 3000):
        o2 = Oracle(b)
        o2.step(n)
        zc = c0[2] + n * dt * v0[2] - g * dt * dt * n * (n + 1) / 2
        vz = v0[2] - g * n * dt
        assert abs(o2.c[0, 2] - zc) < 1e-11 * max(1.0, abs(zc))
        assert abs(o2.v[0, 2] - vz) < 1e-12 * max(1.0, abs(vz))
        np.testing.assert_allclose(o2.c[0, :2], c0[:2] + n * dt * v0[:2], rtol=0, atol=1e-12)
        np.testing.assert_array_equal(o2.v[0, :2], v0[:2])     # horizontal momentum exact


def test_modified_energy_and_angular_momentum_invariant():
    b = scenes.single_body()
    b = b.with_(origin=np.array([[0.0, 0.0, 50.0]], np.float32))
    o = Oracle(b)
    M, g = 1.0, -b.gravity[2]
    L0 = o.L[0].copy()
    E0 = 0.5 * M * o.v[0] @ o.v[0] + M * g * o.c[0, 2] - 0.5 * M * g * b.dt * o.v[0, 2]
    for _ in range(20):
        o.step(100)
        E = 0.5 * M * o.v[0] @ o.v[0] + M * g * o.c[0, 2] - 0.5 * M * g * b.dt * o.v[0, 2]
        assert abs(E - E0) < 1e-9 * abs(E0)
        np.testing.assert_array_equal(o.L[0], L0)                # no torque: L exactly constant
        assert abs(np.linalg.norm(o.q[0]) - 1.0) < 1e-14


def test_isotropic_body_rotates_by_exponential_map():
    """A cubic lattice (coordinates exact in binary) has isotropic inertia, so omega = L / I is constant and the orientation
    after n steps is exp(n dt omega) applied on the left of the initial one (world-frame
    angular velocity), which scipy evaluates independently."""
    w = np.array([1.3, -2.1, 0.7], np.float32).astype(np.float64)   # inputs are float32
    b = scenes.block_batch(extent=(0.25, 0.25, 0.25), counts=(3, 3, 3), omega=w, z_gap=20.0)
    q0 = scenes.random_unit_quat(np.random.default_rng(5), 1)
    b = b.with_(quat=q0)
    o = Oracle(b)
    R0 = Rotation.from_quat(np.roll(o.q[0], -1))   # scipy wants (x, y, z, w)
    n = 500
    o.step(n)
    Rn = Rotation.from_rotvec(n * b.dt * w) * R0
    np.testing.assert_allclose(quat_matrix(o.q[0]), Rn.as_matrix(), atol=1e-11)
    np.testing.assert_allclose(o.omega()[0], w, atol=1e-12)


def test_rotation_about_principal_axis_is_steady():
    """Spin about the long symmetry axis of a box lattice: omega stays along that axis."""
    b = scenes.block_batch(extent=(0.3, 0.1, 0.05), counts=(4, 2, 2), omega=(5.0, 0.0, 0.0),
                           z_gap=20.0)
    o = Oracle(b)
    o.step(2000)
    np.testing.assert_allclose(o.omega()[0], [5.0, 0.0, 0.0], atol=1e-10)


# ----------------------------------------------------------------------------- mass properties

def _lattice_inertia(extent, counts, mass):
    """Closed form for a box lattice of equal masses centred at its CoG: sum over the lattice
    factorises per axis, sum_k x_k^2 = n e^2 (n+1) / (12 (n-1)) for n points spanning e."""
    s2 = []
    for e, n in zip(extent, counts):
        s2.append(0.0 if n == 1 else e * e * n * (n + 1) / (12.0 * (n - 1)))
    N = np.prod(counts)
    m = mass / N
    # sum over the lattice of x^2 = (sum_k x_k^2) * (points along the other two axes)
    Sx = s2[0] * N / counts[0]
    Sy = s2[1] * N / counts[1]
    Sz = s2[2] * N / counts[2]
    # plus each point's own sphere inertia (radius 1 mm): 2/5 M r^2 on the diagonal
    return np.diag([m * (Sy + Sz), m * (Sx + Sz), m * (Sx + Sy)]) + 0.4 * mass * 1e-6 * np.eye(3)


@pytest.mark.parametrize("extent,counts", [((0.3, 0.18, 0.06), (4, 4, 4)),
                                           ((0.02, 0.02, 0.15), (2, 2, 4)),
                                           ((0.2, 0.2, 0.1), (3, 3, 2))])
def test_lattice_mass_properties(extent, counts):
    b = scenes.block_batch(extent=extent, counts=counts, mass=1.7)
    o = Oracle(b)
    g, Ib, M = o.mass_props(0)
    assert abs(M - 1.7) < 1e-6
    np.testing.assert_allclose(g, 0.0, atol=1e-8)
    M32 = float(np.sum(np.float32(1.7 / np.prod(counts)) * np.ones(np.prod(counts), np.float32).astype(np.float64)))
    np.testing.assert_allclose(Ib, _lattice_inertia(extent, counts, M32), rtol=1e-6, atol=1e-12)


def test_hexapod_rest_mass_properties_brute_force():
    """CoG and inertia of the whole hexapod at rest from a direct numpy sum over its points."""
    b = scenes.hexapod_batch(1)
    o = Oracle(b)
    g, Ib, M = o.mass_props(0)
    p = b.p0.astype(np.float64)
    m = b.m.astype(np.float64)
    gg = (m[:, None] * p).sum(0) / m.sum()
    r = p - gg
    I = sum(mi * (ri @ ri * np.eye(3) - np.outer(ri, ri)) for mi, ri in zip(m, r))
    I += 0.4 * m.sum() * 1e-6 * np.eye(3)         # point spheres of radius 1 mm
    assert abs(M - 2.34) < 1e-5
    np.testing.assert_allclose(g, gg, atol=1e-12)
    np.testing.assert_allclose(Ib, I, rtol=1e-10, atol=1e-14)


# ----------------------------------------------------------------------------- kinematics

def _recover_angle(Qp, Qc, u):
    """Angle of the rotation Qp^T Qc about the unit axis u."""
    Rj = Qp.T @ Qc
    vee = np.array([Rj[2, 1] - Rj[1, 2], Rj[0, 2] - Rj[2, 0], Rj[1, 0] - Rj[0, 1]]) / 2
    return math.atan2(vee @ u, (np.trace(Rj) - 1) / 2)


def test_forward_kinematics_recovers_joint_angles():
    b = scenes.hexapod_batch(1)
    rng = np.random.default_rng(11)
    th = rng.uniform(-1.0, 1.0, b.n_joints).astype(np.float32)
    b = b.with_(theta0=th)
    o = Oracle(b)
    np.testing.assert_array_equal(o.theta, th.astype(np.float64))
    Q, T = o.link_frames(0)
    for l in range(1, 19):
        P = b.parent[l]
        u = b.axis[l].astype(np.float64)
        u /= np.linalg.norm(u)
        a = b.anchor[l].astype(np.float64)
        # the hinge rotation equals scipy's rotation vector u * theta (right-hand rule)
        Rj = Q[P].T @ Q[l]
        np.testing.assert_allclose(Rj, Rotation.from_rotvec(u * th[l - 1]).as_matrix(), atol=1e-12)
        assert abs(_recover_angle(Q[P], Q[l], u) - th[l - 1]) < 1e-12
        # the anchor is a fixed point of the joint: both links carry it to the same place
        np.testing.assert_allclose(Q[l] @ a + T[l], Q[P] @ a + T[P], atol=1e-12)


def test_joint_angles_recovered_from_world_points():
    """A tibia point's direction from the knee, measured in the femur's frame, turns by exactly
    the knee angle about the knee axis."""
    b = scenes.hexapod_batch(1)
    th = np.zeros(b.n_joints, np.float32)
    th[2] = 0.7          # first leg's knee (tibia) joint
    o0 = Oracle(b)
    o1 = Oracle(b.with_(theta0=th))
    x0, x1 = o0.points_world(0), o1.points_world(0)
    pl = b.plink
    tib = np.where(pl == 3)[0]
    a = b.anchor[3].astype(np.float64)
    u = b.axis[3].astype(np.float64)
    # femur frame in the world: both scenes share the femur pose up to the CoG shift, so use
    # the femur's own points to build it
    fem = np.where(pl == 2)[0]

    def local(x):
        c = x[fem].mean(0)
        c0 = b.p0[fem].astype(np.float64).mean(0)
        return x[tib] - c - (a - c0)      # vectors from the knee anchor, femur frame = world here
    v0, v1 = local(x0), local(x1)
    for p, q_ in zip(v0, v1):
        pp = p - (p @ u) * u
        qq = q_ - (q_ @ u) * u
        if np.linalg.norm(pp) < 1e-6:
            continue
        ang = math.atan2(np.cross(pp, qq) @ u, pp @ qq)
        assert abs(ang - float(th[2])) < 1e-9


def test_actuator_target_phase():
    """bias + A sin(2 pi f t + phi) with the phase quantised to 2^-32 turns per step: agrees with
    the continuous sinusoid to the quantisation bound n * 2^-33 turns."""
    b = scenes.hexapod_batch(2)
    o = Oracle(b)
    for s in range(2):
        for j in (0, 5, 17):
            A, f, ph, bias = b.act_params[s * 18 + j].astype(np.float64)
            for n in (0, 1, 80, 12345, 60000, 10 ** 7):
                exact = bias + A * math.sin(2 * math.pi * f * n * b.dt + ph)
                bound = A * 2 * math.pi * (n * 2.0 ** -33 + 1e-12) + 1e-12
                assert abs(o.target(s, j, n) - exact) <= bound * 1.0001


def test_joint_update_schedule():
    """Angles change only on steps n = 0 (mod K) and then equal the clamped target."""
    b = scenes.hexapod_batch(1, K=80)
    o = Oracle(b)
    o.step(1)
    lo, hi = b.lo[1:], b.hi[1:]
    want = np.clip([o.target(0, j, 0) for j in range(18)], lo, hi)
    np.testing.assert_array_equal(o.theta, want)
    th1 = o.theta.copy()
    o.step(79)
    np.testing.assert_array_equal(o.theta, th1)
    o.step(1)
    want = np.clip([o.target(0, j, 80) for j in range(18)], lo, hi)
    np.testing.assert_array_equal(o.theta, want)


def test_joint_limits_clamp():
    b = scenes.hexapod_batch(1)
    ap = b.act_params.copy()
    ap[:, 0] = 0.0
    ap[:, 3] = 3.0            # bias far beyond the +-60 deg limit
    o = Oracle(b.with_(act_params=ap))
    o.step(1)
    np.testing.assert_allclose(o.theta, math.radians(60), rtol=1e-6)


# ----------------------------------------------------------------------------- height map

def test_lut_hand_computed():
    """Scale 10 (0.1 m cells, Sec. III-A), origin (-0.2, -0.1), a 4 x 3 map whose value encodes
    its cell: h[iy][ix] = 10 iy + ix.  Expected cells are worked out by hand from floor and
    clamping to the map."""
    maps = (10 * np.arange(3)[:, None] + np.arange(4)[None, :]).astype(np.float32)[None]
    b = scenes.single_body().with_(heightmaps=maps, hmap=np.zeros(1, np.int32), hm_scale=10.0,
                                   hm_origin=(-0.2, -0.1))
    o = Oracle(b)
    cases = [((-0.2, -0.1), 0), ((-0.15, -0.05), 0), ((-0.1, -0.1), 1), ((0.0, 0.0), 12),
             ((0.05, 0.09), 12), ((0.15, 0.15), 23), ((0.19, 0.19), 23), ((-1.0, -1.0), 0),
             ((5.0, -5.0), 3), ((-5.0, 5.0), 20), ((0.5, 0.5), 23), ((-0.21, 0.0), 10),
             ((0.0999, 0.0501), 12)]
    for (x, y), want in cases:
        assert o.lut(0, x, y) == want, (x, y)


# ----------------------------------------------------------------------------- contact

def test_block_rests_on_plane():
    """A 3x3x2 lattice block (9 bottom points) settles to the static sink d = M g / (9 m w_c^2)
    and stays at rest."""
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=0.5)
    o = Oracle(b)
    o.step(1000)
    w2 = b.contact_omega ** 2
    m_pt = float(np.float32(1.0 / 18))
    d = 18 * m_pt * -b.gravity[2] / (9 * m_pt * w2)
    assert abs(o.c[0, 2] - (0.05 - d)) < 1e-9
    assert np.abs(o.v[0]).max() < 1e-6
    np.testing.assert_allclose(o.c[0, :2], 0.0, atol=1e-12)
    c1 = o.c[0].copy()
    o.step(2000)
    assert np.abs(o.v[0]).max() < 1e-6
    assert np.abs(o.c[0] - c1).max() < 1e-9
    assert o.sensors[0] == 1


# ----------------------------------------------------------------------------- friction LS

def _paper_normal_equations(s, e):
    """Eqs. 4-6 written out with the paper's (x, z) as the horizontal (x, y): with source
    (x, y), target (x', y') = (x, y) + e and residuals r1 = x - a3 y + a1 - x',
    r2 = a3 x + y + a2 - y' (Eq. 3), setting the three derivatives to zero gives
        n a1            - a3 sum y          = sum (x' - x)
                n a2    + a3 sum x          = sum (y' - y)
        -a1 sum y + a2 sum x + a3 sum(x^2 + y^2) = sum (x y' - y x')
    which numpy solves as a plain 3 x 3 system."""
    x, y = s[:, 0], s[:, 1]
    xt, yt = x + e[:, 0], y + e[:, 1]
    n = len(x)
    A = np.array([[n, 0.0, -y.sum()],
                  [0.0, n, x.sum()],
                  [-y.sum(), x.sum(), (x * x + y * y).sum()]])
    rhs = np.array([(xt - x).sum(), (yt - y).sum(), (x * yt - y * xt).sum()])
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("n", [2, 3, 7, 40])
def test_friction_ls_matches_paper_equations(n):
    rng = np.random.default_rng(100 + n)
    s = rng.normal(0, 0.3, (n, 2)) + rng.normal(0, 2, 2)
    e = rng.normal(0, 0.01, (n, 2))
    t, a3 = friction_ls(s, e)
    sb = s.mean(0)
    a12 = t - a3 * np.array([-sb[1], sb[0]])
    sol = _paper_normal_equations(s, e)
    np.testing.assert_allclose([*a12, a3], sol, rtol=1e-9, atol=1e-12)


def test_friction_ls_recovers_linear_motion_and_translation():
    rng = np.random.default_rng(3)
    s = rng.normal(0, 0.2, (9, 2))
    a, a3 = np.array([0.01, -0.02]), 0.003
    e = a + a3 * np.stack([-s[:, 1], s[:, 0]], 1)
    t, got = friction_ls(s, e)
    sb = s.mean(0)
    assert abs(got - a3) < 1e-14
    np.testing.assert_allclose(t - got * np.array([-sb[1], sb[0]]), a, atol=1e-14)
    t, got = friction_ls(s, np.tile([-0.004, 0.001], (9, 1)))
    assert got == pytest.approx(0.0, abs=1e-15)
    np.testing.assert_allclose(t, [-0.004, 0.001], atol=1e-16)
    t, got = friction_ls(s[:1], np.array([[0.3, 0.2]]))      # one point: translation only
    assert got == 0.0 and np.allclose(t, [0.3, 0.2])


def _incline_run(theta, mu, steps=3000):
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=mu)
    b = scenes.tilted_gravity(b, theta)
    o = Oracle(b)
    xs, vs = [], []
    for _ in range(steps // 10):
        o.step(10)
        xs.append(o.c[0, 0])
        vs.append(o.v[0, 0])
    return np.array(xs), np.array(vs), b


def test_incline_sticks_below_friction_angle():
    theta, mu = math.radians(20), 0.5     # tan 20 deg = 0.364 < 0.5
    xs, vs, b = _incline_run(theta, mu)
    assert np.abs(vs[50:]).max() < 1e-9
    assert abs(xs[-1] - xs[50]) < 1e-9


@pytest.mark.parametrize("theta_deg,mu", [(35, 0.5), (30, 0.3), (45, 0.8)])
def test_incline_slips_with_coulomb_acceleration(theta_deg, mu):
    theta = math.radians(theta_deg)
    xs, vs, b = _incline_run(theta, mu)
    gx, gz = b.gravity[0], -b.gravity[2]
    want = gx - float(np.float32(mu)) * gz
    acc = (vs[-1] - vs[100]) / ((len(vs) - 1 - 100) * 10 * b.dt)
    assert abs(acc - want) < 1e-3 * want


def test_spinning_block_decelerates_at_the_rotational_coulomb_limit():
    """Maximum static friction on a pure spin (Sec. III-C, reading R8).  A 3 x 3 x 2 lattice block
    rests on the plane (normal force M g on its nine bottom points), then spins about the vertical
    with no translation.  Each step the integration turns it by phi = dt w; the least squares of
    Eqs. 4-6 recovers a3 = -sin(phi) about the contact centroid (t = 0), so the impulse that would
    undo the slip is M u / dt with u = 2 sin(phi / 2) r_rms, r_rms^2 the mean squared horizontal
    distance of the contact points from their centroid.  The cap mu M g dt scales the correction by
    sc = mu g dt^2 / u, and the angular momentum changes by (sc alpha / dt) Iw z, so
        w_(k+1) = w_k - mu g dt (phi / 2) / (sin(phi / 2) r_rms)
    while the spin is fast enough to slip (w r_rms > mu g dt): a constant deceleration
    mu g / r_rms up to a factor 1 + phi^2 / 24.  Once slow enough, one step stops it and it
    sticks.  The yaw turned each step is dt w_(k+1).  A wrong factor in the rotational part of u
    or in the angular-momentum update changes the rate."""
    mu_in = 0.4
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=mu_in)
    o = Oracle(b)
    o.step(1000)                                    # settle: the normal force is M g
    mu, g, dt = float(np.float32(mu_in)), -b.gravity[2], b.dt
    _, Ib, M = o.mass_props(0)
    R = quat_matrix(o.q[0])
    w0 = 3.0
    o.L[0] = R @ Ib @ R.T @ np.array([0.0, 0.0, w0])
    x = o.points_world(0)
    bottom = x[np.argsort(x[:, 2])[:9], :2]
    r_rms = math.sqrt(((bottom - bottom.mean(0)) ** 2).sum(1).mean())
    assert r_rms == pytest.approx(0.1 * math.sqrt(4.0 / 3.0), rel=1e-6)

    def yaw():
        return Rotation.from_quat(np.roll(o.q[0], -1)).as_euler("xyz")[2]

    w, yaw0, n_slip, turned = w0, yaw(), 0, 0.0
    while w * r_rms > mu * g * dt:
        phi = dt * w
        want = w - mu * g * dt * (0.5 * phi) / (math.sin(0.5 * phi) * r_rms)
        o.step(1)
        got = o.omega()[0]
        assert got[2] == pytest.approx(want, rel=1e-9, abs=1e-12), n_slip
        np.testing.assert_allclose(got[:2], 0.0, atol=1e-12)
        np.testing.assert_allclose(o.v[0], 0.0, atol=1e-12)      # no translation appears
        turned += dt * got[2]
        w, n_slip = got[2], n_slip + 1
    # the closed form of a constant deceleration mu g / r_rms
    t_stop = w0 * r_rms / (mu * g)
    assert abs(n_slip * dt - t_stop) <= dt + 1e-3 * t_stop
    assert w == pytest.approx(w0 - n_slip * mu * g * dt / r_rms, rel=1e-3)
    o.step(1)                                       # slow enough: stopped in one step
    turned += dt * o.omega()[0, 2]
    assert abs(o.omega()[0, 2]) < 1e-12
    assert yaw() - yaw0 == pytest.approx(turned, abs=1e-12)
    y1 = yaw()
    o.step(200)                                     # and it sticks
    assert abs(o.omega()[0, 2]) < 1e-12 and abs(yaw() - y1) < 1e-12


def _energy(o, b):
    """Kinetic (translation + rotation) + potential + penalty-spring energy per scene."""
    w2 = b.contact_omega ** 2
    E = []
    om = o.omega()
    for s in range(b.n_scenes):
        g, Ib, M = o.mass_props(s)
        x = o.points_world(s)
        m = b.m[b.point_off[s]:b.point_off[s + 1]].astype(np.float64)
        d = np.maximum(0.0, -x[:, 2])
        E.append(0.5 * M * o.v[s] @ o.v[s] + 0.5 * om[s] @ o.L[s] - M * np.dot(b.gravity, o.c[s])
                 + 0.5 * w2 * (m * d * d).sum())
    return np.array(E)


def test_friction_dissipates_energy():
    """A block sliding and spinning flat on the plane: with friction its total energy never rises
    above its running minimum by more than the frictionless run's integrator noise, and ends
    below the frictionless run.  (The least squares of Eqs. 1-6 holds translation and yaw only;
    sliding caused by roll or pitch is outside what it models, as the text below Eq. 6 says.)"""
    def trace(mu):
        b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=mu,
                               vel=(1.0, 0.5, 0.0), omega=(0.0, 0.0, 3.0))
        o = Oracle(b)
        out = []
        for _ in range(150):
            o.step(4)
            out.append(_energy(o, b)[0])
        return np.array(out)
    e0, e1 = trace(0.0), trace(0.4)
    noise0 = np.max(e0 - np.minimum.accumulate(e0))
    rise1 = np.max(e1 - np.minimum.accumulate(e1))
    assert rise1 <= 2 * noise0 + 1e-9
    assert e1[-1] < e0[-1] - 0.5        # friction took most of the 0.625 J kinetic energy
    assert e1[-1] <= e1.min() + 2 * noise0 + 1e-9


def test_kinematic_correction_keeps_a_turning_foot_in_place():
    """A light body standing on one flat 4-point foot joined by a vertical hinge through the
    foot's centre: turning the hinge by theta turns the foot's contact points about their
    centroid; the least-squares correction (a3 = -sin theta, applied as a rotation by asin a3)
    turns the whole robot back by theta, so the foot stays exactly where it was."""
    body = scenes.box_lattice((0.06, 0.06, 0.02), (0.15, 0.0, 0.1), (2, 2, 2))
    foot = scenes.box_lattice((0.1, 0.1, 0.0), (0.0, 0.0, 0.0), (2, 2, 1))
    links = [((0.06, 0.06, 0.02), (0.15, 0, 0.1), 0.1, -1, None, None, -1),
             ((0.1, 0.1, 0.0), (0, 0, 0), 1.0, 0, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 0)]
    b = scenes._assemble([(links, [body, foot])], mu=[5.0], origin=[(0, 0, 0.0)],
                         quat=[(1, 0, 0, 0)], vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
                         act_params=np.zeros((1, 4)), K=200, name="turning_foot")
    o = Oracle(b)
    o.step(200 * 5)                          # settle with the hinge held at 0
    is_foot = b.plink == 1
    xf0 = o.points_world(0)[is_foot]
    yaw0 = Rotation.from_quat(np.roll(o.q[0], -1)).as_euler("xyz")[2]
    th = 0.4
    ap = o._keep[-1]
    ap[0, 3] = th                            # hinge bias: the next tick turns it by 0.4 rad
    o.step(1)
    xf1 = o.points_world(0)[is_foot]
    yaw1 = Rotation.from_quat(np.roll(o.q[0], -1)).as_euler("xyz")[2]
    assert o.theta[0] == pytest.approx(th)
    assert o.sensors[0] == 1
    np.testing.assert_allclose(xf1[:, :2], xf0[:, :2], atol=1e-7)
    assert abs((yaw1 - yaw0) - (-th)) < 1e-6


def test_point_and_rod_bodies_have_invertible_inertia():
    """A single mass point (createPoint) and a line of points are legal robots: their inertia is
    that of their point spheres, so rotation stays defined and free flight follows the closed
    form."""
    one = ([((0, 0, 0), (0, 0, 0), 0.5, -1, None, None, -1)], [np.zeros((1, 3), np.float32)])
    rod = ([((0.3, 0, 0), (0, 0, 0), 0.5, -1, None, None, -1)],
           [scenes.box_lattice((0.3, 0.0, 0.0), (0, 0, 0), (4, 1, 1))])
    b = scenes._assemble([one, rod], mu=[0.5, 0.5], origin=[(0, 0, 5.0), (0, 0, 5.0)],
                         quat=[(1, 0, 0, 0)] * 2, vel=[(0.1, 0.2, 0.0)] * 2,
                         omega=[(0.0, 0.0, 1.0), (3.0, 0.0, 0.0)], act_params=None, name="pts",
                         act_mode=scenes.ACT_HOLD)
    o = Oracle(b)
    g, Ib, M = o.mass_props(0)
    np.testing.assert_allclose(Ib, 0.4 * M * 1e-6 * np.eye(3), rtol=1e-12)
    o.step(100)
    assert (o.status == 0).all()
    np.testing.assert_allclose(o.omega()[0], [0, 0, 1.0], atol=1e-9)
    np.testing.assert_allclose(o.omega()[1], [3.0, 0, 0], atol=1e-9)
    np.testing.assert_allclose(o.c[:, 0], 0.1 * 100 * b.dt, atol=1e-9)
