"""Pins of the oracle's two friction-model options, the refinements the paper names after Eq. 6:
the least-squares rows weighted by the force pressing each point against the ground, and the
torque of the friction impulse about the horizontal axes.  The weighted solver is checked against
a library least-squares solve of the uncentred model; the torque against its closed form r x J
on a sliding block; both options against the Coulomb law and energy dissipation."""
import numpy as np
import pytest

from oracle.oracle import FRIC_TILT, FRIC_WEIGHTED, Oracle, friction_ls, friction_ls_w
from paper_2411_05799_gb300 import scenes
from tests.parity import clone

G = 9.81


def _lstsq_uncentred(s, e, w):
    """Weighted least squares of e_i ~ a + a3 (-y_i, x_i) by numpy (rows scaled by sqrt(w))."""
    A = np.zeros((2 * len(s), 3))
    A[0::2, 0] = 1.0
    A[1::2, 1] = 1.0
    A[0::2, 2] = -s[:, 1]
    A[1::2, 2] = s[:, 0]
    sw = np.repeat(np.sqrt(w), 2)
    sol, *_ = np.linalg.lstsq(A * sw[:, None], e.reshape(-1) * sw, rcond=None)
    return sol


@pytest.mark.parametrize("n", [2, 3, 7, 40])
def test_weighted_ls_matches_library_least_squares(n):
    rng = np.random.default_rng(200 + n)
    s = rng.normal(0, 0.3, (n, 2)) + rng.normal(0, 2, 2)
    e = rng.normal(0, 0.01, (n, 2))
    w = rng.uniform(0.1, 5.0, n)
    t, a3 = friction_ls_w(s, e, w)
    sb = (w[:, None] * s).sum(0) / w.sum()
    a12 = t - a3 * np.array([-sb[1], sb[0]])       # back to the uncentred parameters
    np.testing.assert_allclose([*a12, a3], _lstsq_uncentred(s, e, w), rtol=1e-8, atol=1e-12)


def test_weighted_ls_special_cases():
    rng = np.random.default_rng(7)
    s = rng.normal(0, 0.2, (9, 2))
    e = rng.normal(0, 0.01, (9, 2))
    # equal weights, of any size, give the unweighted solution
    t0, a0 = friction_ls(s, e)
    for c in (1.0, 3.7, 1e-3):
        t, a = friction_ls_w(s, e, np.full(9, c))
        np.testing.assert_allclose(t, t0, rtol=1e-12, atol=1e-15)
        assert a == pytest.approx(a0, rel=1e-12)
    # a zero weight removes its row
    w = rng.uniform(0.5, 2.0, 9)
    w[4] = 0.0
    t, a = friction_ls_w(s, e, w)
    keep = np.arange(9) != 4
    t2, a2 = friction_ls_w(s[keep], e[keep], w[keep])
    np.testing.assert_allclose(t, t2, rtol=1e-12, atol=1e-15)
    assert a == pytest.approx(a2, rel=1e-12)
    # all weight on one point: that point's residual, no rotation; no weight: nothing
    w = np.zeros(9)
    w[2] = 4.0
    t, a = friction_ls_w(s, e, w)
    np.testing.assert_allclose(t, e[2], atol=1e-16)
    assert a == 0.0
    t, a = friction_ls_w(s, e, np.zeros(9))
    assert a == 0.0 and np.all(t == 0.0)
    # the rotation needs a centre of pressure spread over more than a millimetre (mean squared
    # spread above 1e-6 m^2): two points 0.5 mm apart, or 5 cm apart with the weight nearly all on
    # one, give a translation only; 5 cm apart with equal weights, a rotation
    two = np.array([[0.0, 0.0], [5e-4, 0.0]])
    e2 = np.array([[0.0, -1e-5], [0.0, 1e-5]])
    assert friction_ls_w(two, e2, np.ones(2))[1] == 0.0
    two = np.array([[0.0, 0.0], [0.05, 0.0]])
    assert friction_ls_w(two, e2, np.array([1.0, 1e-4]))[1] == 0.0
    assert friction_ls_w(two, e2, np.ones(2))[1] == pytest.approx(2e-5 / 0.05)
    # a rigid motion in the model's family is recovered exactly whatever the weights
    a, a3 = np.array([0.01, -0.02]), 0.003
    e = a + a3 * np.stack([-s[:, 1], s[:, 0]], 1)
    w = rng.uniform(0.1, 9.0, 9)
    t, got = friction_ls_w(s, e, w)
    sb = (w[:, None] * s).sum(0) / w.sum()
    assert got == pytest.approx(a3, abs=1e-14)
    np.testing.assert_allclose(t - got * np.array([-sb[1], sb[0]]), a, atol=1e-14)


def _sliding_block(vel):
    """A lattice block settled on the plane, then given a horizontal velocity."""
    b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=0.5)
    o = Oracle(b)
    o.step(2000)
    assert np.abs(o.v).max() < 1e-6
    o.v[0, :2] = vel
    return b, o


def test_tilt_torque_is_the_moment_of_the_friction_impulse():
    """One step of a sliding block with and without the horizontal-axis torque: position,
    velocity and orientation agree, and the angular momenta differ by the moment about the CoG of
    the friction impulse J = M dv applied at the bottom face's centre, 0.05 m below the CoG:
    dL = r x J with r = (0, 0, -0.05), i.e. (0.05 Jy, -0.05 Jx, 0): a block braked at its base
    pitches forward."""
    vel = (0.5, -0.2)
    b, o = _sliding_block(vel)
    off, on = clone(o), Oracle(b, fric_mode=FRIC_TILT)
    on.copy_state_from(o)
    off.step(1)
    on.step(1)
    np.testing.assert_allclose(on.c, off.c, atol=1e-15)
    np.testing.assert_allclose(on.v, off.v, atol=1e-15)
    np.testing.assert_allclose(on.q, off.q, atol=1e-15)
    J = 1.0 * (off.v[0, :2] - np.array(vel))      # no horizontal gravity: the friction impulse
    assert np.linalg.norm(J) > 1e-3                 # the block is braked
    dL = on.L[0] - off.L[0]
    np.testing.assert_allclose(dL, [0.05 * J[1], -0.05 * J[0], 0.0], rtol=1e-6, atol=1e-12)
    assert dL[1] > 0 and dL[0] > 0                  # braked along +x and -y: tips toward them


def _incline_velocity(theta, mu, fric_mode, steps=3000):
    b = scenes.tilted_gravity(scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2),
                                                 mass=1.0, mu=mu), theta)
    o = Oracle(b, fric_mode=fric_mode)
    vs = []
    for _ in range(steps // 10):
        o.step(10)
        vs.append(o.v[0, 0])
    return np.array(vs)


@pytest.mark.parametrize("fric_mode", [FRIC_WEIGHTED, FRIC_TILT, FRIC_WEIGHTED | FRIC_TILT])
def test_options_keep_the_coulomb_law(fric_mode):
    """On an incline (gravity tilted by theta on flat ground) the block sticks below the friction
    angle and slides with acceleration g (sin theta - mu cos theta) above it, with either option:
    neither changes the total friction impulse the cap allows."""
    v = _incline_velocity(np.radians(20), 0.5, fric_mode)
    assert np.abs(v[-50:]).max() < 1e-4
    theta, mu = np.radians(35), 0.5
    v = _incline_velocity(theta, mu, fric_mode)
    acc = np.polyfit(np.arange(150, 300) * 10e-3, v[150:], 1)[0]
    assert acc == pytest.approx(G * (np.sin(theta) - mu * np.cos(theta)), rel=1e-3)


def _energy(o, b):
    from tests.test_oracle_pins import _energy as energy
    return energy(o, b)


@pytest.mark.parametrize("fric_mode", [FRIC_WEIGHTED, FRIC_TILT, FRIC_WEIGHTED | FRIC_TILT])
def test_options_dissipate_energy(fric_mode):
    """A block sliding and spinning flat on the plane loses its kinetic energy to friction with
    either option, the total energy never rising above its running minimum by more than the
    frictionless run's integrator noise."""
    def trace(mu, mode):
        b = scenes.block_batch(extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0, mu=mu,
                               vel=(1.0, 0.5, 0.0), omega=(0.0, 0.0, 3.0))
        o = Oracle(b, fric_mode=mode)
        out = []
        for _ in range(150):
            o.step(4)
            out.append(_energy(o, b)[0])
        return np.array(out)
    e0, e1 = trace(0.0, fric_mode), trace(0.4, fric_mode)
    noise0 = np.max(e0 - np.minimum.accumulate(e0))
    rise1 = np.max(e1 - np.minimum.accumulate(e1))
    assert rise1 <= 2 * noise0 + 1e-9
    assert e1[-1] < e0[-1] - 0.5
