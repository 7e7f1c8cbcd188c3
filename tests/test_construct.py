"""Robot construction from primitives (the paper's construction calls and simplifyMode): point
placement, masses and inertia of the primitives in every simplify mode against closed forms,
roll-pitch-yaw against scipy, joints in the first body's frame, the link tree, and robots built
this way stepping in the oracle."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle.oracle import Oracle
from paper_2411_05799_gb300 import construct


def _inertia(pts, m):
    c = (m[:, None] * pts).sum(0) / m.sum()
    d = pts - c
    return c, np.diag([(m * (d[:, 1] ** 2 + d[:, 2] ** 2)).sum(), (m * (d[:, 0] ** 2 + d[:, 2] ** 2)).sum(),
                       (m * (d[:, 0] ** 2 + d[:, 1] ** 2)).sum()])


def test_box_is_its_corners():
    r = construct.Robot()
    b = r.create_box(0.3, 0.2, 0.1, 1.0, 2.0, 3.0, 2.0)
    pts = r.body_points(b)
    assert len(pts) == 8
    c, I = _inertia(pts, np.full(8, 0.25))
    np.testing.assert_allclose(c, [1, 2, 3], atol=1e-15)
    # corners (+-w/2, +-h/2, +-d/2), mass m/8 each: Ixx = m (h^2 + d^2) / 4
    np.testing.assert_allclose(np.diag(I), [2 * (0.04 + 0.01) / 4, 2 * (0.09 + 0.01) / 4, 2 * (0.09 + 0.04) / 4],
                               rtol=1e-12)


@pytest.mark.parametrize("mode,n", [(0, 16), (1, 8), (2, 2), (3, 1), (7, 1)])
def test_cylinder_in_every_simplify_mode(mode, n):
    r = construct.Robot()
    r.simplify_mode(mode)
    p1, p2, rr = np.array([0.1, -0.2, 0.3]), np.array([0.4, 0.2, -0.1]), 0.05
    b = r.create_cylinder(*p1, *p2, rr, 0.6)
    pts = r.body_points(b)
    assert len(pts) == n
    u = (p2 - p1) / np.linalg.norm(p2 - p1)
    mid = 0.5 * (p1 + p2)
    np.testing.assert_allclose(pts.mean(0), mid, atol=1e-14)          # the centre of mass
    along = (pts - mid) @ u
    perp = np.linalg.norm((pts - mid) - along[:, None] * u, axis=1)
    L = np.linalg.norm(p2 - p1)
    if mode == 0:          # two rims of 8 at radius rr at the end faces
        np.testing.assert_allclose(np.sort(np.abs(along)), np.full(16, L / 2), atol=1e-14)
        np.testing.assert_allclose(perp, rr, atol=1e-14)
    elif mode == 1:        # the box around it, aligned with the axis: corners at rr sqrt 2
        np.testing.assert_allclose(np.abs(along), L / 2, atol=1e-14)
        np.testing.assert_allclose(perp, rr * math.sqrt(2), atol=1e-14)
    elif mode == 2:        # the end centres
        np.testing.assert_allclose(sorted(map(tuple, pts)), sorted([tuple(p1), tuple(p2)]), atol=1e-14)
    else:                  # one point at the centre
        np.testing.assert_allclose(pts[0], mid, atol=1e-15)


@pytest.mark.parametrize("mode,n", [(0, 12), (1, 8), (2, 2), (3, 1)])
def test_sphere_in_every_simplify_mode(mode, n):
    r = construct.Robot()
    r.simplify_mode(mode)
    b = r.create_sphere(0.5, -0.5, 1.0, 0.1, 1.2)
    pts = r.body_points(b)
    assert len(pts) == n
    c, I = _inertia(pts, np.full(n, 1.2 / n))
    np.testing.assert_allclose(c, [0.5, -0.5, 1.0], atol=1e-15)
    if mode == 0:          # 12 icosahedron vertices on the sphere: isotropic, (2/3) m r^2
        np.testing.assert_allclose(np.linalg.norm(pts - c, axis=1), 0.1, rtol=1e-14)
        np.testing.assert_allclose(np.diag(I), np.full(3, 2 / 3 * 1.2 * 0.01), rtol=1e-12)
    if mode == 2:          # top and bottom
        np.testing.assert_allclose(np.sort(pts[:, 2]), [0.9, 1.1], atol=1e-15)


def test_points_and_boxes_ignore_simplify_mode():
    r = construct.Robot()
    r.simplify_mode(3)
    assert len(r.body_points(r.create_box(0.1, 0.1, 0.1, 0, 0, 0, 1.0))) == 8
    assert len(r.body_points(r.create_point(0, 0, 0, 1.0))) == 1


def test_rotate_body_is_fixed_axis_roll_pitch_yaw():
    r = construct.Robot()
    b = r.create_box(0.3, 0.2, 0.1, 0.5, 0.0, 0.0, 1.0)
    before = r.body_points(b) - [0.5, 0, 0]
    a, be, g = 0.3, -0.7, 1.1
    r.rotate_body(b, a, be, g)
    ref = Rotation.from_euler("xyz", [a, be, g]).apply(before) + [0.5, 0, 0]   # extrinsic x, y, z
    np.testing.assert_allclose(r.body_points(b), ref, atol=1e-14)
    r.move_body(b, 1.0, 2.0, 3.0)
    np.testing.assert_allclose(r.body_points(b).mean(0), [1, 2, 3], atol=1e-14)


def test_joint_anchor_and_axis_in_the_first_body_frame():
    r = construct.Robot()
    a = r.create_box(0.2, 0.2, 0.2, 1.0, 0.0, 0.0, 1.0)
    r.rotate_body(a, 0.0, 0.0, math.pi / 2)                 # body a turned 90 degrees about z
    b = r.create_box(0.1, 0.1, 0.1, 1.0, 0.3, 0.0, 0.5)
    r.create_joint(a, b, 0.2, 0.0, 0.0, 1.0, 0.0, 0.0)      # anchor 0.2 along a's x, axis a's x
    L = r.links()
    assert [l[1] for l in L] == [-1, 0]
    np.testing.assert_allclose(L[1][2], [1.0, 0.2, 0.0], atol=1e-15)   # a's x is the world y
    np.testing.assert_allclose(L[1][3], [0.0, 1.0, 0.0], atol=1e-15)


def test_glue_and_tree_errors():
    r = construct.Robot()
    a = r.create_point(0, 0, 0, 1.0)
    b = r.create_point(0.1, 0, 0, 1.0)
    r.connect_bodies(a, b)
    assert len(r.links()) == 1 and len(r.links()[0][0]) == 2
    r.create_joint(a, b, 0, 0, 0, 0, 0, 1)
    with pytest.raises(ValueError):          # a hinge inside one rigid link
        r.links()
    r = construct.Robot()
    a, b = r.create_point(0, 0, 0, 1.0), r.create_point(1, 0, 0, 1.0)
    with pytest.raises(ValueError):          # two roots
        r.links()
    with pytest.raises(ValueError):
        r.create_box(1, 1, 1, 0, 0, 0, 0.0)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_cylinder_hexapod_steps_in_the_oracle(mode):
    """The hexapod built from a torso box and 18 cylinders walks in every simplify mode: its
    points drop from 296 to 26, its mass stays, it settles on its feet without freezing."""
    rb = construct.cylinder_hexapod(mode)
    n_pts = {0: 8 + 18 * 16, 1: 8 + 18 * 8, 2: 8 + 18 * 2, 3: 8 + 18}[mode]
    b = rb.batch(2, origin=(0.0, 0.0, -float(rb.batch(1).p0[:, 2].min()) + 0.01))
    assert b.n_points == 2 * n_pts
    assert b.m.sum() == pytest.approx(2 * (1.2 + 6 * (0.05 + 0.08 + 0.06)), rel=1e-6)
    assert sorted(set(b.sensor.tolist()) - {-1}) == list(range(6))
    o = Oracle(b)
    o.step(1500)
    assert (o.status == 0).all()
    assert (o.sensors != 0).all()            # some foot touches the ground
