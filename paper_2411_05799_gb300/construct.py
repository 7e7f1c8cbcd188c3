"""Robot construction from primitives, as the paper's construction calls describe it (Appendix:
createPoint, createBox, createCylinder, createSphere, connectBodies, createJoint, moveBody,
rotateBody, finalizeConstruction; Sec. III-D: simplifyMode), producing the point clouds, links and
hinges of a scene batch.

Bodies stay on the host until `batch()`: bodies glued with connect_bodies form one rigid link, and
create_joint hangs the link of its second body from the link of its first by a hinge.  A body's
own frame is its centre (the position it was created at, or moved to) with the orientation
rotate_body gave it; joint anchors and axes are given in the first body's frame.

Readings where the text is silent:
  - a box is its 8 corners ("consists of 8 points"), extents (w, h, d) along x, y, z;
  - without simplification a cylinder is its two end rims of 8 points each and a sphere the 12
    vertices of the inscribed icosahedron (an isotropic inertia);
  - simplify mode 1 turns cylinders and spheres into their bounding boxes (8 corners, the box of a
    cylinder aligned with its axis), mode 2 into two points (a cylinder's end centres, a sphere's
    top and bottom), mode >= 3 into one point at the centre; points and boxes are unchanged;
  - rotate_body is roll-pitch-yaw about the fixed construction axes x, then y, then z
    (R = Rz(gamma) Ry(beta) Rx(alpha)), right-handed, about the body's centre; move_body puts the
    body's centre at the given position;
  - a body's mass is spread equally over its points; rays (render-only, no collision) have no
    points and are not built.
"""
from __future__ import annotations

import math

import numpy as np

from . import scenes

DEG = math.pi / 180.0


def _rpy(alpha, beta, gamma):
    ca, sa, cb, sb, cg, sg = (math.cos(alpha), math.sin(alpha), math.cos(beta), math.sin(beta),
                              math.cos(gamma), math.sin(gamma))
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _perp_frame(u):
    """An orthonormal frame (e1, e2, u) for the unit vector u (deterministic)."""
    a = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    return e1, e2


def _icosahedron(r):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-t, t):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    return v / np.linalg.norm(v, axis=1, keepdims=True) * r


def _box_corners(ext):
    w, h, d = ext
    return np.array([(sx * w / 2, sy * h / 2, sz * d / 2)
                     for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], np.float64)


class Robot:
    """One robot built from primitives (the construction calls of the paper's appendix)."""

    def __init__(self):
        self._pts = []          # per body: points in the body's own frame [n, 3]
        self._mass = []         # per body: total mass
        self._pos = []          # per body: centre in the construction frame
        self._rot = []          # per body: orientation (3x3)
        self._glue = []         # union-find parents
        self._joints = []       # (body1, body2, anchor in body-1 frame, axis in body-1 frame, lo, hi)
        self._sensor = {}
        self._mode = 0

    # -- simplification (Sec. III-D)
    def simplify_mode(self, mode: int):
        """0: none; 1: cylinders and spheres become boxes; 2: two points; >= 3: one point.
        Applies to the bodies created after the call."""
        self._mode = int(mode)

    def _add(self, pts, mass, centre, rot=None) -> int:
        if not (mass > 0):
            raise ValueError("a body needs a positive mass")
        self._pts.append(np.asarray(pts, np.float64).reshape(-1, 3))
        self._mass.append(float(mass))
        self._pos.append(np.asarray(centre, np.float64))
        self._rot.append(np.eye(3) if rot is None else np.asarray(rot, np.float64))
        self._glue.append(len(self._glue))
        return len(self._pts) - 1

    # -- primitives (Appendix)
    def create_point(self, x, y, z, m) -> int:
        return self._add([[0.0, 0.0, 0.0]], m, (x, y, z))

    def create_box(self, w, h, d, x, y, z, m) -> int:
        return self._add(_box_corners((w, h, d)), m, (x, y, z))

    def create_cylinder(self, x1, y1, z1, x2, y2, z2, rr, m) -> int:
        p1, p2 = np.array([x1, y1, z1], float), np.array([x2, y2, z2], float)
        c = 0.5 * (p1 + p2)
        axis = p2 - p1
        L = float(np.linalg.norm(axis))
        u = axis / L if L > 0 else np.array([0.0, 0.0, 1.0])
        e1, e2 = _perp_frame(u)
        R = np.stack([e1, e2, u], 1)            # body frame: z along the axis
        if self._mode == 0:
            ang = np.arange(8) * (2 * math.pi / 8)
            rim = np.stack([rr * np.cos(ang), rr * np.sin(ang), np.zeros(8)], 1)
            pts = np.concatenate([rim + [0, 0, -L / 2], rim + [0, 0, L / 2]])
        elif self._mode == 1:
            pts = _box_corners((2 * rr, 2 * rr, L))
        elif self._mode == 2:
            pts = np.array([[0.0, 0.0, -L / 2], [0.0, 0.0, L / 2]])
        else:
            pts = np.zeros((1, 3))
        return self._add(pts, m, c, R)

    def create_sphere(self, x, y, z, rr, m) -> int:
        if self._mode == 0:
            pts = _icosahedron(rr)
        elif self._mode == 1:
            pts = _box_corners((2 * rr, 2 * rr, 2 * rr))
        elif self._mode == 2:
            pts = np.array([[0.0, 0.0, -rr], [0.0, 0.0, rr]])
        else:
            pts = np.zeros((1, 3))
        return self._add(pts, m, (x, y, z))

    # -- assembly
    def _root(self, i):
        while self._glue[i] != i:
            self._glue[i] = self._glue[self._glue[i]]
            i = self._glue[i]
        return i

    def connect_bodies(self, id1, id2):
        """Glue two bodies into one rigid link."""
        a, b = self._root(id1), self._root(id2)
        if a != b:
            self._glue[max(a, b)] = min(a, b)

    def create_joint(self, id1, id2, anx, any_, anz, ax, ay, az, lo=-60 * DEG, hi=60 * DEG) -> int:
        """A hinge between the link of id1 (parent) and that of id2 (child), anchor and axis in
        the frame of body id1."""
        self._joints.append((id1, id2, np.array([anx, any_, anz], float), np.array([ax, ay, az], float),
                             float(lo), float(hi)))
        return len(self._joints) - 1

    def add_sensor(self, body, bit):
        """The foot-contact sensor bit of the body's link."""
        self._sensor[body] = int(bit)

    def move_body(self, body, tx, ty, tz):
        self._pos[body] = np.array([tx, ty, tz], float)

    def rotate_body(self, body, alpha, beta, gamma):
        self._rot[body] = _rpy(alpha, beta, gamma) @ self._rot[body]

    def max_body_id(self) -> int:
        return len(self._pts)

    def body_points(self, body) -> np.ndarray:
        """The body's points in the construction frame."""
        return self._pts[body] @ self._rot[body].T + self._pos[body]

    # -- finalizeConstruction
    def links(self):
        """Links (groups of glued bodies) in tree order, root first: list of (bodies, parent link,
        anchor, axis, lo, hi, sensor) with anchor and axis in the construction frame."""
        roots = sorted({self._root(i) for i in range(len(self._pts))})
        group = {r: [i for i in range(len(self._pts)) if self._root(i) == r] for r in roots}
        child_of = {}
        for id1, id2, an, ax, lo, hi in self._joints:
            p, c = self._root(id1), self._root(id2)
            if p == c:
                raise ValueError("a joint inside one rigid link")
            if c in child_of:
                raise ValueError("a link hangs from two joints (the links must form a tree)")
            R1 = self._rot[id1]
            axw = R1 @ ax
            child_of[c] = (p, R1 @ an + self._pos[id1], axw / np.linalg.norm(axw), lo, hi)
        tops = [r for r in roots if r not in child_of]
        if len(tops) != 1:
            raise ValueError(f"{len(tops)} root links: every link but one must hang from a joint")
        order, index = [], {}
        stack = [tops[0]]
        while stack:                             # parents before children
            r = stack.pop(0)
            index[r] = len(order)
            order.append(r)
            stack += [c for c in roots if c in child_of and child_of[c][0] == r]
        if len(order) != len(roots):
            raise ValueError("the joints do not connect every link to the root")
        out = []
        for r in order:
            sen = [self._sensor[b] for b in group[r] if b in self._sensor]
            if r in child_of:
                p, an, ax, lo, hi = child_of[r]
                out.append((group[r], index[p], an, ax, lo, hi, sen[0] if sen else -1))
            else:
                out.append((group[r], -1, np.zeros(3), np.array([0.0, 0.0, 1.0]), 0.0, 0.0,
                            sen[0] if sen else -1))
        return out

    def batch(self, n_scenes=1, origin=(0.0, 0.0, 0.0), mu=0.8, act_params=None,
              act_mode=None, name="constructed", **kw) -> "scenes.SceneBatch":
        """n_scenes copies of the robot as a SceneBatch (finalizeConstruction)."""
        L = self.links()
        p0, m, plink, parent, anchor, axis, lo, hi, sensor = [], [], [], [], [], [], [], [], []
        for k, (bodies, par, an, ax, l, h, sen) in enumerate(L):
            for b in bodies:
                pts = self.body_points(b)
                p0.append(pts)
                m.append(np.full(len(pts), self._mass[b] / len(pts)))
                plink.append(np.full(len(pts), k))
            parent.append(par)
            anchor.append(an)
            axis.append(ax)
            lo.append(l)
            hi.append(h)
            sensor.append(sen)
        P1, L1 = sum(len(a) for a in p0), len(L)
        S = n_scenes
        J = (L1 - 1) * S
        f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
        i32 = lambda a: np.ascontiguousarray(np.asarray(a, np.int32))
        tile = lambda a, reps: np.concatenate([np.asarray(a)] * reps)
        if act_params is None:
            act_params = np.zeros((J, 4))
        if act_mode is None:
            act_mode = scenes.ACT_SINUSOID if J else scenes.ACT_HOLD
        r32 = lambda x: float(np.float32(x))
        return scenes.SceneBatch(
            dt=r32(kw.get("dt", 1e-3)), gravity=(0.0, 0.0, r32(-9.81)), joint_update_steps=kw.get("K", 80),
            contact_omega=300.0, contact_zeta=1.0,
            link_off=i32(np.arange(S + 1) * L1), point_off=i32(np.arange(S + 1) * P1),
            p0=f32(tile(np.concatenate(p0), S)), m=f32(tile(np.concatenate(m), S)),
            plink=i32(tile(np.concatenate(plink), S)), parent=i32(tile(parent, S)),
            anchor=f32(tile(anchor, S)), axis=f32(tile(axis, S)), lo=f32(tile(lo, S)), hi=f32(tile(hi, S)),
            sensor=i32(tile(sensor, S)), mu=f32(np.full(S, mu)), hmap=-np.ones(S, np.int32),
            origin=f32(np.tile(origin, (S, 1))), quat=f32(np.tile([1.0, 0, 0, 0], (S, 1))),
            vel=np.zeros((S, 3), np.float32), omega=np.zeros((S, 3), np.float32),
            theta0=np.zeros(J, np.float32), act_mode=act_mode, act_params=f32(act_params), name=name)


def cylinder_hexapod(mode: int) -> Robot:
    """The benchmark's 18-DoF hexapod (torso box, coxa / femur / tibia per leg, foot sensors on
    the tibiae) with its leg segments built as cylinders of 1 cm radius and the torso as a box,
    under simplify mode `mode`."""
    r = Robot()
    t = scenes.TORSO
    torso = r.create_box(*t["extent"], 0.0, 0.0, 0.0, t["mass"])
    r.simplify_mode(mode)
    bit = 0
    for xh in scenes.LEG_X[6]:
        for side in (1.0, -1.0):
            y0 = side * scenes.HIP_Y
            y1 = side * (scenes.HIP_Y + scenes.COXA["length"])
            y2 = side * (scenes.HIP_Y + scenes.COXA["length"] + scenes.FEMUR["length"])
            coxa = r.create_cylinder(xh, y0, 0.0, xh, y1, 0.0, 0.01, scenes.COXA["mass"])
            femur = r.create_cylinder(xh, y1, 0.0, xh, y2, 0.0, 0.01, scenes.FEMUR["mass"])
            tibia = r.create_cylinder(xh, y2, 0.0, xh, y2, -scenes.TIBIA["length"], 0.01, scenes.TIBIA["mass"])
            # anchors and axes in the first body's own frame
            r.create_joint(torso, coxa, xh, y0, 0.0, 0.0, 0.0, 1.0)
            R = r._rot[coxa]
            r.create_joint(coxa, femur, *(R.T @ (np.array([xh, y1, 0.0]) - r._pos[coxa])), *(R.T @ [side, 0.0, 0.0]))
            R = r._rot[femur]
            r.create_joint(femur, tibia, *(R.T @ (np.array([xh, y2, 0.0]) - r._pos[femur])), *(R.T @ [side, 0.0, 0.0]))
            r.add_sensor(tibia, bit)
            bit += 1
    return r
