"""Seeded synthetic scene generators: the inputs that both the CUDA path and the CPU oracle consume.

This module holds input data only -- point clouds, link trees, joint definitions, initial poses,
actuator parameters and height fields -- and none of the simulation arithmetic (no centre of
gravity, inertia, kinematics, contact or friction).  Every array is float32 or int32, so the FP64
oracle and the FP32 kernels read bit-identical inputs.

Robot model (NeoPhysIx, Sec. III-B "Joint Angle Determination" and Appendix "createJoint"): a
scene is one robot made of links; every link is a cloud of mass points (Sec. III-A); link 0 is the
root (torso); every other link l hangs from one parent link by a hinge whose anchor and axis are
given in the construction frame (the parent's frame at rest, all joint angles zero).  Joint j of a
scene is the hinge of link j+1.

The hexapod geometry is synthetic: the paper's robot figure (Sec. IV, Fig. "hexapod") carries no
dimensions.  The torso is a 0.30 x 0.18 x 0.06 m box of 1.2 kg; each leg is coxa (0.05 m, 0.05 kg,
yaw hinge), femur (0.10 m, 0.08 kg, pitch hinge) and tibia (0.15 m, 0.06 kg, pitch hinge, pointing
down at rest); joint limits are +-60 deg; each tibia carries one foot-contact sensor.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

ROOT_SEED = 2411_05799

# actuator modes (mirrors NPX_ACT_* in include/npx.h; values are part of the C-ABI)
ACT_HOLD = 0
ACT_SINUSOID = 1

DEG = math.pi / 180.0


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([ROOT_SEED, *key])))


@dataclass
class SceneBatch:
    """Flat structure-of-arrays description of S independent scenes (all float32 / int32).

    Per scene s: links link_off[s]..link_off[s+1]-1, points point_off[s]..point_off[s+1]-1,
    joints joint_off[s]..joint_off[s+1]-1 with joint_off[s] = link_off[s] - s.
    Per link (global index l, scene-local index k = l - link_off[s]): parent (scene-local, -1 for
    the root), hinge anchor/axis in the construction frame, limits lo/hi [rad], sensor id or -1.
    Per point: construction-frame position p0, mass m [kg], scene-local link index plink.
    """
    dt: float
    gravity: tuple
    joint_update_steps: int          # K: joint angles are recomputed every K steps (Sec. III-B)
    contact_omega: float             # penalty natural frequency [rad/s]
    contact_zeta: float              # penalty damping ratio
    link_off: np.ndarray
    point_off: np.ndarray
    p0: np.ndarray
    m: np.ndarray
    plink: np.ndarray
    parent: np.ndarray
    anchor: np.ndarray
    axis: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    sensor: np.ndarray
    mu: np.ndarray
    hmap: np.ndarray                 # per scene height-map index, -1 = flat ground z = 0
    origin: np.ndarray               # initial construction-frame origin in the world [S,3]
    quat: np.ndarray                 # initial orientation (w,x,y,z) [S,4]
    vel: np.ndarray                  # initial CoG velocity [S,3]
    omega: np.ndarray                # initial angular velocity (world) [S,3]
    theta0: np.ndarray               # initial joint angles [J]
    act_mode: int = ACT_SINUSOID
    act_params: np.ndarray = None    # [J,4] (amplitude rad, frequency Hz, phase rad, bias rad)
    heightmaps: np.ndarray = None    # [H, ny, nx] float32 or None
    hm_scale: float = 10.0           # cells per metre (Sec. III-A: factor 10 -> 0.1 m cells)
    hm_origin: tuple = (0.0, 0.0)    # world (x, y) of the map's cell (0, 0) corner
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_scenes(self) -> int:
        return len(self.link_off) - 1

    @property
    def n_points(self) -> int:
        return int(self.point_off[-1])

    @property
    def n_links(self) -> int:
        return int(self.link_off[-1])

    @property
    def joint_off(self) -> np.ndarray:
        return (self.link_off - np.arange(len(self.link_off))).astype(np.int32)

    @property
    def n_joints(self) -> int:
        return int(self.joint_off[-1])

    def subset(self, scenes) -> "SceneBatch":
        """Scenes `scenes` (ascending indices) as a batch of their own, inputs unchanged."""
        scenes = np.asarray(scenes, dtype=np.int64)
        lo_, po_, jo_ = self.link_off, self.point_off, self.joint_off
        lidx = np.concatenate([np.arange(lo_[s], lo_[s + 1]) for s in scenes])
        pidx = np.concatenate([np.arange(po_[s], po_[s + 1]) for s in scenes])
        jidx = np.concatenate([np.arange(jo_[s], jo_[s + 1]) for s in scenes]).astype(np.int64)
        nl = lo_[scenes + 1] - lo_[scenes]
        npt = po_[scenes + 1] - po_[scenes]
        hm = self.hmap[scenes]
        maps = None
        if self.heightmaps is not None:
            used = np.unique(hm[hm >= 0])
            remap = -np.ones(len(self.heightmaps), np.int32)
            remap[used] = np.arange(len(used), dtype=np.int32)
            maps = np.ascontiguousarray(self.heightmaps[used])
            hm = np.where(hm >= 0, remap[np.maximum(hm, 0)], -1).astype(np.int32)
        return SceneBatch(
            dt=self.dt, gravity=self.gravity, joint_update_steps=self.joint_update_steps,
            contact_omega=self.contact_omega, contact_zeta=self.contact_zeta,
            link_off=np.concatenate([[0], np.cumsum(nl)]).astype(np.int32),
            point_off=np.concatenate([[0], np.cumsum(npt)]).astype(np.int32),
            p0=self.p0[pidx].copy(), m=self.m[pidx].copy(), plink=self.plink[pidx].copy(),
            parent=self.parent[lidx].copy(), anchor=self.anchor[lidx].copy(),
            axis=self.axis[lidx].copy(), lo=self.lo[lidx].copy(), hi=self.hi[lidx].copy(),
            sensor=self.sensor[lidx].copy(), mu=self.mu[scenes].copy(), hmap=hm,
            origin=self.origin[scenes].copy(), quat=self.quat[scenes].copy(),
            vel=self.vel[scenes].copy(), omega=self.omega[scenes].copy(),
            theta0=self.theta0[jidx].copy(), act_mode=self.act_mode,
            act_params=None if self.act_params is None else self.act_params[jidx].copy(),
            heightmaps=maps, hm_scale=self.hm_scale, hm_origin=self.hm_origin,
            name=self.name + f"[subset {len(scenes)}]", meta=dict(self.meta))

    def with_(self, **kw) -> "SceneBatch":
        d = dict(self.__dict__)
        d.update(kw)
        return SceneBatch(**d)


# ----------------------------------------------------------------------------- point lattices

def box_lattice(extent, center, counts) -> np.ndarray:
    """Points of an nx x ny x nz lattice spanning a box (corners included), float32 [n,3]."""
    axes = []
    for e, c, n in zip(extent, center, counts):
        axes.append(np.array([c]) if n == 1 else c - e / 2 + e * np.arange(n) / (n - 1))
    g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    return g.astype(np.float32)


def box_corners(w, h, d, x, y, z) -> np.ndarray:
    """createBox (Appendix): the 8 corner mass points of a w x h x d box centred at (x,y,z).
    (w,h,d) are the extents along the construction frame's (x,y,z)."""
    return box_lattice((w, h, d), (x, y, z), (2, 2, 2))


def box_uniform(rng, extent, center, n) -> np.ndarray:
    e = np.asarray(extent, np.float64)
    c = np.asarray(center, np.float64)
    return (c + (rng.random((n, 3)) - 0.5) * e).astype(np.float32)


def random_unit_quat(rng, n) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1
    return q.astype(np.float32)


# ----------------------------------------------------------------------------- legged robots

TORSO = dict(extent=(0.30, 0.18, 0.06), mass=1.2)
SEG_XSEC = 0.02
COXA = dict(length=0.05, mass=0.05)
FEMUR = dict(length=0.10, mass=0.08)
TIBIA = dict(length=0.15, mass=0.06)
HIP_Y = 0.09
LIMIT = 60 * DEG
LEG_X = {6: (-0.12, 0.0, 0.12), 4: (-0.12, 0.12), 2: (0.0,)}


def _robot_links(n_legs):
    """Link boxes of a legged robot: list of (extent, center, mass, parent, anchor, axis, sensor).
    Hips at x in LEG_X[n_legs], y = +-HIP_Y; coxa/femur extend outward along y, tibia down."""
    links = [(TORSO["extent"], (0.0, 0.0, 0.0), TORSO["mass"], -1, None, None, -1)]
    sensor = 0
    for xh in LEG_X[n_legs]:
        for side in (1.0, -1.0):
            y0 = side * HIP_Y
            y1 = side * (HIP_Y + COXA["length"])
            y2 = side * (HIP_Y + COXA["length"] + FEMUR["length"])
            base = len(links)
            links.append(((SEG_XSEC, COXA["length"], SEG_XSEC), (xh, (y0 + y1) / 2, 0.0), COXA["mass"],
                          0, (xh, y0, 0.0), (0.0, 0.0, 1.0), -1))
            links.append(((SEG_XSEC, FEMUR["length"], SEG_XSEC), (xh, (y1 + y2) / 2, 0.0), FEMUR["mass"],
                          base, (xh, y1, 0.0), (side, 0.0, 0.0), -1))
            links.append(((SEG_XSEC, SEG_XSEC, TIBIA["length"]), (xh, y2, -TIBIA["length"] / 2),
                          TIBIA["mass"], base + 1, (xh, y2, 0.0), (side, 0.0, 0.0), sensor))
            sensor += 1
    return links


FOOT_Z = -TIBIA["length"]        # lowest construction-frame z of a leg at rest


def _lattice_counts(extent):
    """4x4x4 for the torso; 2x2x4 (4 along the long axis) for a leg segment."""
    if extent[0] > 0.1:
        return (4, 4, 4)
    return tuple(4 if e == max(extent) else 2 for e in extent)


def _assemble(robots, mu, origin, quat, vel, omega, act_params, name, dt=1e-3, K=80,
              hmap=None, heightmaps=None, hm_scale=10.0, hm_origin=(0.0, 0.0), meta=None,
              gravity=(0.0, 0.0, -9.81), act_mode=ACT_SINUSOID):
    """robots: list of per-scene (links, points_per_link list of float32 [n,3])."""
    S = len(robots)
    link_off = [0]
    point_off = [0]
    p0, m, plink, parent, anchor, axis, lo, hi, sensor = [], [], [], [], [], [], [], [], []
    for links, pts in robots:
        for k, (ext, ctr, mass, par, anc, ax, sen) in enumerate(links):
            n = len(pts[k])
            p0.append(pts[k])
            m.append(np.full(n, mass / n, np.float32))
            plink.append(np.full(n, k, np.int32))
            parent.append(par)
            anchor.append(anc if anc is not None else (0.0, 0.0, 0.0))
            axis.append(ax if ax is not None else (0.0, 0.0, 1.0))
            lo.append(-LIMIT if par >= 0 else 0.0)
            hi.append(LIMIT if par >= 0 else 0.0)
            sensor.append(sen)
        link_off.append(link_off[-1] + len(links))
        point_off.append(point_off[-1] + sum(len(p) for p in pts))
    J = link_off[-1] - S
    r32 = lambda x: float(np.float32(x))      # world parameters are single precision inputs
    dt, hm_scale = r32(dt), r32(hm_scale)
    gravity = tuple(r32(g) for g in gravity)
    hm_origin = tuple(r32(o) for o in hm_origin)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    i32 = lambda a: np.ascontiguousarray(np.asarray(a, np.int32))
    return SceneBatch(
        dt=dt, gravity=tuple(gravity), joint_update_steps=K, contact_omega=300.0, contact_zeta=1.0,
        link_off=i32(link_off), point_off=i32(point_off),
        p0=f32(np.concatenate(p0)), m=f32(np.concatenate(m)), plink=i32(np.concatenate(plink)),
        parent=i32(parent), anchor=f32(anchor), axis=f32(axis), lo=f32(lo), hi=f32(hi),
        sensor=i32(sensor), mu=f32(mu), hmap=i32(hmap if hmap is not None else -np.ones(S)),
        origin=f32(origin), quat=f32(quat), vel=f32(vel), omega=f32(omega),
        theta0=np.zeros(J, np.float32), act_mode=act_mode,
        act_params=f32(act_params) if act_params is not None else np.zeros((J, 4), np.float32),
        heightmaps=None if heightmaps is None else f32(heightmaps), hm_scale=hm_scale,
        hm_origin=tuple(hm_origin), name=name, meta=meta or {})


def _sinusoid_params(rng, J, amp_max=30 * DEG, fmin=0.5, fmax=2.0):
    A = rng.uniform(0.0, amp_max, J)
    f = rng.uniform(fmin, fmax, J)
    ph = rng.uniform(0.0, 2 * math.pi, J)
    return np.stack([A, f, ph, np.zeros(J)], 1)


# ----------------------------------------------------------------------------- the workloads

def single_body(seed_key: int = 0, n_points: int = 32) -> SceneBatch:
    """One rigid body: 32 points uniform in a 0.2 x 0.1 x 0.05 m box (1 kg), random orientation,
    origin 0.5 m above flat ground, v ~ N(0, 0.5^2), omega ~ N(0, 2^2) per component, mu = 0.6."""
    rng = _rng(1, seed_key)
    pts = box_uniform(rng, (0.2, 0.1, 0.05), (0.0, 0.0, 0.0), n_points)
    links = [((0.2, 0.1, 0.05), (0, 0, 0), 1.0, -1, None, None, -1)]
    q = random_unit_quat(rng, 1)
    v = rng.normal(0.0, 0.5, (1, 3))
    w = rng.normal(0.0, 2.0, (1, 3))
    return _assemble([(links, [pts])], mu=[0.6], origin=[(0.0, 0.0, 0.5)], quat=q, vel=v,
                     omega=w, act_params=None, name="single_body_32pt", act_mode=ACT_HOLD)


def legged_batch(n_scenes: int, n_legs=6, seed_key: int = 0, mu=0.8, lattice=True,
                 pts_range=(8, 64), K=80, amp_max=30 * DEG, fmin=0.5, fmax=2.0,
                 name=None, cfg=2) -> SceneBatch:
    """n_scenes copies of a legged robot (hexapod by default, Sec. IV's 18-DoF six-sensor walker),
    feet 1 cm above flat ground, at rest, each joint driven by its own seeded sinusoid."""
    rng = _rng(cfg, seed_key)
    robots = []
    links = _robot_links(n_legs)
    if lattice:
        # identical robots: assemble one and tile its arrays
        pts = [box_lattice(e, c, _lattice_counts(e)) for e, c, *_ in links]
        one = _assemble([(links, pts)], mu=[0.0], origin=np.zeros((1, 3)), quat=[(1, 0, 0, 0)],
                        vel=np.zeros((1, 3)), omega=np.zeros((1, 3)), act_params=None, K=K,
                        name="template")
        S, nl, npt = n_scenes, len(links), one.n_points
        J = (nl - 1) * S
        mu_arr = np.full(S, mu) if np.isscalar(mu) else np.asarray(mu)
        act = _sinusoid_params(rng, J, amp_max, fmin, fmax)
        return one.with_(
            link_off=(np.arange(S + 1) * nl).astype(np.int32),
            point_off=(np.arange(S + 1) * npt).astype(np.int32),
            p0=np.tile(one.p0, (S, 1)), m=np.tile(one.m, S), plink=np.tile(one.plink, S),
            parent=np.tile(one.parent, S), anchor=np.tile(one.anchor, (S, 1)),
            axis=np.tile(one.axis, (S, 1)), lo=np.tile(one.lo, S), hi=np.tile(one.hi, S),
            sensor=np.tile(one.sensor, S), mu=mu_arr.astype(np.float32),
            hmap=-np.ones(S, np.int32),
            origin=np.tile(np.float32([0.0, 0.0, -FOOT_Z + 0.01]), (S, 1)),
            quat=np.tile(np.float32([1.0, 0.0, 0.0, 0.0]), (S, 1)),
            vel=np.zeros((S, 3), np.float32), omega=np.zeros((S, 3), np.float32),
            theta0=np.zeros(J, np.float32), act_mode=ACT_SINUSOID,
            act_params=act.astype(np.float32), name=name or f"legged{n_legs}x{n_scenes}")
    else:
        for _ in range(n_scenes):
            pts = [box_uniform(rng, e, c, int(rng.integers(pts_range[0], pts_range[1] + 1)))
                   for e, c, *_ in links]
            robots.append((links, pts))
    J = (len(links) - 1) * n_scenes
    S = n_scenes
    mu_arr = np.full(S, mu) if np.isscalar(mu) else mu
    origin = np.tile([0.0, 0.0, -FOOT_Z + 0.01], (S, 1))
    quat = np.tile([1.0, 0.0, 0.0, 0.0], (S, 1))
    act = _sinusoid_params(rng, J, amp_max, fmin, fmax)
    return _assemble(robots, mu=mu_arr, origin=origin, quat=quat, vel=np.zeros((S, 3)),
                     omega=np.zeros((S, 3)), act_params=act, K=K,
                     name=name or f"legged{n_legs}x{n_scenes}")


def hexapod_batch(n_scenes: int = 4096, seed_key: int = 0, K: int = 80) -> SceneBatch:
    """The 18-DoF hexapod workload: torso 64 points + 18 segments x 16 points = 352 points,
    18 hinges (+-60 deg) tracking A sin(2 pi f t + phi) with A ~ U(0, 30 deg), f ~ U(0.5, 2) Hz,
    phi ~ U(0, 2 pi); flat ground, mu = 0.8, dt = 1 ms."""
    return legged_batch(n_scenes, 6, seed_key, mu=0.8, K=K, name=f"hexapod_{n_scenes}")


def _robots_vectorized(rng, legs_per_scene, pts_lo=8, pts_hi=64):
    """Flat arrays for scenes of legged robots with U{pts_lo..pts_hi} points per link, uniform in
    each link's box (vectorised over all scenes)."""
    templates = {n: _robot_links(n) for n in np.unique(legs_per_scene)}
    tl = [templates[n] for n in legs_per_scene]
    nl = np.array([len(t) for t in tl], np.int64)
    ext = np.concatenate([[l[0] for l in t] for t in tl]).reshape(-1, 3)
    ctr = np.concatenate([[l[1] for l in t] for t in tl]).reshape(-1, 3)
    lmass = np.concatenate([[l[2] for l in t] for t in tl])
    parent = np.concatenate([[l[3] for l in t] for t in tl]).astype(np.int32)
    anchor = np.concatenate([[l[4] if l[4] is not None else (0, 0, 0) for l in t] for t in tl]).reshape(-1, 3)
    axis = np.concatenate([[l[5] if l[5] is not None else (0, 0, 1) for l in t] for t in tl]).reshape(-1, 3)
    sensor = np.concatenate([[l[6] for l in t] for t in tl]).astype(np.int32)
    counts = rng.integers(pts_lo, pts_hi + 1, len(parent))
    u = rng.random((int(counts.sum()), 3))
    p0 = (np.repeat(ctr, counts, 0) + (u - 0.5) * np.repeat(ext, counts, 0)).astype(np.float32)
    m = np.repeat(lmass / counts, counts).astype(np.float32)
    link_off = np.concatenate([[0], np.cumsum(nl)]).astype(np.int32)
    scene_of_link = np.repeat(np.arange(len(nl)), nl)
    local = (np.arange(len(parent)) - link_off[scene_of_link]).astype(np.int32)
    plink = np.repeat(local, counts).astype(np.int32)
    pts_per_scene = np.add.reduceat(counts, link_off[:-1])
    point_off = np.concatenate([[0], np.cumsum(pts_per_scene)]).astype(np.int32)
    root = parent < 0
    lo = np.where(root, 0.0, -LIMIT).astype(np.float32)
    hi = np.where(root, 0.0, LIMIT).astype(np.float32)
    return dict(link_off=link_off, point_off=point_off, p0=p0, m=m, plink=plink, parent=parent,
                anchor=anchor.astype(np.float32), axis=axis.astype(np.float32), lo=lo, hi=hi,
                sensor=sensor)


def uneven_batch(n_scenes: int = 65536, seed_key: int = 0) -> SceneBatch:
    """Mixed batch: hexapods (19 links) / quadrupeds (13 links) / bipeds (7 links) in seeded
    50/30/20 proportions, 8..64 points per link uniform in the link box, mu ~ U(0.3, 1.0)."""
    rng = _rng(3, seed_key)
    kinds = rng.choice([6, 4, 2], size=n_scenes, p=[0.5, 0.3, 0.2])
    mu = rng.uniform(0.3, 1.0, n_scenes)
    arr = _robots_vectorized(rng, kinds)
    S = n_scenes
    J = int(arr["link_off"][-1]) - S
    act = _sinusoid_params(rng, J)
    r32 = lambda x: float(np.float32(x))
    return SceneBatch(
        dt=r32(1e-3), gravity=(0.0, 0.0, r32(-9.81)), joint_update_steps=80, contact_omega=300.0,
        contact_zeta=1.0, **arr, mu=mu.astype(np.float32), hmap=-np.ones(S, np.int32),
        origin=np.tile(np.float32([0.0, 0.0, -FOOT_Z + 0.01]), (S, 1)),
        quat=np.tile(np.float32([1.0, 0, 0, 0]), (S, 1)), vel=np.zeros((S, 3), np.float32),
        omega=np.zeros((S, 3), np.float32), theta0=np.zeros(J, np.float32),
        act_mode=ACT_SINUSOID, act_params=act.astype(np.float32), name=f"uneven_{n_scenes}",
        meta={"legs": kinds.astype(np.int32)})


def rough_heightfields(rng, n_maps, n=128, cell=0.05, sigma_cells=2.0, std=0.02):
    """Per-scene n x n FP32 height fields: N(0,1) noise, periodic Gaussian blur (sigma in cells),
    rescaled to the given standard deviation [m]."""
    import scipy.fft as sfft
    ky = np.fft.fftfreq(n)
    kx = np.fft.rfftfreq(n)
    g = np.exp(-2 * (math.pi * sigma_cells) ** 2 * (ky[:, None] ** 2 + kx[None, :] ** 2))
    out = np.empty((n_maps, n, n), np.float32)
    chunk = 1024
    for i in range(0, n_maps, chunk):
        z = rng.standard_normal((min(chunk, n_maps - i), n, n), dtype=np.float32)
        z = sfft.irfft2(sfft.rfft2(z, workers=-1) * g, s=(n, n), workers=-1)
        z /= z.std(axis=(1, 2), keepdims=True)
        out[i:i + len(z)] = (z * std).astype(np.float32)
    return out


def cpg_batch(n_scenes: int = 16384, seed_key: int = 0, n_cells=128, cell=0.05) -> SceneBatch:
    """Evolution-scale rollout: hexapods with per-leg CPG parameters (f ~ U(0.5, 3) Hz,
    phi ~ U(0, 2 pi), A ~ U(5, 35 deg); coxa/femur/tibia phase offsets 0, pi/2, pi/2) on a
    per-scene 128 x 128 rough height field with 5 cm cells (scale 20, Sec. III-A), robot
    started at the map centre."""
    rng = _rng(4, seed_key)
    base = legged_batch(n_scenes, 6, seed_key, mu=0.8, name=f"cpg_rough_{n_scenes}", cfg=4)
    S = n_scenes
    f = rng.uniform(0.5, 3.0, (S, 6))
    ph = rng.uniform(0.0, 2 * math.pi, (S, 6))
    A = rng.uniform(5 * DEG, 35 * DEG, (S, 6))
    offs = np.array([0.0, math.pi / 2, math.pi / 2])
    act = np.zeros((S, 6, 3, 4))
    act[..., 0] = A[..., None]
    act[..., 1] = f[..., None]
    act[..., 2] = ph[..., None] + offs
    maps = rough_heightfields(rng, S, n_cells, cell)
    half = n_cells * cell / 2
    # start above the highest cell under the robot's footprint (0.6 m square at the centre)
    c0 = n_cells // 2
    r = int(round(0.3 / cell))
    hmax = maps[:, c0 - r:c0 + r, c0 - r:c0 + r].max(axis=(1, 2))
    origin = np.zeros((S, 3))
    origin[:, 2] = hmax - FOOT_Z + 0.01
    return base.with_(act_params=act.reshape(-1, 4).astype(np.float32),
                      origin=origin.astype(np.float32), heightmaps=maps,
                      hmap=np.arange(S, dtype=np.int32), hm_scale=float(np.float32(1.0 / cell)),
                      hm_origin=(float(np.float32(-half)), float(np.float32(-half))))


def tilted_gravity(batch: SceneBatch, theta: float, g: float = 9.81) -> SceneBatch:
    """An incline of angle theta realised by tilting gravity about the y axis on flat ground."""
    return batch.with_(gravity=(float(np.float32(g * math.sin(theta))), 0.0,
                                float(np.float32(-g * math.cos(theta)))))


def ragged_bodies(counts, seed_key: int = 0, mu: float = 0.6) -> SceneBatch:
    """Single-link bodies with the given point counts (uniform in a 0.2 x 0.1 x 0.05 m box, 1 kg),
    random orientation, dropped from 0.3 m with random linear and angular velocity onto flat
    ground: ragged batches from one point up to the largest scene a world holds."""
    rng = _rng(7, seed_key)
    S = len(counts)
    robots = []
    for n in counts:
        pts = box_uniform(rng, (0.2, 0.1, 0.05), (0.0, 0.0, 0.0), int(n))
        robots.append(([((0.2, 0.1, 0.05), (0, 0, 0), 1.0, -1, None, None, -1)], [pts]))
    origin = np.column_stack([rng.uniform(-1, 1, S), rng.uniform(-1, 1, S), np.full(S, 0.3)])
    return _assemble(robots, mu=np.full(S, mu), origin=origin, quat=random_unit_quat(rng, S),
                     vel=rng.normal(0.0, 0.5, (S, 3)), omega=rng.normal(0.0, 2.0, (S, 3)),
                     act_params=None, name="ragged_bodies", act_mode=ACT_HOLD)


def block_batch(n_scenes=1, mu=0.5, extent=(0.2, 0.2, 0.1), counts=(3, 3, 2), mass=1.0,
                z_gap=0.0, vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), name="block") -> SceneBatch:
    """A single-link lattice block resting (bottom face at z = z_gap) on flat ground."""
    pts = box_lattice(extent, (0, 0, 0), counts)
    links = [(extent, (0, 0, 0), mass, -1, None, None, 0)]
    S = n_scenes
    origin = np.tile([0.0, 0.0, extent[2] / 2 + z_gap], (S, 1))
    return _assemble([(links, [pts])] * S, mu=np.full(S, mu), origin=origin,
                     quat=np.tile([1.0, 0, 0, 0], (S, 1)), vel=np.tile(vel, (S, 1)),
                     omega=np.tile(omega, (S, 1)), act_params=None, name=name,
                     act_mode=ACT_HOLD)


def concat(batches) -> SceneBatch:
    """The scenes of several batches (same step, gravity, contact law, actuator mode; flat ground)
    as one batch, in order."""
    b0 = batches[0]
    for b in batches[1:]:
        if (b.dt, b.gravity, b.joint_update_steps, b.contact_omega, b.contact_zeta, b.act_mode) != \
                (b0.dt, b0.gravity, b0.joint_update_steps, b0.contact_omega, b0.contact_zeta, b0.act_mode):
            raise ValueError("batches differ in their world parameters")
    if any(b.heightmaps is not None for b in batches):
        raise ValueError("concat takes flat-ground batches")
    offs = lambda key: np.concatenate([[0]] + [getattr(b, key)[1:] + sum(int(getattr(c, key)[-1])
                                                                         for c in batches[:i])
                                               for i, b in enumerate(batches)]).astype(np.int32)
    cat = lambda key: np.ascontiguousarray(np.concatenate([getattr(b, key) for b in batches]))
    return b0.with_(link_off=offs("link_off"), point_off=offs("point_off"),
                    **{k: cat(k) for k in ("p0", "m", "plink", "parent", "anchor", "axis", "lo", "hi",
                                           "sensor", "mu", "hmap", "origin", "quat", "vel", "omega",
                                           "theta0", "act_params")},
                    name="+".join(b.name for b in batches), meta={})


# Arena layouts (robot-robot collision): hexapod k of an arena is placed at ARENA_XY[size][k].
# Side by side along y, 0.44 m apart, the legs of the two rows overlap by 4 cm and are staggered
# by 6 cm along x, so that swinging coxae drive legs into each other's; in the 2 x 2 layout the
# torsos of a row are 4 cm apart.
ARENA_XY = {2: ((0.0, -0.22), (0.06, 0.22)),
            4: ((-0.17, -0.22), (0.17, -0.22), (-0.11, 0.22), (0.23, 0.22))}


def arena_batch(n_arenas: int, size: int = 4, seed_key: int = 0) -> SceneBatch:
    """n_arenas arenas of `size` hexapods (scenes a*size .. a*size + size - 1), each robot with its
    own seeded sinusoid gaits, laid out by ARENA_XY (every arena at the same place: arenas do not
    interact)."""
    base = hexapod_batch(n_arenas * size, seed_key=seed_key)
    xy = np.tile(np.asarray(ARENA_XY[size], np.float64), (n_arenas, 1))
    origin = base.origin.astype(np.float64).copy()
    origin[:, :2] = xy
    return base.with_(origin=origin.astype(np.float32), name=f"hexapod_arenas_{n_arenas}x{size}",
                      meta={"arena": size})
