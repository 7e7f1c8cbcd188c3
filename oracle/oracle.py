"""Python handle on the FP64 CPU oracle (oracle/npxo.c) -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this module.  It
shares no code with the CUDA library; it reads the same seeded inputs (a SceneBatch of float32 /
int32 arrays) and keeps its own double-precision state.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpxo.so")
COUNT_LIB_PATH = os.path.join(HERE, "libnpxo_count.so")
SOURCES = [os.path.join(HERE, "npxo.c")]
HEADERS = [os.path.join(HERE, "npxo.h"), os.path.join(HERE, "opcount.h")]


def _compile(out: str, cmd_head: list, force: bool) -> str:
    newest = max(os.path.getmtime(p) for p in SOURCES + HEADERS)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run([*cmd_head, "-o", tmp, *SOURCES, "-lm", "-lpthread"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction so that x86 and Arm agree), and
    its counting build (the same source as C++ with every double counting its operations)."""
    _compile(COUNT_LIB_PATH, ["g++", "-O2", "-std=c++17", "-x", "c++", "-DNPXO_OPCOUNT", "-D_GNU_SOURCE",
                              "-ffp-contract=off", "-fPIC", "-shared"], force)
    return _compile(LIB_PATH, ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC",
                               "-shared"], force)


class _Model(C.Structure):
    _fields_ = [
        ("n_scenes", C.c_int), ("dt", C.c_double), ("gravity", C.c_double * 3), ("K", C.c_int),
        ("omega_c", C.c_double), ("zeta", C.c_double),
        ("link_off", C.c_void_p), ("point_off", C.c_void_p),
        ("p0", C.c_void_p), ("m", C.c_void_p), ("plink", C.c_void_p),
        ("parent", C.c_void_p), ("anchor", C.c_void_p), ("axis", C.c_void_p),
        ("lo", C.c_void_p), ("hi", C.c_void_p), ("sensor", C.c_void_p),
        ("mu", C.c_void_p), ("hmap", C.c_void_p),
        ("heightmaps", C.c_void_p), ("hm_nx", C.c_int), ("hm_ny", C.c_int),
        ("hm_scale", C.c_double), ("hm_origin", C.c_double * 2),
        ("act_mode", C.c_int), ("act_params", C.c_void_p),
        ("fric_mode", C.c_int),
        ("gp_prog", C.c_void_p),
        ("arena", C.c_int), ("arena_radius", C.c_double),
    ]


class _State(C.Structure):
    _fields_ = [("c", C.c_void_p), ("q", C.c_void_p), ("v", C.c_void_p), ("L", C.c_void_p),
                ("theta", C.c_void_p), ("kappa", C.c_void_p), ("sensors", C.c_void_p),
                ("status", C.c_void_p), ("gp_pc", C.c_void_p), ("gp_acc", C.c_void_p),
                ("gp_k", C.c_void_p)]


class Counts(C.Structure):
    _fields_ = [("scene_steps", C.c_ulonglong), ("points", C.c_ulonglong),
                ("contacts", C.c_ulonglong), ("friction_pts", C.c_ulonglong),
                ("ticks", C.c_ulonglong), ("tick_points", C.c_ulonglong)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None
_count_lib = None


def _declare(L):
    P = C.c_void_p
    L.npxo_init.argtypes = [P, P, P, P, P, P, P]
    L.npxo_step.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_longlong, P]
    L.npxo_step_mt.argtypes = [P, P, C.c_int, C.c_longlong, C.c_int, P]
    L.npxo_points_world.argtypes = [P, P, C.c_int, P]
    L.npxo_mass_props.argtypes = [P, P, C.c_int, P, P, P]
    L.npxo_link_frames.argtypes = [P, P, C.c_int, P]
    L.npxo_target.argtypes = [P, C.c_int, C.c_int, C.c_longlong]
    L.npxo_target.restype = C.c_double
    L.npxo_lut.argtypes = [P, C.c_int, C.c_double, C.c_double, P]
    L.npxo_friction_ls.argtypes = [C.c_int, P, P, P, P]
    L.npxo_friction_ls_w.argtypes = [C.c_int, P, P, P, P, P]
    L.npxo_gp_run.argtypes = [P, P, P, P, C.c_int, C.c_uint, C.c_int]
    L.npxo_gp_run.restype = None
    L.npxo_arena_forces.argtypes = [C.c_int, P, P, P, P, P, P, P, C.c_double, C.c_double,
                                    C.c_double, P]
    L.npxo_arena_forces.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def count_lib():
    """The counting build of the oracle (opcount.h): same results, operations counted."""
    global _count_lib
    if _count_lib is None:
        build()
        L = _declare(C.CDLL(COUNT_LIB_PATH))
        L.npxo_opcount_reset.argtypes = []
        L.npxo_opcount_reset.restype = None
        L.npxo_opcount_get.argtypes = [C.c_void_p]
        L.npxo_opcount_get.restype = None
        _count_lib = L
    return _count_lib


# the counting build's regions of a step and kinds of operation (opcount.h)
OP_REGIONS = ("other", "scene", "point", "contact", "friction", "tick")
OP_KINDS = ("add", "mul", "div", "sqrt", "transc", "cmp")
FLOP_KINDS = ("add", "mul", "div", "sqrt", "transc")    # comparisons are not floating-point work


def _ptr(a):
    return None if a is None else a.ctypes.data


def friction_ls(src_xy: np.ndarray, e_xy: np.ndarray):
    """The oracle's solution of Eqs. 4-6: (t, a3) of the centred problem."""
    s = np.ascontiguousarray(src_xy, np.float64)
    e = np.ascontiguousarray(e_xy, np.float64)
    t = np.zeros(2)
    a3 = np.zeros(1)
    lib().npxo_friction_ls(len(s), _ptr(s), _ptr(e), _ptr(t), _ptr(a3))
    return t, float(a3[0])


def friction_ls_w(src_xy: np.ndarray, e_xy: np.ndarray, w: np.ndarray):
    """The oracle's weighted least squares (rows weighted by w >= 0): (t, a3) of the problem
    centred on the weighted centroid."""
    s = np.ascontiguousarray(src_xy, np.float64)
    e = np.ascontiguousarray(e_xy, np.float64)
    ww = np.ascontiguousarray(w, np.float64)
    t = np.zeros(2)
    a3 = np.zeros(1)
    lib().npxo_friction_ls_w(len(s), _ptr(s), _ptr(e), _ptr(ww), _ptr(t), _ptr(a3))
    return t, float(a3[0])


ACT_GP = 2                # actuator mode of the machine-code controller (Sec. IV, Table I)
GP_LEN, GP_PER_UPDATE = 32, 32


def gp_run(prog, pc: int, acc: int, k, sensors: int, n_instr: int = GP_PER_UPDATE):
    """The oracle's interpreter on one program: returns (pc, acc, k) after n_instr instructions."""
    p = np.ascontiguousarray(prog, np.uint8)
    pcs = np.array([pc], np.uint8)
    accs = np.array([acc], np.uint8)
    kk = np.ascontiguousarray(np.array(k, np.int8))
    lib().npxo_gp_run(_ptr(p), _ptr(pcs), _ptr(accs), _ptr(kk), len(kk), int(sensors), int(n_instr))
    return int(pcs[0]), int(accs[0]), kk


def arena_forces(x, m, c, v, om, active, radius: float, omega_c: float, zeta: float) -> np.ndarray:
    """The oracle's robot-robot contact wrenches: x[k] ([n_k, 3] world points) and m[k] ([n_k]
    masses) of robot k, with its CoG c[k], velocity v[k] and angular velocity om[k]; returns
    [n_robots, 6] force and torque about each CoG."""
    n = len(x)
    xs = [np.ascontiguousarray(a, np.float64) for a in x]
    ms = [np.ascontiguousarray(a, np.float32) for a in m]
    npts = np.array([len(a) for a in xs], np.int32)
    xp = (C.c_void_p * n)(*[a.ctypes.data for a in xs])
    mp = (C.c_void_p * n)(*[a.ctypes.data for a in ms])
    cc, vv, ww = (np.ascontiguousarray(a, np.float64).reshape(n, 3) for a in (c, v, om))
    act = np.ascontiguousarray(active, np.int32)
    out = np.zeros((n, 6))
    lib().npxo_arena_forces(n, _ptr(npts), C.cast(xp, C.c_void_p), C.cast(mp, C.c_void_p), _ptr(cc), _ptr(vv),
                            _ptr(ww), _ptr(act), radius, omega_c, zeta, _ptr(out))
    return out


# friction-model options (bits of fric_mode): least-squares rows weighted by the points' normal
# forces; the friction impulse's torque about the horizontal axes.  0 = Eqs. 1-6 as written.
FRIC_WEIGHTED, FRIC_TILT = 1, 2


class Oracle:
    """FP64 state of every scene of a SceneBatch, advanced by the C oracle."""

    def __init__(self, batch, threads: int = 1, fric_mode: int = 0, gp_programs=None, arena: int = 1,
                 arena_radius: float = 0.0, counting: bool = False):
        self.batch = b = batch
        self.threads = threads
        # the counting build steps identically and counts every operation (one thread only)
        self.counting = bool(counting)
        if self.counting and threads != 1:
            raise ValueError("the counting build of the oracle runs on one thread")
        self._L = count_lib() if self.counting else lib()
        self.fric_mode = int(fric_mode)
        # robots per arena (consecutive scenes colliding with one another) and the point radius
        self.arena, self.arena_radius = int(arena), float(arena_radius)
        S, P, J = b.n_scenes, b.n_points, b.n_joints
        self._keep = [np.ascontiguousarray(a) for a in
                      (b.link_off, b.point_off, b.p0, b.m, b.plink, b.parent, b.anchor, b.axis,
                       b.lo, b.hi, b.sensor, b.mu, b.hmap)]
        (lo_, po_, p0, m, pl, par, anc, ax, lo, hi, sen, mu, hm) = self._keep
        maps = None if b.heightmaps is None else np.ascontiguousarray(b.heightmaps, np.float32)
        act = np.ascontiguousarray(b.act_params if b.act_params is not None
                                   else np.zeros((J, 4), np.float32), np.float32)
        # the machine-code controller replaces the batch's actuators when programs are given
        self.gp_prog = None if gp_programs is None else np.ascontiguousarray(gp_programs, np.uint8).reshape(S, GP_LEN)
        self._keep += [maps, act]
        self.model = _Model(
            n_scenes=S, dt=b.dt, gravity=(C.c_double * 3)(*b.gravity), K=b.joint_update_steps,
            omega_c=b.contact_omega, zeta=b.contact_zeta,
            link_off=_ptr(lo_), point_off=_ptr(po_), p0=_ptr(p0), m=_ptr(m), plink=_ptr(pl),
            parent=_ptr(par), anchor=_ptr(anc), axis=_ptr(ax), lo=_ptr(lo), hi=_ptr(hi),
            sensor=_ptr(sen), mu=_ptr(mu), hmap=_ptr(hm), heightmaps=_ptr(maps),
            hm_nx=0 if maps is None else maps.shape[2], hm_ny=0 if maps is None else maps.shape[1],
            hm_scale=b.hm_scale, hm_origin=(C.c_double * 2)(*b.hm_origin),
            act_mode=ACT_GP if self.gp_prog is not None else b.act_mode, act_params=_ptr(act),
            fric_mode=int(fric_mode), gp_prog=_ptr(self.gp_prog) if self.gp_prog is not None else None,
            arena=self.arena, arena_radius=self.arena_radius)
        self.c = np.zeros((S, 3))
        self.q = np.zeros((S, 4))
        self.v = np.zeros((S, 3))
        self.L = np.zeros((S, 3))
        self.theta = np.zeros(J)
        self.kappa = np.zeros(P, np.uint8)
        self.sensors = np.zeros(S, np.uint32)
        self.status = np.zeros(S, np.uint32)
        self.gp_pc = np.zeros(S, np.uint8)
        self.gp_acc = np.zeros(S, np.uint8)
        self.gp_k = np.zeros(J, np.int8)
        self.state = _State(*[_ptr(a) for a in (self.c, self.q, self.v, self.L, self.theta,
                                                 self.kappa, self.sensors, self.status,
                                                 self.gp_pc, self.gp_acc, self.gp_k)])
        self.n = 0
        rc = self._L.npxo_init(C.byref(self.model), _ptr(b.origin), _ptr(b.quat), _ptr(b.vel),
                             _ptr(b.omega), _ptr(np.ascontiguousarray(b.theta0, np.float32)),
                             C.byref(self.state))
        if rc:
            raise ValueError(f"oracle rejected the scene batch (rc={rc})")

    def step(self, n_steps: int, threads: int | None = None) -> dict:
        cnt = Counts()
        th = self.threads if threads is None else threads
        if th > 1 and not self.counting:
            rc = self._L.npxo_step_mt(C.byref(self.model), C.byref(self.state), n_steps, self.n, th,
                                      C.byref(cnt))
        else:
            rc = self._L.npxo_step(C.byref(self.model), C.byref(self.state), 0, self.batch.n_scenes,
                                   n_steps, self.n, C.byref(cnt))
        if rc:
            raise RuntimeError(f"oracle step failed (rc={rc})")
        self.n += n_steps
        return cnt.as_dict()

    # -- views
    def omega(self) -> np.ndarray:
        """World angular velocity of every scene, from L and the current shape."""
        out = np.zeros((self.batch.n_scenes, 3))
        for s in range(self.batch.n_scenes):
            g, Ib, M = self.mass_props(s)
            R = quat_matrix(self.q[s])
            out[s] = R @ np.linalg.solve(Ib, R.T @ self.L[s])
        return out

    def points_world(self, s: int) -> np.ndarray:
        b = self.batch
        out = np.zeros((int(b.point_off[s + 1] - b.point_off[s]), 3))
        lib().npxo_points_world(C.byref(self.model), C.byref(self.state), s, _ptr(out))
        return out

    def mass_props(self, s: int):
        g = np.zeros(3)
        Ib = np.zeros(9)
        M = np.zeros(1)
        lib().npxo_mass_props(C.byref(self.model), C.byref(self.state), s, _ptr(g), _ptr(Ib),
                              _ptr(M))
        return g, Ib.reshape(3, 3), float(M[0])

    def link_frames(self, s: int):
        b = self.batch
        nl = int(b.link_off[s + 1] - b.link_off[s])
        out = np.zeros((nl, 12))
        lib().npxo_link_frames(C.byref(self.model), C.byref(self.state), s, _ptr(out))
        return out[:, :9].reshape(nl, 3, 3), out[:, 9:]

    def target(self, s: int, j: int, n: int) -> float:
        return lib().npxo_target(C.byref(self.model), s, j, n)

    def lut(self, s: int, x: float, y: float) -> float:
        h = np.zeros(1)
        lib().npxo_lut(C.byref(self.model), s, x, y, _ptr(h))
        return float(h[0])

    def copy_state_from(self, other: "Oracle"):
        for a, b_ in ((self.c, other.c), (self.q, other.q), (self.v, other.v), (self.L, other.L),
                      (self.theta, other.theta), (self.kappa, other.kappa),
                      (self.sensors, other.sensors), (self.status, other.status),
                      (self.gp_pc, other.gp_pc), (self.gp_acc, other.gp_acc), (self.gp_k, other.gp_k)):
            a[...] = b_
        self.n = other.n


def count_ops(batch, n_steps: int, warm_steps: int = 0) -> dict:
    """Floating-point operations of the oracle's step, counted by its counting build: every scene
    of `batch` advanced by warm_steps (not counted), then n_steps counted.  Returns the event
    counts of the counted steps, the operations per region and kind ({region: {kind: n}}), and
    flops = additions, multiplications, divisions, square roots and transcendental calls."""
    o = Oracle(batch, counting=True)
    if warm_steps:
        o.step(warm_steps)
    L = count_lib()
    L.npxo_opcount_reset()
    events = o.step(n_steps)
    raw = np.zeros(len(OP_REGIONS) * len(OP_KINDS), np.uint64)
    L.npxo_opcount_get(raw.ctypes.data)
    raw = raw.reshape(len(OP_REGIONS), len(OP_KINDS))
    ops = {r: {k: int(raw[i, j]) for j, k in enumerate(OP_KINDS)} for i, r in enumerate(OP_REGIONS)}
    flops = sum(ops[r][k] for r in OP_REGIONS for k in FLOP_KINDS)
    return {"events": events, "ops": ops, "flops": flops, "oracle": o}


def quat_matrix(q) -> np.ndarray:
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def time_oracle(batch, n_steps: int, threads: int) -> dict:
    """Wall-clock throughput of the oracle on `batch` for n_steps (CPU baseline)."""
    o = Oracle(batch, threads=threads)
    t0 = time.perf_counter()
    cnt = o.step(n_steps)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "scene_steps": cnt["scene_steps"], "counts": cnt,
            "scene_steps_per_s": cnt["scene_steps"] / dt if dt > 0 else float("nan")}


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
