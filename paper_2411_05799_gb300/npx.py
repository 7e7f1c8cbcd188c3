"""Thin Python binding of libnpx (include/npx.h): argument marshalling only.

Every step of the simulation runs in the CUDA library; this module converts numpy arrays to the
C-ABI's pointers and back.  There is no CPU fallback: if the compiled library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpx.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
HEADER = os.path.join(INCLUDE, "npx.h")

NPX_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ESTATE", -4: "ECUDA", -5: "ETIMEOUT", -6: "ERANGE"}
ACT_HOLD = 0
ACT_SINUSOID = 1
ACT_GP = 2            # targets from each scene's machine-code program (World.set_gp_programs)
FRIC_WEIGHTED = 1     # friction rows weighted by the normal forces (npx_world_set_friction_model)
FRIC_TILT = 2         # the friction impulse also turns the body about the horizontal axes


class NpxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class WorldDesc(C.Structure):
    _fields_ = [("n_scenes", C.c_int), ("dt", C.c_float), ("gravity", C.c_float * 3),
                ("joint_update_steps", C.c_int), ("contact_omega", C.c_float),
                ("contact_zeta", C.c_float), ("hm_count", C.c_int), ("hm_nx", C.c_int),
                ("hm_ny", C.c_int), ("hm_scale", C.c_float), ("hm_origin", C.c_float * 2),
                ("hm_data", C.c_void_p), ("stream", C.c_void_p), ("device", C.c_int)]


class SceneBatchC(C.Structure):
    _fields_ = [("first", C.c_int), ("count", C.c_int), ("link_off", C.c_void_p),
                ("point_off", C.c_void_p), ("parent", C.c_void_p), ("anchor", C.c_void_p),
                ("axis", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p),
                ("sensor", C.c_void_p), ("p0", C.c_void_p), ("m", C.c_void_p),
                ("plink", C.c_void_p), ("mu", C.c_void_p), ("hmap", C.c_void_p)]


class Sensors(C.Structure):
    _fields_ = [("cog", C.c_void_p), ("quat", C.c_void_p), ("vel", C.c_void_p),
                ("omega", C.c_void_p), ("angmom", C.c_void_p), ("theta", C.c_void_p),
                ("contacts", C.c_void_p), ("status", C.c_void_p), ("step", C.c_void_p)]


class WorldInfo(C.Structure):
    _fields_ = [("n_scenes", C.c_int), ("n_links", C.c_int), ("n_joints", C.c_int),
                ("n_points", C.c_int), ("max_points", C.c_int), ("max_links", C.c_int),
                ("lanes_per_scene", C.c_int), ("warps_per_block", C.c_int), ("blocks", C.c_int),
                ("chunk_steps", C.c_int), ("step", C.c_int64), ("kernel_launches", C.c_int64),
                ("size_classes", C.c_int), ("hm_window_tma", C.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class DeviceWorld(C.Structure):
    """npx_device_world: device pointers to caller-owned arrays for npx_step_noalloc."""
    _fields_ = [("n_scenes", C.c_int), ("max_points", C.c_int), ("max_links", C.c_int),
                ("link_off", C.c_void_p), ("point_off", C.c_void_p), ("p0m", C.c_void_p),
                ("plink", C.c_void_p), ("links", C.c_void_p), ("gref", C.c_void_p),
                ("mu", C.c_void_p), ("hmap", C.c_void_p), ("hm", C.c_void_p),
                ("hm_max", C.c_void_p), ("hm_nx", C.c_int), ("hm_ny", C.c_int),
                ("hm_scale", C.c_float), ("hm_origin", C.c_float * 2), ("dt", C.c_float),
                ("gravity", C.c_float * 3), ("joint_update_steps", C.c_int),
                ("contact_omega", C.c_float), ("contact_zeta", C.c_float), ("act_mode", C.c_int),
                ("act", C.c_void_p), ("act_nu", C.c_void_p), ("state", C.c_void_p),
                ("theta", C.c_void_p), ("contact", C.c_void_p), ("omega", C.c_void_p),
                ("sensors", C.c_void_p), ("status", C.c_void_p), ("step", C.c_int64),
                ("lanes_per_scene", C.c_int), ("warps_per_block", C.c_int)]


def step_noalloc(device_world: DeviceWorld, n_steps: int, stream=None):
    """npx_step_noalloc: step caller-owned device arrays without any allocation."""
    load()
    _check(_lib.npx_step_noalloc(C.byref(device_world), int(n_steps), stream))


EPI_BIAS, EPI_BIAS_GELU, EPI_F32, EPI_DGELU = 0, 1, 2, 3


class GemmEpilogue(C.Structure):
    """npx_gemm_epilogue (include/npx_mlp.h)."""
    _fields_ = [("mode", C.c_int), ("bias", C.c_void_p), ("out", C.c_void_p), ("ldo", C.c_int),
                ("outT", C.c_void_p), ("ldt", C.c_int), ("outf", C.c_void_p), ("ldf", C.c_int),
                ("split_stride", C.c_longlong), ("zsave", C.c_void_p), ("ldz", C.c_int),
                ("zin", C.c_void_p), ("ldzi", C.c_int)]


def gemm_wait_selftest(use_abort: bool, stream=None):
    """The GEMM's bounded barrier wait on a barrier that nothing completes: (gave_up, microseconds)
    after the two-second limit, or after a second warp raises the abort flag (use_abort)."""
    load()
    t, us = C.c_int(), C.c_int()
    _check(_lib.npx_gemm_wait_selftest(1 if use_abort else 0, C.byref(t), C.byref(us),
                                       C.c_void_p(stream or 0)))
    return t.value, us.value


def window_wait_selftest(stream=None):
    """The step kernel's bounded window-copy wait on its own: (lanes that gave up, lanes that saw
    their barrier complete, microseconds), two of its four 8-lane groups waiting on copies that are
    never issued."""
    load()
    up, ok, us = C.c_int(), C.c_int(), C.c_int()
    _check(_lib.npx_window_wait_selftest(C.byref(up), C.byref(ok), C.byref(us), C.c_void_p(stream or 0)))
    return up.value, ok.value, us.value


def gemm_bf16(A, B, M, N, K, epilogue: GemmEpilogue, err, splits=1, stream=None):
    """npx_gemm_bf16: C = A B^T on the tensor cores (device pointers as integers)."""
    load()
    _check(_lib.npx_gemm_bf16(A, B, M, N, K, splits, C.byref(epilogue), err, stream))


P = C.c_void_p
I = C.c_int
F = C.c_float
_SIGS = {
    "npx_world_create": [P, P],
    "npx_world_destroy": [P],
    "npx_body_add_pointcloud": [P, I, P, P, F, I, P],
    "npx_body_connect": [P, I, I, I],
    "npx_joint_add": [P, I, I, I, P, P, F, F, P],
    "npx_sensor_add": [P, I, I, I],
    "npx_scene_set_friction": [P, I, F],
    "npx_scene_set_heightmap": [P, I, I],
    "npx_scene_clone": [P, I, I, I],
    "npx_scenes_add": [P, P],
    "npx_world_finalize": [P],
    "npx_state_set": [P, P, P, P, P, P],
    "npx_actuator_set": [P, I, P],
    "npx_state_write": [P, P, P, P, P, P, P, C.c_int64],
    "npx_contacts_read": [P, P, C.c_size_t],
    "npx_world_step": [P, I],
    "npx_world_sync": [P],
    "npx_sensors_read": [P, P],
    "npx_points_read": [P, I, P, I],
    "npx_state_export": [P, P, P],
    "npx_state_import": [P, P, C.c_size_t],
    "npx_world_info_get": [P, P],
    "npx_world_configure": [P, I, I, I, I],
    "npx_world_autotune": [P, I, P],
    "npx_world_use_graphs": [P, I],
    "npx_step_noalloc": [P, I, P],
    "npx_gemm_bf16": [P, P, I, I, I, I, P, P, P],
    "npx_gemm_wait_selftest": [I, P, P, P],
    "npx_window_wait_selftest": [P, P, P, P],
    "npx_world_set_friction_model": [P, I],
    "npx_world_set_arenas": [P, I, C.c_float],
    "npx_gp_programs_set": [P, P],
    "npx_gp_state_read": [P, P, P, P],
    "npx_gp_state_write": [P, P, P, P],
    "npx_mlp_create": [P, P],
    "npx_mlp_destroy": [P],
    "npx_mlp_params_set": [P, P, C.c_size_t],
    "npx_mlp_params_get": [P, P, C.c_size_t],
    "npx_mlp_grads_get": [P, P, C.c_size_t],
    "npx_mlp_forward": [P, P, P, I],
    "npx_mlp_backward": [P, P, P, I, P],
    "npx_mlp_adam_step": [P],
    "npx_mlp_set_lr": [P, F],
    "npx_surrogate_dims": [P, P, P],
    "npx_surrogate_collect": [P, P, I, I, P, P],
    "npx_world_step_surrogate": [P, P, P, I, I, P],
    "npx_surrogate_fallback_counts": [P, P],
    "npx_surrogate_set_fallback": [P, I],
    "npx_column_moments": [P, C.c_longlong, I, P, P, P],
}

_lib = None


def header_functions() -> list[str]:
    """Names of every function the public headers (include/*.h) declare."""
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            text = open(os.path.join(INCLUDE, h)).read()
            names |= set(re.findall(r"^\s*(?:int|size_t|const char \*)\s*(npx_\w+)\s*\(", text, re.M))
    return sorted(names)


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libnpx.so (build it first with paper_2411_05799_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libnpx.so not built at {path}; run paper_2411_05799_gb300/build.py")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.npx_last_error.argtypes = []
    lib.npx_last_error.restype = C.c_char_p
    lib.npx_mlp_param_count.argtypes = [P]
    lib.npx_mlp_param_count.restype = C.c_size_t
    _lib = lib
    return lib


def _check(rc):
    if rc != NPX_OK:
        raise NpxError(rc, _lib.npx_last_error().decode())
    return rc


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data


class World:
    """A world of independent scenes on one GPU (a handle on npx_world)."""

    def __init__(self, n_scenes, dt=1e-3, gravity=(0.0, 0.0, -9.81), joint_update_steps=80,
                 contact_omega=300.0, contact_zeta=1.0, heightmaps=None, hm_scale=10.0,
                 hm_origin=(0.0, 0.0), stream=None, device=0):
        lib = load()
        self._h = P()
        maps = None if heightmaps is None else _f32(heightmaps)
        d = WorldDesc(n_scenes=n_scenes, dt=dt, gravity=(F * 3)(*gravity),
                      joint_update_steps=joint_update_steps, contact_omega=contact_omega,
                      contact_zeta=contact_zeta,
                      hm_count=0 if maps is None else maps.shape[0],
                      hm_nx=0 if maps is None else maps.shape[2],
                      hm_ny=0 if maps is None else maps.shape[1], hm_scale=hm_scale,
                      hm_origin=(F * 2)(*hm_origin), hm_data=_p(maps), stream=stream,
                      device=device)
        _check(lib.npx_world_create(C.byref(d), C.byref(self._h)))
        self.n_scenes = n_scenes
        self.dt = float(np.float32(dt))
        self._info = None

    @classmethod
    def from_batch(cls, batch, stream=None, device=0, configure=None) -> "World":
        """World built from a SceneBatch: bulk construction, finalize, initial state, actuators."""
        b = batch
        w = cls(b.n_scenes, dt=b.dt, gravity=b.gravity, joint_update_steps=b.joint_update_steps,
                contact_omega=b.contact_omega, contact_zeta=b.contact_zeta,
                heightmaps=b.heightmaps, hm_scale=b.hm_scale, hm_origin=b.hm_origin,
                stream=stream, device=device)
        w.add_scenes(b)
        w.finalize()
        if configure:
            w.configure(**configure)
        w.set_state(b.origin, b.quat, b.vel, b.omega, b.theta0)
        w.set_actuators(b.act_mode, b.act_params)
        return w

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.npx_world_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- construction
    def add_scenes(self, b, first=0):
        keep = [_i32(b.link_off), _i32(b.point_off), _i32(b.parent), _f32(b.anchor),
                _f32(b.axis), _f32(b.lo), _f32(b.hi), _i32(b.sensor), _f32(b.p0), _f32(b.m),
                _i32(b.plink), _f32(b.mu), _i32(b.hmap)]
        sb = SceneBatchC(first, b.n_scenes, *[_p(a) for a in keep])
        _check(_lib.npx_scenes_add(self._h, C.byref(sb)))

    def add_body(self, scene, xyz, mass=None, total_mass=1.0) -> int:
        xyz = _f32(xyz).reshape(-1, 3)
        m = None if mass is None else _f32(mass)
        out = C.c_int()
        _check(_lib.npx_body_add_pointcloud(self._h, scene, _p(xyz), _p(m), total_mass,
                                            len(xyz), C.byref(out)))
        return out.value

    def connect(self, scene, b1, b2):
        _check(_lib.npx_body_connect(self._h, scene, b1, b2))

    def add_joint(self, scene, b1, b2, anchor, axis, lo, hi) -> int:
        a, u = _f32(anchor), _f32(axis)
        out = C.c_int()
        _check(_lib.npx_joint_add(self._h, scene, b1, b2, _p(a), _p(u), lo, hi, C.byref(out)))
        return out.value

    def add_sensor(self, scene, body, bit):
        _check(_lib.npx_sensor_add(self._h, scene, body, bit))

    def set_friction(self, scene, mu):
        _check(_lib.npx_scene_set_friction(self._h, scene, mu))

    def set_heightmap(self, scene, hm):
        _check(_lib.npx_scene_set_heightmap(self._h, scene, hm))

    def clone(self, src, first, count):
        _check(_lib.npx_scene_clone(self._h, src, first, count))

    def finalize(self):
        _check(_lib.npx_world_finalize(self._h))
        self._info = self.info()

    # -- state
    def set_state(self, origin, quat, vel, omega, theta=None):
        S = self.n_scenes
        o, q, v, w = (_f32(origin).reshape(S, 3), _f32(quat).reshape(S, 4),
                      _f32(vel).reshape(S, 3), _f32(omega).reshape(S, 3))
        th = None if theta is None else _f32(theta)
        _check(_lib.npx_state_set(self._h, _p(o), _p(q), _p(v), _p(w), _p(th)))

    def write_state(self, cog, quat, vel, angmom, theta=None, contact_prev=None, step=0):
        S = self.n_scenes
        c, q, v, L = (_f32(cog).reshape(S, 3), _f32(quat).reshape(S, 4),
                      _f32(vel).reshape(S, 3), _f32(angmom).reshape(S, 3))
        th = None if theta is None else _f32(theta)
        k = None if contact_prev is None else np.ascontiguousarray(contact_prev, np.uint8)
        _check(_lib.npx_state_write(self._h, _p(c), _p(q), _p(v), _p(L), _p(th), _p(k),
                                    int(step)))

    def contacts(self, out: np.ndarray | None = None) -> np.ndarray:
        """Per-point contact flags of the last step, in the caller's point order (npx_contacts_read),
        into a new array or into out (uint8, n_points)."""
        if out is None:
            out = np.zeros(self._info["n_points"], np.uint8)
        _check(_lib.npx_contacts_read(self._h, _p(out), out.size))
        return out

    def set_gp_programs(self, programs):
        """One 32-byte machine-code program per scene (uint8 [S, 32]); resets the controllers."""
        p = np.ascontiguousarray(programs, np.uint8)
        if p.shape != (self.n_scenes, 32):
            raise ValueError(f"programs must be uint8 [{self.n_scenes}, 32]")
        _check(_lib.npx_gp_programs_set(self._h, p.ctypes.data))

    def gp_state(self) -> dict:
        """Controller state: program counters and accumulators [S], joint targets in 5-degree
        steps [J]."""
        info = self.info()
        pc = np.zeros(self.n_scenes, np.uint8)
        acc = np.zeros(self.n_scenes, np.uint8)
        k = np.zeros(max(info["n_joints"], 1), np.int8)
        _check(_lib.npx_gp_state_read(self._h, pc.ctypes.data, acc.ctypes.data, k.ctypes.data))
        return {"pc": pc, "acc": acc, "k": k[:info["n_joints"]]}

    def write_gp_state(self, pc, acc, k):
        pc = np.ascontiguousarray(pc, np.uint8)
        acc = np.ascontiguousarray(acc, np.uint8)
        k = np.ascontiguousarray(k, np.int8)
        _check(_lib.npx_gp_state_write(self._h, pc.ctypes.data, acc.ctypes.data, k.ctypes.data))

    def set_friction_model(self, flags: int):
        """FRIC_WEIGHTED | FRIC_TILT (0: Eqs. 1-6 as written)."""
        _check(_lib.npx_world_set_friction_model(self._h, int(flags)))

    def set_arenas(self, size: int, radius: float = 0.01):
        """Robot-robot collision within arenas of `size` consecutive scenes (1 = off, 2 or 4);
        every mass point is a sphere of `radius` metres."""
        _check(_lib.npx_world_set_arenas(self._h, int(size), float(radius)))

    def set_actuators(self, mode, params=None):
        p = None if params is None else _f32(params)
        _check(_lib.npx_actuator_set(self._h, mode, _p(p)))

    def step(self, n: int):
        _check(_lib.npx_world_step(self._h, int(n)))

    def sync(self):
        _check(_lib.npx_world_sync(self._h))

    def read_buffers(self) -> dict:
        """Arrays for read(out=...): allocate them once (pinned memory makes the copies DMA)."""
        S, J = self.n_scenes, self._info["n_joints"]
        return {"cog": np.zeros((S, 3), np.float32), "quat": np.zeros((S, 4), np.float32),
                "vel": np.zeros((S, 3), np.float32), "omega": np.zeros((S, 3), np.float32),
                "angmom": np.zeros((S, 3), np.float32), "theta": np.zeros(J, np.float32),
                "contacts": np.zeros(S, np.uint32), "status": np.zeros(S, np.uint32),
                "step": np.zeros(1, np.int64)}

    def read(self, out: dict | None = None) -> dict:
        """State and sensors (npx_sensors_read) into new arrays, or into out's arrays (same
        shapes and dtypes as read_buffers(); returned with "step" as an int)."""
        if out is None:
            out = self.read_buffers()
        else:
            out = dict(out)
            if not isinstance(out.get("step"), np.ndarray):
                out["step"] = np.zeros(1, np.int64)
        s = Sensors(*[_p(out[k]) for k in ("cog", "quat", "vel", "omega", "angmom", "theta",
                                           "contacts", "status", "step")])
        _check(_lib.npx_sensors_read(self._h, C.byref(s)))
        out["step"] = int(out["step"][0])
        return out

    def points(self, scene: int) -> np.ndarray:
        n = self._info["max_points"]
        buf = np.zeros((n, 3), np.float32)
        _check(_lib.npx_points_read(self._h, scene, _p(buf), n))
        return buf

    def export_state(self) -> bytes:
        size = C.c_size_t()
        _check(_lib.npx_state_export(self._h, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        _check(_lib.npx_state_export(self._h, buf, C.byref(size)))
        return buf.raw[:size.value]

    def import_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(_lib.npx_state_import(self._h, buf, len(blob)))

    # -- tuning
    def info(self) -> dict:
        i = WorldInfo()
        _check(_lib.npx_world_info_get(self._h, C.byref(i)))
        return i.as_dict()

    def configure(self, lanes_per_scene=0, warps_per_block=0, blocks=0, chunk_steps=0):
        _check(_lib.npx_world_configure(self._h, lanes_per_scene, warps_per_block, blocks,
                                        chunk_steps))
        self._info = self.info()

    def autotune(self, n_steps=200) -> dict:
        i = WorldInfo()
        _check(_lib.npx_world_autotune(self._h, n_steps, C.byref(i)))
        self._info = i.as_dict()
        return self._info

    def use_graphs(self, on: bool):
        _check(_lib.npx_world_use_graphs(self._h, 1 if on else 0))


class MLPDesc(C.Structure):
    _fields_ = [("n_in", C.c_int), ("n_hidden", C.c_int), ("n_hidden_layers", C.c_int),
                ("n_out", C.c_int), ("max_batch", C.c_int), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("seed", C.c_ulonglong), ("stream", C.c_void_p)]


class MLP:
    """The surrogate network (npx_mlp): tensor-core forward, backward and Adam.  Arrays passed
    to forward/backward are device pointers (integers, e.g. torch tensors' data_ptr())."""

    def __init__(self, n_in, n_out, n_hidden=512, n_hidden_layers=4, max_batch=8192, lr=1e-3,
                 beta1=0.9, beta2=0.999, eps=1e-8, seed=0, stream=None):
        lib = load()
        self._h = P()
        d = MLPDesc(n_in, n_hidden, n_hidden_layers, n_out, max_batch, lr, beta1, beta2, eps,
                    seed, stream)
        _check(lib.npx_mlp_create(C.byref(d), C.byref(self._h)))
        self.n_in, self.n_out = n_in, n_out
        self.sizes = [n_in] + [n_hidden] * n_hidden_layers + [n_out]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.npx_mlp_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_params(self) -> int:
        return int(_lib.npx_mlp_param_count(self._h))

    def set_params(self, Ws, bs):
        flat = np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(),
                                               np.asarray(b, np.float32).ravel()])
                               for W, b in zip(Ws, bs)]).astype(np.float32)
        _check(_lib.npx_mlp_params_set(self._h, _p(flat), flat.size))

    def _unflat(self, flat):
        Ws, bs, off = [], [], 0
        for fi, fo in zip(self.sizes[:-1], self.sizes[1:]):
            Ws.append(flat[off:off + fi * fo].reshape(fo, fi)); off += fi * fo
            bs.append(flat[off:off + fo]); off += fo
        return Ws, bs

    def get_params(self):
        flat = np.zeros(self.n_params, np.float32)
        _check(_lib.npx_mlp_params_get(self._h, _p(flat), flat.size))
        return self._unflat(flat)

    def get_grads(self):
        flat = np.zeros(self.n_params, np.float32)
        _check(_lib.npx_mlp_grads_get(self._h, _p(flat), flat.size))
        return self._unflat(flat)

    def forward(self, x_ptr, y_ptr, M):
        _check(_lib.npx_mlp_forward(self._h, x_ptr, y_ptr, M))

    def backward(self, x_ptr, t_ptr, M, loss_ptr):
        _check(_lib.npx_mlp_backward(self._h, x_ptr, t_ptr, M, loss_ptr))

    def adam_step(self):
        _check(_lib.npx_mlp_adam_step(self._h))

    def set_lr(self, lr: float):
        _check(_lib.npx_mlp_set_lr(self._h, float(lr)))


class SurrogateNorm(C.Structure):
    """npx_surrogate_norm: device pointers to the standardisation vectors."""
    _fields_ = [("x_mu", C.c_void_p), ("x_isd", C.c_void_p), ("t_mu", C.c_void_p),
                ("t_sd", C.c_void_p)]


def surrogate_dims(world: "World"):
    nf, nt = C.c_int(), C.c_int()
    _check(_lib.npx_surrogate_dims(world._h, C.byref(nf), C.byref(nt)))
    return nf.value, nt.value


def surrogate_collect(world: "World", n_windows, X_ptr, T_ptr, norm: SurrogateNorm = None, stride: int = 1):
    _check(_lib.npx_surrogate_collect(world._h, C.byref(norm) if norm else None, int(stride),
                                      int(n_windows), X_ptr, T_ptr))


def world_step_surrogate(world: "World", net: "MLP", norm: SurrogateNorm, n_steps, stride: int = 1) -> int:
    fb = C.c_longlong()
    _check(_lib.npx_world_step_surrogate(world._h, net._h, C.byref(norm), int(stride), int(n_steps),
                                         C.byref(fb)))
    return fb.value


def surrogate_fallback_counts(world: "World") -> np.ndarray:
    """npx_surrogate_fallback_counts: windows of each scene that fell back since the last call."""
    out = np.zeros(world.n_scenes, np.int32)
    _check(_lib.npx_surrogate_fallback_counts(world._h, _p(out)))
    return out


def surrogate_set_fallback(world: "World", max_changed_bits: int) -> None:
    """npx_surrogate_set_fallback: a surrogate window falls back when more than max_changed_bits
    contact sensors change over it (0: any change, the default; -1: never)."""
    _check(_lib.npx_surrogate_set_fallback(world._h, max_changed_bits))


def column_moments(X_ptr, rows: int, cols: int, sum_ptr, sumsq_ptr, stream=None):
    """npx_column_moments: adds the FP64 column sums and sums of squares of X [rows x cols] (device
    FP32) to sum / sumsq (device FP64 [cols])."""
    load()
    _check(_lib.npx_column_moments(X_ptr, int(rows), int(cols), sum_ptr, sumsq_ptr, stream))
