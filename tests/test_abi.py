"""The C-ABI library: it builds, loads, exports every function include/npx.h declares, and its
host-side construction logic rejects bad input with the documented codes.  Nothing here needs a
GPU: construction is host-only until npx_world_finalize."""
import ctypes as C
import shutil

import numpy as np
import pytest

from paper_2411_05799_gb300 import build as npx_build
from paper_2411_05799_gb300 import npx


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not npx_build.os.path.exists(npx_build.LIB):
        pytest.skip("nvcc not available to build libnpx.so")
    npx_build.build()
    return npx.load()


def test_every_header_function_is_exported(lib):
    names = npx.header_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    missing = set(npx.header_functions()) - set(npx._SIGS) - {"npx_last_error", "npx_mlp_param_count"}
    assert not missing, missing


def _desc(**kw):
    d = npx.WorldDesc(n_scenes=2, dt=1e-3, gravity=(C.c_float * 3)(0, 0, -9.81),
                      joint_update_steps=80, contact_omega=300.0, contact_zeta=1.0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _create(lib, **kw):
    h = C.c_void_p()
    rc = lib.npx_world_create(C.byref(_desc(**kw)), C.byref(h))
    return rc, h


def test_create_validates_description(lib):
    assert lib.npx_world_create(None, None) == npx_build_codes("EINVAL")
    assert _create(lib, n_scenes=0)[0] == -1
    assert _create(lib, dt=0.0)[0] == -1
    assert _create(lib, joint_update_steps=0)[0] == -1
    assert _create(lib, contact_omega=0.0)[0] == -1
    assert _create(lib, hm_count=1)[0] == -1          # maps without data
    assert b"maps" in lib.npx_last_error()
    rc, h = _create(lib)
    assert rc == 0 and h.value
    assert lib.npx_world_destroy(h) == 0
    assert lib.npx_world_destroy(None) == 0


def npx_build_codes(name):
    return {v: k for k, v in npx.ERRORS.items()}[name]


def test_construction_errors_are_host_side(lib):
    rc, h = _create(lib)
    assert rc == 0
    pts = np.zeros((4, 3), np.float32)
    b = C.c_int()
    P = lambda a: a.ctypes.data
    # bad scene index, no points, no mass
    assert lib.npx_body_add_pointcloud(h, 5, P(pts), None, 1.0, 4, C.byref(b)) == -1
    assert lib.npx_body_add_pointcloud(h, 0, P(pts), None, 1.0, 0, C.byref(b)) == -1
    assert lib.npx_body_add_pointcloud(h, 0, P(pts), None, 0.0, 4, C.byref(b)) == -1
    assert lib.npx_body_add_pointcloud(h, 0, P(pts), None, 1.0, 4, C.byref(b)) == 0 and b.value == 0
    assert lib.npx_body_add_pointcloud(h, 0, P(pts), None, 1.0, 4, C.byref(b)) == 0 and b.value == 1
    a = np.zeros(3, np.float32)
    u = np.array([0, 0, 1], np.float32)
    j = C.c_int()
    assert lib.npx_joint_add(h, 0, 0, 7, P(a), P(u), -1.0, 1.0, C.byref(j)) == -1   # no body 7
    assert lib.npx_joint_add(h, 0, 0, 1, P(a), P(u), 1.0, -1.0, C.byref(j)) == -1   # lo > hi
    assert lib.npx_joint_add(h, 0, 0, 1, P(a), P(u), -1.0, 1.0, C.byref(j)) == 0
    assert lib.npx_sensor_add(h, 0, 1, 40) == -6                                 # bit >= 32
    assert lib.npx_scene_set_friction(h, 0, -1.0) == -1
    assert lib.npx_scene_set_heightmap(h, 0, 0) == -1                             # no maps
    # calls that need a finalized world
    assert lib.npx_world_step(h, 1) == -3
    assert lib.npx_state_set(h, None, None, None, None, None) == -3
    # scene 1 undefined: finalize refuses before touching the GPU
    assert lib.npx_world_finalize(h) == -3
    assert b"scene 1" in lib.npx_last_error()
    assert lib.npx_scene_clone(h, 0, 1, 1) == 0
    lib.npx_world_destroy(h)


def test_joint_tree_must_reach_every_link(lib):
    rc, h = _create(lib, n_scenes=1)
    P = lambda a: a.ctypes.data
    pts = np.zeros((2, 3), np.float32)
    for _ in range(3):
        lib.npx_body_add_pointcloud(h, 0, P(pts), None, 1.0, 2, None)
    a = np.zeros(3, np.float32)
    u = np.array([1, 0, 0], np.float32)
    # joints 1->2 and 2->1 leave link 0 detached and close a loop
    lib.npx_joint_add(h, 0, 1, 2, P(a), P(u), -1, 1, None)
    lib.npx_joint_add(h, 0, 2, 1, P(a), P(u), -1, 1, None)
    assert lib.npx_world_finalize(h) == -1
    lib.npx_world_destroy(h)


def test_batched_construction_validates(lib):
    from paper_2411_05799_gb300 import scenes
    b = scenes.hexapod_batch(2)
    rc, h = _create(lib, n_scenes=2)
    keep = [npx._i32(b.link_off), npx._i32(b.point_off), npx._i32(b.parent), npx._f32(b.anchor),
            npx._f32(b.axis), npx._f32(b.lo), npx._f32(b.hi), npx._i32(b.sensor),
            npx._f32(b.p0), npx._f32(b.m), npx._i32(b.plink), npx._f32(b.mu), npx._i32(b.hmap)]
    sb = npx.SceneBatchC(0, 2, *[a.ctypes.data for a in keep])
    assert lib.npx_scenes_add(h, C.byref(sb)) == 0
    bad = keep[2].copy()
    bad[3] = 5                      # a parent index that is not an earlier link
    keep2 = list(keep)
    keep2[2] = bad
    sb2 = npx.SceneBatchC(0, 2, *[a.ctypes.data for a in keep2])
    assert lib.npx_scenes_add(h, C.byref(sb2)) == -1
    sb3 = npx.SceneBatchC(1, 2, *[a.ctypes.data for a in keep])
    assert lib.npx_scenes_add(h, C.byref(sb3)) == -1          # scenes 1..2 exceed n_scenes
    lib.npx_world_destroy(h)


def test_scene_size_limit_is_checked_on_the_host(lib):
    from paper_2411_05799_gb300 import scenes
    b = scenes.ragged_bodies([2049])
    rc, h = _create(lib, n_scenes=1)
    keep = [npx._i32(b.link_off), npx._i32(b.point_off), npx._i32(b.parent), npx._f32(b.anchor),
            npx._f32(b.axis), npx._f32(b.lo), npx._f32(b.hi), npx._i32(b.sensor),
            npx._f32(b.p0), npx._f32(b.m), npx._i32(b.plink), npx._f32(b.mu), npx._i32(b.hmap)]
    sb = npx.SceneBatchC(0, 1, *[a.ctypes.data for a in keep])
    assert lib.npx_scenes_add(h, C.byref(sb)) == npx_build_codes("ERANGE")   # at most 2048 points
    lib.npx_world_destroy(h)
    # the largest scene is accepted
    b = scenes.ragged_bodies([2048])
    rc, h = _create(lib, n_scenes=1)
    keep = [npx._i32(b.link_off), npx._i32(b.point_off), npx._i32(b.parent), npx._f32(b.anchor),
            npx._f32(b.axis), npx._f32(b.lo), npx._f32(b.hi), npx._i32(b.sensor),
            npx._f32(b.p0), npx._f32(b.m), npx._i32(b.plink), npx._f32(b.mu), npx._i32(b.hmap)]
    sb = npx.SceneBatchC(0, 1, *[a.ctypes.data for a in keep])
    assert lib.npx_scenes_add(h, C.byref(sb)) == 0
    lib.npx_world_destroy(h)
