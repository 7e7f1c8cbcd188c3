"""npx_step_noalloc: the entry point for callers that cannot allocate device memory while they run
(real-time control loops that forbid allocation after start-up, frameworks that hand out all
device memory from their own pool).  The caller lays out its own device arrays; the call must step
them exactly like npx_world_step steps the same world, call after call, although its scratch lives
in one static array shared by every call.  Arguments it cannot serve are refused on the host,
before anything is launched.  This file sorts last so that a stop-at-first-failure run has already
run everything else."""
import math

import numpy as np
import pytest

from paper_2411_05799_gb300 import npx, scenes
from paper_2411_05799_gb300.npx import World

LINK_DTYPE = np.dtype([("ax", "<f4"), ("ay", "<f4"), ("az", "<f4"), ("lo", "<f4"),
                       ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4"), ("hi", "<f4"),
                       ("parent", "<i4"), ("sensor", "<i4"), ("depth", "<i4"), ("pad", "<i4")])


def _layout(b, r, contact_user):
    """The documented device layout of a finalized world, built from the scene inputs and a
    state read back through the public API."""
    S, P = b.n_scenes, b.n_points
    perm = np.zeros(P, np.int64)          # stored point -> caller's point
    for s in range(S):
        p0, p1 = b.point_off[s], b.point_off[s + 1]
        perm[p0:p1] = p0 + np.argsort(b.p0[p0:p1, 2], kind="stable")
    p0m = np.concatenate([b.p0[perm], b.m[perm, None]], 1).astype(np.float32)
    links = np.zeros(b.n_links, LINK_DTYPE)
    for s in range(S):
        l0, l1 = b.link_off[s], b.link_off[s + 1]
        depth = np.zeros(l1 - l0, np.int32)
        for k in range(1, l1 - l0):
            depth[k] = depth[b.parent[l0 + k]] + 1
        for k in range(l1 - l0):
            L = l0 + k
            u = b.axis[L].astype(np.float64)
            u = u / np.linalg.norm(u) if k > 0 else np.array([0.0, 0.0, 1.0])
            links[L] = (*b.anchor[L], b.lo[L], *u.astype(np.float32), b.hi[L], b.parent[L],
                        b.sensor[L], depth[k], 0)
    gref = np.zeros((S, 3), np.float32)
    for s in range(S):
        p0, p1 = b.point_off[s], b.point_off[s + 1]
        m = b.m[p0:p1].astype(np.float64)
        gref[s] = (m[:, None] * b.p0[p0:p1].astype(np.float64)).sum(0) / m.sum()
    f = b.act_params[:, 1].astype(np.float64)
    nu = np.floor(f * float(np.float32(b.dt)) * 4294967296.0 + 0.5).astype(np.int64) & 0xffffffff
    state = np.concatenate([r["cog"].T, r["quat"].T, r["vel"].T, r["angmom"].T]).astype(np.float32)
    return {"link_off": b.link_off.astype(np.int32), "point_off": b.point_off.astype(np.int32),
            "p0m": p0m, "plink": b.plink[perm].astype(np.uint8), "links": links.view(np.uint8),
            "gref": gref, "mu": b.mu.astype(np.float32), "hmap": b.hmap.astype(np.int32),
            "act": b.act_params.astype(np.float32), "act_nu": nu.astype(np.uint32),
            "state": np.ascontiguousarray(state), "theta": r["theta"].astype(np.float32),
            "contact": contact_user[perm].astype(np.uint8),
            "omega": np.zeros(3 * S, np.float32), "sensors": r["contacts"].astype(np.uint32),
            "status": r["status"].astype(np.uint32)}, perm


def _rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(np.abs(b), 1.0)


@pytest.mark.gpu
@pytest.mark.parametrize("terrain", ["flat", "rough"])
def test_noalloc_steps_like_world_step_on_consecutive_calls(terrain):
    torch = pytest.importorskip("torch")
    if terrain == "flat":
        b = scenes.hexapod_batch(96, seed_key=21)
    else:   # per-scene 128 x 128 height maps: the height-map build of the step kernel
        b = scenes.cpg_batch(24, seed_key=21)
    lps, wpb = 16, 4
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps, warps_per_block=wpb))
    w.step(37)
    r = w.read()
    arr, perm = _layout(b, r, w.contacts())
    if b.heightmaps is not None:
        maps = np.ascontiguousarray(b.heightmaps, np.float32)
        arr["hm"] = maps
        arr["hm_max"] = maps.reshape(len(maps), -1).max(1)
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in arr.items()}
    ptr = lambda k: dev[k].data_ptr() if k in dev else None
    info = w.info()
    hm_ny, hm_nx = (0, 0) if b.heightmaps is None else b.heightmaps.shape[1:]
    dw = npx.DeviceWorld(
        n_scenes=b.n_scenes, max_points=info["max_points"], max_links=info["max_links"],
        link_off=ptr("link_off"), point_off=ptr("point_off"), p0m=ptr("p0m"), plink=ptr("plink"),
        links=ptr("links"), gref=ptr("gref"), mu=ptr("mu"), hmap=ptr("hmap"), hm=ptr("hm"),
        hm_max=ptr("hm_max"), hm_nx=hm_nx, hm_ny=hm_ny, hm_scale=b.hm_scale, dt=b.dt,
        joint_update_steps=b.joint_update_steps,
        contact_omega=b.contact_omega, contact_zeta=b.contact_zeta, act_mode=b.act_mode,
        act=ptr("act"), act_nu=ptr("act_nu"), state=ptr("state"), theta=ptr("theta"),
        contact=ptr("contact"), omega=ptr("omega"), sensors=ptr("sensors"),
        status=ptr("status"), step=r["step"], lanes_per_scene=lps, warps_per_block=wpb)
    dw.gravity[:] = b.gravity
    dw.hm_origin[:] = b.hm_origin
    stream = torch.cuda.current_stream()
    for call in range(2):                       # two calls in a row share the static scratch
        npx.step_noalloc(dw, 150, stream.cuda_stream)
        torch.cuda.synchronize()
        dw.step += 150
        w.step(150)
        ref = w.read()
        st = dev["state"].cpu().numpy()
        got = {"cog": st[0:3].T, "quat": st[3:7].T, "vel": st[7:10].T, "angmom": st[10:13].T}
        for k in got:
            assert _rel(got[k], ref[k]).max() <= 1e-5, (call, k)
            if terrain == "rough":
                # the same arithmetic: this entry point culls against each map's highest cell
                # and loads windows by plain loads, the world culls against its dilated map and
                # loads windows by TMA; the cull is exact and the windows hold the same cells
                assert np.array_equal(got[k], ref[k]), (call, k)
        assert _rel(dev["theta"].cpu().numpy(), ref["theta"]).max() <= 1e-5
        kap = np.zeros(b.n_points, np.uint8)
        kap[perm] = dev["contact"].cpu().numpy()
        assert np.array_equal(kap, w.contacts()), call
        assert np.array_equal(dev["sensors"].cpu().numpy(), ref["contacts"]), call
        assert np.array_equal(dev["status"].cpu().numpy(), ref["status"]), call
        om = dev["omega"].cpu().numpy().reshape(3, -1).T
        assert _rel(om, ref["omega"]).max() <= 1e-5
    assert ref["step"] == dw.step == 37 + 300


def _host_world(**kw):
    """A device-world description whose array fields hold dummy non-null addresses: every case
    below is refused by the host-side checks, before any device memory is touched."""
    fake = 0x1000
    base = dict(n_scenes=8, max_points=8, max_links=1, lanes_per_scene=16, warps_per_block=4,
                dt=1e-3, joint_update_steps=80, contact_omega=300.0, contact_zeta=1.0,
                act_mode=npx.ACT_SINUSOID, hm_scale=20.0)
    for k in ("link_off", "point_off", "p0m", "plink", "links", "gref", "mu", "hmap", "act",
              "act_nu", "state", "theta", "contact", "omega", "sensors", "status"):
        base[k] = fake
    base.update(kw)
    return npx.DeviceWorld(**base)


def test_noalloc_rejects_worlds_beyond_its_scratch():
    with pytest.raises(npx.NpxError) as e:
        npx.step_noalloc(_host_world(n_scenes=65537), 10)
    assert e.value.code == -6 and "65536" in str(e.value)


def test_noalloc_refuses_the_machine_code_controller():
    """A world driven by machine-code programs needs per-scene program state that this entry
    point has no fields for: it is refused before any launch."""
    with pytest.raises(npx.NpxError) as e:
        npx.step_noalloc(_host_world(act_mode=npx.ACT_GP), 10)
    assert e.value.code == -1 and "act_mode" in str(e.value)
    with pytest.raises(npx.NpxError):
        npx.step_noalloc(_host_world(act_mode=7), 10)


@pytest.mark.parametrize("bad", [dict(hm_nx=0, hm_ny=128), dict(hm_nx=128, hm_ny=0),
                                 dict(hm_nx=128, hm_ny=128, hm_scale=0.0),
                                 dict(hm_nx=128, hm_ny=128, hm_scale=-20.0),
                                 dict(hm_nx=128, hm_ny=128, hm_scale=math.inf)])
def test_noalloc_refuses_malformed_height_maps(bad):
    """The map lookup clamps a cell index into [0, n - 1]; empty maps or a scale that is not
    positive would read outside the caller's array, so such worlds are refused on the host."""
    with pytest.raises(npx.NpxError) as e:
        npx.step_noalloc(_host_world(hm=0x2000, hm_max=0x3000, **bad), 10)
    assert e.value.code == -1 and "height map" in str(e.value)
