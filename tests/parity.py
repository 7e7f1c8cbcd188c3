"""Helpers shared by the GPU parity tests: moving the oracle's FP64 state into the GPU world and
comparing the two.  Imports the oracle (test infrastructure) and the binding; nothing here runs
simulation arithmetic of its own."""
import numpy as np

from oracle.oracle import Oracle

# per-step tolerance: |gpu - oracle| / max(|oracle|, 1) per component
STEP_RTOL = 1e-5
# a point closer than this to the ground decides its contact bit by rounding
NEAR = 1e-5


def to_gpu(world, o: Oracle):
    """Write the oracle's whole dynamic state (rounded to float32) into the GPU world."""
    world.write_state(o.c, o.q, o.v, o.L, o.theta, o.kappa, o.n)


def clone(o: Oracle) -> Oracle:
    c = Oracle(o.batch, threads=o.threads, fric_mode=o.fric_mode, gp_programs=o.gp_prog, arena=o.arena,
               arena_radius=o.arena_radius)
    c.copy_state_from(o)
    return c


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(np.abs(b), 1.0)


def quat_angle(qa, qb):
    """Rotation angle between orientations given as (w, x, y, z) rows (well conditioned for
    small angles: 2 atan2(|a - b|, |a + b|) with b's sign matched to a)."""
    a = np.asarray(qa, np.float64)
    b = np.asarray(qb, np.float64)
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    b = b * np.where(np.sum(a * b, axis=1, keepdims=True) < 0, -1.0, 1.0)
    return 2 * np.arctan2(np.linalg.norm(a - b, axis=1), np.linalg.norm(a + b, axis=1))


def ground_height(b, s, xy):
    if b.heightmaps is None or b.hmap[s] < 0:
        return np.zeros(len(xy))
    maps = b.heightmaps[b.hmap[s]]
    ny, nx = maps.shape
    fx = (xy[:, 0].astype(np.float32) - np.float32(b.hm_origin[0])) * np.float32(b.hm_scale)
    fy = (xy[:, 1].astype(np.float32) - np.float32(b.hm_origin[1])) * np.float32(b.hm_scale)
    ix = np.clip(np.floor(fx).astype(np.int64), 0, nx - 1)
    iy = np.clip(np.floor(fy).astype(np.int64), 0, ny - 1)
    return maps[iy, ix].astype(np.float64)


def near_threshold(o_before: Oracle, o_after: Oracle, theta_new=None) -> np.ndarray:
    """Scenes in which some point lies within NEAR of the ground at the step start, after the
    joint update (theta_new), or after the step: their contact bits are decided by rounding."""
    b = o_before.batch
    near = np.zeros(b.n_scenes, bool)
    probes = [o_before, o_after]
    if theta_new is not None:
        mid = clone(o_before)
        mid.theta[:] = theta_new
        probes.append(mid)
    for s in range(b.n_scenes):
        for o in probes:
            x = o.points_world(s)
            if np.min(np.abs(x[:, 2] - ground_height(b, s, x))) < NEAR:
                near[s] = True
                break
    return near


def per_step_compare(world, o: Oracle, threads=8):
    """One step from the oracle's state on both sides.  Returns (errors dict per scene, near)."""
    to_gpu(world, o)
    o2 = clone(o)
    o2.step(1, threads=threads)
    world.step(1)
    r = world.read()
    near = near_threshold(o, o2, o2.theta)
    err = {
        "cog": rel(r["cog"], o2.c).max(1),
        "quat": np.minimum(rel(r["quat"], o2.q), rel(-r["quat"], o2.q)).max(1),
        "vel": rel(r["vel"], o2.v).max(1),
        "angmom": rel(r["angmom"], o2.L).max(1),
    }
    jo = o.batch.joint_off
    th_err = rel(r["theta"], o2.theta)
    err["theta"] = np.array([th_err[jo[s]:jo[s + 1]].max(initial=0.0) for s in range(o.batch.n_scenes)])
    kap = world.contacts()
    po = o.batch.point_off
    err["contacts"] = np.array([np.count_nonzero(kap[po[s]:po[s + 1]] != o2.kappa[po[s]:po[s + 1]])
                                for s in range(o.batch.n_scenes)], np.float64)
    err["sensors"] = (r["contacts"] != o2.sensors).astype(np.float64)
    return err, near, o2, r
