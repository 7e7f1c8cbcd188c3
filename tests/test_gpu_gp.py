"""The machine-code controller (Sec. IV, Table I) on the GPU against the oracle's: from the
oracle's state at joint updates, the controller state after the update is exact (integer logic on
the same foot bits) and the joint angles and body state agree per step; the state blob carries
the controller state."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2411_05799_gb300 import scenes
from paper_2411_05799_gb300.npx import World
from tests.parity import STEP_RTOL, clone, near_threshold, rel, to_gpu

pytestmark = pytest.mark.gpu

THREADS = 8


def random_programs(n, seed):
    """Uniformly random programs (every byte an opcode)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (n, 32), dtype=np.uint8)


def _to_gpu_with_controller(w, o):
    to_gpu(w, o)
    w.write_gp_state(o.gp_pc, o.gp_acc, o.gp_k)


@pytest.mark.parametrize("lps, terrain", [(8, "flat"), (32, "flat"), (16, "rough")])
def test_controller_per_joint_update(lps, terrain):
    """Flat ground, and hexapods on per-scene rough height maps (the height-map build of the step
    kernel runs the same controller)."""
    b = scenes.hexapod_batch(128, seed_key=21) if terrain == "flat" else scenes.cpg_batch(64, seed_key=23)
    progs = random_programs(b.n_scenes, 5)
    o = Oracle(b, threads=THREADS, gp_programs=progs)
    w = World.from_batch(b, configure=dict(lanes_per_scene=lps))
    w.set_gp_programs(progs)
    jo = b.joint_off
    K = b.joint_update_steps
    moved = 0
    for n in [0, K, 2 * K, 10 * K, 20 * K, 20 * K + 1, 40 * K]:
        o.step(n - o.n, threads=THREADS)
        _to_gpu_with_controller(w, o)
        o2 = clone(o)
        o2.step(1, threads=THREADS)
        w.step(1)
        g = w.gp_state()
        np.testing.assert_array_equal(g["pc"], o2.gp_pc)
        np.testing.assert_array_equal(g["acc"], o2.gp_acc)
        np.testing.assert_array_equal(g["k"], o2.gp_k)
        moved += int(np.count_nonzero(o2.gp_k != o.gp_k))
        r = w.read()
        near = near_threshold(o, o2, o2.theta)
        ok = ~near
        assert rel(r["theta"], o2.theta).max() <= STEP_RTOL
        for k, ref in (("cog", o2.c), ("vel", o2.v), ("angmom", o2.L)):
            assert rel(r[k], ref).max(1)[ok].max(initial=0.0) <= STEP_RTOL, (n, k)
    assert moved > 50 * b.n_scenes // 64     # the programs did move motors


def test_controller_state_in_the_blob():
    b = scenes.hexapod_batch(64, seed_key=22)
    w = World.from_batch(b)
    w.set_gp_programs(random_programs(64, 6))
    w.step(400)
    blob = w.export_state()
    w.step(800)
    a = w.read(), w.gp_state()
    w.import_state(blob)
    w.step(800)
    bb = w.read(), w.gp_state()
    for key in ("cog", "quat", "vel", "angmom", "theta"):
        np.testing.assert_array_equal(a[0][key], bb[0][key])
    for key in ("pc", "acc", "k"):
        np.testing.assert_array_equal(a[1][key], bb[1][key])


def test_evolution_keeps_its_best():
    """Two populations of 20 controllers, 5-second evaluations, 4 generations: the survivors'
    programs replay bit-identical trajectories wherever they sit in the world, so each
    population's best fitness never falls; the best half of the last generation is the parents'
    best half carried over unchanged."""
    from paper_2411_05799_gb300.evolution import evolve
    res = evolve(n_groups=2, pop=20, keep=10, generations=4, eval_seconds=5.0, seed=3)
    best = res["best_fitness"]
    assert best.shape == (4, 2)
    assert (np.diff(best, axis=0) >= 0).all(), best
    assert (best[-1] > 0).all()
    assert np.isfinite(res["fitness"]).all()
