"""The oracle's operation counter (oracle/opcount.h): the counting build of npxo.c must step
exactly like the plain build, and its counts must equal operation counts derived by hand from the
oracle's source.  The benchmark's algorithmic flops per scene-step are this counter's total."""
import ctypes as C

import numpy as np
import pytest

from oracle.oracle import FLOP_KINDS, Oracle, count_lib, count_ops
from paper_2411_05799_gb300 import scenes


def _flops(ops: dict) -> int:
    return sum(ops[k] for k in FLOP_KINDS)


@pytest.mark.parametrize("make,steps", [(lambda: scenes.hexapod_batch(6, seed_key=3), 250),
                                        (lambda: scenes.cpg_batch(3, seed_key=3), 250),
                                        (lambda: scenes.uneven_batch(8, seed_key=3), 170)])
def test_counting_build_steps_bit_identically(make, steps):
    """Same IEEE operations in the same order: the counted run's state equals the plain run's
    bit for bit (joint updates, contacts and friction included)."""
    b = make()
    plain, counted = Oracle(b), Oracle(b, counting=True)
    e1, e2 = plain.step(steps), counted.step(steps)
    assert e1 == e2 and e1["contacts"] > 0 and e1["ticks"] > 0
    for a, c in ((plain.c, counted.c), (plain.q, counted.q), (plain.v, counted.v),
                 (plain.L, counted.L), (plain.theta, counted.theta), (plain.kappa, counted.kappa)):
        np.testing.assert_array_equal(a, c)


def test_counter_matches_a_hand_count_of_the_least_squares():
    """npxo_friction_ls on n points (Eqs. 4-6, centred): the first loop adds 4 per point, four
    divisions make the centroids; the second loop takes 2 subtractions, then S2 += sx sx + sy sy
    and X += sx ey - sy ex (4 multiplications, 4 additions) per point; one comparison and one
    division give a3."""
    L = count_lib()
    for n in (2, 5, 33):
        rng = np.random.default_rng(n)
        s, e = rng.normal(size=(n, 2)), rng.normal(size=(n, 2)) * 0.01
        t, a3 = np.zeros(2), np.zeros(1)
        L.npxo_opcount_reset()
        L.npxo_friction_ls(n, s.ctypes.data, e.ctypes.data, t.ctypes.data, a3.ctypes.data)
        raw = np.zeros(36, np.uint64)
        L.npxo_opcount_get(raw.ctypes.data)
        other = raw.reshape(6, 6)[0]
        assert list(other) == [10 * n, 4 * n, 5, 0, 0, 1], n


def test_per_event_operation_counts():
    """Per-event costs read off the oracle's source, checked against the counter on hexapod steps:
    - every point, every step: its world position c + R r (9 multiplications, 6 + 3 additions);
      on a height map also the cell index (2 subtractions, 2 multiplications, single precision);
    - every point in contact: rho = x - c (3), v_z (2 mul, 2 add), depth (1), the penalty force
      (3 mul, 1 sub), FN (1 add) and two torque terms (2 mul, 2 add): 10 additions, 7 mults;
    - the fixed per-scene work (rotation, angular velocity, integration, exponential map, freeze
      check) is the same for every robot: one hexapod's equals one single body's."""
    r = count_ops(scenes.hexapod_batch(8, seed_key=5), 300, warm_steps=50)
    ev, ops = r["events"], r["ops"]
    assert ops["point"] == {"add": 9 * ev["points"], "mul": 9 * ev["points"], "div": 0, "sqrt": 0,
                            "transc": 0, "cmp": 0}
    assert ev["contacts"] > 0
    assert ops["contact"] == {"add": 10 * ev["contacts"], "mul": 7 * ev["contacts"], "div": 0,
                              "sqrt": 0, "transc": 0, "cmp": ev["contacts"]}
    rough = count_ops(scenes.cpg_batch(2, seed_key=5), 100)
    n = rough["events"]["points"]
    assert _flops(rough["ops"]["point"]) == (18 + 4) * n
    per_scene = {k: v // ev["scene_steps"] for k, v in ops["scene"].items()}
    assert all(v % ev["scene_steps"] == 0 for v in ops["scene"].values())
    one = count_ops(scenes.single_body(), 200)
    assert {k: v // 200 for k, v in one["ops"]["scene"].items()} == per_scene
    assert r["flops"] == sum(_flops(ops[k]) for k in ops)
