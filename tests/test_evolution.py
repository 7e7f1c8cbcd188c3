"""Host logic of the controller evolution (Sec. IV): mutation and selection, no GPU."""
import numpy as np

from paper_2411_05799_gb300.evolution import PROG_LEN, mutate, select


def test_mutation_changes_every_copy_and_about_one_byte():
    rng = np.random.default_rng(0)
    parents = rng.integers(0, 256, (5000, PROG_LEN), dtype=np.uint8)
    kids = mutate(rng, parents)
    changed = (kids != parents).sum(axis=1)
    assert (changed >= 1).all()             # at least one byte replaced by another
    assert 1.0 <= changed.mean() <= 2.2     # about one in 32 otherwise
    assert parents.dtype == kids.dtype == np.uint8


def test_selection_keeps_the_best_half_unchanged_and_mutates_a_copy():
    rng = np.random.default_rng(1)
    progs = rng.integers(0, 256, (10, PROG_LEN), dtype=np.uint8)
    fit = np.array([0.3, 2.0, 0.1, 2.0, 5.0, 0.0, 1.0, 0.7, 3.0, 0.2])
    nxt = select(rng, progs, fit, 5)
    best = [4, 8, 1, 3, 6]                  # by fitness, ties by index
    np.testing.assert_array_equal(nxt[:5], progs[best])
    assert ((nxt[5:] != progs[best]).sum(axis=1) >= 1).all()
    assert nxt.shape == progs.shape
