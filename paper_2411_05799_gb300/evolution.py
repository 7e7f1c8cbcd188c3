"""Evolution of machine-code controllers (Sec. IV): many independent populations evaluated at once.

The paper evolves one population of 100 hexapods whose 32-byte machine-code programs (Table I)
drive the joints, with mutation as the only variation operator: every generation each robot walks
for two minutes, the best 50 of 100 are kept, duplicated and mutated.  Here a world holds
n_groups such populations side by side (one scene per individual, all starting from the same
rest state); one `npx_world_step` evaluates every individual of every population, and the
selection of each population is a few numpy lines on the host.

Readings where the text is silent: the fitness is the horizontal distance of the robot's CoG from
its start after the evaluation (a frozen scene scores 0); of the best half, one copy survives
unchanged and the other is mutated, every byte replaced by another random byte with probability
1/32 and at least one byte replaced.
"""
from __future__ import annotations

import time

import numpy as np

from . import npx, scenes

PROG_LEN = 32


def mutate(rng: np.random.Generator, parents: np.ndarray, rate: float = 1.0 / PROG_LEN) -> np.ndarray:
    """Copies of the parents with every byte replaced by another byte (uniform over the 255 others)
    with probability `rate`, at least one byte per copy."""
    kids = parents.copy()
    hit = rng.random(kids.shape) < rate
    none = ~hit.any(axis=1)
    hit[np.flatnonzero(none), rng.integers(0, PROG_LEN, int(none.sum()))] = True
    shift = rng.integers(1, 256, int(hit.sum()))
    kids[hit] = ((kids[hit].astype(np.int64) + shift) % 256).astype(np.uint8)
    return kids


def select(rng: np.random.Generator, programs: np.ndarray, fitness: np.ndarray, keep: int) -> np.ndarray:
    """One population's next generation: the best `keep` programs unchanged, then a mutated copy
    of each (ties broken by index, so the selection is deterministic)."""
    order = np.lexsort((np.arange(len(fitness)), -fitness))
    parents = programs[order[:keep]]
    return np.concatenate([parents, mutate(rng, parents)])


def evolve(n_groups: int = 1, pop: int = 100, keep: int = 50, generations: int = 10,
           eval_seconds: float = 120.0, seed: int = 0, world: "npx.World | None" = None,
           batch: "scenes.SceneBatch | None" = None, stream=None, log=None) -> dict:
    """Evolve n_groups independent populations of `pop` machine-code controllers of the 18-DoF
    hexapod on flat ground (or `batch`, n_groups * pop scenes of equal robots).

    Returns the final programs [n_groups * pop, 32], the best fitness of every population in every
    generation [generations, n_groups], the last generation's fitness, and the GPU time spent
    stepping (seconds) with the scene-steps it simulated."""
    if keep * 2 != pop:
        raise ValueError("the next generation is the best half and a mutated copy of it: pop = 2 keep")
    S = n_groups * pop
    rng = np.random.default_rng(seed)
    if world is None:
        if batch is None:
            batch = scenes.hexapod_batch(S, seed_key=seed)
        world = npx.World.from_batch(batch, stream=stream)
        world.autotune(200)     # the launch shape for this many scenes (the state is kept)
    if world.n_scenes != S:
        raise ValueError(f"the world must hold n_groups * pop = {S} scenes")
    n_steps = int(round(eval_seconds / world.dt))
    start = world.export_state()
    c0 = world.read()["cog"][:, :2].copy()
    programs = rng.integers(0, 256, (S, PROG_LEN), dtype=np.uint8)
    best = np.zeros((generations, n_groups))
    step_s = 0.0
    fit = np.zeros(S)
    for g in range(generations):
        world.import_state(start)
        world.set_gp_programs(programs)
        t0 = time.perf_counter()
        world.step(n_steps)
        world.sync()
        step_s += time.perf_counter() - t0
        r = world.read()
        fit = np.linalg.norm(r["cog"][:, :2] - c0, axis=1)
        fit[(r["status"] != 0) | ~np.isfinite(fit)] = 0.0
        groups = fit.reshape(n_groups, pop)
        best[g] = groups.max(axis=1)
        if log:
            log(f"generation {g}: best {best[g].max():.3f} m, median of the populations' best {np.median(best[g]):.3f} m")
        if g + 1 < generations:
            programs = np.concatenate([select(rng, programs[i * pop:(i + 1) * pop], groups[i], keep)
                                       for i in range(n_groups)])
    return {"programs": programs, "best_fitness": best, "fitness": fit, "step_seconds": step_s,
            "scene_steps": float(S) * n_steps * generations, "world": world}
