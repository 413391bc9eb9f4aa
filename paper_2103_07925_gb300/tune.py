"""Autotuner of the cell layout and the launch shape of the interaction sweep.

Two groups of knobs decide how fast a step runs without changing what it computes:

* the cell layout, fixed when a scene is created: cell-key order (Morton or row-major),
  cells per warp group of the neighbour search (row-major only) and the Verlet skin
  (cell edge r_c + skin; neighbour lists rebuilt only when a particle has moved more
  than half the skin);
* the launch shape, changeable at any time: threads per block of the pair sweeps
  (density, extrapolation, force/heat) and resident blocks per SM of the sweeps and of
  the search.

The search is staged: every cell layout is timed on a fresh scene with the default
launch shape, then the launch shape is refined on the winner one knob at a time
(coordinate descent).  Every time is a device measurement (CUDA events around graph
replays, inside libsph) of whole steps after a warm-up; the tuner itself only chooses.
Results are kept per (dimension, precision, size class, bodies yes/no) so that similar
scenes reuse them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

# cells_per_group = -1: row-major keys searched in windows of 32 consecutive particles
LAYOUTS = [dict(key_order=0, cells_per_group=0)] + [dict(key_order=1, cells_per_group=g) for g in (1, 2, 3, -1)]
SKINS_H = (0.0, 0.1, 0.15, 0.2, 0.3, 0.5, 0.7, 1.0)
SWEEP_BLOCKS = (64, 128, 256)
WAVES = (0, 1, 2, 4)

_cache: dict = {}


@dataclass
class Tuned:
    params: dict                      # creation overrides: key_order, cells_per_group, skin
    launch: dict                      # sweep_block, sweep_waves, search_waves
    ms_per_step: float
    table: list = field(default_factory=list)  # (knobs, ms per step) of every trial


def size_class(scene):
    p = scene["params"]
    n = len(scene["particles"]["mass"])
    has_bodies = len(scene["bodies"]["quat"]) > 0
    return (p["dim"], int(p.get("precision", 64)), int(round(math.log2(max(n, 1)))), has_bodies)


def _time(g, steps, warmup):
    g.step(warmup)
    return g.time_steps(steps) / steps


def tune_scene(scene, precision=32, steps=12, warmup=3, skins_h=SKINS_H, layouts=LAYOUTS,
               blocks=SWEEP_BLOCKS, waves=WAVES, use_cache=True):
    """Best cell layout and launch shape for this scene (and scenes of its size class)."""
    from .sph import Scene, SphError
    key = size_class(dict(scene, params=dict(scene["params"], precision=precision)))
    if use_cache and key in _cache:
        return _cache[key]
    h = scene["params"]["h"]
    table = []
    best = None
    for lay in layouts:
        for s in skins_h:
            knobs = dict(lay, skin=s * h)
            try:
                g = Scene(scene, precision=precision, **knobs)
            except SphError:
                continue  # layout not valid for this box (e.g. too few periodic cells)
            try:
                ms = _time(g, steps, warmup)
            finally:
                g.close()
            table.append((dict(knobs), ms))
            if best is None or ms < best[1]:
                best = (knobs, ms)
    params = best[0]
    launch = dict(sweep_block=256, sweep_waves=0, search_waves=0)
    g = Scene(scene, precision=precision, **params)
    try:
        g.step(warmup)
        cur = g.time_steps(steps) / steps
        for knob, values in (("sweep_block", blocks), ("sweep_waves", waves), ("search_waves", waves)):
            start = launch[knob]  # timed already
            for v in values:
                if v == start:
                    continue
                trial = dict(launch, **{knob: v})
                g.set_launch(**trial)
                g.step(1)  # re-capture outside the timed region
                ms = g.time_steps(steps) / steps
                table.append((dict(params, **trial), ms))
                if ms < cur:
                    cur, launch = ms, trial
            g.set_launch(**launch)
    finally:
        g.close()
    res = Tuned(params=params, launch=launch, ms_per_step=cur, table=table)
    if use_cache:
        _cache[key] = res
    return res


def tune_batch(batch, scenes, precision=32, steps=6, warmup=2, **kw):
    """Cell layout per dimension from the largest scene of that dimension, then the launch
    shape of each dimension's engine on the running batch itself (jobs must be admitted
    with no step limit while it runs).  Returns {dim: Tuned}."""
    out = {}
    for dim in (2, 3):
        mine = [sc for sc in scenes if sc["params"]["dim"] == dim]
        if not mine:
            continue
        big = max(mine, key=lambda sc: len(sc["particles"]["mass"]))
        out[dim] = tune_scene(big, precision=precision, **kw)
    if batch is not None:
        batch.step(warmup)
        for dim, t in out.items():
            launch = dict(sweep_block=256, sweep_waves=0, search_waves=0)
            batch.set_launch(dim, **launch)
            batch.step(1)
            cur = batch.time_steps(steps) / steps
            for knob, values in (("sweep_block", SWEEP_BLOCKS), ("sweep_waves", WAVES), ("search_waves", WAVES)):
                start = launch[knob]  # timed already
                for v in values:
                    if v == start:
                        continue
                    trial = dict(launch, **{knob: v})
                    batch.set_launch(dim, **trial)
                    batch.step(1)
                    ms = batch.time_steps(steps) / steps
                    t.table.append((dict(dim=dim, batch=True, **trial), ms))
                    if ms < cur:
                        cur, launch = ms, trial
            batch.set_launch(dim, **launch)
            t.launch = launch
            t.ms_per_step = cur
    return out
