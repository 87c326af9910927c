"""Schedule autotuner for imexds contexts.

Candidates: the per-step kernel schedule (one launch per kernel and step, replayed from a CUDA graph),
the lockstep instance-group schedule (one resident launch per call) at several group sizes and CTA widths
(the number of sweep warps beside the warp that solves the blocks), and the independent instance groups
(each instance of a group at its own pace, tiles dealt to whichever instance is open).
Each candidate gets a context of its own loaded with the batch; one untimed run (graph build, caches) is
followed by imexds_reset and a timed run, host clock around the call, which returns when the device is
done: the whole run_to for a batch with an end time (the early steps of a run are not representative of
its cost), else `steps` steps. A candidate whose run leaves an instance with an error status is skipped.
The fastest is kept. Choices are cached per configuration (instance sizes, boundary counts, options) in
memory and, optionally, in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

CANDIDATES = [
    {"schedule": 1},
    {"schedule": 2, "group_threads": 128, "group_cells": 16384},
    {"schedule": 2, "group_threads": 256, "group_cells": 16384},
    {"schedule": 2, "group_threads": 256, "group_cells": 24576},
    {"schedule": 2, "group_threads": 256, "group_cells": 8192},
    {"schedule": 2, "group_threads": 192, "group_cells": 16384},
    {"schedule": 2, "group_threads": 128, "group_cells": 8192},
    {"schedule": 2, "group_threads": 96, "group_cells": 16384},
    {"schedule": 2, "group_threads": 64, "group_cells": 4096},
    {"schedule": 3, "group_threads": 128, "group_cells": 16384},
    {"schedule": 3, "group_threads": 128, "group_cells": 8192},
]

_cache: dict = {}


def config_key(batch) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(batch.n_lattice).tobytes())
    flips = np.diff(batch.phase.astype(np.int16)) != 0
    h.update(np.int64(flips.sum()).tobytes())
    h.update(json.dumps(batch.options.__dict__, sort_keys=True).encode())
    return h.hexdigest()[:16]


def tune(batch, steps: int = 64, cache_file: str | None = None, candidates=None) -> dict:
    """Return the fastest candidate for this batch (and remember it). A batch with an end time is timed over
    a whole run_to (the early steps of a run are not representative of its cost); otherwise over `steps`
    steps. The returned dict carries every candidate's time under "timings"."""
    from .imexds import Imexds
    key = config_key(batch)
    if cache_file and os.path.exists(cache_file):
        try:
            with open(cache_file) as f:
                _cache.update(json.load(f))
        except (OSError, ValueError):
            pass
    if key in _cache:
        return _cache[key]
    best, best_t = None, float("inf")
    timings = []
    for cand in candidates or CANDIDATES:
        ctx = Imexds.from_batch(batch, schedule=cand["schedule"], group_threads=cand.get("group_threads", 0),
                                group_cells=cand.get("group_cells", 0))
        run = (lambda: ctx.run_to(batch.t_end)) if batch.t_end > 0 else (lambda: ctx.step(steps))
        run()                            # warm-up (graph build, caches)
        ctx.reset()
        ctx.get_states()                 # synchronises
        t0 = time.perf_counter()
        run()
        st = ctx.get_states()            # synchronises
        dt = time.perf_counter() - t0
        ctx.close()
        if (st["status"] != 0).any():
            continue
        timings.append({**cand, "seconds": dt})
        if dt < best_t:
            best, best_t = cand, dt
    if best is None:
        best = CANDIDATES[0]
    choice = dict(best)
    choice["seconds"] = best_t
    choice["timings"] = timings
    _cache[key] = choice
    if cache_file:
        try:
            with open(cache_file, "w") as f:
                json.dump(_cache, f, indent=1)
        except OSError:
            pass
    return choice
