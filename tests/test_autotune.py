"""Host logic of the schedule autotuner (paper_2211_00705_gb300/autotune.py) with a stand-in for the library
context: the fastest candidate is chosen, candidates whose run leaves an instance with an error status are
skipped, choices are cached per configuration in memory and in a JSON file, and the configuration key follows
the instance sizes, the boundary count and the options. No GPU is involved."""
import dataclasses
import json

import numpy as np

from paper_2211_00705_gb300 import autotune
from paper_2211_00705_gb300 import imexds as imexds_mod
from paper_2211_00705_gb300 import inputs as I


class _Clock:
    t = 0.0


def _fake_imexds(cost, failing=(), created=None):
    """A context class whose runs advance a fake clock by cost[(schedule, threads, cells)] seconds."""

    class Ctx:
        def __init__(self, key):
            self.key = key
            self.n = 1

        @classmethod
        def from_batch(cls, batch, schedule=0, group_threads=0, group_cells=0, **kw):
            key = (schedule, group_threads, group_cells)
            if created is not None:
                created.append(key)
            c = cls(key)
            c.n = batch.n_inst
            return c

        def run_to(self, t_end):
            _Clock.t += cost[self.key]

        def step(self, n):
            _Clock.t += cost[self.key]

        def reset(self):
            pass

        def get_states(self):
            bad = self.key in failing
            return {"status": np.full(self.n, 3 if bad else 0, dtype=np.int32)}

        def close(self):
            pass

    return Ctx


CANDS = [{"schedule": 1}, {"schedule": 2, "group_threads": 128, "group_cells": 16384},
         {"schedule": 2, "group_threads": 96, "group_cells": 16384},
         {"schedule": 3, "group_threads": 128, "group_cells": 8192}]
COST = {(1, 0, 0): 1.4, (2, 128, 16384): 0.95, (2, 96, 16384): 0.94, (3, 128, 8192): 0.5}


def _setup(monkeypatch, failing=(), created=None):
    monkeypatch.setattr(imexds_mod, "Imexds", _fake_imexds(COST, failing, created))
    monkeypatch.setattr(autotune.time, "perf_counter", lambda: _Clock.t)
    monkeypatch.setattr(autotune, "_cache", {})


def test_fastest_candidate_is_chosen_and_failing_ones_are_skipped(monkeypatch):
    _setup(monkeypatch, failing={(3, 128, 8192)})
    b = I.workload(1, scale=8 / 4096)
    choice = autotune.tune(b, candidates=CANDS)
    assert (choice["schedule"], choice["group_threads"], choice["group_cells"]) == (2, 96, 16384)
    assert abs(choice["seconds"] - 0.94) < 1e-12
    timed = {(t["schedule"], t.get("group_threads", 0), t.get("group_cells", 0)) for t in choice["timings"]}
    assert timed == {(1, 0, 0), (2, 128, 16384), (2, 96, 16384)}    # the failing candidate is not listed


def test_choice_is_cached_in_memory_and_in_a_file(monkeypatch, tmp_path):
    created = []
    _setup(monkeypatch, created=created)
    b = I.workload(1, scale=8 / 4096)
    f = tmp_path / "tune.json"
    first = autotune.tune(b, candidates=CANDS, cache_file=str(f))
    assert first["schedule"] == 3 and len(created) == len(CANDS)
    again = autotune.tune(b, candidates=CANDS, cache_file=str(f))
    assert again == first and len(created) == len(CANDS)           # memory cache: no new context
    saved = json.loads(f.read_text())
    assert saved[autotune.config_key(b)]["schedule"] == 3
    monkeypatch.setattr(autotune, "_cache", {})                     # a new process: the file answers
    from_file = autotune.tune(b, candidates=CANDS, cache_file=str(f))
    assert from_file["schedule"] == 3 and len(created) == len(CANDS)


def test_every_candidate_failing_falls_back_to_the_first(monkeypatch):
    _setup(monkeypatch, failing=set(COST))
    b = I.workload(1, scale=8 / 4096)
    choice = autotune.tune(b, candidates=CANDS)
    assert choice["schedule"] == autotune.CANDIDATES[0]["schedule"] and choice["timings"] == []


def test_configuration_key():
    a = I.workload(1, scale=8 / 4096)
    b = I.workload(1, scale=8 / 4096)
    assert autotune.config_key(a) == autotune.config_key(b)
    c = dataclasses.replace(a, options=dataclasses.replace(a.options, block_solver=1))
    assert autotune.config_key(c) != autotune.config_key(a)
    d = I.workload(1, scale=16 / 4096)
    assert autotune.config_key(d) != autotune.config_key(a)
