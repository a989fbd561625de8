"""Autotuner for batched applies: picks the group's stream count and the mixed
kernels' right-hand-side blocking by timing candidates, and caches the choice.

Cache: a JSON file (``$IFGF_TUNE_CACHE`` or ``~/.cache/ifgf_gb300/tune.json``)
keyed by device name, precision, total-point bucket (power of two) and the
number of right-hand sides per plan.  The timer is pluggable so the selection
and cache logic run without a GPU.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from dataclasses import dataclass

DEFAULT_CANDIDATES = [{"nstreams": s, "rhs_block": rb} for s, rb in itertools.product((1, 2, 4, 8), (1, 4))]


def cache_path() -> str:
    return os.environ.get("IFGF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ifgf_gb300", "tune.json"))


def tune_key(device: str, precision: str, total_points: int, nrhs: int) -> str:
    bucket = 1 << max(0, int(math.ceil(math.log2(max(total_points, 1)))))
    return f"{device}|{precision}|N<={bucket}|nrhs={nrhs}"


@dataclass
class TuneResult:
    config: dict
    ms: float
    table: list
    cached: bool


class Autotuner:
    def __init__(self, path: str | None = None):
        self.path = path or cache_path()
        self._db = None

    def _load(self) -> dict:
        if self._db is None:
            try:
                with open(self.path) as f:
                    self._db = json.load(f)
            except (OSError, ValueError):
                self._db = {}
        return self._db

    def _save(self):
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self._db, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def lookup(self, key: str):
        return self._load().get(key)

    def tune(self, key: str, run, candidates=None, reps: int = 3, force: bool = False) -> TuneResult:
        """run(config) -> milliseconds of one timed apply with that config (median of reps taken here)."""
        db = self._load()
        if not force and key in db:
            e = db[key]
            return TuneResult(e["config"], e["ms"], e.get("table", []), True)
        table = []
        for cfg in candidates or DEFAULT_CANDIDATES:
            ts = sorted(run(cfg) for _ in range(reps))
            table.append((cfg, ts[len(ts) // 2]))
        best, ms = min(table, key=lambda t: t[1])
        db[key] = {"config": best, "ms": ms, "table": [[c, t] for c, t in table]}
        self._save()
        return TuneResult(best, ms, table, False)


def gpu_timer(group, plans, sigmas, outs, warmup: int = 1):
    """Timer for Autotuner.tune: applies `config` to the group and its plans and
    returns the CUDA-event time of one group apply (after `warmup` untimed ones)."""
    import torch

    def run(cfg):
        group.set_streams(cfg["nstreams"])
        for p in plans:
            p.set_rhs_block(cfg["rhs_block"])
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            group.apply(sigmas, outs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        group.apply(sigmas, outs)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    return run
