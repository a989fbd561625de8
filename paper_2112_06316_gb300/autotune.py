"""Autotuner: picks launch settings by timing candidates, and caches the choice.

* Batched applies (``gpu_timer``): the group's stream count and the mixed kernels'
  right-hand-side blocking.
* One plan's apply (``plan_timer`` / ``tune_plan``): the kernel choices of the mixed
  path -- the tile-fill threshold above which a propagation level runs on the tensor
  cores, the tensor-core engine (tcgen05 over the angular contraction, tcgen05 per pair,
  or mma.sync), the CUDA-core interpolation engine (cone-stationary or
  point-stationary) and the right-hand-side blocking.  Every candidate computes the
  same operator (each engine is parity-tested); only the time differs.

Cache: a JSON file (``$IFGF_TUNE_CACHE`` or ``~/.cache/ifgf_gb300/tune.json``)
keyed by device name, precision, total-point bucket (power of two) and the
number of right-hand sides per plan (plans add their level count and orders).
The timer is pluggable so the selection and cache logic run without a GPU.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from dataclasses import dataclass

DEFAULT_CANDIDATES = [{"nstreams": s, "rhs_block": rb} for s, rb in itertools.product((1, 2, 4, 8), (1, 4))]

# kernel choices of one plan: tensor-core fill threshold (0: every propagation level on the tensor cores,
# 2: none), tensor-core engine, interpolation engine; right-hand-side blocking is added when nrhs > 1
PLAN_CANDIDATES = [{"tc_fill": f, "tc_engine": e, "interp_engine": i}
                   for f, e, i in itertools.product((0.0, 0.4, 0.7, 2.0), (1, 2, 0), (1, 0))
                   if not (f == 2.0 and e != 1)]  # with no tensor-core level the engine does not matter


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


def plan_key(device: str, precision: str, info: dict, orders, nrhs: int) -> str:
    """Cache key of one plan's apply: the point bucket, the level count and the interpolation orders."""
    return tune_key(device, precision, info["N"], nrhs) + f"|D={info['D']}|orders={orders[0]}x{orders[1]}"


def plan_candidates(nrhs: int) -> list:
    if nrhs <= 1:
        return [dict(c) for c in PLAN_CANDIDATES]
    return [dict(c, rhs_block=rb) for c in PLAN_CANDIDATES for rb in (1, 4)]


def apply_plan_config(plan, cfg: dict):
    plan.set_tc_fill(cfg["tc_fill"])
    plan.set_tc_engine(cfg["tc_engine"])
    plan.set_interp_engine(cfg["interp_engine"])
    if "rhs_block" in cfg:
        plan.set_rhs_block(cfg["rhs_block"])


def plan_timer(plan, sigma, out, warmup: int = 1):
    """Timer for Autotuner.tune: applies `config` to the plan and returns the CUDA-event time of one
    apply of sigma (after `warmup` untimed ones)."""
    import torch

    def run(cfg):
        apply_plan_config(plan, cfg)
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            plan.apply(sigma, out=out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.apply(sigma, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    return run


def tune_plan(plan, sigma, tuner: Autotuner | None = None, reps: int = 3, force: bool = False) -> TuneResult:
    """Time the plan's kernel choices on sigma (a CUDA tensor of the precision to tune), cache the
    fastest and leave the plan configured with it."""
    import torch

    tuner = tuner or Autotuner()
    prec = "fp64" if sigma.dtype == torch.complex128 else "mixed"
    nrhs = 1 if sigma.dim() == 1 else int(sigma.shape[0])
    p = plan.params
    key = plan_key(torch.cuda.get_device_name(sigma.device), prec, plan.info(), (p.Ps, p.Pang), nrhs)
    out = torch.empty_like(sigma)
    r = tuner.tune(key, plan_timer(plan, sigma, out), candidates=plan_candidates(nrhs), reps=reps, force=force)
    apply_plan_config(plan, r.config)
    return r
