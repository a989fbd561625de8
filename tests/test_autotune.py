"""Host logic of the autotuner: candidate selection, medians, JSON cache, keys."""
import json

from paper_2112_06316_gb300.autotune import DEFAULT_CANDIDATES, Autotuner, tune_key


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def run(cfg):
        calls.append(cfg)
        # fake cost: 4 streams and rhs_block 4 are best
        return 10.0 + abs(cfg["nstreams"] - 4) + (0 if cfg["rhs_block"] == 4 else 3)

    t = Autotuner(str(tmp_path / "tune.json"))
    key = tune_key("GB300", "mixed", 3_854_976, 4)
    r = t.tune(key, run, reps=3)
    assert r.config == {"nstreams": 4, "rhs_block": 4} and not r.cached
    assert len(calls) == 3 * len(DEFAULT_CANDIDATES)
    db = json.load(open(tmp_path / "tune.json"))
    assert db[key]["config"] == r.config
    # a second tuner reads the cache and does not time again
    calls.clear()
    r2 = Autotuner(str(tmp_path / "tune.json")).tune(key, run)
    assert r2.cached and r2.config == r.config and not calls
    r3 = Autotuner(str(tmp_path / "tune.json")).tune(key, run, force=True, candidates=[{"nstreams": 1, "rhs_block": 1}])
    assert r3.config == {"nstreams": 1, "rhs_block": 1} and not r3.cached


def test_median_of_reps(tmp_path):
    seq = iter([5.0, 100.0, 6.0, 1.0, 9.0, 8.0])

    def run(cfg):
        return next(seq)

    r = Autotuner(str(tmp_path / "t.json")).tune("k", run, reps=3,
                                                 candidates=[{"nstreams": 1, "rhs_block": 1}, {"nstreams": 2, "rhs_block": 1}])
    # medians: (5, 100, 6) -> 6 and (1, 9, 8) -> 8
    assert r.config["nstreams"] == 1 and r.ms == 6.0


def test_key_buckets():
    assert tune_key("d", "fp64", 1000, 1) == tune_key("d", "fp64", 1024, 1)
    assert tune_key("d", "fp64", 1025, 1) != tune_key("d", "fp64", 1024, 1)
    assert tune_key("d", "mixed", 1000, 4) != tune_key("d", "fp64", 1000, 4)


def test_plan_candidates_and_key():
    from paper_2112_06316_gb300.autotune import PLAN_CANDIDATES, plan_candidates, plan_key

    # every knob takes each of its values somewhere; no duplicate candidates
    assert {c["tc_fill"] for c in PLAN_CANDIDATES} == {0.0, 0.4, 0.7, 2.0}
    assert {c["tc_engine"] for c in PLAN_CANDIDATES} == {0, 1, 2}
    assert {c["interp_engine"] for c in PLAN_CANDIDATES} == {0, 1}
    keys = [tuple(sorted(c.items())) for c in plan_candidates(4)]
    assert len(keys) == len(set(keys)) == 2 * len(PLAN_CANDIDATES)
    assert all("rhs_block" not in c for c in plan_candidates(1))
    info = {"N": 393216, "D": 6}
    assert plan_key("GB300", "mixed", info, (5, 8), 1) != plan_key("GB300", "mixed", info, (3, 5), 1)
    assert plan_key("GB300", "mixed", info, (5, 8), 1) != plan_key("GB300", "mixed", dict(info, D=5), (5, 8), 1)


def test_tune_plan_logic_with_fake_plan(tmp_path, monkeypatch):
    """tune_plan's selection and configuration on a stand-in plan (the timer reads the settings)."""
    from paper_2112_06316_gb300 import autotune as at

    class FakePlan:
        def __init__(self):
            self.s = {}

        def set_tc_fill(self, v):
            self.s["tc_fill"] = v

        def set_tc_engine(self, v):
            self.s["tc_engine"] = v

        def set_interp_engine(self, v):
            self.s["interp_engine"] = v

        def set_rhs_block(self, v):
            self.s["rhs_block"] = v

    plan = FakePlan()

    def run(cfg):
        at.apply_plan_config(plan, cfg)
        # fake cost: all levels on tcgen05 engine 1 with the cone-stationary interpolation is best
        return 5.0 + (0 if plan.s["tc_fill"] == 0.0 else 1) + (0 if plan.s["tc_engine"] == 1 else 2) + \
            (0 if plan.s["interp_engine"] == 1 else 3)

    r = at.Autotuner(str(tmp_path / "t.json")).tune("k", run, candidates=at.plan_candidates(1))
    assert r.config == {"tc_fill": 0.0, "tc_engine": 1, "interp_engine": 1}
    at.apply_plan_config(plan, r.config)
    assert plan.s == r.config
