"""Host logic of the autotuner: search space and conditional, baseline as
best of repeats, time limit, resumable database, and that both strategies find
the optimum of a synthetic objective (no GPU needed)."""
import json
import math

import pytest

from paper_2402_09222_b300 import tuner


def synthetic_objective(calls=None, timeout_above=None):
    """Run time with an optimum at queued, 2e6 in flight, 20000 bins, period 2."""
    def f(cfg, limit):
        if calls is not None:
            calls.append(dict(cfg))
        t = 1.0
        t += 0.3 * (cfg["mode"] != tuner.QUEUED)
        t += 0.2 * abs(math.log(cfg["particles_in_flight"] / 2e6))
        t += 0.1 * abs(math.log(cfg["hash_bins"] / 2e4))
        if cfg["mode"] == tuner.QUEUED:
            t += 0.05 * abs(cfg["sort_period"] - 2)
        t += 0.02 * (cfg["block_size"] != 256)
        if limit and t > limit:
            raise TimeoutError
        return t
    return f


def test_space_defaults_and_condition():
    space = tuner.transport_space()
    d = {p.name: p.default for p in space}
    assert d["mode"] == tuner.QUEUED and d["particles_in_flight"] == 1_000_000
    assert d["hash_bins"] == 4000 and d["sort_threshold"] == 20_000
    c = tuner.canonical(space, dict(d, mode=tuner.QUEUELESS))
    assert "sort_threshold" not in c and "sort_period" not in c
    c = tuner.canonical(space, d)
    assert c["sort_threshold"] == 20_000
    import random
    rng = random.Random(0)
    for p in space:
        for _ in range(50):
            v = p.sample(rng)
            if p.kind != "choice":
                assert p.lo <= v <= p.hi and v % p.q == 0


def test_baseline_is_best_of_five_and_limit_is_one_and_a_half(tmp_path):
    calls = []
    seen_limits = []
    f = synthetic_objective(calls)

    def obj(cfg, limit):
        seen_limits.append(limit)
        return f(cfg, limit)

    t = tuner.Tuner(tuner.transport_space(), obj, db_path=str(tmp_path / "db.jsonl"))
    base = t.run_baseline()
    assert len(calls) == 5 and seen_limits == [0.0] * 5
    t.evaluate(t.random_config(), "random")
    assert seen_limits[-1] == pytest.approx(1.5 * base)


def test_random_plus_coordinate_descent_finds_the_optimum(tmp_path):
    t = tuner.Tuner(tuner.transport_space(), synthetic_objective(), db_path=str(tmp_path / "db.jsonl"),
                    seed=3)
    best = t.tune(n_random=24, max_evals=120)
    assert best.seconds < 1.12
    assert best.config["mode"] == tuner.QUEUED
    rep = t.report()
    assert rep["improvement_pct"] > 0 and rep["evaluations"] <= 120


def test_timeouts_are_recorded_and_the_search_continues(tmp_path):
    t = tuner.Tuner(tuner.transport_space(), synthetic_objective(), seed=5, timeout_factor=1.05,
                    db_path=str(tmp_path / "db.jsonl"))
    t.tune(n_random=20, max_evals=30)
    assert any(r.status == "timeout" for r in t.records)
    assert t.best().seconds is not None


def test_database_resumes_without_repeating(tmp_path):
    db = str(tmp_path / "db.jsonl")
    calls = []
    t1 = tuner.Tuner(tuner.transport_space(), synthetic_objective(calls), db_path=db, seed=7)
    t1.tune(n_random=10, max_evals=10)
    n1 = len(calls)
    lines = [json.loads(l) for l in open(db)]
    assert len(lines) == n1
    calls2 = []
    t2 = tuner.Tuner(tuner.transport_space(), synthetic_objective(calls2), db_path=db, seed=7)
    assert t2.baseline == t1.baseline
    t2.tune(n_random=10, max_evals=14)
    assert len(calls2) == 4            # only the new evaluations ran
    keys = [tuner.key_of(c) for c in calls2]
    old = {tuner.key_of(r.config) for r in t1.records if r.kind != "baseline"}
    assert not (set(keys) & old)


def test_bayesian_optimisation_with_random_forest_and_lcb(tmp_path):
    """The surrogate's mean alone (kappa = 0) leads to the optimum; with the
    paper's kappa = 1.96 the search explores more and still improves on the
    baseline."""
    t = tuner.Tuner(tuner.transport_space(), synthetic_objective(), seed=11,
                    db_path=str(tmp_path / "db.jsonl"))
    best = t.tune(n_random=12, max_evals=60, strategy="bo", kappa=0.0)
    assert best.seconds < 1.06
    assert any(r.kind == "bo" for r in t.records)
    t2 = tuner.Tuner(tuner.transport_space(), synthetic_objective(), seed=11)
    best2 = t2.tune(n_random=12, max_evals=60, strategy="bo")
    assert best2.seconds < 0.95 * t2.baseline


def test_rejected_configurations_count_as_failures(tmp_path):
    def obj(cfg, limit):
        if cfg["block_size"] == 512:
            raise ValueError("rejected")
        return 1.0 + cfg["particles_in_flight"] * 1e-9
    t = tuner.Tuner(tuner.transport_space(), obj, seed=2)
    t.tune(n_random=16, max_evals=16)
    assert all(r.seconds is not None or r.status.startswith("error") or r.status == "timeout"
               for r in t.records)


def test_energy_metric_keeps_the_time_limit_in_seconds(tmp_path):
    """With an energy objective the limit is still 1.5 x the baseline's run
    time, not 1.5 x its joules."""
    limits = []

    def obj(cfg, limit):
        limits.append(limit)
        t = 2.0 + 0.1 * (cfg["block_size"] != 256)
        if limit and t > limit:
            raise TimeoutError
        return 500.0 * t, t          # (joules, seconds)

    t = tuner.Tuner(tuner.transport_space(), obj, db_path=str(tmp_path / "db.jsonl"), seed=4)
    t.run_baseline()
    assert t.baseline == pytest.approx(1000.0) and t.baseline_runtime == pytest.approx(2.0)
    t.tune(n_random=4, max_evals=4)
    assert limits[-1] == pytest.approx(3.0)
    t2 = tuner.Tuner(tuner.transport_space(), obj, db_path=str(tmp_path / "db.jsonl"), seed=4)
    assert t2.baseline_runtime == pytest.approx(2.0)


def test_energy_meter_with_a_fake_counter():
    from paper_2402_09222_b300 import energy

    class FakeNvml:
        def __init__(self):
            self.mj = 1_000_000
            self.calls = []

        def nvmlInit(self):
            self.calls.append("init")

        def nvmlShutdown(self):
            self.calls.append("shutdown")

        def nvmlDeviceGetHandleByIndex(self, i):
            return ("dev", i)

        def nvmlDeviceGetTotalEnergyConsumption(self, h):
            self.mj += 250_000          # 250 J per reading
            return self.mj

    nv = FakeNvml()
    with energy.EnergyMeter(3, nvml=nv) as m:
        pass
    assert m.joules == pytest.approx(250.0)
    assert m.edp == pytest.approx(m.joules * m.seconds)
    assert nv.calls == ["init", "shutdown"]
    assert energy.objective_value("edp", 2.0, 10.0) == 20.0
    assert energy.objective_value("time", 2.0, None) == 2.0
    with pytest.raises(ValueError):
        energy.objective_value("energy", 2.0, None)


def test_random_forest_surrogate_fits_and_spreads():
    import random
    rng = random.Random(0)
    X = [[rng.uniform(0, 1), rng.uniform(0, 1)] for _ in range(80)]
    y = [3 * x0 + (x1 > 0.5) for x0, x1 in X]
    rf = tuner.RandomForest(n_trees=50, seed=1).fit(X, y)
    pred = rf.predict_trees([[0.2, 0.9], [0.8, 0.1]])
    mu = [sum(col) / len(col) for col in zip(*pred)]
    assert abs(mu[0] - 1.6) < 0.35 and abs(mu[1] - 2.4) < 0.35
    # far from the data the trees disagree more than at a dense point
    spread = lambda i: max(p[i] for p in pred) - min(p[i] for p in pred)
    assert spread(0) >= 0.0 and len(pred) == 50


def test_device_scheduling_space_keeps_sort_parameters_for_both_queued_modes():
    space = tuner.transport_space(device_scheduling=True)
    mode = next(p for p in space if p.name == "mode")
    assert set(mode.choices) == {tuner.QUEUED, tuner.QUEUELESS, tuner.QUEUED_FULLEST}
    d = {p.name: p.default for p in space}
    for m in (tuner.QUEUED, tuner.QUEUED_FULLEST):
        c = tuner.canonical(space, dict(d, mode=m))
        assert "sort_threshold" in c and "sort_period" in c
    c = tuner.canonical(space, dict(d, mode=tuner.QUEUELESS))
    assert "sort_threshold" not in c
    # the paper's two-mode space is unchanged by default
    assert tuner.QUEUED_FULLEST not in next(p for p in tuner.transport_space() if p.name == "mode").choices
