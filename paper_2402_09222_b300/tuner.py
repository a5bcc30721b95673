"""Autotuner for the event loop and the lookup (the role ytopt plays for OpenMC
in the paper, Sec. 2-5, on this one GPU).

Search space (Table 1 of the paper, mapped to this implementation):
  mode              queued | queueless                     (P0; with
                    device_scheduling=True also the fullest-queue mode,
                    the paper's queued policy decided on the device)
  particles_in_flight  1e5 .. 8e6, log scale, step 1000     (P1)
  hash_bins         100 .. 100000, log scale, step 100      (P2)
  sort_threshold    0 .. 1e6, step 1000; active only in queued modes (P3,
                    the paper's EqualsCondition(P3, P0, queued))
  sort_period       0, 1, 2, 4, 8, 16; queued modes only   (this GPU's binning)
  block_size        64, 128, 256, 512                      (replaces the paper's
                    host-thread and MPI-rank parameters P4-P6, which have no
                    counterpart on one GPU)

Strategies:
  "random+cd"  the minimum tuner: the default configuration as baseline
               (best of `baseline_repeats` runs; Sec. 6: best of five), then
               random samples, then coordinate descent from the best point;
  "bo"         Bayesian optimisation with a random-forest surrogate and the
               lower-confidence-bound acquisition a(x) = mu(x) - kappa sigma(x),
               kappa = 1.96 (Sec. 2.1, Eq. 1), minimising run time.
Every evaluation runs under a time limit of `timeout_factor` x the baseline
time (Sec. 3: 1.5x); a run that exceeds it is recorded as a timeout with a very
bad objective and the search continues.  The performance database is a JSONL
file; an interrupted search resumes without repeating recorded evaluations.
"""
from __future__ import annotations

import json
import math
import os
import random
import time
from dataclasses import dataclass, field
from typing import Callable

QUEUELESS, QUEUED, QUEUED_FULLEST = 0, 1, 2


@dataclass
class Param:
    name: str
    kind: str                    # "int_log" | "int" | "choice"
    lo: float = 0
    hi: float = 0
    q: int = 1
    choices: tuple = ()
    default: object = None
    active_if: tuple | None = None   # (other_param, value or tuple of values)

    def active(self, cfg: dict) -> bool:
        if self.active_if is None:
            return True
        name, want = self.active_if
        return cfg.get(name) in want if isinstance(want, tuple) else cfg.get(name) == want

    def sample(self, rng: random.Random):
        if self.kind == "choice":
            return rng.choice(self.choices)
        if self.kind == "int_log":
            v = math.exp(rng.uniform(math.log(self.lo), math.log(self.hi)))
        else:
            v = rng.uniform(self.lo, self.hi)
        return self.quantise(v)

    def quantise(self, v):
        if self.kind == "choice":
            return v
        v = int(round(v / self.q)) * self.q
        return int(min(max(v, self.lo), self.hi))

    def neighbours(self, v):
        """Values one coordinate step away (for coordinate descent)."""
        if self.kind == "choice":
            return [c for c in self.choices if c != v]
        if self.kind == "int_log":
            return sorted({self.quantise(v * 2), self.quantise(v / 2)} - {v})
        step = max(self.q, (self.hi - self.lo) / 8)
        return sorted({self.quantise(v + step), self.quantise(v - step)} - {v})

    def encode(self, v) -> float:
        """Numeric feature for the surrogate."""
        if self.kind == "choice":
            return float(self.choices.index(v))
        if self.kind == "int_log":
            return math.log(max(v, 1))
        return float(v)


class RandomForest:
    """A small random-forest regressor (the surrogate of Sec. 2.1): bootstrap
    samples, CART regression trees split on the largest decrease of squared
    error over a random subset of features, leaves of at least
    `min_leaf` samples.  `predict_trees` returns each tree's predictions, whose
    mean and spread give mu(x) and sigma(x) for the LCB acquisition."""

    def __init__(self, n_trees: int = 100, max_features: float = 0.6, min_leaf: int = 1,
                 max_depth: int = 12, seed: int = 0):
        self.n_trees, self.max_features = n_trees, max_features
        self.min_leaf, self.max_depth = min_leaf, max_depth
        self.rng = random.Random(seed)
        self.trees = []

    def fit(self, X, y):
        n = len(X)
        self.trees = []
        for _ in range(self.n_trees):
            idx = [self.rng.randrange(n) for _ in range(n)]
            self.trees.append(self._grow([X[i] for i in idx], [y[i] for i in idx], 0))
        return self

    def _grow(self, X, y, depth):
        mean = sum(y) / len(y)
        if depth >= self.max_depth or len(y) < 2 * self.min_leaf or max(y) - min(y) < 1e-12:
            return mean
        d = len(X[0])
        feats = self.rng.sample(range(d), max(1, int(round(self.max_features * d))))
        best = None
        total_sq = sum(v * v for v in y)
        for f in feats:
            order = sorted(range(len(y)), key=lambda i: X[i][f])
            s_left = sq_left = 0.0
            s_all = sum(y)
            for k in range(len(order) - 1):
                v = y[order[k]]
                s_left += v
                sq_left += v * v
                nl, nr = k + 1, len(order) - k - 1
                if nl < self.min_leaf or nr < self.min_leaf:
                    continue
                a, b = X[order[k]][f], X[order[k + 1]][f]
                if a == b:
                    continue
                s_right = s_all - s_left
                sse = (sq_left - s_left * s_left / nl) + ((total_sq - sq_left) - s_right * s_right / nr)
                if best is None or sse < best[0]:
                    best = (sse, f, 0.5 * (a + b))
        if best is None:
            return mean
        _, f, thr = best
        left = [i for i in range(len(y)) if X[i][f] <= thr]
        right = [i for i in range(len(y)) if X[i][f] > thr]
        return (f, thr, self._grow([X[i] for i in left], [y[i] for i in left], depth + 1),
                self._grow([X[i] for i in right], [y[i] for i in right], depth + 1))

    @staticmethod
    def _predict_one(node, x):
        while isinstance(node, tuple):
            f, thr, l, r = node
            node = l if x[f] <= thr else r
        return node

    def predict_trees(self, X):
        return [[self._predict_one(t, x) for x in X] for t in self.trees]


def transport_space(max_in_flight: int = 8_000_000, device_scheduling: bool = False) -> list[Param]:
    modes = (QUEUED, QUEUELESS, QUEUED_FULLEST) if device_scheduling else (QUEUED, QUEUELESS)
    queued = (QUEUED, QUEUED_FULLEST)
    return [
        Param("mode", "choice", choices=modes, default=QUEUED),
        Param("particles_in_flight", "int_log", 100_000, max_in_flight, 1000, default=1_000_000),
        Param("hash_bins", "int_log", 100, 100_000, 100, default=4000),
        Param("sort_threshold", "int", 0, 1_000_000, 1000, default=20_000, active_if=("mode", queued)),
        Param("sort_period", "choice", choices=(0, 1, 2, 4, 8, 16), default=4, active_if=("mode", queued)),
        Param("block_size", "choice", choices=(64, 128, 256, 512), default=256),
    ]


def lookup_space() -> list[Param]:
    return [
        Param("hash_bins", "int_log", 100, 100_000, 100, default=4000),
        Param("binned", "choice", choices=(1, 0), default=1),
    ]


def canonical(space: list[Param], cfg: dict) -> dict:
    """Inactive conditional parameters are dropped (the paper's 'nan')."""
    out = {}
    for p in space:
        if not p.active(cfg):
            continue
        out[p.name] = cfg[p.name]
    return out


def key_of(cfg: dict) -> str:
    return json.dumps(cfg, sort_keys=True)


@dataclass
class Record:
    config: dict
    seconds: float | None      # the objective (run time, energy or EDP); None: timed out or failed
    status: str                # "ok" | "timeout" | "error"
    kind: str                  # "baseline" | "random" | "cd" | "bo"
    runtime: float | None = None   # wall seconds of the run (for the time limit)


@dataclass
class Tuner:
    """objective(config, time_limit_s) -> value, or (value, run seconds) when
    the value is not a time (energy, EDP); raises TimeoutError past the limit.
    The limit is timeout_factor x the baseline's run seconds."""
    space: list[Param]
    objective: Callable[[dict, float], float]
    db_path: str | None = None
    seed: int = 1234
    timeout_factor: float = 1.5
    baseline_repeats: int = 5
    bad_seconds: float = 1e9
    records: list[Record] = field(default_factory=list)

    def __post_init__(self):
        self.rng = random.Random(self.seed)
        self._done: dict[str, Record] = {}
        if self.db_path and os.path.exists(self.db_path):
            for line in open(self.db_path):
                if line.strip():
                    d = json.loads(line)
                    r = Record(d["config"], d["seconds"], d["status"], d["kind"], d.get("runtime"))
                    self.records.append(r)
                    if r.kind != "baseline":
                        self._done[key_of(r.config)] = r
        self.baseline = None
        self.baseline_runtime = None
        base = [r for r in self.records if r.kind == "baseline" and r.seconds]
        if len(base) >= self.baseline_repeats:
            self._set_baseline(base)

    def _set_baseline(self, base):
        self.baseline = min(r.seconds for r in base)
        rts = [r.runtime for r in base if r.runtime]
        self.baseline_runtime = min(rts) if rts else self.baseline

    # -- bookkeeping
    def default_config(self) -> dict:
        return canonical(self.space, {p.name: p.default for p in self.space})

    def _log(self, r: Record):
        self.records.append(r)
        if self.db_path:
            with open(self.db_path, "a") as f:
                f.write(json.dumps({"config": r.config, "seconds": r.seconds, "status": r.status,
                                    "kind": r.kind, "runtime": r.runtime, "time": time.time()}) + "\n")

    def evaluate(self, cfg: dict, kind: str) -> Record:
        cfg = canonical(self.space, cfg)
        k = key_of(cfg)
        if kind != "baseline" and k in self._done:
            return self._done[k]
        limit = (self.timeout_factor * self.baseline_runtime
                 if (self.baseline_runtime and kind != "baseline") else 0.0)
        try:
            v = self.objective(cfg, limit)
            if isinstance(v, tuple):
                r = Record(cfg, float(v[0]), "ok", kind, float(v[1]))
            else:
                r = Record(cfg, float(v), "ok", kind, float(v))
        except TimeoutError:
            r = Record(cfg, None, "timeout", kind)
        except Exception as e:  # a configuration the library rejects counts as a failure
            r = Record(cfg, None, f"error: {e}"[:200], kind)
        self._log(r)
        if kind != "baseline":
            self._done[k] = r
        return r

    def score(self, r: Record) -> float:
        return r.seconds if r.seconds is not None else self.bad_seconds

    def best(self) -> Record:
        cand = [r for r in self.records if r.seconds is not None]
        return min(cand, key=lambda r: r.seconds)

    # -- strategies
    def run_baseline(self):
        have = [r for r in self.records if r.kind == "baseline" and r.seconds]
        for _ in range(self.baseline_repeats - len(have)):
            self.evaluate(self.default_config(), "baseline")
        base = [r for r in self.records if r.kind == "baseline" and r.seconds]
        if not base:
            raise RuntimeError("the default configuration failed")
        self._set_baseline(base)
        return self.baseline

    def random_config(self) -> dict:
        cfg = {p.name: p.sample(self.rng) for p in self.space}
        return canonical(self.space, cfg)

    def tune(self, n_random: int = 24, max_evals: int = 64, strategy: str = "random+cd",
             kappa: float = 1.96) -> Record:
        """kappa: exploration weight of the LCB acquisition (the paper's
        default 1.96; 0 exploits the surrogate's mean only)."""
        if self.baseline is None:
            self.run_baseline()
        n_eval = lambda: sum(1 for r in self.records if r.kind != "baseline")
        if strategy == "bo":
            return self._bo(n_random, max_evals, n_eval, kappa=kappa)
        while n_eval() < min(n_random, max_evals):
            self.evaluate(self.random_config(), "random")
        improved = True
        while improved and n_eval() < max_evals:
            improved = False
            cur = self.best()
            full = {p.name: cur.config.get(p.name, p.default) for p in self.space}
            for p in self.space:
                if not p.active(full):
                    continue
                for v in p.neighbours(full[p.name]):
                    if n_eval() >= max_evals:
                        break
                    trial = dict(full)
                    trial[p.name] = v
                    r = self.evaluate(trial, "cd")
                    if r.seconds is not None and r.seconds < cur.seconds:
                        improved = True
                        break
                if improved:
                    break
        return self.best()

    def _features(self, cfg: dict) -> list[float]:
        return [p.encode(cfg.get(p.name, p.default)) for p in self.space]

    def _bo(self, n_init, max_evals, n_eval, kappa: float = 1.96, n_candidates: int = 512):
        while n_eval() < min(n_init, max_evals):
            self.evaluate(self.random_config(), "random")
        while n_eval() < max_evals:
            data = [(self._features(r.config), math.log(self.score(r)))
                    for r in self.records]
            X = [d[0] for d in data]
            y = [d[1] for d in data]
            rf = RandomForest(n_trees=100, seed=self.rng.randrange(2**31)).fit(X, y)
            cands = [self.random_config() for _ in range(n_candidates)]
            # local candidates around the best configurations so far: every
            # single-coordinate neighbour and random two-coordinate moves
            top = sorted((r for r in self.records if r.seconds is not None), key=lambda r: r.seconds)[:5]
            for rec in top:
                full = {p.name: rec.config.get(p.name, p.default) for p in self.space}
                for p in self.space:
                    for v in p.neighbours(full[p.name]):
                        c = dict(full)
                        c[p.name] = v
                        cands.append(canonical(self.space, c))
                for _ in range(32):
                    c = dict(full)
                    for p in self.rng.sample(self.space, 2):
                        c[p.name] = self.rng.choice(p.neighbours(c[p.name]) or [c[p.name]])
                    cands.append(canonical(self.space, c))
            cands = [c for c in cands if key_of(c) not in self._done]
            if not cands:
                break
            Xc = [self._features(c) for c in cands]
            per_tree = rf.predict_trees(Xc)
            mu = [sum(col) / len(col) for col in zip(*per_tree)]
            sd = [math.sqrt(max(sum((v - m) ** 2 for v in col) / len(col), 0.0))
                  for col, m in zip(zip(*per_tree), mu)]
            acq = [m - kappa * s for m, s in zip(mu, sd)]
            i = min(range(len(cands)), key=lambda j: acq[j])
            self.evaluate(cands[i], "bo")
        return self.best()

    def report(self) -> dict:
        b = self.best()
        return {"baseline_s": self.baseline, "best_s": b.seconds, "best_config": b.config,
                "improvement_pct": 100.0 * (self.baseline / b.seconds - 1.0),
                "evaluations": sum(1 for r in self.records if r.kind != "baseline"),
                "timeouts": sum(1 for r in self.records if r.status == "timeout")}


# ---------------------------------------------------------------------------
# objectives on the GPU
# ---------------------------------------------------------------------------

def transport_objective(prob, seed: int = 1, precision: int = 1, device: int = 0,
                        max_in_flight: int | None = None, metric: str = "time"):
    """The objective of one run of `prob` under a configuration: its seconds
    (CUDA events around mcx_run_batch), or with metric "energy"/"edp" the GPU
    energy in joules (NVML counter) or energy x seconds (the paper's Sec. 7
    objectives).  Raises TimeoutError when the library reports its time limit
    (the limit is in seconds whatever the metric)."""
    import torch
    from . import energy, mcx
    handles = {}

    def objective(cfg: dict, limit: float) -> float:
        H = cfg["hash_bins"]
        if H not in handles:
            handles.clear()
            handles[H] = mcx.make_problem(prob, precision=precision, hash_bins=H, device=device)
        p = handles[H]
        p.set_tuning(mode=cfg["mode"], block_size=cfg["block_size"],
                     sort_period=cfg.get("sort_period", 0), sort_threshold=cfg.get("sort_threshold", 0),
                     time_limit_s=limit)
        pif = cfg["particles_in_flight"]
        if max_in_flight:
            pif = min(pif, max_in_flight)
        p.zero_tallies()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        meter = energy.EnergyMeter(device) if metric != "time" else None
        if meter:
            meter.__enter__()
        a.record()
        try:
            p.run(particles_in_flight=pif, seed=seed)
        except mcx.McxError as e:
            if meter:
                meter.__exit__(None, None, None)
            if e.code == mcx.ERR_TIMEOUT:
                raise TimeoutError(str(e)) from e
            raise
        b.record()
        torch.cuda.synchronize()
        seconds = a.elapsed_time(b) / 1e3
        joules = None
        if meter:
            meter.__exit__(None, None, None)
            joules = meter.joules
        value = energy.objective_value(metric, seconds, joules)
        return value if metric == "time" else (value, seconds)

    return objective


def batched_objective(lib, mats, probs, seed: int = 9, precision: int = 1, device: int = 0):
    """Seconds of one event loop over many problems (mcx_batch_run: one global
    work list, shared tables) under a configuration; the tuning of the first
    handle governs the loop.  Hash-bin changes rebuild the shared tables'
    hash grid in place."""
    import torch
    from . import mcx
    base = mcx.Problem(probs[0], device=device).load_tables(lib, mats, precision=precision, hash_bins=4000)
    hs = [base] + [mcx.Problem(pr, device=device).share_tables(base) for pr in probs[1:]]
    nh = [pr.n_histories for pr in probs]
    state = {"H": 4000}

    def objective(cfg: dict, limit: float) -> float:
        if cfg["hash_bins"] != state["H"]:
            base.set_hash_bins(cfg["hash_bins"])
            state["H"] = cfg["hash_bins"]
        base.set_tuning(mode=cfg["mode"], block_size=cfg["block_size"],
                        sort_period=cfg.get("sort_period", 0), sort_threshold=cfg.get("sort_threshold", 0),
                        time_limit_s=limit)
        for h in hs:
            h.zero_tallies()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        try:
            mcx.batch_run(hs, nh, cfg["particles_in_flight"], seed)
        except mcx.McxError as e:
            if e.code == mcx.ERR_TIMEOUT:
                raise TimeoutError(str(e)) from e
            raise
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    return objective


def lookup_objective(lib, mats, E, mat, precision: int = 1, device: int = 0, fast: bool = True):
    """Seconds of one binned-or-not lookup pass over device inputs E, mat."""
    import torch
    from . import mcx
    dE = torch.as_tensor(E, device=f"cuda:{device}")
    dm = torch.as_tensor(mat, device=f"cuda:{device}")
    out = torch.empty((len(E), lib.n_ch), dtype=torch.float64, device=dE.device)
    perm = torch.empty(len(E), dtype=torch.int32, device=dE.device)
    h = mcx.Problem(None, device=device).load_tables(lib, mats, precision=precision, hash_bins=4000)
    state = {"H": 4000}

    def objective(cfg: dict, limit: float) -> float:
        if cfg["hash_bins"] != state["H"]:
            h.set_hash_bins(cfg["hash_bins"])
            state["H"] = cfg["hash_bins"]
        flags = mcx.LOOKUP_FAST if fast else mcx.LOOKUP_EXACT
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        if cfg["binned"]:
            h.xs_sort(dE, dm, perm)
            h.xs_lookup_ordered(dE, dm, perm, out=out, flags=flags)
        else:
            h.xs_lookup_ordered(dE, dm, None, out=out, flags=flags)
        b.record()
        torch.cuda.synchronize()
        s = a.elapsed_time(b) / 1e3
        if limit and s > limit:
            raise TimeoutError(f"{s:.3f} s > {limit:.3f} s")
        return s

    return objective


def main(argv=None):
    """python -m paper_2402_09222_b300.tuner --workload transport|lookup|batched ..."""
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=["transport", "lookup", "batched"], default="transport")
    ap.add_argument("--histories", type=int, default=10_000_000)
    ap.add_argument("--lookups", type=int, default=100_000_000)
    ap.add_argument("--strategy", choices=["random+cd", "bo"], default="random+cd")
    ap.add_argument("--random", type=int, default=24)
    ap.add_argument("--evals", type=int, default=40)
    ap.add_argument("--db", default=None, help="JSONL performance database (resumable)")
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--metric", choices=["time", "energy", "edp"], default="time",
                    help="transport objective (the time limit is always 1.5x baseline seconds)")
    ap.add_argument("--device-scheduling", action="store_true",
                    help="add the fullest-queue mode (queue chosen on the device) to the mode choices")
    args = ap.parse_args(argv)
    from . import synth
    if args.workload == "transport":
        prob = synth.config3_problem(n_histories=args.histories)
        space = transport_space(device_scheduling=args.device_scheduling)
        obj = transport_objective(prob, seed=5, precision=1, metric=args.metric)
    elif args.workload == "batched":
        # 64 uneven lattices over the 12-material set (the batched workload)
        lib = synth.species_library(355, 11_303, 1236).channels([synth.CH_SCATTER, synth.CH_ABSORB])
        mats = synth.lookup_materials(355, 1236)
        probs = synth.config5_problems(lib, mats, n_problems=64)
        space = transport_space(device_scheduling=args.device_scheduling)
        obj = batched_objective(lib, mats, probs, seed=9)
    else:
        lib = synth.species_library(355, 11_303, 1236)
        mats = synth.lookup_materials(355, 1236)
        E, mat = synth.lookup_inputs(args.lookups, mats.n_materials, 1336)
        space = lookup_space()
        obj = lookup_objective(lib, mats, E, mat)
    t = Tuner(space, obj, db_path=args.db, seed=args.seed)
    t.tune(n_random=args.random, max_evals=args.evals, strategy=args.strategy)
    print(json.dumps(t.report()))


if __name__ == "__main__":
    main()
