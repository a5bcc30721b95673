#!/usr/bin/env python
"""Benchmark of the macroscopic cross-section lookup (and, alongside it, the
event-based transport) on one B300 per rank.

One step = one pass of the lookup hot path over one batch of 1e8 synthetic
lookups (355 species x 11,303 points, 5 channels, 12 materials of 4-321
species; energies log-uniform on [1e-5, 2e7] eV, materials uniform): binning
by material and log-energy, then the gather-interpolate-sum kernel, FP32
tables, 4000 hash bins.  Inputs (1.2 GB) and outputs (4 GB) are far larger
than the 126 MB L2, so no flush is needed between steps.

Printed: one JSON line (rank 0) with the contract keys plus `roofline`
(lookup kernel, algorithmic bytes over its CUDA-event time against the
measured HBM copy bandwidth), `cpu_baseline` (the CPU oracle on a bounded
sample of the same workload), `e2e` (the same lookups through the C-ABI host
entry point, copies included), `plain` (the FP64 exact full-search form) and
`transport` (particles/s on the 17x17 lattice, tuned and plain).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mcx|reference]
Under torchrun each rank runs its own batch (weak scaling, no collective on
the data path; a barrier and a max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LOOKUPS = 100_000_000
E2E_CALLS = 3        # timed end-to-end calls from host buffers (after one untimed call)
N_SPECIES, N_POINTS = 355, 11_303
LIB_SEED, MAT_SEED, INPUT_SEED = 1236, 1236, 1336
# FP32 tables, fast arithmetic, binned; hash bins from a sweep of the tuner's
# range on this step (best of 5: 4000 bins 39.1 ms, 45600 35.6 ms, 68400
# 33.3 ms, 100000 33.5 ms, 200000 34.3 ms)
# flags: fast arithmetic with the round-linear sums (MCX_LOOKUP_FAST |
# MCX_LOOKUP_LINEAR); PER_LOOKUP_FLAGS is the bit-identical per-lookup form
TUNED = dict(precision=1, hash_bins=68_400, flags=17)
PER_LOOKUP_FLAGS = 1
# the host pipeline (2M/4M-lookup chunks, each binned on its own into about
# 11-21 lookups per bucket, so a round spans several buckets): the per-lookup
# form, binned (measured 73.6 against 73.8 ms with FP64 outputs, 43.2 against
# 48.3 ms with FP32 outputs for the round-linear form)
HOST_FLAGS = 1 | 2
PLAIN = dict(precision=0, hash_bins=0, flags=0)           # FP64 tables, exact, full binary search
TRANSPORT_HIST = 10_000_000
# chosen by paper_2402_09222_b300.tuner (random + coordinate descent, 40
# evaluations on this workload, 1.5x-baseline time limit): 1.326 s against
# 1.855 s for the default configuration (best of 5), +39.9 %
TRANSPORT_TUNED = dict(precision=1, hash_bins=37_100, pif=1_600_000,
                       tune=dict(mode=1, block_size=256, sort_period=1, sort_threshold=400_000))
TRANSPORT_PLAIN = dict(precision=0, hash_bins=0, pif=1_000_000, tune=dict(mode=0, block_size=256))
TRANSPORT_FULLEST = dict(TRANSPORT_TUNED, tune=dict(TRANSPORT_TUNED["tune"], mode=2))
# the 64 uneven lattices of the batched workload in one event loop, chosen by
# paper_2402_09222_b300.tuner on that workload (Bayesian optimisation with the
# random-forest surrogate and LCB, three modes, 45 evaluations, 1.5x-baseline
# time limit): 3.56 s against 5.29 s for the default configuration (best of 5),
# +48.6 %; the lattice's own point (1.6e6 in flight, 4000 bins, block 256)
# measured 3.60 s on the same workload
BATCHED_TUNED = dict(precision=1, hash_bins=2600, pif=3_090_000,
                     tune=dict(mode=1, block_size=512, sort_period=1, sort_threshold=817_000))
WORKLOAD = ("macroscopic XS lookup, 355 species x 11,303 points x 5 channels, 12 materials "
            "(4-321 species), 1e8 lookups per step")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def workload_inputs(rank: int):
    from paper_2402_09222_b300 import synth
    lib = synth.species_library(N_SPECIES, N_POINTS, LIB_SEED)
    mats = synth.lookup_materials(N_SPECIES, MAT_SEED)
    E, mat = synth.lookup_inputs(N_LOOKUPS, mats.n_materials, INPUT_SEED + rank)
    return lib, mats, E, mat


def algorithmic_bytes(mats, mat, sigma_bytes: int, n_ch: int = 5) -> float:
    """Per-lookup bytes of the definition: per species the two bracketing
    energies (16 B) and the two table rows (2 n_ch sigma), plus E (8), the
    material id (4) and the output row (8 n_ch)."""
    counts = np.bincount(mat, minlength=mats.n_materials)
    sizes = np.diff(mats.offsets)
    species_visits = float((counts * sizes).sum())
    return species_visits * (16 + 2 * n_ch * sigma_bytes) + len(mat) * (8 + 4 + 8 * n_ch)


def compulsory_bytes(lib, mats, n: int, n_ch: int = 5, hash_bins: int = None) -> float:
    """Bytes one binned launch cannot avoid moving: per lookup the energy (8),
    material (4), permutation entry (4) and output row (8 n_ch); once per
    launch every point record (32 B, FP32) and hash-window column (4 B per
    bin) of the species the materials hold."""
    H = TUNED["hash_bins"] if hash_bins is None else hash_bins
    used = np.unique(mats.species)
    pts = float(sum(lib.grid_offsets[s + 1] - lib.grid_offsets[s] for s in used))
    return n * (8 + 4 + 4 + 8 * n_ch) + pts * 32 + len(used) * (H + 1) * 4


def host_link_bandwidth(host_buf, dev_buf, nbytes: int = 1 << 30) -> dict:
    """Pinned host <-> device copy bandwidth (GB/s, one direction at a time,
    best of 3), the bound of the end-to-end path: its 4 GB of FP64 outputs
    leave through the device-to-host direction."""
    import torch
    del host_buf   # a dedicated pinned buffer: views of another may copy through a pageable path
    hb = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    db = dev_buf.reshape(-1).view(torch.uint8)[:nbytes]
    assert db.numel() == nbytes and hb.numel() == nbytes
    res = {}
    for name, (dst, src) in (("h2d", (db, hb)), ("d2h", (hb, db))):
        best = None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            s = time.perf_counter() - t0
            best = s if best is None else min(best, s)
        res[name + "_GBs"] = nbytes / best / 1e9
    return res


def lookup_traffic():
    """DRAM bytes per launch of the binned lookup kernel at this workload,
    from the ncu summary in profiles/ -- only while the kernel source and the
    hash-bin count are those the capture measured."""
    path = os.path.join(ROOT, "profiles", "lookup_traffic.json")
    if not os.path.exists(path):
        return None
    tr = json.load(open(path))
    if (tr.get("kernel_source_hash") != kernel_source_hash() or tr.get("hash_bins") != TUNED["hash_bins"]
            or N_LOOKUPS != 100_000_000):
        return None
    return tr


def cpu_baseline(lib, mats, E, mat, n_sample: int = 8_000_000, n_single: int = 200_000):
    import oracle
    cores = os.cpu_count() or 1
    oracle.xs_lookup(lib, mats, E[:1000], mat[:1000], n_threads=cores)   # warm
    t0 = time.perf_counter()
    oracle.xs_lookup(lib, mats, E[:n_sample], mat[:n_sample], n_threads=cores)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.xs_lookup(lib, mats, E[:n_single], mat[:n_single], n_threads=1)
    d1 = time.perf_counter() - t1
    return {"value": n_sample / dt, "unit": "lookups/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample:,} lookups of the step's batch, FP64 tables, "
                      f"full binary search, OpenMP over lookups on {cores} host cores ({dt:.1f} s)",
            "single_thread": {"value": n_single / d1, "unit": "lookups/s",
                              "sample": f"first {n_single:,} lookups, 1 thread ({d1:.1f} s)"}}


def cpu_transport(synth, lib3, n_sample: int = 200_000):
    """The oracle's lattice transport on all host cores (a bounded sample of
    the 1e7-history workload)."""
    import oracle
    cores = os.cpu_count() or 1
    prob = synth.config3_problem(n_histories=TRANSPORT_HIST, lib=lib3)
    t0 = time.perf_counter()
    oracle.transport(prob, seed=5, first=0, count=n_sample, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "particles/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample:,} histories of the 17x17 lattice, FP64, "
                      f"OpenMP over histories ({dt:.1f} s)"}


def time_inflight_sweep(mcx, synth, lib3, seed=5):
    """Particles/s of the tuned lattice transport against the number of
    particles in flight (the paper's P1 range, 1e5 to 8e6)."""
    import torch
    prob = synth.config3_problem(n_histories=TRANSPORT_HIST, lib=lib3)
    p = mcx.make_problem(prob, precision=1, hash_bins=TRANSPORT_TUNED["hash_bins"])
    p.set_tuning(**TRANSPORT_TUNED["tune"])
    out = {}
    for pif in (100_000, 250_000, 500_000, 1_000_000, 2_000_000, 4_000_000, 8_000_000):
        p.run(count=TRANSPORT_HIST // 20, particles_in_flight=pif, seed=seed)   # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        p.run(particles_in_flight=pif, seed=seed)
        b.record()
        torch.cuda.synchronize()
        out[str(pif)] = TRANSPORT_HIST / (a.elapsed_time(b) / 1e3)
    p.close()
    return {"unit": "particles/s", "histories": TRANSPORT_HIST, "by_particles_in_flight": out}


def time_derivatives(mcx, synth, lib3, n=2_000_000, seed=13, n_lookups=10_000_000):
    """Overhead of the likelihood-ratio derivative tallies (3 material
    density scales) on the lattice, and the lookup's backward pass into the
    FP32 sigma tables."""
    import torch
    prob = synth.config3_problem(n_histories=n, lib=lib3)
    res = {}
    dtal = {}
    for name, flags, prec in (("plain", 0, 1), ("derivatives", mcx.FLAG_DERIVATIVES, 1),
                              ("derivatives_fp64", mcx.FLAG_DERIVATIVES, 0)):
        p = mcx.make_problem(prob, precision=prec, hash_bins=TRANSPORT_TUNED["hash_bins"], flags=flags)
        p.set_tuning(**TRANSPORT_TUNED["tune"])
        p.run(count=n // 10, particles_in_flight=TRANSPORT_TUNED["pif"], seed=seed)
        p.zero_tallies()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        p.run(particles_in_flight=TRANSPORT_TUNED["pif"], seed=seed)
        b.record()
        torch.cuda.synchronize()
        res[name] = n / (a.elapsed_time(b) / 1e3)
        if flags:
            dtal[prec] = p.tallies()["dabsorb"]
        p.close()
    lib = synth.species_library(N_SPECIES, N_POINTS, LIB_SEED)
    mats = synth.lookup_materials(N_SPECIES, MAT_SEED)
    E, mat = synth.lookup_inputs(n_lookups, mats.n_materials, INPUT_SEED)
    q = mcx.Problem(None).load_tables(lib, mats, precision=1, hash_bins=TUNED["hash_bins"])
    dE = torch.as_tensor(E, device="cuda")
    dm = torch.as_tensor(mat, device="cuda")
    g = torch.ones((n_lookups, 5), dtype=torch.float64, device="cuda")
    gd, gs = q.xs_lookup_backward(dE, dm, g)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    q.xs_lookup_backward(dE, dm, g, gd, gs)
    b.record()
    torch.cuda.synchronize()
    q.close()
    B = dtal[1].shape[0]
    return {"unit": "particles/s", "histories": n, "plain": res["plain"],
            "with_derivative_tallies": res["derivatives"],
            "overhead": res["plain"] / res["derivatives"] - 1.0,
            "fp32_vs_fp64_tables_dabsorb_se": tally_z(dtal[1].reshape(B, -1), dtal[0].reshape(B, -1)),
            "lookup_backward": {"lookups_per_s": n_lookups / (a.elapsed_time(b) / 1e3),
                                "form": "binned (material, log-E bucket); per warp and species, FP64 sums per "
                                        "grid interval before one atomic per point and channel; densities summed "
                                        "per block in shared memory"}}


def run_reference(args, rank: int, world: int):
    """The reference arm: the CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    lib, mats, E, mat = workload_inputs(0)
    import oracle
    cores = os.cpu_count() or 1
    sample = 1_000_000
    times = []
    for s in range(args.warmup + args.steps):
        lo = (s * sample) % (N_LOOKUPS - sample)
        t0 = time.perf_counter()
        oracle.xs_lookup(lib, mats, E[lo:lo + sample], mat[lo:lo + sample], n_threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample * args.steps / tot
    line = {"impl": "reference", "metric": "XS lookups/s", "value": value, "unit": "lookups/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "CPU FP64 oracle, bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample:,} lookups of the workload per step"},
            "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_transport(mcx, synth, lib3, spec, seed, reps=1):
    import torch
    prob = synth.config3_problem(n_histories=TRANSPORT_HIST, lib=lib3)
    p = mcx.make_problem(prob, precision=spec["precision"], hash_bins=spec["hash_bins"])
    p.set_tuning(**spec["tune"])
    p.run(count=TRANSPORT_HIST // 10, particles_in_flight=spec["pif"], seed=seed)   # warm-up
    best = None
    for _ in range(reps):
        p.zero_tallies()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        p.run(particles_in_flight=spec["pif"], seed=seed)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    st = p.stats()
    tal = p.tallies()
    out = tal["outcome"].sum(0)
    p.close()
    return {"particles_per_s": TRANSPORT_HIST / (best / 1e3), "ms": best,
            "collisions_per_history": float(out[4] / TRANSPORT_HIST),
            "iterations": st["iterations"], "kernels": st["kernels"], "_tallies": tal}


# Algorithmic HBM bytes per event of the transport's event kernels: the
# particle-state fields each kernel reads and writes in the structure-of-
# arrays layout (table gathers are L2-resident and queue appends are left
# out).  Lookup: queue entry 4, E 8, material 4, flags 1 + 1, {Sigma_t,
# Sigma_a} 16, plus 8 bytes per running-sum entry it stores (rows of the
# material's species count rounded up to 4).  Flight: flags 1, problem 4,
# x y z u v w 48, cell 4, history 8, draw counter 4, {Sigma_t, Sigma_a} 16,
# material 4 read; x y z 24, draw counter 4, flags 1 written.  Collision:
# queue entry 4, flags 1, problem 4, E 8, material 4, u v w 24, history 8,
# draw counter 4, collision count 4, one 32-byte sector of the running sums
# read; E 8, u v w 24, draw counter 4, collision count 4, flags 1 written.
EVENT_BYTES = {"lookup": 34, "flight": 118, "collision": 138}
# What bounds each event kernel instead of HBM, from ncu in the bulk of the
# timed run (profiles/transport_config3_kernels.md): the unit and its share of
# its peak.
EVENT_BOUND = {"lookup": {"unit": "L1TEX (load latency: 10.9 long-scoreboard stalls per issue)", "pct_of_peak": 56.2},
               "flight": {"unit": "FP64 pipe", "pct_of_peak": 81.3},
               "collision": {"unit": "FP64 pipe", "pct_of_peak": 74.5}}


def transport_roofline(mcx, synth, lib3, peak, seed=5):
    """Per event kernel of the tuned lattice transport: device time from a
    run with kernel timing on (plain launches with CUDA events around each
    kernel), events counted on the device, algorithmic bytes per event
    (EVENT_BYTES), achieved GB/s and the fraction of the HBM peak."""
    spec = TRANSPORT_TUNED
    prob = synth.config3_problem(n_histories=TRANSPORT_HIST, lib=lib3)
    p = mcx.make_problem(prob, precision=spec["precision"], hash_bins=spec["hash_bins"])
    p.set_tuning(**spec["tune"])
    p.set_kernel_timing(True)
    p.run(count=TRANSPORT_HIST // 10, particles_in_flight=spec["pif"], seed=seed)   # warm-up
    p.zero_tallies()
    p.run(particles_in_flight=spec["pif"], seed=seed)
    ks = p.kernel_stats()
    p.close()
    ev = ks["events"]
    nbytes = {"lookup": EVENT_BYTES["lookup"] * ev["lookups"] + 8 * ev["row_entries"],
              "flight": EVENT_BYTES["flight"] * ev["flights"],
              "collision": EVENT_BYTES["collision"] * ev["collisions"]}
    counts = {"lookup": ev["lookups"], "flight": ev["flights"], "collision": ev["collisions"]}
    res = {"config": "17x17 lattice, 1e7 histories, tuned settings, kernel timing on (no graphs)"}
    for k in ("lookup", "flight", "collision"):
        ms = ks["ms"][k]
        ach = nbytes[k] / (ms / 1e3) / 1e9
        res[k] = {"bound": "hbm", "events": counts[k], "bytes_per_event": nbytes[k] / max(counts[k], 1),
                  "kernel_ms_total": ms, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                  "measured_bound": dict(EVENT_BOUND[k], source="ncu, bulk iteration of the 1e7-history run")}
    return res


def tally_z(a, b):
    """max and median over bins of |mean_a - mean_b| in standard errors of the
    difference of the two batch means (per-batch tallies [B][bins])."""
    B = a.shape[0]
    se = np.sqrt(a.var(axis=0, ddof=1) / B + b.var(axis=0, ddof=1) / B)
    d = np.abs(a.sum(0) - b.sum(0)) / B
    m = se > 0
    z = d[m] / se[m]
    return {"max": float(z.max()) if z.size else 0.0, "median": float(np.median(z)) if z.size else 0.0,
            "bins": int(m.sum())}


def time_large_library(mcx, synth, dE, dm, mat, out, perm, stream, reps=3):
    """The tuned lookup step on a library three times larger (1065 species x
    11,303 points): the 12 materials then touch ~3x the table bytes, more than
    the 126 MB L2 holds, so the records come from HBM instead of L2."""
    import torch
    lib = synth.species_library(3 * N_SPECIES, N_POINTS, LIB_SEED + 7)
    mats = synth.lookup_materials(3 * N_SPECIES, MAT_SEED + 7)
    p = mcx.Problem(None).load_tables(lib, mats, precision=TUNED["precision"], hash_bins=TUNED["hash_bins"])
    used = np.unique(mats.species)
    table_bytes = float(sum(lib.grid_offsets[s + 1] - lib.grid_offsets[s] for s in used)) * (16 + 5 * 4)

    def timed(binned):
        best = None
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if binned:
                p.xs_sort(dE, dm, perm)
            p.xs_lookup_ordered(dE, dm, perm if binned else None, out=out, flags=TUNED["flags"])
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)   # the first pass is a warm-up
        return best

    ms_b = timed(True)
    ms_n = timed(False)
    alg = algorithmic_bytes(mats, mat, 4)
    p.close()
    return {"config": "1065 species x 11,303 points x 5 channels, 12 materials (4-321 species), 1e8 lookups",
            "touched_table_bytes": table_bytes,
            "binned": {"lookups_per_s": N_LOOKUPS / (ms_b / 1e3), "ms_per_step": ms_b,
                       "achieved_alg_GBs": alg / (ms_b / 1e3) / 1e9},
            "natural_order": {"lookups_per_s": N_LOOKUPS / (ms_n / 1e3), "ms": ms_n,
                              "achieved_alg_GBs": alg / (ms_n / 1e3) / 1e9}}


def time_infinite_medium(mcx, synth, n_hist=10_000_000, seed=3):
    """Particles/s of the 8-species infinite medium (50 energy-bin flux
    tally, FP64 tables that stay in L1/L2) at 1e7 histories."""
    import torch
    prob = synth.config1_problem(n_hist)
    res = {}
    for name, tune in (("queued", dict(mode=1, block_size=128, sort_period=0)),
                       ("fullest_queue", dict(mode=2, block_size=128, sort_period=0))):
        p = mcx.make_problem(prob, precision=0, hash_bins=4000)
        p.set_tuning(**tune)
        p.run(count=n_hist // 20, particles_in_flight=2_000_000, seed=seed)   # warm-up
        p.zero_tallies()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        p.run(particles_in_flight=2_000_000, seed=seed)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out = p.tallies()["outcome"].sum(0)
        p.close()
        res[name] = {"particles_per_s": n_hist / (ms / 1e3), "ms": ms,
                     "collisions_per_history": float(out[4] / n_hist)}
    res["config"] = "8 species x 2000 points, FP64 tables, infinite medium, 1e7 histories, 2e6 in flight"
    return res


def time_eigenvalue(mcx, synth, n=1_000_000, gens=12, inactive=2, seed=11):
    """k-eigenvalue power iteration of the 17x17 lattice (fuel species
    fissile): 1e6 histories per generation, 12 generations (2 inactive),
    FP32 tables and the tuned transport settings."""
    import torch
    prob = synth.eigen_problem(n_per_gen=n)
    p = mcx.make_problem(prob, precision=1, hash_bins=TRANSPORT_TUNED["hash_bins"])
    p.set_tuning(**TRANSPORT_TUNED["tune"])
    p.run_eigenvalue(n // 10, 2, 1, particles_in_flight=TRANSPORT_TUNED["pif"], seed=seed)   # warm-up
    p.zero_tallies()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = p.run_eigenvalue(n, gens, inactive, particles_in_flight=TRANSPORT_TUNED["pif"], seed=seed)
    s = time.perf_counter() - t0        # synchronous call: the host clock brackets the device work
    p.close()
    act = slice(inactive, None)
    se = lambda a: float(a[act].std(ddof=1) / np.sqrt(len(a[act])))
    return {"config": "17x17 lattice, fuel species fissile (nu = 2.43), Maxwellian T = 1.2895 MeV, "
                      f"{n:.0e} histories x {gens} generations ({inactive} inactive), FP32 tables",
            "particles_per_s": n * gens / s, "s": s,
            "k": {"site_count": float(r["k"][act].mean()), "se": se(r["k"]),
                  "collision": float(r["k_col"][act].mean()), "collision_se": se(r["k_col"]),
                  "track_length": float(r["k_tl"][act].mean()), "track_length_se": se(r["k_tl"])},
            "sites_per_generation": [int(x) for x in r["sites"]]}


def time_batched(mcx, synth, seed=9):
    """64 lattices of uneven size (3x3 .. 17x17, 1e4 .. 2e6 histories) over the
    12-material set: one event loop over all problems (tuned) against one
    plain run per problem (FP64, full search, queueless)."""
    import torch
    lib = synth.species_library(N_SPECIES, N_POINTS, LIB_SEED).channels([synth.CH_SCATTER, synth.CH_ABSORB])
    mats = synth.lookup_materials(N_SPECIES, MAT_SEED)
    probs = synth.config5_problems(lib, mats, n_problems=64)
    total = sum(p.n_histories for p in probs)
    res = {"config": f"64 lattices, n in 3..17, {total:,} histories, 12 materials of 4-321 species"}
    # tuned: one persistent loop, shared FP32 tables
    spec = BATCHED_TUNED
    base = mcx.Problem(probs[0]).load_tables(lib, mats, precision=spec["precision"], hash_bins=spec["hash_bins"])
    hs = [base] + [mcx.Problem(pr).share_tables(base) for pr in probs[1:]]
    base.set_tuning(**spec["tune"])
    nh = [pr.n_histories for pr in probs]
    mcx.batch_run(hs, [max(1, n // 50) for n in nh], spec["pif"], seed)   # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    mcx.batch_run(hs, nh, spec["pif"], seed)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    res["tuned"] = {"particles_per_s": total / (ms / 1e3), "ms": ms, "stats": base.stats()}
    for h in hs:
        h.close()
    # plain: one run per problem
    plain = mcx.Problem(probs[0]).load_tables(lib, mats, precision=0, hash_bins=0)
    ph = [plain] + [mcx.Problem(pr).share_tables(plain) for pr in probs[1:]]
    for h in ph:
        h.set_tuning(**TRANSPORT_PLAIN["tune"])
    ph[0].run(count=1000, particles_in_flight=TRANSPORT_PLAIN["pif"], seed=seed)     # warm-up
    torch.cuda.synchronize()
    a.record()
    for h, pr in zip(ph, probs):
        h.run(particles_in_flight=TRANSPORT_PLAIN["pif"], seed=seed)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    res["plain"] = {"particles_per_s": total / (ms / 1e3), "ms": ms}
    for h in ph:
        h.close()
    return res


def run_leg(args):
    """One transport or eigenvalue leg alone (tuned settings), one JSON line."""
    global TRANSPORT_HIST
    from paper_2402_09222_b300 import mcx, synth
    TRANSPORT_HIST = args.histories
    if args.workload == "transport":
        r = time_transport(mcx, synth, synth.config3_library(), TRANSPORT_TUNED, seed=5)
        r.pop("_tallies")
    else:
        r = time_eigenvalue(mcx, synth, n=args.histories)
    print(json.dumps({"workload": args.workload, **r}), flush=True)


def main():
    global N_LOOKUPS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcx", choices=["mcx", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain form, e2e, transport and CPU legs (profiling runs)")
    ap.add_argument("--lookups", type=int, default=N_LOOKUPS,
                    help="lookups per step (smaller cases for profiler captures)")
    ap.add_argument("--workload", default="lookup", choices=["lookup", "transport", "eigenvalue"],
                    help="transport / eigenvalue: time only that leg (profiler captures)")
    ap.add_argument("--histories", type=int, default=TRANSPORT_HIST,
                    help="histories of the transport leg")
    args = ap.parse_args()
    if args.lookups != N_LOOKUPS:
        N_LOOKUPS = args.lookups
        WORKLOAD = WORKLOAD.replace("1e8 lookups", f"{N_LOOKUPS:.3g} lookups")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "lookup":
        return run_leg(args)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2402_09222_b300 import mcx, synth

    lib, mats, E, mat = workload_inputs(rank)
    dE = torch.as_tensor(E, device="cuda")
    dm = torch.as_tensor(mat, device="cuda")
    out = torch.empty((N_LOOKUPS, 5), dtype=torch.float64, device="cuda")
    perm = torch.empty(N_LOOKUPS, dtype=torch.int32, device="cuda")
    Eb = torch.empty(N_LOOKUPS, dtype=torch.float64, device="cuda")   # inputs in the binned order
    mb = torch.empty(N_LOOKUPS, dtype=torch.int32, device="cuda")
    p = mcx.Problem(None, device=local).load_tables(lib, mats, precision=TUNED["precision"],
                                                    hash_bins=TUNED["hash_bins"])
    stream = torch.cuda.current_stream()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        p.xs_sort_inputs(dE, dm, perm, Eb, mb)
        if evs:
            evs[1].record(stream)
        p.xs_lookup_ordered(Eb, mb, perm, out=out, flags=TUNED["flags"] | mcx.LOOKUP_BINNED_INPUTS)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    lookup_ms = [e[1].elapsed_time(e[2]) for e in evs]
    sort_ms = [e[0].elapsed_time(e[1]) for e in evs]
    if world > 1:
        from paper_2402_09222_b300 import shard
        total_ms = shard.max_over_ranks(total_ms)
    value = world * N_LOOKUPS * args.steps / (total_ms / 1e3)

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(mats, mat, 4)
    comp = compulsory_bytes(lib, mats, len(mat))
    lk = sum(lookup_ms) / len(lookup_ms)
    tr = lookup_traffic()
    traffic = tr["dram_bytes_per_launch"] if tr else None
    # the roof: HBM; achieved = DRAM bytes one launch moved (ncu, this kernel
    # source) over the launch's CUDA-event time
    achieved = traffic / (lk / 1e3) / 1e9 if traffic else comp / (lk / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_xs_lookup_warp2, round-linear sums (binned order)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "frac_basis": ("DRAM bytes per launch (ncu dram__bytes_read + write, this kernel source) / "
                               "the launch's CUDA-event time" if traffic else
                               "compulsory bytes / the launch's CUDA-event time (no current ncu traffic)"),
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json)" if peak_kind == "measured"
                else "fallback 6400 GB/s",
                "lookup_kernel_ms": lk, "sort_ms": sum(sort_ms) / len(sort_ms),
                "compulsory_bytes_per_launch": comp,
                "compulsory_frac": comp / (lk / 1e3) / 1e9 / peak,
                "work_rate_GBs": alg / (lk / 1e3) / 1e9,
                "algorithmic_bytes_per_launch": alg}
    if tr:
        roofline["traffic_source"] = tr.get("source")
        if tr.get("binning_per_step"):
            # the whole step: binning kernels and the lookup, DRAM bytes over the step's time
            sb = sum(v["dram_read"] + v["dram_write"] for v in tr["binning_per_step"].values()) + traffic
            roofline["step"] = {"dram_bytes": sb, "ms": total_ms / args.steps,
                                "achieved": sb / (total_ms / args.steps / 1e3) / 1e9,
                                "frac": sb / (total_ms / args.steps / 1e3) / 1e9 / peak}
        if tr.get("issue_active_frac") is not None:
            roofline["issue_active_frac"] = tr["issue_active_frac"]
    roofline["note"] = ("frac: DRAM traffic measured by ncu over the kernel's own time. compulsory_bytes: the "
                        "inputs, permutation and outputs once plus every table record and hash window the "
                        "materials touch once. work_rate_GBs: the definition's bytes (every species' "
                        "records and energies per lookup, 4,568 B per lookup on average) per second; binning "
                        "lets a warp's lookups share each species' records, so that rate is not an HBM figure "
                        "and exceeds the peak. issue_active_frac: the share of cycles the kernel issued an "
                        "instruction (ncu, a 2e7-lookup capture): the binned kernel is bound by instruction "
                        "issue and load latency, not by HBM")

    # the same kernel family on the natural (unbinned) order, where every
    # species' records are a real gather from L2/HBM: the per-lane kernel
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p.xs_lookup_ordered(dE, dm, None, out=out, flags=TUNED["flags"])
    a.record(stream)
    p.xs_lookup_ordered(dE, dm, None, out=out, flags=TUNED["flags"])
    b.record(stream)
    torch.cuda.synchronize()
    nat_ms = a.elapsed_time(b)
    roofline["natural_order"] = {"kernel": "k_xs_lookup_fast (per-lane form)", "lookup_kernel_ms": nat_ms,
                                 "lookups_per_s": N_LOOKUPS / (nat_ms / 1e3),
                                 "work_rate_GBs": alg / (nat_ms / 1e3) / 1e9}
    # the bit-identical per-lookup form on the same binned order (every
    # species' term per lookup), beside the round-linear sums timed above
    p.xs_lookup_ordered(Eb, mb, perm, out=out, flags=PER_LOOKUP_FLAGS | mcx.LOOKUP_BINNED_INPUTS)
    a.record(stream)
    p.xs_lookup_ordered(Eb, mb, perm, out=out, flags=PER_LOOKUP_FLAGS | mcx.LOOKUP_BINNED_INPUTS)
    b.record(stream)
    torch.cuda.synchronize()
    pl_ms = a.elapsed_time(b)
    roofline["per_lookup_form"] = {"kernel": "k_xs_lookup_warp2, per-lookup sums (bit-identical to the "
                                             "per-lane form)", "lookup_kernel_ms": pl_ms,
                                   "lookups_per_s": N_LOOKUPS / (pl_ms / 1e3)}
    if tr and tr.get("natural_dram_bytes_per_launch"):
        nd = tr["natural_dram_bytes_per_launch"]
        roofline["natural_order"].update(traffic=nd, achieved=nd / (nat_ms / 1e3) / 1e9,
                                         frac=nd / (nat_ms / 1e3) / 1e9 / peak)

    line = {"metric": "XS lookups/s",
            "value": value, "unit": "lookups/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 tables, f64 energies and search",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "tables": "FP32", "hash_bins": TUNED["hash_bins"],
                       "arithmetic": "fast (<=1e-6 rel), round-linear sums",
                       "binning": "material x log-E buckets, ~128 lookups each, in two levels; energies and "
                                  "materials carried into the binned order",
                       "l2": "inputs 1.2 GB + outputs 4 GB per step exceed the 126 MB L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": roofline, "gpu_launches": 6 * args.steps,
            "clocks": clocks.summary()}

    if not args.no_extras:
        # end to end through the C ABI with host buffers (copies in the timed region)
        Eh = torch.as_tensor(E).pin_memory()
        mh = torch.as_tensor(mat).pin_memory()
        oh = torch.empty((N_LOOKUPS, 5), dtype=torch.float64).pin_memory()
        # one untimed full-size call (it allocates the pipeline's staging),
        # then the mean of E2E_CALLS timed calls
        p.xs_lookup_host(Eh, mh, oh, flags=HOST_FLAGS)
        if world > 1:
            dist.barrier()
        t0w = time.perf_counter()
        for _ in range(E2E_CALLS):
            p.xs_lookup_host(Eh, mh, oh, flags=HOST_FLAGS)
        e2e_s = (time.perf_counter() - t0w) / E2E_CALLS
        if world > 1:
            from paper_2402_09222_b300 import shard
            e2e_s = shard.max_over_ranks(e2e_s)
        line["e2e"] = {"value": world * N_LOOKUPS / e2e_s, "unit": "lookups/s",
                       "h2d_bytes_per_step": N_LOOKUPS * 12, "d2h_bytes_per_step": N_LOOKUPS * 40,
                       "path": "mcx_xs_lookup_host, pinned host buffers, 2M-lookup chunks binned and looked up on 3 streams; mean of 3 calls after one untimed call",
                       "host_link": host_link_bandwidth(oh, out)}
        del oh
        # the same with FP32 outputs (the compensated sums rounded once; still
        # within 1e-6 of the definition): half the device-to-host bytes
        oh32 = torch.empty((N_LOOKUPS, 5), dtype=torch.float32).pin_memory()
        f32 = HOST_FLAGS | mcx.LOOKUP_OUT32
        p.xs_lookup_host(Eh, mh, oh32, flags=f32)
        t0w = time.perf_counter()
        for _ in range(E2E_CALLS):
            p.xs_lookup_host(Eh, mh, oh32, flags=f32)
        e2e32 = (time.perf_counter() - t0w) / E2E_CALLS
        if world > 1:
            e2e32 = shard.max_over_ranks(e2e32)
        out32 = torch.empty((N_LOOKUPS, 5), dtype=torch.float32, device="cuda")
        p.xs_lookup_ordered(dE, dm, perm, out=out32, flags=TUNED["flags"] | mcx.LOOKUP_OUT32)
        a32, b32 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a32.record(stream)
        p.xs_sort(dE, dm, perm)
        p.xs_lookup_ordered(dE, dm, perm, out=out32, flags=TUNED["flags"] | mcx.LOOKUP_OUT32)
        b32.record(stream)
        torch.cuda.synchronize()
        line["fp32_outputs"] = {
            "e2e": {"value": world * N_LOOKUPS / e2e32, "unit": "lookups/s", "h2d_bytes_per_step": N_LOOKUPS * 12,
                    "d2h_bytes_per_step": N_LOOKUPS * 20,
                    "path": "4M-lookup chunks on 3 streams; mean of 3 calls after one untimed call"},
            "device_step_lookups_per_s": N_LOOKUPS / (a32.elapsed_time(b32) / 1e3),
            "note": "MCX_LOOKUP_OUT32: outputs rounded once to FP32 (within the 1e-6 bound); "
                    "the headline value keeps FP64 outputs"}
        del Eh, mh, oh32, out32
    if rank == 0 and world == 1 and not args.no_extras:
        # plain form: FP64 tables, exact arithmetic, full binary search, natural order
        # the tuned output (FP32 tables, fast arithmetic, binned) for the precision block
        p.xs_sort(dE, dm, perm)
        p.xs_lookup_ordered(dE, dm, perm, out=out, flags=TUNED["flags"])
        out64 = torch.empty_like(out)
        pp = mcx.Problem(None, device=local).load_tables(lib, mats, precision=0, hash_bins=0)
        pp.xs_lookup(dE, dm, out=out64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pp.xs_lookup(dE, dm, out=out64)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        line["plain"] = {"lookups_per_s": N_LOOKUPS / (pms / 1e3), "ms": pms,
                         "form": "FP64 tables, exact FP64 arithmetic, full binary search, unsorted",
                         "work_rate_GBs": algorithmic_bytes(mats, mat, 8) / (pms / 1e3) / 1e9}
        pp.close()
        # FP64 against FP32 tables at equal algorithm (hash grid, binned order,
        # exact arithmetic), and the errors of FP32 tables against the FP64
        # definition (the plain form's outputs equal the definition bit for bit)
        p64 = mcx.Problem(None, device=local).load_tables(lib, mats, precision=0, hash_bins=TUNED["hash_bins"])
        out_e = torch.empty_like(out)

        def timed_exact(h, o):
            h.xs_lookup_ordered(dE, dm, perm, out=o, flags=mcx.LOOKUP_EXACT)
            a.record(stream)
            h.xs_lookup_ordered(dE, dm, perm, out=o, flags=mcx.LOOKUP_EXACT)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        ms64 = timed_exact(p64, out_e)
        p64.close()
        ms32 = timed_exact(p, out_e)

        def rel_err(o, ref=out64):
            r = ((o - ref).abs() / ref.abs().clamp_min(1e-300))
            return {"max": [float(x) for x in r.max(0).values.cpu()],
                    "median": [float(x) for x in r.median(0).values.cpu()]}

        line["precision_error"] = {
            "reference": "FP64 tables, exact arithmetic, full search (equal to the FP64 definition bit for bit)",
            "channels": ["total", "scatter", "absorb", "fission", "nu-fission"],
            "lookup_fp32_tables_exact": rel_err(out_e),
            "lookup_fp32_tables_fast_binned": rel_err(out),
            "fast_binned_vs_exact_on_fp32_tables": rel_err(out, out_e),
            "bound": "2^-24 = 5.96e-8 (exact) and 1e-6 + 2^-24 (fast), relative"}
        line["fp64_vs_fp32_tables"] = {
            "form": "exact arithmetic, 68,400 hash bins, binned order (the same permutation)",
            "fp64_tables": {"ms": ms64, "lookups_per_s": N_LOOKUPS / (ms64 / 1e3)},
            "fp32_tables": {"ms": ms32, "lookups_per_s": N_LOOKUPS / (ms32 / 1e3)},
            "fp32_tables_fast_arithmetic": {"ms": lk, "lookups_per_s": N_LOOKUPS / (lk / 1e3)}}
        del out64, out_e
        # transport, 17x17 lattice, 1e7 histories
        lib3 = synth.config3_library()
        line["transport"] = {
            "metric": "particles/s", "config": "17x17 lattice, 40/4/3-species materials, 1e7 histories",
            "tuned": time_transport(mcx, synth, lib3, TRANSPORT_TUNED, seed=5),
            "plain": time_transport(mcx, synth, lib3, TRANSPORT_PLAIN, seed=5),
            "tuned_settings": {k: v for k, v in TRANSPORT_TUNED.items()},
            # the same settings with the fullest-queue policy decided on the device
            "tuned_fullest_queue": time_transport(mcx, synth, lib3, TRANSPORT_FULLEST, seed=5),
        }
        tt, tp = line["transport"]["tuned"].pop("_tallies"), line["transport"]["plain"].pop("_tallies")
        line["transport"]["tuned_fullest_queue"].pop("_tallies", None)
        line["precision_error"]["lattice_tallies_fp32_vs_fp64_tables_se"] = {
            k: tally_z(tt[k], tp[k]) for k in ("flux", "absorb")}
        line["transport"]["roofline"] = transport_roofline(mcx, synth, lib3, peak)
        line["transport"]["cpu_baseline"] = cpu_transport(synth, lib3)
        line["transport"]["inflight_sweep"] = time_inflight_sweep(mcx, synth, lib3)
        line["derivatives"] = time_derivatives(mcx, synth, lib3)
        line["precision_error"]["derivative_tallies_fp32_vs_fp64_tables_se"] = \
            line["derivatives"].pop("fp32_vs_fp64_tables_dabsorb_se")
        line["infinite_medium"] = time_infinite_medium(mcx, synth)
        line["eigenvalue"] = time_eigenvalue(mcx, synth)
        line["large_library"] = time_large_library(mcx, synth, dE, dm, mat, out, perm, stream)
        line["batched"] = time_batched(mcx, synth)
        line["cpu_baseline"] = cpu_baseline(lib, mats, E, mat)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def kernel_source_hash() -> str:
    """Hash of the lookup kernel's source and of the binning parameters that
    set the order it reads in, with comments and blank space removed: the
    recorded DRAM traffic stays valid across comment edits and reads null
    after any change to the code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("xs_fast.cu", "mcx_internal.cuh", "kernels.h"):
        src = open(os.path.join(ROOT, "paper_2402_09222_b300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
