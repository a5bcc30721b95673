"""GPU parity of event-based transport against the CPU oracle.

Histories are matched through the shared Philox stream definition: per-history
collision counts must be identical, tallies within 1e-9 relative, and nothing
may depend on the particles-in-flight count, queueing mode, binning, hash bins,
block size or graph replay (the paper: the in-flight count does not affect the
numerical characteristics; sorting only improves locality).
"""
import numpy as np
import pytest

import bench   # the launch settings the benchmark times
import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

TALLY_RTOL = 1e-9


@pytest.fixture(scope="module")
def mcx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx as m
    return m


def run_gpu(mcx, prob, precision=0, H=4000, flags=None, pif=100_000, seed=7, first=0, count=None,
            **tune):
    flags = mcx.FLAG_HISTORY_DEBUG if flags is None else flags
    p = mcx.make_problem(prob, precision=precision, hash_bins=H, flags=flags)
    p.set_tuning(**tune)
    count = prob.n_histories - first if count is None else count
    p.run(first=first, count=count, particles_in_flight=pif, seed=seed)
    res = p.tallies()
    if flags & mcx.FLAG_HISTORY_DEBUG:
        res["ncoll"] = p.history_debug(count)
    res["stats"] = p.stats()
    p.close()
    return res


def assert_tallies_close(g, o, keys=("flux", "absorb", "outcome")):
    for k in keys:
        scale = max(np.abs(o[k]).max(), 1e-300)
        np.testing.assert_allclose(g[k], o[k], rtol=TALLY_RTOL, atol=TALLY_RTOL * scale, err_msg=k)


@pytest.fixture(scope="module")
def config1():
    prob = synth.config1_problem(10_000)
    return prob, oracle.transport(prob, seed=7, history_debug=True, n_threads=8)


TUNINGS = [
    dict(mode=0, pif=10_000, sort_period=0, block_size=256, H=4000, use_graph=1),
    dict(mode=0, pif=777, sort_period=0, block_size=128, H=0, use_graph=0),
    dict(mode=1, pif=3000, sort_period=0, block_size=256, H=100, use_graph=1),
    dict(mode=1, pif=3000, sort_period=2, sort_threshold=0, block_size=512, H=4000, use_graph=1),
    dict(mode=1, pif=200_000, sort_period=1, sort_threshold=10, block_size=64, H=100_000, use_graph=1,
         iters_per_sync=3),
    # fullest-queue mode: a small buffer makes every ring wrap many times
    dict(mode=2, pif=10_000, sort_period=0, block_size=256, H=4000, use_graph=1),
    dict(mode=2, pif=333, sort_period=1, sort_threshold=0, block_size=128, H=100, use_graph=1,
         iters_per_sync=5),
    dict(mode=2, pif=5000, sort_period=2, sort_threshold=100, block_size=64, H=0, use_graph=0),
]


@pytest.mark.parametrize("tu", TUNINGS, ids=lambda t: "-".join(f"{k}{v}" for k, v in t.items()))
def test_config1_history_matched_for_every_tuning(mcx, config1, tu):
    prob, ref = config1
    tu = dict(tu)
    pif, H = tu.pop("pif"), tu.pop("H")
    g = run_gpu(mcx, prob, H=H, pif=pif, **tu)
    assert np.array_equal(g["ncoll"], ref["ncoll"])
    assert_tallies_close(g, ref)
    assert g["stats"]["iterations"] > 0


def test_config1_fp32_tables(mcx):
    prob = synth.config1_problem(4000)
    ref_prob = synth.config1_problem(4000)
    ref_prob.lib = prob.lib.fp32_rounded()
    ref = oracle.transport(ref_prob, seed=9, history_debug=True, n_threads=8)
    g = run_gpu(mcx, prob, precision=mcx.FP32, pif=1500, seed=9, mode=1, sort_period=3, sort_threshold=0)
    assert np.array_equal(g["ncoll"], ref["ncoll"])
    assert_tallies_close(g, ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_source_above_the_grids(mcx, precision):
    """A source at 5e7 eV, above every species' grid (top 2e7): the first
    lookups fall in the grids' last intervals, where the transport lookup
    clamps the interpolation fraction to 1 instead of using the stored
    slopes; history-matched against the oracle's clamped definition."""
    prob = synth.config1_problem(3000)
    prob.E0 = 5.0e7
    ref_prob = synth.config1_problem(3000)
    ref_prob.E0 = 5.0e7
    if precision:
        ref_prob.lib = prob.lib.fp32_rounded()
    ref = oracle.transport(ref_prob, seed=13, history_debug=True, n_threads=8)
    g = run_gpu(mcx, prob, precision=precision, pif=1000, seed=13, mode=1, sort_period=0)
    assert np.array_equal(g["ncoll"], ref["ncoll"])
    assert_tallies_close(g, ref)


@pytest.fixture(scope="module")
def lattice():
    prob = synth.config3_problem(n_histories=5000)
    return prob, oracle.transport(prob, seed=11, history_debug=True, n_threads=8)


@pytest.mark.parametrize("mode,sort_period", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_lattice_history_matched(mcx, lattice, mode, sort_period):
    prob, ref = lattice
    g = run_gpu(mcx, prob, pif=1234, seed=11, mode=mode, sort_period=sort_period, sort_threshold=0)
    match = np.mean(g["ncoll"] == ref["ncoll"])
    assert match >= 0.9999, match
    if match == 1.0:
        assert_tallies_close(g, ref)
    out = g["outcome"].sum(0)
    assert out[:4].sum() == prob.n_histories


@pytest.mark.parametrize("mode", [1, 2])
def test_lattice_derivative_tallies(mcx, mode):
    prob = synth.config3_problem(n_histories=3000, lattice_n=9)
    ref = oracle.transport(prob, seed=13, derivatives=True, history_debug=True, n_threads=8)
    g = run_gpu(mcx, prob, pif=1000, seed=13, flags=mcx.FLAG_DERIVATIVES | mcx.FLAG_HISTORY_DEBUG, mode=mode)
    assert np.array_equal(g["ncoll"], ref["ncoll"])
    assert_tallies_close(g, ref, keys=("flux", "absorb", "outcome", "dflux", "dabsorb", "doutcome"))


def test_slab_and_infinite_closed_forms_on_gpu(mcx):
    Sa, L = 1.3, 1.1
    lib = synth.flat_library(0.0, Sa)
    mats = synth.make_materials([[0]], [[1.0]])
    prob = synth.slab_problem(lib, mats, L, 20_000)
    ref = oracle.transport(prob, seed=15, derivatives=True)
    g = run_gpu(mcx, prob, H=0, pif=4096, seed=15, flags=mcx.FLAG_DERIVATIVES, mode=1)
    assert_tallies_close(g, ref, keys=("flux", "absorb", "outcome", "dflux", "dabsorb", "doutcome"))
    k = g["outcome"][:, 1].sum()
    dk = g["doutcome"][:, 1, 0].sum()
    assert abs(dk - (-Sa * L) * k) <= 1e-9 * abs(dk)


def test_resume_from_a_history_offset(mcx, config1):
    prob, ref = config1
    p = mcx.make_problem(prob, flags=mcx.FLAG_HISTORY_DEBUG)
    p.run(first=0, count=4321, particles_in_flight=2000, seed=7)
    n1 = p.history_debug(4321)
    p.run(first=4321, count=prob.n_histories - 4321, particles_in_flight=2000, seed=7)
    n2 = p.history_debug(prob.n_histories - 4321)
    assert np.array_equal(np.concatenate([n1, n2]), ref["ncoll"])
    assert_tallies_close(p.tallies(), ref)


def test_reused_handle_honours_a_smaller_in_flight_count(mcx, config1):
    """A handle keeps its largest particle buffer; a later run with fewer
    particles in flight must still use only that many slots."""
    prob, ref = config1
    p = mcx.make_problem(prob, flags=mcx.FLAG_HISTORY_DEBUG)
    p.run(particles_in_flight=5000, seed=7)
    it_big = p.stats()["iterations"]
    p.zero_tallies()
    p.run(particles_in_flight=500, seed=7)
    it_small = p.stats()["iterations"]
    assert it_small > 2 * it_big, (it_small, it_big)
    assert np.array_equal(p.history_debug(prob.n_histories), ref["ncoll"])
    fresh = mcx.make_problem(prob)
    fresh.run(particles_in_flight=500, seed=7)
    assert abs(fresh.stats()["iterations"] - it_small) <= 0.05 * it_small


@pytest.mark.parametrize("mode", [0, 2])
def test_iteration_cap_returns_an_error_and_the_handle_stays_usable(mcx, config1, mode):
    prob, ref = config1
    p = mcx.make_problem(prob)
    p.set_tuning(mode=mode, max_event_iters=5, iters_per_sync=2)
    with pytest.raises(mcx.McxError, match="ITER_LIMIT"):
        p.run(particles_in_flight=1000, seed=7)
    p.zero_tallies()
    p.set_tuning(mode=mode)
    p.run(particles_in_flight=1000, seed=7)
    assert_tallies_close(p.tallies(), ref)


def test_fullest_queue_steps(mcx, config1):
    """Fullest-queue mode: every step runs exactly one event kernel, all three
    are chosen, and the step count is close to three event sweeps per
    iteration of the plain queued loop on the same buffer."""
    prob, ref = config1
    q = run_gpu(mcx, prob, pif=2000, mode=1)
    f = run_gpu(mcx, prob, pif=2000, mode=2)
    assert np.array_equal(f["ncoll"], ref["ncoll"])
    sel = f["stats"]["selected"]
    assert sum(sel.values()) == f["stats"]["iterations"]
    assert min(sel.values()) > 0
    assert q["stats"]["selected"] == dict(lookup=0, flight=0, collision=0)
    assert f["stats"]["iterations"] <= 6 * q["stats"]["iterations"]


@pytest.mark.parametrize("mode", [1, 2])
def test_batched_uneven_problems(mcx, mode):
    lib = synth.species_library(60, 1500, 301).channels([synth.CH_SCATTER, synth.CH_ABSORB])
    mats = synth.lookup_materials(60, 302, n_materials=6)
    probs = synth.config5_problems(lib, mats, n_problems=7, seed=303, hist_lo=100, hist_hi=3000)
    refs = [oracle.transport(pr, seed=21, history_debug=True, n_threads=8) for pr in probs]
    base = mcx.Problem(probs[0], flags=mcx.FLAG_HISTORY_DEBUG).load_tables(lib, mats, hash_bins=1000)
    handles = [base] + [mcx.Problem(pr, flags=mcx.FLAG_HISTORY_DEBUG).share_tables(base) for pr in probs[1:]]
    base.set_tuning(mode=mode, sort_period=2, sort_threshold=0)
    mcx.batch_run(handles, [pr.n_histories for pr in probs], particles_in_flight=2500, seed=21)
    for h, pr, ref in zip(handles, probs, refs):
        nc = h.history_debug(pr.n_histories)
        assert np.mean(nc == ref["ncoll"]) >= 0.9999
        if np.array_equal(nc, ref["ncoll"]):
            assert_tallies_close(h.tallies(), ref)


N_SAMPLED = 10_000
MATCH_MIN = 0.9999


def _assert_batch_matches(g, ref, b, ncoll_match):
    """Tallies of batch b against the oracle's run of that batch alone:
    within 1e-9 relative where every history's collision count matched,
    else within 3 standard errors (from the spread of the GPU's batches)."""
    for k in ("flux", "absorb", "outcome"):
        got, want = g[k][b], ref[k][b]
        if ncoll_match:
            scale = max(np.abs(want).max(), 1e-300)
            np.testing.assert_allclose(got, want, rtol=TALLY_RTOL, atol=TALLY_RTOL * scale, err_msg=k)
        else:
            se = g[k].std(axis=0, ddof=1)
            assert np.all(np.abs(got - want) <= 3 * se + 1e-9 * np.abs(want)), k


@pytest.mark.parametrize("mode", [1, 2])
def test_config3_full_size_sampled(mcx, mode):
    """1e7 histories of the 17x17 lattice in exactly the launch the benchmark
    times (FP32 tables, its hash bins, particles in flight, block size, sort
    period and threshold; mode 2 is the fullest-queue variant of the same
    settings).  10,000 sampled histories re-run one by one in the oracle
    (FP32-rounded tables) must match their collision counts at >= 99.99 %
    (a flight-length logarithm one ulp away from the host's can flip a
    collision-versus-surface decision); the first batch (500,000 contiguous
    histories) is run whole in the oracle and its tallies compared; the
    outcome balance holds on the whole run."""
    import os
    spec = bench.TRANSPORT_TUNED if mode == 1 else bench.TRANSPORT_FULLEST
    n = bench.TRANSPORT_HIST
    prob = synth.config3_problem(n_histories=n)
    g = run_gpu(mcx, prob, precision=spec["precision"], H=spec["hash_bins"], pif=spec["pif"], seed=5,
                **spec["tune"])
    rp = synth.config3_problem(n_histories=n, lib=prob.lib.fp32_rounded())
    cores = os.cpu_count() or 1
    idx = np.sort(np.random.default_rng(6).choice(n, N_SAMPLED, replace=False))
    ref = oracle.transport_histories(rp, 5, idx, n_threads=cores)
    rate = float(np.mean(g["ncoll"][idx] == ref))
    print(f"\nconfig3 mode {mode}: sampled collision-count match {rate:.6f} "
          f"({int(np.sum(g['ncoll'][idx] != ref))} of {N_SAMPLED} differ)")
    assert rate >= MATCH_MIN, rate
    nb = n // prob.n_batches
    rb = oracle.transport(rp, seed=5, first=0, count=nb, history_debug=True, n_threads=cores)
    same = g["ncoll"][:nb] == rb["ncoll"]
    print(f"config3 mode {mode}: batch 0 ({nb} histories) collision-count match {np.mean(same):.6f}")
    assert np.mean(same) >= MATCH_MIN
    _assert_batch_matches(g, rb, 0, bool(same.all()))
    out = g["outcome"].sum(0)
    assert out[:4].sum() == prob.n_histories
    assert out[4] == g["ncoll"].sum()
    d = g["absorb"].sum(1) - g["outcome"][:, 0]
    assert abs(d.mean()) <= 3 * d.std(ddof=1) / np.sqrt(len(d))


def test_config5_full_size_sampled(mcx):
    """The 64 uneven lattices of the batched benchmark (2.76e7 histories) in
    one event loop with the benchmark's own settings: 10,000 histories
    sampled over the problems (in proportion to their sizes) re-run one by
    one in the oracle (FP32-rounded tables) match their collision counts at
    >= 99.99 %, the smallest problem is compared whole (tallies too), and
    each problem's histories all end in its own outcome tallies."""
    import os
    spec = bench.BATCHED_TUNED
    lib = synth.species_library(bench.N_SPECIES, bench.N_POINTS, bench.LIB_SEED).channels(
        [synth.CH_SCATTER, synth.CH_ABSORB])
    mats = synth.lookup_materials(bench.N_SPECIES, bench.MAT_SEED)
    probs = synth.config5_problems(lib, mats, n_problems=64)
    base = mcx.Problem(probs[0], flags=mcx.FLAG_HISTORY_DEBUG).load_tables(
        lib, mats, precision=spec["precision"], hash_bins=spec["hash_bins"])
    hs = [base] + [mcx.Problem(pr, flags=mcx.FLAG_HISTORY_DEBUG).share_tables(base) for pr in probs[1:]]
    base.set_tuning(**spec["tune"])
    nh = np.array([pr.n_histories for pr in probs])
    mcx.batch_run(hs, list(nh), particles_in_flight=spec["pif"], seed=9)
    lib32 = lib.fp32_rounded()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(17)
    picks = np.sort(rng.choice(int(nh.sum()), N_SAMPLED, replace=False))
    starts = np.concatenate([[0], np.cumsum(nh)])
    matched = total = 0
    smallest = int(np.argmin(nh))
    for i, (h, pr) in enumerate(zip(hs, probs)):
        nc = h.history_debug(pr.n_histories)
        tal = h.tallies()
        out = tal["outcome"].sum(0)
        assert out[:4].sum() == pr.n_histories
        assert out[4] == nc.sum()
        rp = synth.Problem(pr.geometry, lib32, pr.mats, lattice_n=pr.lattice_n,
                           region_material=pr.region_material, problem_id=pr.problem_id,
                           n_histories=pr.n_histories)
        mine = picks[(picks >= starts[i]) & (picks < starts[i + 1])] - starts[i]
        if len(mine):
            ref = oracle.transport_histories(rp, 9, mine, n_threads=cores)
            matched += int(np.sum(nc[mine] == ref))
            total += len(mine)
        if i == smallest:
            whole = oracle.transport(rp, seed=9, history_debug=True, n_threads=cores)
            same = nc == whole["ncoll"]
            assert np.mean(same) >= MATCH_MIN
            if same.all():
                assert_tallies_close(tal, whole)
    rate = matched / total
    print(f"\nconfig5: sampled collision-count match {rate:.6f} ({total - matched} of {total} differ)")
    assert total == N_SAMPLED
    assert rate >= MATCH_MIN, (matched, total)
    for h in hs:
        h.close()


def test_simulated_allocation_failures_are_errors_and_leave_handles_usable(mcx, config1, monkeypatch):
    """Host-side fault injection (MCX_FAIL_ALLOC_AFTER): an allocation that
    fails inside problem creation, table loading or the particle buffer
    returns MCX_ERR_OOM, and the handles work again once it is lifted."""
    prob, ref = config1
    monkeypatch.setenv("MCX_FAIL_ALLOC_AFTER", "0")
    with pytest.raises(mcx.McxError, match="OOM"):
        mcx.Problem(prob)
    monkeypatch.delenv("MCX_FAIL_ALLOC_AFTER")
    p = mcx.Problem(prob)
    monkeypatch.setenv("MCX_FAIL_ALLOC_AFTER", "3")
    with pytest.raises(mcx.McxError, match="OOM"):
        p.load_tables(prob.lib, prob.mats, hash_bins=4000)
    monkeypatch.delenv("MCX_FAIL_ALLOC_AFTER")
    p.load_tables(prob.lib, prob.mats, hash_bins=4000)
    monkeypatch.setenv("MCX_FAIL_ALLOC_AFTER", "0")
    with pytest.raises(mcx.McxError, match="OOM"):
        p.run(particles_in_flight=1000, seed=7)
    monkeypatch.delenv("MCX_FAIL_ALLOC_AFTER")
    p.zero_tallies()
    p.run(particles_in_flight=1000, seed=7)
    assert_tallies_close(p.tallies(), ref)
    p.close()


def test_kernel_timing_mode_changes_nothing(mcx, lattice):
    """With kernel timing on (plain launches, events around the event
    kernels) the run is history-matched as before; the per-kernel times are
    positive and the event counts add up (queued mode)."""
    prob, ref = lattice
    p = mcx.make_problem(prob, flags=mcx.FLAG_HISTORY_DEBUG)
    p.set_tuning(mode=1, sort_period=1, sort_threshold=0)
    p.set_kernel_timing(True)
    p.run(particles_in_flight=1234, seed=11)
    nc = p.history_debug(prob.n_histories)
    assert np.mean(nc == ref["ncoll"]) >= 0.9999
    g = p.tallies()
    if np.array_equal(nc, ref["ncoll"]):
        assert_tallies_close(g, ref)
    ks = p.kernel_stats()
    assert all(v > 0 for v in ks["ms"].values()), ks
    ev = ks["events"]
    assert ev["collisions"] == int(g["outcome"][:, 4].sum())
    assert ev["lookups"] >= prob.n_histories and ev["flights"] >= max(ev["collisions"], prob.n_histories)
    sizes = np.diff(prob.mats.offsets)
    assert 4 * ev["lookups"] <= ev["row_entries"] <= ((sizes.max() + 3) // 4 * 4) * ev["lookups"]
    p.set_kernel_timing(False)
    p.zero_tallies()
    p.run(particles_in_flight=1234, seed=11)
    assert p.kernel_stats()["ms"]["lookup"] == -1.0
    assert np.array_equal(p.history_debug(prob.n_histories), nc)
    p.close()
