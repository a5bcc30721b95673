"""The autotuner driving the real event loop on the GPU: the default
configuration is the baseline, a configuration that runs past 1.5x the
baseline is stopped by the library's host time limit (no GPU work is killed)
and recorded as a timeout, and the best configuration found is no slower
than the baseline."""
import pytest

from paper_2402_09222_b300 import synth, tuner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx as m
    return m


def test_time_limit_stops_a_run_and_the_handle_recovers(mcx):
    prob = synth.config3_problem(n_histories=400_000)
    p = mcx.make_problem(prob, precision=mcx.FP32)
    p.set_tuning(mode=mcx.QUEUELESS, time_limit_s=1e-4, iters_per_sync=1)
    with pytest.raises(mcx.McxError) as e:
        p.run(particles_in_flight=100_000, seed=3)
    assert e.value.code == mcx.ERR_TIMEOUT
    p.zero_tallies()
    p.set_tuning(mode=mcx.QUEUED)
    p.run(particles_in_flight=100_000, seed=3)
    assert p.tallies()["outcome"].sum(0)[:4].sum() == prob.n_histories


def test_short_search_on_the_lattice(mcx, tmp_path):
    prob = synth.config3_problem(n_histories=300_000)
    obj = tuner.transport_objective(prob, seed=5, max_in_flight=300_000)
    t = tuner.Tuner(tuner.transport_space(max_in_flight=300_000), obj, db_path=str(tmp_path / "db.jsonl"),
                    baseline_repeats=2, seed=3)
    best = t.tune(n_random=4, max_evals=8)
    rep = t.report()
    assert best.seconds <= t.baseline * 1.05
    assert rep["evaluations"] == 8
    assert all(r.status in ("ok", "timeout") for r in t.records), [r.status for r in t.records]


def test_energy_meter_reads_the_board_counter(mcx):
    """The NVML total-energy counter (pynvml, or the driver library through
    ctypes) brackets a run: positive joules at a plausible board power."""
    from paper_2402_09222_b300 import energy
    prob = synth.config3_problem(n_histories=300_000, lattice_n=9, n_points=2000)
    p = mcx.make_problem(prob, precision=mcx.FP32, hash_bins=4000)
    p.set_tuning(mode=mcx.QUEUED)
    import time
    with energy.EnergyMeter(0) as m:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 0.6:     # the counter ticks every few tens of ms
            p.run(particles_in_flight=300_000, seed=2)
    p.close()
    assert m.joules > 0 and m.seconds > 0
    assert 20.0 < m.watts < 2000.0, m.watts
