"""GPU parity of the k-eigenvalue power iteration against the CPU oracle.

Generations are history-matched through the shared Philox streams and the
canonical bank order, so the site counts, the site-count k (formed from
integers on the host), the ordered bank and the per-history collision counts
must be identical; the collision and track-length estimators and the tallies
are FP64 sums in a different order (1e-12 and 1e-9 relative).
"""
import numpy as np
import pytest

import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx as m
    return m


def flat_problem(n, nu_sig_f=1.2):
    lib = synth.flat_fission_library(3.0, 1.0, nu_sig_f, A=1e6)
    mats = synth.make_materials([np.array([0])], [np.array([1.0])])
    return synth.infinite_problem(lib, mats, n_histories=n)


def run_gpu(mcx, prob, n, gens, inactive, k0=1.0, pif=100_000, seed=5, H=1000, precision=0, **tune):
    p = mcx.make_problem(prob, precision=precision, hash_bins=H, flags=mcx.FLAG_HISTORY_DEBUG)
    p.set_tuning(**tune)
    r = p.run_eigenvalue(n, gens, inactive, k0=k0, particles_in_flight=pif, seed=seed)
    r.update(p.tallies())
    r["bank"] = p.fission_bank()
    r["ncoll"] = p.history_debug(n)
    r["stats"] = p.stats()
    p.close()
    return r


def assert_matched(g, o):
    assert np.array_equal(g["sites"], o["sites"])
    assert np.array_equal(g["k"], o["k"])
    np.testing.assert_allclose(g["k_col"], o["k_col"], rtol=1e-12)
    np.testing.assert_allclose(g["k_tl"], o["k_tl"], rtol=1e-12)
    # site positions: the same FP64 expressions, but CUDA's log and the host
    # libm's may differ in the last bit, which moves a collision point by an
    # ulp without changing any decision; cells and flags are exact
    gb, ob = g["bank"], o["bank"]
    assert gb.shape == ob.shape
    assert np.array_equal(gb[:, 3:], ob[:, 3:])
    np.testing.assert_allclose(gb[:, :3], ob[:, :3], rtol=1e-12, atol=1e-12)
    assert np.array_equal(g["ncoll"], o["ncoll"])
    for key in ("flux", "absorb", "outcome"):
        scale = max(np.abs(o[key]).max(), 1e-300)
        np.testing.assert_allclose(g[key], o[key], rtol=1e-9, atol=1e-9 * scale, err_msg=key)


@pytest.mark.parametrize("tu", [dict(mode=0, pif=4000), dict(mode=1, pif=777, sort_period=1, sort_threshold=0),
                                dict(mode=2, pif=50_000, sort_period=2, sort_threshold=10)],
                         ids=["queueless", "queued", "fullest"])
def test_flat_infinite_medium_matches_the_oracle(mcx, tu):
    tu = dict(tu)
    pif = tu.pop("pif")
    n = 5000
    prob = flat_problem(n)
    o = oracle.eigenvalue(prob, seed=5, n_per_gen=n, n_generations=5, n_inactive=2, n_threads=8,
                          bank=True, history_debug=True)
    g = run_gpu(mcx, prob, n, 5, 2, pif=pif, **tu)
    assert_matched(g, o)
    assert abs(np.mean(g["k_col"][2:]) / 1.2 - 1) < 0.02


@pytest.fixture(scope="module")
def lattice():
    prob = synth.eigen_problem(n_per_gen=3000, lattice_n=9, n_points=2000)
    o = oracle.eigenvalue(prob, seed=8, n_per_gen=3000, n_generations=4, n_inactive=1, n_threads=8,
                          bank=True, history_debug=True)
    return prob, o


@pytest.mark.parametrize("precision", [0, 1])
def test_lattice_generations_match_the_oracle(mcx, lattice, precision):
    prob, o = lattice
    if precision == 1:
        rp = synth.eigen_problem(n_per_gen=3000, lattice_n=9, lib=prob.lib.fp32_rounded())
        o = oracle.eigenvalue(rp, seed=8, n_per_gen=3000, n_generations=4, n_inactive=1, n_threads=8,
                              bank=True, history_debug=True)
    g = run_gpu(mcx, prob, 3000, 4, 1, seed=8, precision=precision, pif=1500, mode=1, sort_period=1,
                sort_threshold=0)
    assert_matched(g, o)


def test_initial_guess_far_below_k_grows_the_bank(mcx):
    """k0 = 0.04 makes generation 0 bank ~30 N sites, beyond the 4 N bank: the
    inactive generation is run again with room for all of them."""
    n = 2000
    prob = flat_problem(n)
    o = oracle.eigenvalue(prob, seed=3, n_per_gen=n, n_generations=3, n_inactive=1, k0=0.04,
                          bank=True, history_debug=True)
    assert o["sites"][0] > 4 * 4096
    g = run_gpu(mcx, prob, n, 3, 1, k0=0.04, seed=3, mode=1)
    assert_matched(g, o)


def test_overflow_in_an_active_generation_is_an_error(mcx):
    n = 2000
    prob = flat_problem(n)
    p = mcx.make_problem(prob, hash_bins=0)
    with pytest.raises(mcx.McxError, match="BOUNDS"):
        p.run_eigenvalue(n, 2, 0, k0=0.04, particles_in_flight=4000, seed=3)
    # the handle stays usable
    r = p.run_eigenvalue(n, 2, 0, k0=1.0, particles_in_flight=4000, seed=3)
    assert r["sites"][0] > 0
    p.close()


def test_no_fission_and_bad_arguments(mcx):
    prob = flat_problem(500, nu_sig_f=0.0)
    p = mcx.make_problem(prob, hash_bins=0)
    with pytest.raises(mcx.McxError, match="STATE"):
        p.run_eigenvalue(500, 3, 1, particles_in_flight=1000)
    with pytest.raises(mcx.McxError, match="ARG"):
        p.run_eigenvalue(500, 3, 3)
    with pytest.raises(mcx.McxError, match="ARG"):
        p.run_eigenvalue(500, 3, 1, k0=0.0)
    p.close()
    two = synth.config1_problem(100)
    q = mcx.make_problem(two)
    with pytest.raises(mcx.McxError, match="ARG"):
        q.run_eigenvalue(100, 2, 1)
    q.close()


def test_fixed_source_runs_are_unchanged_after_an_eigenvalue_run(mcx):
    """An eigenvalue run and a fixed-source run on the same handle: the
    fixed-source tallies still match the oracle (no fission state leaks)."""
    prob = synth.eigen_problem(n_per_gen=2000, lattice_n=9, n_points=2000)
    ref = oracle.transport(prob, seed=4, history_debug=True, n_threads=8)
    p = mcx.make_problem(prob, flags=mcx.FLAG_HISTORY_DEBUG)
    p.set_tuning(mode=1)
    p.run_eigenvalue(2000, 2, 1, particles_in_flight=3000, seed=9)
    p.zero_tallies()
    p.run(particles_in_flight=3000, seed=4)
    assert np.array_equal(p.history_debug(2000), ref["ncoll"])
    t = p.tallies()
    np.testing.assert_allclose(t["flux"], ref["flux"], rtol=1e-9, atol=1e-9 * ref["flux"].max())
    p.close()


def test_full_lattice_power_iteration(mcx):
    """The 17x17 lattice, 2e5 histories per generation, FP32 tables, tuned
    queue settings: the three k estimators agree, the bank stays near N once
    the source has settled, every site lies in a fuel pin, and the active
    generations' histories all end in the tallies."""
    n = 200_000
    prob = synth.eigen_problem(n_per_gen=n)
    g = run_gpu(mcx, prob, n, 6, 2, precision=1, H=37_100, pif=400_000, mode=1, sort_period=1,
                sort_threshold=20_000)
    act = slice(2, None)
    kk, kc, kt = g["k"][act].mean(), g["k_col"][act].mean(), g["k_tl"][act].mean()
    assert abs(kc / kk - 1) < 0.02 and abs(kt / kk - 1) < 0.02
    assert np.all(np.abs(g["sites"][2:] / n - 1) < 0.1)    # after the source settles
    bank = g["bank"]
    assert np.all(bank[:, 5] == 1)                       # fuel pins only
    assert g["outcome"][:, :4].sum() == 4 * n
