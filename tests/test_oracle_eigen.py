"""Pins of the oracle's k-eigenvalue power iteration (CPU only).

Each pin comes from outside the oracle's text: the closed form k = nuSigma_f /
Sigma_a of an infinite homogeneous medium with energy-independent cross
sections (every estimator must converge to it), the scaling of the first
generation's bank with the initial guess k0, the Maxwellian fission spectrum
(Gamma(3/2, T): mean 1.5 T, variance 1.5 T^2, CDF P(3/2, E/T)), geometric
facts about where fission sites can lie, and invariance under threading.
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2402_09222_b300 import synth


def flat_problem(sig_s=3.0, sig_a=1.0, nu_sig_f=1.2, n=20_000, A=1e6):
    lib = synth.flat_fission_library(sig_s, sig_a, nu_sig_f, A=A)
    mats = synth.make_materials([np.array([0])], [np.array([1.0])])
    return synth.infinite_problem(lib, mats, n_histories=n)


def test_fission_spectrum_is_the_maxwellian():
    T = 1.2895e6
    e = oracle.fission_energies(11, 0, 3, T, 100_000)
    assert abs(e.mean() / (1.5 * T) - 1) < 0.01
    assert abs(e.var() / (1.5 * T * T) - 1) < 0.03
    ks = stats.kstest(e / T, lambda x: special.gammainc(1.5, x))
    assert ks.pvalue > 1e-3


@pytest.mark.parametrize("nu_sig_f", [0.8, 1.2])
def test_infinite_medium_k_is_nu_sigma_f_over_sigma_a(nu_sig_f):
    prob = flat_problem(nu_sig_f=nu_sig_f)
    r = oracle.eigenvalue(prob, seed=5, n_per_gen=20_000, n_generations=12, n_inactive=2, n_threads=8)
    k_true = nu_sig_f / 1.0
    for key in ("k", "k_col", "k_tl"):
        act = r[key][2:]
        se = act.std(ddof=1) / np.sqrt(len(act))
        assert abs(act.mean() - k_true) < 4 * se + 2e-3, (key, act.mean(), se)
    # the bank stays near N once renormalised by the previous generation's k
    assert np.all(np.abs(r["sites"][1:] / 20_000 - 1) < 0.05)
    # track-length and collision estimators are far less noisy than the site count
    assert r["k_col"][2:].std() < r["k"][2:].std()


def test_first_bank_scales_with_the_initial_guess():
    prob = flat_problem(nu_sig_f=1.2, n=40_000)
    lo = oracle.eigenvalue(prob, seed=7, n_per_gen=40_000, n_generations=1, n_inactive=0, k0=0.5)
    hi = oracle.eigenvalue(prob, seed=7, n_per_gen=40_000, n_generations=1, n_inactive=0, k0=2.0)
    # M_0 has mean N k / k0; the site-count k estimate is M_0 k0 / N either way
    assert abs(lo["sites"][0] / (40_000 * 1.2 / 0.5) - 1) < 0.02
    assert abs(hi["sites"][0] / (40_000 * 1.2 / 2.0) - 1) < 0.03
    assert abs(lo["k"][0] / 1.2 - 1) < 0.02 and abs(hi["k"][0] / 1.2 - 1) < 0.03
    # the collision estimator does not depend on k0 at all (same histories)
    assert lo["k_col"][0] == hi["k_col"][0]


def test_no_fissile_material_ends_the_iteration():
    prob = flat_problem(nu_sig_f=0.0, n=500)
    with pytest.raises(RuntimeError, match="no fission site"):
        oracle.eigenvalue(prob, seed=1, n_per_gen=500, n_generations=3, n_inactive=1)


@pytest.fixture(scope="module")
def lattice_run():
    prob = synth.eigen_problem(n_per_gen=1500, lattice_n=9, n_points=2000)
    return prob, oracle.eigenvalue(prob, seed=9, n_per_gen=1500, n_generations=4, n_inactive=1,
                                   n_threads=8, bank=True, history_debug=True)


def test_fission_sites_lie_in_fuel_pins(lattice_run):
    prob, r = lattice_run
    bank = r["bank"]
    assert len(bank) == r["sites"][-1] > 0
    x, y, z, ci, cj, inpin = bank.T
    n, p, rad = prob.lattice_n, prob.pitch, prob.radius
    half = 0.5 * n * p
    cx = -half + p * (ci + 0.5)
    cy = -half + p * (cj + 0.5)
    assert np.all((0 <= ci) & (ci < n) & (0 <= cj) & (cj < n))
    assert np.all(np.abs(x - cx) <= p / 2 + 1e-9) and np.all(np.abs(y - cy) <= p / 2 + 1e-9)
    assert np.all((z >= 0) & (z <= prob.height))
    # only the fuel (material 0, in pins that are not guide tubes) has nu-fission
    assert np.all(inpin == 1)
    assert np.all(np.hypot(x - cx, y - cy) <= rad * (1 + 1e-9))
    guide = (ci.astype(int) % 3 == 2) & (cj.astype(int) % 3 == 2)
    assert not np.any(guide)


def test_estimators_agree_on_the_lattice(lattice_run):
    prob, r = lattice_run
    for key in ("k_col", "k_tl"):
        assert np.all(np.abs(r[key] / r["k"] - 1) < 0.25)
    assert r["outcome"][:, :4].sum() == 3 * 1500      # active generations only
    assert len(r["ncoll"]) == 1500


def test_threads_change_nothing():
    prob = synth.eigen_problem(n_per_gen=800, lattice_n=9, n_points=1000)
    a = oracle.eigenvalue(prob, seed=4, n_per_gen=800, n_generations=3, n_inactive=1, n_threads=1,
                          bank=True)
    b = oracle.eigenvalue(prob, seed=4, n_per_gen=800, n_generations=3, n_inactive=1, n_threads=6,
                          bank=True)
    assert np.array_equal(a["sites"], b["sites"]) and np.array_equal(a["k"], b["k"])
    assert np.array_equal(a["bank"], b["bank"])
    np.testing.assert_allclose(a["k_col"], b["k_col"], rtol=1e-13)
    np.testing.assert_allclose(a["flux"], b["flux"], rtol=1e-12, atol=1e-12 * a["flux"].max())


@pytest.mark.parametrize("n_per_gen", [700, 3000])
def test_next_source_is_a_systematic_resample_of_the_bank(n_per_gen):
    """Generation 1 starts from generation 0's bank resampled to N sites:
    every source site is a bank site, taken in bank order, and every bank site
    is used floor(N/M) or ceil(N/M) times (0 or 1 when M > N)."""
    prob = flat_problem(nu_sig_f=1.2, n=n_per_gen)
    g0 = oracle.eigenvalue(prob, seed=2, n_per_gen=n_per_gen, n_generations=1, n_inactive=0,
                           k0=0.4 if n_per_gen == 700 else 3.0, bank=True)
    g1 = oracle.eigenvalue(prob, seed=2, n_per_gen=n_per_gen, n_generations=2, n_inactive=0,
                           k0=0.4 if n_per_gen == 700 else 3.0, bank=True)
    bank, src = g0["bank"], g1["source"]
    M, N = len(bank), n_per_gen
    assert (M > N) == (n_per_gen == 700)
    pos = {tuple(r): i for i, r in enumerate(bank)}
    assert len(pos) == M                     # collision points are distinct
    idx = np.array([pos[tuple(r)] for r in src])
    assert np.all(np.diff(idx) >= 0)
    use = np.bincount(idx, minlength=M)
    assert use.min() >= N // M and use.max() <= -(-N // M)
    assert use.sum() == N


def test_a_history_starts_at_its_site_isotropic_with_fission_energy():
    prob = synth.eigen_problem(n_per_gen=10, lattice_n=9, n_points=500)
    n, p = prob.lattice_n, prob.pitch
    half = 0.5 * n * p
    ci, cj = 4, 1
    site = [-half + p * (ci + 0.5) + 0.1, -half + p * (cj + 0.5) - 0.2, 37.5, ci, cj, 1]
    st = np.array([oracle.site_source_state(prob, 3, h, site) for h in range(4000)])
    assert np.all(st[:, :3] == np.array(site[:3]))
    assert np.all(st[:, 7] == ci * n + cj)                 # the pin's region
    assert np.allclose(np.linalg.norm(st[:, 3:6], axis=1), 1.0)
    assert stats.kstest(st[:, 5], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = np.arctan2(st[:, 4], st[:, 3])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3
    assert stats.kstest(st[:, 6] / prob.T_fission, lambda x: special.gammainc(1.5, x)).pvalue > 1e-3
    # outside the pin (moderator) the region is the moderator's
    out = oracle.site_source_state(prob, 3, 0, [site[0] + 0.45, site[1], 1.0, ci, cj, 0])
    assert out[7] == n * n
