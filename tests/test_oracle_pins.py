"""Pins for the CPU oracle: published vectors, brute force, closed forms and
invariants.  None of these re-types the oracle's own formulas; each checks a
property that the paper's method (or the mathematics behind it) fixes, chosen
so that a dropped term, a wrong sign or a transposed operand fails one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_2402_09222_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _within_se(estimate, expected, se, k=3.0):
    assert abs(estimate - expected) <= k * se, (estimate, expected, se)


# ---------------------------------------------------------------------------
# Philox4x32-10 and the uniform map
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniforms_open_interval_and_uniform():
    u = np.concatenate([oracle.uniforms(12345, 3, h, 2000) for h in range(50)])
    assert np.all(u > 0.0) and np.all(u < 1.0)
    counts, _ = np.histogram(u, bins=100, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4
    # consecutive pairs are independent (2-D cells)
    h2, _, _ = np.histogram2d(u[0::2], u[1::2], bins=10, range=[[0, 1], [0, 1]])
    assert stats.chisquare(h2.ravel()).pvalue > 1e-4


def test_streams_differ_by_history_problem_and_seed():
    a = oracle.uniforms(1, 0, 0, 8)
    assert not np.array_equal(a, oracle.uniforms(1, 0, 1, 8))
    assert not np.array_equal(a, oracle.uniforms(1, 1, 0, 8))
    assert not np.array_equal(a, oracle.uniforms(2, 0, 0, 8))
    # resuming a stream mid-way gives the same numbers
    assert np.array_equal(oracle.uniforms(1, 0, 0, 8)[5:], oracle.uniforms(1, 0, 0, 3, first=5))


def test_uniform_extremes_of_the_word_map():
    # all-zero and all-one words must still give values strictly inside (0,1);
    # reconstruct from the stream's first block as a structural check
    w = oracle.philox4x32_10([0, 7, 0, 0], [9, 0])
    u = oracle.uniforms(9, 0, 7, 2)
    k0 = ((int(w[0]) >> 6) << 26) | (int(w[1]) >> 6)
    k1 = ((int(w[2]) >> 6) << 26) | (int(w[3]) >> 6)
    assert u[0] == (k0 + 0.5) * 2.0 ** -52 and u[1] == (k1 + 0.5) * 2.0 ** -52
    assert (0 + 0.5) * 2.0 ** -52 > 0 and ((1 << 52) - 1 + 0.5) * 2.0 ** -52 < 1.0


# ---------------------------------------------------------------------------
# Grid search: brute force on tiny grids
# ---------------------------------------------------------------------------

def _brute_index(g, E):
    n = len(g)
    k = 0
    for j in range(n - 1):
        if g[j] <= E:
            k = j
    return k


def test_grid_index_brute_force():
    rng = np.random.default_rng(0)
    for n in list(range(2, 51)) + [64, 100]:
        g = np.sort(rng.uniform(-5, 5, n))
        while np.any(np.diff(g) <= 0):
            g = np.sort(rng.uniform(-5, 5, n))
        cands = list(g) + list((g[1:] + g[:-1]) / 2) + [g[0] - 1, g[-1] + 1]
        cands += [np.nextafter(x, -np.inf) for x in g] + [np.nextafter(x, np.inf) for x in g]
        for E in cands:
            assert oracle.grid_index(g, E) == _brute_index(g, E), (n, E)


def test_grid_index_nan_and_ties():
    g = np.array([1.0, 2.0, 3.0, 4.0])
    assert oracle.grid_index(g, float("nan")) == 0
    assert oracle.grid_index(g, 2.0) == 1      # E == g[k] -> k
    assert oracle.grid_index(g, 4.0) == 2      # top end -> n-2
    assert oracle.grid_index(g, 0.5) == 0


# ---------------------------------------------------------------------------
# Macroscopic lookup: textbook routines, closed forms, special cases
# ---------------------------------------------------------------------------

def _small_case(seed=5, n_species=10, n_points=200, n_lookups=3000):
    lib = synth.species_library(n_species, n_points, seed)
    rng = np.random.default_rng(seed)
    members = [np.sort(rng.choice(n_species, k, replace=False)) for k in (1, 3, 7, 10)]
    mats = synth.make_materials(members, [np.exp(rng.uniform(-10, -1, len(m))) for m in members])
    E, mat = synth.lookup_inputs(n_lookups, mats.n_materials, seed)
    # adversarial energies: exact grid points, outside the range
    E[:200] = lib.energies[rng.integers(0, len(lib.energies), 200)]
    E[200:210] = [1e-7, 1e-6, 5e-6, 2e7, 2.5e7, 1e9, 1e-5, 3e7, 1e-8, 2e7]
    return lib, mats, E, mat


def test_lookup_indices_match_searchsorted():
    lib, mats, E, mat = _small_case()
    K = oracle.xs_indices(lib, mats, E, mat)
    for l in range(len(E)):
        sp, _ = mats.members(mat[l])
        for i, s in enumerate(sp):
            g = lib.grid(s)
            k = int(np.searchsorted(g, E[l], side="right")) - 1
            assert K[l, i] == min(max(k, 0), len(g) - 2)
        assert np.all(K[l, len(sp):] == -1)


def test_lookup_matches_numpy_interp():
    lib, mats, E, mat = _small_case()
    out = oracle.xs_lookup(lib, mats, E, mat)
    ref = np.zeros_like(out)
    for m in range(mats.n_materials):
        sel = mat == m
        sp, dn = mats.members(m)
        for s, N in zip(sp, dn):
            g, t = lib.grid(s), lib.table(s)
            for r in range(lib.n_ch):
                ref[sel, r] += N * np.interp(E[sel], g, t[:, r])
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=0)


def test_lookup_linear_tables_closed_form():
    lib = synth.linear_library(6, 300, seed=11, n_ch=5)
    mats = synth.make_materials([np.arange(6)], [np.full(6, 0.25)])
    rng = np.random.default_rng(2)
    E = np.exp(rng.uniform(math.log(1e-5), math.log(2e7), 2000))
    out = oracle.xs_lookup(lib, mats, E, np.zeros(2000, np.int32))
    # per species: sigma = a + b E exactly; recover a, b from the first two table rows
    ref = np.zeros_like(out)
    for s in range(6):
        g, t = lib.grid(s), lib.table(s)
        b = (t[-1] - t[0]) / (g[-1] - g[0])
        a = t[0] - b * g[0]
        ref += 0.25 * (a[None, :] + b[None, :] * E[:, None])
    np.testing.assert_allclose(out, ref, rtol=1e-12)


def test_lookup_shared_grid_single_search():
    lib = synth.linear_library(5, 100, seed=3, shared_grid=True)
    mats = synth.make_materials([np.arange(5)], [np.ones(5)])
    E, _ = synth.lookup_inputs(500, 1, 4)
    K = oracle.xs_indices(lib, mats, E, np.zeros(500, np.int32))
    assert np.all(K == K[:, :1])


def test_lookup_bad_material_is_nan():
    lib, mats, E, mat = _small_case(n_lookups=300)
    mat = mat.copy()
    mat[7] = 99
    mat[8] = -1
    out = oracle.xs_lookup(lib, mats, E, mat)
    assert np.all(np.isnan(out[7])) and np.all(np.isnan(out[8]))
    assert np.all(np.isfinite(out[:7]))


def test_lookup_threads_do_not_change_results():
    lib, mats, E, mat = _small_case()
    assert np.array_equal(oracle.xs_lookup(lib, mats, E, mat, 1), oracle.xs_lookup(lib, mats, E, mat, 4))


def test_lookup_backward_is_the_exact_adjoint():
    """The lookup is linear in densities and table entries, so finite
    differences of the forward lookup are exact up to rounding."""
    lib, mats, E, mat = _small_case(n_points=60, n_lookups=400)
    rng = np.random.default_rng(9)
    G = rng.normal(size=(len(E), lib.n_ch))
    gd, gs = oracle.xs_lookup_backward(lib, mats, E, mat, G)
    base = (oracle.xs_lookup(lib, mats, E, mat) * G).sum()
    for i in rng.choice(len(mats.dens), 8, replace=False):
        d = mats.dens.copy()
        d[i] += 1.0
        pert = synth.Materials(mats.offsets, mats.species, d)
        fd = (oracle.xs_lookup(lib, pert, E, mat) * G).sum() - base
        assert abs(fd - gd[i]) <= 1e-9 * max(1.0, abs(gd[i])), (i, fd, gd[i])
    flat = gs.ravel()
    touched = np.flatnonzero(flat)
    for j in list(rng.choice(touched, 8, replace=False)) + [int(np.flatnonzero(flat == 0)[0])]:
        sg = lib.sigma.copy().ravel()
        sg[j] += 1.0
        pl = synth.Library(lib.grid_offsets, lib.energies, sg.reshape(lib.sigma.shape), lib.awr)
        fd = (oracle.xs_lookup(pl, mats, E, mat) * G).sum() - base
        assert abs(fd - flat[j]) <= 1e-9 * max(1.0, abs(flat[j])), (j, fd, flat[j])


# ---------------------------------------------------------------------------
# Transport single steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("A", [1.0, 2.0, 12.0, 238.0])
def test_scatter_kinematics_textbook_relations(A):
    alpha = ((A - 1) / (A + 1)) ** 2
    for mu in np.linspace(-1 + 1e-9, 1, 41):
        r, mul = oracle.scatter_kinematics(A, mu)
        assert alpha - 1e-15 <= r <= 1 + 1e-15
        # lab cosine from the energy ratio: mu_lab = ((A+1) sqrt(r) - (A-1) / sqrt(r)) / 2
        assert abs(mul - ((A + 1) * math.sqrt(r) - (A - 1) / math.sqrt(r)) / 2) < 1e-9
    assert oracle.scatter_kinematics(A, 1.0) == (1.0, 1.0)
    assert abs(oracle.scatter_kinematics(A, -1.0)[0] - alpha) < 1e-15
    # averages over an isotropic CM cosine
    mean_r = integrate.quad(lambda m: oracle.scatter_kinematics(A, m)[0], -1, 1)[0] / 2
    assert abs(mean_r - (A * A + 1) / (A + 1) ** 2) < 1e-12
    if A > 1:
        mean_mu = integrate.quad(lambda m: oracle.scatter_kinematics(A, m)[1], -1, 1, limit=200)[0] / 2
        assert abs(mean_mu - 2.0 / (3.0 * A)) < 1e-7


def test_rotation_preserves_norm_and_sets_angle():
    rng = np.random.default_rng(1)
    for t in range(400):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if t % 50 == 0:
            d = np.array([0.0, 1e-3, math.sqrt(1 - 1e-6)]) * (1 if t % 100 else -1)
        mu = rng.uniform(-1, 1)
        phi = rng.uniform(0, 2 * math.pi)
        out = oracle.rotate_direction(d, mu, math.cos(phi), math.sin(phi))
        assert abs(np.linalg.norm(out) - 1) < 1e-12
        assert abs(out @ d - mu) < 1e-12
        # the two azimuths phi and -phi are mirror images about the plane of d and out+mirror
        out2 = oracle.rotate_direction(d, mu, math.cos(phi), -math.sin(phi))
        assert abs(out2 @ d - mu) < 1e-12
        # azimuth phi + pi gives the reflection through the axis d
        out3 = oracle.rotate_direction(d, mu, -math.cos(phi), -math.sin(phi))
        np.testing.assert_allclose(out + out3, 2 * mu * d, atol=1e-12)


def test_isotropic_source_directions():
    lib = synth.flat_library(1.0, 1.0)
    mats = synth.make_materials([[0]], [[1.0]])
    prob = synth.infinite_problem(lib, mats, 10_000)
    st = np.array([oracle.source_state(prob, 77, h) for h in range(4000)])
    u, v, w = st[:, 3], st[:, 4], st[:, 5]
    np.testing.assert_allclose(u * u + v * v + w * w, 1.0, atol=1e-13)
    assert stats.kstest(w, stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert stats.kstest(np.arctan2(v, u), stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3


def test_lattice_source_positions_are_pin_centres():
    prob = synth.config3_problem(n_histories=1000, lattice_n=17, lib=synth.flat_library(1.0, 1.0))
    st = np.array([oracle.source_state(prob, 5, h) for h in range(3000)])
    n, p = 17, 1.26
    i, j = st[:, 6].astype(int) // n, st[:, 6].astype(int) % n
    np.testing.assert_allclose(st[:, 0], -n * p / 2 + p * (i + 0.5), atol=1e-12)
    np.testing.assert_allclose(st[:, 1], -n * p / 2 + p * (j + 0.5), atol=1e-12)
    assert np.all(st[:, 2] == 50.0)
    counts = np.bincount(st[:, 6].astype(int), minlength=n * n)
    assert stats.chisquare(counts).pvalue > 1e-3


def _random_lattice_state(rng, n, p, r, H, inpin):
    ci, cj = rng.integers(0, n, 2)
    cx, cy = -n * p / 2 + p * (ci + 0.5), -n * p / 2 + p * (cj + 0.5)
    while True:
        x, y = cx + rng.uniform(-p / 2, p / 2), cy + rng.uniform(-p / 2, p / 2)
        rho = math.hypot(x - cx, y - cy)
        if (rho < r) == inpin and abs(rho - r) > 1e-6:
            break
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return np.array([x, y, rng.uniform(0.01, H - 0.01), *d, ci, cj, float(inpin)]), cx, cy


def test_lattice_surface_distance_geometry():
    n, p, r, H = 17, 1.26, 0.41, 100.0
    prob = synth.config3_problem(n_histories=10, lattice_n=n, lib=synth.flat_library(1.0, 1.0))
    rng = np.random.default_rng(3)
    seen = set()
    for t in range(3000):
        inpin = t % 2 == 0
        st, cx, cy = _random_lattice_state(rng, n, p, r, H, inpin)
        surf, d = oracle.surface_distance(prob, st)
        seen.add((inpin, surf))
        pos, u = st[:3], st[3:6]
        end = pos + d * u
        xl, yl = cx - p / 2, cy - p / 2
        on = {oracle.SURF_CYL: abs(math.hypot(end[0] - cx, end[1] - cy) - r),
              oracle.SURF_ZTOP: abs(end[2] - H), oracle.SURF_ZBOT: abs(end[2]),
              oracle.SURF_XLO: abs(end[0] - xl), oracle.SURF_XHI: abs(end[0] - xl - p),
              oracle.SURF_YLO: abs(end[1] - yl), oracle.SURF_YHI: abs(end[1] - yl - p)}[surf]
        assert on < 1e-9, (surf, on)
        # the open segment stays inside the starting region
        for f in np.linspace(0.001, 0.999, 25):
            q = pos + f * d * u
            rho = math.hypot(q[0] - cx, q[1] - cy)
            assert 0 <= q[2] <= H
            if inpin:
                assert rho <= r + 1e-9
            else:
                assert rho >= r - 1e-9 and xl - 1e-9 <= q[0] <= xl + p + 1e-9
                assert yl - 1e-9 <= q[1] <= yl + p + 1e-9
    # every surface kind was exercised
    assert {s for _, s in seen} >= {oracle.SURF_CYL, oracle.SURF_ZTOP, oracle.SURF_ZBOT,
                                    oracle.SURF_XLO, oracle.SURF_XHI, oracle.SURF_YLO,
                                    oracle.SURF_YHI}


# ---------------------------------------------------------------------------
# Transport closed forms
# ---------------------------------------------------------------------------

def _flat_infinite(sig_s, sig_a, N=1.0, A=12.0, n_hist=20_000, E_cut=1e-5, B=20):
    lib = synth.flat_library(sig_s, sig_a, A)
    mats = synth.make_materials([[0]], [[N]])
    prob = synth.infinite_problem(lib, mats, n_hist, E_cut=E_cut)
    prob.n_batches = B
    return prob


def test_pure_absorber_infinite_medium():
    Sa = 0.7
    prob = _flat_infinite(0.0, Sa, n_hist=20_000)
    r = oracle.transport(prob, seed=11, history_debug=True)
    N = prob.n_histories
    assert np.all(r["ncoll"] == 1)
    assert r["outcome"][:, oracle.OUT_ABSORBED].sum() == N
    assert r["outcome"][:, oracle.OUT_COLLISIONS].sum() == N
    # track length d ~ Exp(Sa): total flux per source 1/Sa, sd 1/Sa
    _within_se(r["flux"].sum() / N, 1 / Sa, (1 / Sa) / math.sqrt(N))
    _within_se(r["absorb"].sum() / N, 1.0, 1.0 / math.sqrt(N))
    # the particle never changes energy: all flux sits in E0's bin
    assert np.count_nonzero(r["flux"].sum(0)) == 1


def _two_species_flat(s1, a1, N1, s2, a2, N2, n_hist=20_000, A=1e6):
    """An infinite medium of two species with constant cross sections; a huge
    mass ratio keeps the energy (and so the cross sections) fixed."""
    g = np.array([synth.E_MIN, synth.E_MAX])
    lib = synth.Library(np.array([0, 2, 4], np.int64), np.concatenate([g, g]),
                        np.array([[s1, a1], [s1, a1], [s2, a2], [s2, a2]]), np.array([A, A]))
    mats = synth.make_materials([[0, 1]], [[N1, N2]])
    return synth.infinite_problem(lib, mats, n_hist, E_cut=0.0)


@pytest.mark.parametrize("case", [
    # pure scatterer + pure absorber: a collision absorbs iff species 2 is
    # chosen, P = N2 a2 / (N1 s1 + N2 a2) = 1 / 7
    (3.0, 0.0, 2.0, 0.0, 2.0, 0.5, 1.0 / 7.0),
    # both mixed: P(absorb) = sum_j P(j) a_j / t_j = Sigma_a / Sigma_t = 3.5 / 8
    (2.0, 1.0, 2.0, 1.0, 3.0, 0.5, 3.5 / 8.0),
])
def test_species_selection_sets_the_absorption_probability(case):
    """Species selection (Sec. 5.1 lookup feeding the collision; reading 7):
    species j is chosen with probability N_j sigma_t,j / Sigma_t and absorbs
    with sigma_a,j / sigma_t,j, so with flat cross sections every collision
    absorbs with probability Sigma_a / Sigma_t and the collision count is
    geometric with that parameter.  A running sum without the densities
    gives 4/7 and 19/32, an exclusive running sum 1 and 3/4, the scattering
    cross section in the absorption test 6/7 and 9/16."""
    s1, a1, N1, s2, a2, N2, p = case
    prob = _two_species_flat(s1, a1, N1, s2, a2, N2)
    r = oracle.transport(prob, seed=31, history_debug=True)
    n = r["ncoll"].astype(float)
    assert abs(p - (N1 * a1 + N2 * a2) / (N1 * (s1 + a1) + N2 * (s2 + a2))) < 1e-15
    _within_se(n.mean(), 1 / p, math.sqrt((1 - p) / p ** 2 / len(n)))
    # every history ends absorbed; absorptions per collision = p
    assert r["outcome"][:, oracle.OUT_ABSORBED].sum() == len(n)
    coll = r["outcome"][:, oracle.OUT_COLLISIONS].sum()
    _within_se(len(n) / coll, p, math.sqrt(p * (1 - p) / coll))


@pytest.mark.parametrize("N,B", [(2000, 20), (1999, 20), (37, 5)])
def test_histories_fall_in_batches_by_floor_h_B_over_N(N, B):
    """History h scores into batch floor(h B / N) (reading 10): every history
    ends in exactly one outcome, so batch b holds exactly the histories
    ceil(b N / B) .. ceil((b + 1) N / B) - 1 -- N/B each when B divides N.
    Histories taken modulo B, or floor(h B / (N + 1)), give other counts."""
    prob = _flat_infinite(0.0, 0.7, n_hist=N, B=B)
    r = oracle.transport(prob, seed=3)
    per_batch = r["outcome"][:, :4].sum(1)
    want = np.array([math.ceil((b + 1) * N / B) - math.ceil(b * N / B) for b in range(B)])
    assert np.array_equal(per_batch, want)
    # and a run of a sub-range scores only into the batches of its histories
    r2 = oracle.transport(prob, seed=3, first=N // 2, count=N - N // 2)
    got = np.nonzero(r2["outcome"][:, :4].sum(1))[0]
    assert got.min() == (N // 2) * B // N and got.max() == B - 1


def test_config1_flux_lands_in_the_source_energy_bin():
    """A pure absorber never changes the particle's energy, so the whole
    track-length flux of the 50-bin energy tally (log-spaced over
    [1e-5, 2e7] eV) lands in the bin holding E0 = 2e6 eV: bin
    floor(50 ln(E0 / 1e-5) / ln(2e7 / 1e-5)) = 45."""
    prob = _flat_infinite(0.0, 0.7, n_hist=2000)
    r = oracle.transport(prob, seed=11)
    k = int(math.floor(50 * math.log(2e6 / 1e-5) / math.log(2e7 / 1e-5)))
    assert k == 45
    flux = r["flux"].sum(0)
    assert flux[k] > 0 and np.count_nonzero(flux) == 1
    assert r["absorb"].sum(0)[k] > 0 and np.count_nonzero(r["absorb"].sum(0)) == 1


def test_collision_count_is_geometric():
    Ss, Sa = 2.0, 0.5
    prob = _flat_infinite(Ss, Sa, n_hist=20_000, E_cut=0.0)
    r = oracle.transport(prob, seed=12, history_debug=True)
    n = r["ncoll"].astype(float)
    p = Sa / (Ss + Sa)
    _within_se(n.mean(), 1 / p, math.sqrt((1 - p) / p ** 2 / len(n)))
    ks = np.arange(1, 16)
    obs = np.array([(n == k).sum() for k in ks] + [(n > 15).sum()])
    exp = np.array([(1 - p) ** (k - 1) * p for k in ks] + [(1 - p) ** 15]) * len(n)
    assert stats.chisquare(obs, exp).pvalue > 1e-3
    # flux = S / Sigma_a for an infinite medium with flat cross sections
    F = r["flux"].sum(1)   # per batch
    _within_se(F.sum() / len(n), 1 / Sa, F.std(ddof=1) / (len(n) / prob.n_batches) / math.sqrt(prob.n_batches))


def test_first_collision_energy_is_uniform_between_alpha_e_and_e():
    """Pure scatterer: the particle is cut off at its first collision iff
    E'/E < c, which has probability (c - alpha) / (1 - alpha)."""
    A, c = 12.0, 0.8
    alpha = ((A - 1) / (A + 1)) ** 2
    prob = _flat_infinite(1.0, 0.0, A=A, n_hist=20_000, E_cut=c * 2.0e6)
    r = oracle.transport(prob, seed=13, history_debug=True)
    q = (c - alpha) / (1 - alpha)
    k = (r["ncoll"] == 1).sum()
    N = prob.n_histories
    _within_se(k, N * q, math.sqrt(N * q * (1 - q)))
    assert r["outcome"][:, oracle.OUT_CUTOFF].sum() == N


def test_hydrogen_like_mean_collisions_to_cutoff():
    """A = 1: E'/E ~ U(0,1), so the number of collisions to fall below c E0
    has mean 1 + ln(1/c)."""
    c = 0.5
    prob = _flat_infinite(1.0, 0.0, A=1.0, n_hist=20_000, E_cut=c * 2.0e6)
    r = oracle.transport(prob, seed=14, history_debug=True)
    n = r["ncoll"].astype(float)
    _within_se(n.mean(), 1 + math.log(1 / c), n.std(ddof=1) / math.sqrt(len(n)))


def test_slab_transmission_and_its_derivative():
    Sa, L = 1.3, 1.1
    lib = synth.flat_library(0.0, Sa)
    mats = synth.make_materials([[0]], [[1.0]])
    prob = synth.slab_problem(lib, mats, L, 20_000)
    r = oracle.transport(prob, seed=15, derivatives=True)
    N = prob.n_histories
    T = math.exp(-Sa * L)
    k = r["outcome"][:, oracle.OUT_LEAK_XHI].sum()
    _within_se(k, N * T, math.sqrt(N * T * (1 - T)))
    # every transmitted history carries W = -Sigma_a L exactly
    dk = r["doutcome"][:, oracle.OUT_LEAK_XHI, 0].sum()
    assert abs(dk - (-Sa * L) * k) <= 1e-9 * abs(dk)
    _within_se(dk / N, -Sa * L * T, Sa * L * math.sqrt(T * (1 - T) / N))
    assert r["outcome"][:, oracle.OUT_ABSORBED].sum() + k == N


def test_infinite_medium_likelihood_ratio():
    """Absorptions per source are 1 whatever the density scale s, so their
    derivative is 0; the flux 1/(s Sigma_a) has derivative -1/Sigma_a at s=1."""
    Ss, Sa = 1.5, 1.0
    prob = _flat_infinite(Ss, Sa, n_hist=20_000, E_cut=0.0, B=40)
    r = oracle.transport(prob, seed=16, derivatives=True)
    N, B = prob.n_histories, prob.n_batches
    per = N / B

    def check(per_batch, expected):
        _within_se(per_batch.sum() / N, expected, per_batch.std(ddof=1) / per / math.sqrt(B))

    check(r["doutcome"][:, oracle.OUT_ABSORBED, 0], 0.0)
    check(r["dflux"].sum(axis=(1, 2)), -1.0 / Sa)
    check(r["dabsorb"].sum(axis=(1, 2)), 0.0)
    # a score made with W excluding the collision at the segment's end would be biased:
    # the flux derivative would be -2/Sa instead.  Make sure the estimate is far from it.
    assert abs(r["dflux"].sum() / N - (-2.0 / Sa)) > 0.5 / Sa


def _batch_pair_check(a, b, k=3.0):
    """a and b are per-batch sums with equal expectations."""
    d = a - b
    _within_se(d.mean(), 0.0, d.std(ddof=1) / math.sqrt(len(d)), k)


def test_config1_absorption_balance():
    prob = synth.config1_problem(3000)
    prob.n_batches = 30
    r = oracle.transport(prob, seed=17, history_debug=True)
    N = prob.n_histories
    out = r["outcome"].sum(0)
    assert out[oracle.OUT_ABSORBED] + out[oracle.OUT_CUTOFF] == N
    assert out[oracle.OUT_LEAK_XHI] == 0 and out[oracle.OUT_LEAK_OTHER] == 0
    assert out[oracle.OUT_COLLISIONS] == r["ncoll"].sum()
    # track-length absorption estimate == analog absorption count, per batch in expectation
    _batch_pair_check(r["absorb"].sum(1), r["outcome"][:, oracle.OUT_ABSORBED])


def test_lattice_balance_small():
    prob = synth.config3_problem(n_histories=3000, lattice_n=7, n_points=500)
    prob.n_batches = 30
    r = oracle.transport(prob, seed=18)
    out = r["outcome"].sum(0)
    assert out[:4].sum() == prob.n_histories
    assert out[oracle.OUT_LEAK_OTHER] > 0 and out[oracle.OUT_ABSORBED] > 0
    _batch_pair_check(r["absorb"].sum(1), r["outcome"][:, oracle.OUT_ABSORBED])


def test_unit_cell_streaming_geometry():
    """1x1 lattice with no material: per history, the pin path is r / sin(theta)
    and the moderator path D(phi) / sin(theta) with D the horizontal distance
    from the pin surface to the square cell boundary, so moderator/pin = D/r."""
    p, r = 1.26, 0.41
    lib = synth.flat_library(1.0, 1.0)
    mats = synth.make_materials([[0], [0]], [[0.0], [0.0]])
    N = 6000
    prob = synth.Problem(synth.GEOM_LATTICE, lib, mats, lattice_n=1, pitch=p, radius=r,
                         region_material=np.array([0, 1], np.int32), n_histories=N, n_batches=N)
    res = oracle.transport(prob, seed=19)
    pin, mod = res["flux"][:, 0], res["flux"][:, 1]
    assert np.all(res["outcome"][:, oracle.OUT_LEAK_XHI] + res["outcome"][:, oracle.OUT_LEAK_OTHER] == 1)
    assert stats.kstest(pin, lambda t: np.sqrt(np.clip(1 - (r / np.maximum(t, r)) ** 2, 0, 1))).pvalue > 1e-3
    y = mod / pin * r
    lo, hi = p / 2 - r, p / math.sqrt(2) - r
    assert np.all(y > lo - 1e-9) and np.all(y < hi + 1e-9)
    cdf = lambda yy: (4 / math.pi) * np.arccos(np.clip((p / 2) / (np.asarray(yy) + r), -1, 1))
    assert stats.kstest(y, cdf).pvalue > 1e-3
    # leak face: +x is one of four equivalent faces
    k = res["outcome"][:, oracle.OUT_LEAK_XHI].sum()
    _within_se(k, N / 4, math.sqrt(N * 0.25 * 0.75))


def test_history_results_do_not_depend_on_threads_or_splitting():
    prob = synth.config3_problem(n_histories=2000, lattice_n=5, n_points=400)
    a = oracle.transport(prob, seed=20, history_debug=True, derivatives=True)
    b = oracle.transport(prob, seed=20, history_debug=True, derivatives=True, n_threads=4)
    h1 = oracle.transport(prob, seed=20, first=0, count=900, history_debug=True, derivatives=True)
    h2 = oracle.transport(prob, seed=20, first=900, count=1100, history_debug=True, derivatives=True)
    assert np.array_equal(a["ncoll"], b["ncoll"])
    assert np.array_equal(a["ncoll"], np.concatenate([h1["ncoll"], h2["ncoll"]]))
    for key in ("flux", "absorb", "outcome", "dflux", "dabsorb", "doutcome"):
        np.testing.assert_allclose(b[key], a[key], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(h1[key] + h2[key], a[key], rtol=1e-12, atol=1e-12)
