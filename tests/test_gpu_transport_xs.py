"""The transport's own macroscopic lookup against the oracle's FP64 sums.

Transport evaluates Sigma_t, Sigma_a (and nuSigma_f) at each flight (Sec. 5.1:
the macroscopic cross section is the density-weighted sum of the species'
interpolated microscopic ones, Eq. 1) in FP32 pairs from per-point totals and
interval slopes.  The history-matched transport tests check it only through
collision counts; this test compares the values directly, lookup by lookup,
with an a-priori error bound written from the pair arithmetic:

* an FP64 value split into an FP32 pair keeps it within 2^-48 relative, so the
  energy difference E - g_k carries at most about 2^-46 E, which the slope
  multiplies;
* one pair a + b c is within a few 2^-48 of |a| + |b c|;
* the density-weighted accumulation over n species adds at most n such
  errors of the running sum.

The bound below takes 2^-44 for each of these (4 to 16 times the estimate):
a dropped term, a wrong slope or a wrong interval is off by orders of
magnitude more.
"""
import numpy as np
import pytest

import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -44


@pytest.fixture(scope="module")
def mcx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx as m
    return m


def lookup_inputs(mats, n, seed):
    """Log-uniform energies from half the lowest to twice the highest grid
    energy (so some fall below and above every grid), a few exact grid
    energies, and uniform materials."""
    rng = np.random.default_rng(seed)
    E = np.exp(rng.uniform(np.log(synth.E_MIN * 0.5), np.log(synth.E_MAX * 2.0), n))
    mat = rng.integers(0, mats.n_materials, n).astype(np.int32)
    return E, mat


def channel_bound(lib, mats, E, mat, kk, values):
    """Per-lookup error bound of the pair sum of one channel whose per-point
    values are `values` [P]."""
    go, g = lib.grid_offsets, lib.energies
    bound = np.zeros(len(E))
    total = np.zeros(len(E))
    n_sp = np.diff(mats.offsets)[mat]
    for i in range(kk.shape[1]):
        live = kk[:, i] >= 0
        l = np.nonzero(live)[0]
        ent = mats.offsets[mat[l]] + i
        s = mats.species[ent]
        N = mats.dens[ent]
        p = go[s] + kk[l, i]
        g0, g1 = g[p], g[p + 1]
        v0, v1 = values[p], values[p + 1]
        slope = (v1 - v0) / (g1 - g0)
        d = np.clip(E[l], g0, g1) - g0
        v = np.abs(v0 + slope * d)
        bound[l] += N * (2 * EPS * E[l] * np.abs(slope) + EPS * (np.abs(slope) * d + np.abs(v0)))
        total[l] += N * v
    return bound + n_sp * EPS * total, total


def check(mcx, lib, mats, precision, n=200_000, seed=5):
    import torch
    ref_lib = lib.fp32_rounded() if precision == mcx.FP32 else lib
    E, mat = lookup_inputs(mats, n, seed)
    # exact grid energies of random species of each lookup's material
    kk0 = oracle.xs_indices(ref_lib, mats, E[:1000], mat[:1000])
    for l in range(1000):
        s = mats.species[mats.offsets[mat[l]]]
        E[l] = ref_lib.energies[ref_lib.grid_offsets[s] + max(kk0[l, 0], 0)]
    ref = oracle.xs_lookup(ref_lib, mats, E, mat, n_threads=8)
    kk = oracle.xs_indices(ref_lib, mats, E, mat)
    chans = ([synth.CH_SCATTER, synth.CH_ABSORB] if lib.n_ch == 5 else [0, 1])
    sig = ref_lib.sigma
    tot_pts = sig[:, chans[0]] + sig[:, chans[1]]
    want = [ref[:, chans[0]] + ref[:, chans[1]], ref[:, chans[1]]]
    bounds = [channel_bound(ref_lib, mats, E, mat, kk, tot_pts)[0],
              channel_bound(ref_lib, mats, E, mat, kk, sig[:, chans[1]])[0]]
    nf = {5: synth.CH_NU_FISSION, 3: 2}.get(lib.n_ch)
    if nf is not None:
        want.append(ref[:, nf])
        bounds.append(channel_bound(ref_lib, mats, E, mat, kk, sig[:, nf])[0])

    p = mcx.Problem(None)
    p.load_tables(lib, mats, precision=precision, hash_bins=4000)
    try:
        got = p.debug_transport_xs(torch.from_numpy(E).cuda(), torch.from_numpy(mat).cuda()).cpu().numpy()
    finally:
        p.close()
    worst = []
    for c, (w, b) in enumerate(zip(want, bounds)):
        err = np.abs(got[:, c] - w)
        assert np.all(err <= b), (c, int(np.argmax(err - b)), float(np.max(err / b)))
        rel = err / np.maximum(np.abs(w), 1e-300)
        worst.append((float(np.median(rel)), float(np.max(rel)), float(np.max(err / np.maximum(b, 1e-300)))))
    if nf is None:
        assert np.all(got[:, 2] == 0.0)
    print(f"\nn_ch {lib.n_ch} precision {precision}: (median and max relative error, max error/bound) per channel {worst}")
    return worst


@pytest.mark.parametrize("precision", [0, 1])
def test_lattice_library(mcx, precision):
    """47 species x 11,303 points, materials of 40/4/3 species, 2 channels."""
    check(mcx, synth.config3_library(), synth.config3_materials(), precision)


def test_eigenvalue_library(mcx):
    """The same library with a nu-fission channel (3 channels)."""
    check(mcx, synth.eigen_library(), synth.config3_materials(), 0)


def test_invalid_inputs_give_nan(mcx):
    import torch
    lib, mats = synth.config3_library(2000), synth.config3_materials()
    p = mcx.Problem(None)
    p.load_tables(lib, mats, hash_bins=100)
    try:
        E = torch.tensor([1.0, float("nan"), 1.0, 1.0], dtype=torch.float64, device="cuda")
        mat = torch.tensor([0, 0, -1, mats.n_materials], dtype=torch.int32, device="cuda")
        got = p.debug_transport_xs(E, mat).cpu().numpy()
        assert np.all(np.isfinite(got[0])) and got[0, 0] > 0
        assert np.all(np.isnan(got[1:]))
        assert p.debug_transport_xs(E[:0], mat[:0]).shape == (0, 3)
    finally:
        p.close()
