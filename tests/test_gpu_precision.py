"""The error of FP32 cross-section tables against the FP64 definition.

FP32 tables halve the gathered bytes; energies, the grid search and every
sum stay FP64.  Rounding each table entry to FP32 moves it by at most 2^-24
relative, and a macroscopic value is a sum of non-negative terms
N_i ((1 - f) s_k + f s_{k+1}), so the exact lookup on FP32 tables is within
2^-24 relative of the FP64 definition (plus FP64 rounding); the fast
arithmetic adds its own 1e-6 budget.  Tallies and derivative tallies differ
only through histories whose decisions move with the tables: compared in
standard errors of the batch means.  All against the oracle on the
UNROUNDED FP64 tables."""
import numpy as np
import pytest

import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def mcx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx as m
    return m


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_fp32_table_lookup_error_against_the_fp64_definition(mcx):
    """355 x 11,303 library, 12 materials, 200,000 lookups: per channel the
    exact path on FP32 tables stays within 2^-24 of the FP64 definition and
    the benchmark's fast binned path within 1e-6 + 2^-24; the measured
    maxima and medians are printed."""
    import torch
    lib = synth.species_library(355, 11_303, 1236)
    mats = synth.lookup_materials(355, 1236)
    E, mat = synth.lookup_inputs(200_000, mats.n_materials, 1337)
    ref = oracle.xs_lookup(lib, mats, E, mat, n_threads=8)
    p = mcx.Problem(None).load_tables(lib, mats, precision=mcx.FP32, hash_bins=68_400)
    dE, dm = torch.as_tensor(E, device="cuda"), torch.as_tensor(mat, device="cuda")
    exact = p.xs_lookup(dE, dm).cpu().numpy()
    fast = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT).cpu().numpy()
    re, rf = _rel(exact, ref), _rel(fast, ref)
    print("\nFP32 tables vs FP64 definition, per channel (max, median): exact",
          [(float(re[:, c].max()), float(np.median(re[:, c]))) for c in range(5)],
          "fast", [(float(rf[:, c].max()), float(np.median(rf[:, c]))) for c in range(5)])
    assert re.max() <= U32 + 1e-12
    assert rf.max() <= 1e-6 + U32
    p.close()


def _z(a, b, batches_a, batches_b):
    """|a - b| in standard errors of the difference of the two batch means."""
    B = batches_a.shape[0]
    se = np.sqrt(batches_a.var(axis=0, ddof=1) / B + batches_b.var(axis=0, ddof=1) / B)
    d = np.abs(a - b)
    return np.where(se > 0, d / np.where(se > 0, se, 1.0), np.where(d > 0, np.inf, 0.0))


def test_fp32_table_tallies_against_the_fp64_oracle(mcx):
    """17x17 lattice, 20,000 histories, FP32 tables on the GPU against the
    oracle on the FP64 tables: every region's flux and absorption mean within
    3 standard errors (the two runs share their random numbers, so they
    differ only through histories that a table rounding moves)."""
    prob = synth.config3_problem(n_histories=20_000)
    ref = oracle.transport(prob, seed=19, n_threads=8)
    p = mcx.make_problem(prob, precision=mcx.FP32, hash_bins=37_100)
    p.set_tuning(mode=1, sort_period=1, sort_threshold=0)
    p.run(particles_in_flight=8192, seed=19)
    g = p.tallies()
    zs = {}
    for k in ("flux", "absorb"):
        z = _z(g[k].sum(0), ref[k].sum(0), g[k], ref[k])
        zs[k] = (float(z.max()), float(np.median(z)))
        assert z.max() < 3.0, k
    print("\nFP32-table tallies vs FP64 oracle, |diff| in SE (max, median):", zs)
    p.close()


def test_fp32_table_derivative_tallies_against_the_fp64_oracle(mcx):
    """9x9 lattice with derivative tallies (3 density scales), 6,000
    histories: FP32 tables on the GPU against the oracle on the FP64 tables,
    each region's derivative of the absorption within 3 standard errors."""
    prob = synth.config3_problem(n_histories=6000, lattice_n=9)
    ref = oracle.transport(prob, seed=23, derivatives=True, n_threads=8)
    p = mcx.make_problem(prob, precision=mcx.FP32, flags=mcx.FLAG_DERIVATIVES)
    p.set_tuning(mode=1)
    p.run(particles_in_flight=4096, seed=23)
    g = p.tallies()
    z = _z(g["dabsorb"].sum(0), ref["dabsorb"].sum(0), g["dabsorb"], ref["dabsorb"])
    print("\nFP32-table derivative tallies vs FP64 oracle, |diff| in SE (max, median):",
          float(z.max()), float(np.median(z)))
    assert z.max() < 3.0
    p.close()
