"""GPU parity of the round-linear binned lookup (MCX_LOOKUP_LINEAR) against
the CPU oracle.

Per 64-lookup round of a binned order, species whose grid interval holds the
whole round (or whose grid has one point inside the round's energy range)
are summed as one linear function of E plus a hinge; the rest per lookup.
The outputs must stay within the fast form's 1e-6 relative bound of the
definition (the oracle on the FP32-rounded tables), keep exact zeros, and
treat invalid lookups as the other forms do.  The inputs mix log-uniform
energies (wide rounds: the per-lookup fallback) with narrow bands around
grid points, the grid ends and outside the grid (narrow rounds: the linear
sums, hinges and the clamp exclusions).
"""
import numpy as np
import pytest

import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

FAST_RTOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _handle(lib, mats, precision, H):
    from paper_2402_09222_b300 import mcx
    p = mcx.Problem(None)
    p.load_tables(lib, mats, precision=precision, hash_bins=H)
    return p


def banded_inputs(lib, n_materials, n, seed, frac_banded=0.6, n_bands=40):
    """Log-uniform lookups plus narrow bands (relative widths 1e-6 .. 1e-3)
    centred on random grid points of the library, on both grid ends and just
    outside them; a few exact grid points and out-of-grid energies."""
    rng = np.random.default_rng(seed)
    E, mat = synth.lookup_inputs(n, n_materials, seed + 1)
    nb = int(n * frac_banded)
    centres = lib.energies[rng.integers(0, len(lib.energies), n_bands)]
    centres[:4] = [synth.E_MIN, synth.E_MAX, synth.E_MIN * 0.999, synth.E_MAX * 1.0005]
    widths = 10.0 ** rng.uniform(-6, -3, n_bands)
    which = rng.integers(0, n_bands, nb)
    E[:nb] = centres[which] * (1.0 + widths[which] * rng.uniform(-1, 1, nb))
    E[nb:nb + 200] = lib.energies[rng.integers(0, len(lib.energies), 200)]
    E[nb + 200:nb + 206] = [1e-7, 9.99e-6, 1e-5, 2e7, 2.0000001e7, 1e9]
    perm = rng.permutation(n)
    return E[perm], mat[perm]


def _rel(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)


def _check(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.all(np.isfinite(got[fin]))
    assert np.all((ref == 0) <= (got == 0)), "an exactly-zero channel came out non-zero"
    r = _rel(got[fin], ref[fin])
    assert r.max() <= FAST_RTOL, r.max()
    return r.max()


@pytest.mark.parametrize("n_ch", [1, 2, 3, 5])
@pytest.mark.parametrize("H", [0, 100, 4000])
def test_linear_form_within_tolerance(torch_cuda, n_ch, H):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(40, 700, 701).channels(list(range(n_ch)))
    mats = synth.lookup_materials(40, 702, n_materials=6)
    E, mat = banded_inputs(lib, mats.n_materials, 600_011, 703)
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E, mat, n_threads=8)
    p = _handle(lib, mats, mcx.FP32, H)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    lin = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT | mcx.LOOKUP_LINEAR).cpu().numpy()
    _check(lin, ref)
    # the linear sums ran: some outputs differ from the per-lookup form's in
    # their last bits, by no more than the two forms' bounds allow
    bit = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT).cpu().numpy()
    fin = np.isfinite(bit)
    assert np.any(lin[fin] != bit[fin])
    assert _rel(lin[fin], bit[fin]).max() <= 2 * FAST_RTOL
    # FP32 outputs: the same sums rounded once
    lin32 = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT | mcx.LOOKUP_LINEAR
                        | mcx.LOOKUP_OUT32).cpu().numpy()
    _check(lin32.astype(np.float64), ref)
    p.close()


def test_linear_form_on_an_ordered_call_and_unbinned(torch_cuda):
    """The flag through the caller-binned entry point; without a binned order
    (natural order, no rounds) it changes nothing."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(30, 500, 711)
    mats = synth.lookup_materials(30, 712, n_materials=4)
    E, mat = banded_inputs(lib, mats.n_materials, 300_007, 713)
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E, mat, n_threads=8)
    p = _handle(lib, mats, mcx.FP32, 3000)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm = torch.empty(len(E), dtype=torch.int32, device="cuda")
    p.xs_sort(dE, dm, perm)
    out = torch.empty((len(E), lib.n_ch), dtype=torch.float64, device="cuda")
    p.xs_lookup_ordered(dE, dm, perm, out=out, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_LINEAR)
    _check(out.cpu().numpy(), ref)
    a = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST).cpu().numpy()
    b = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_LINEAR).cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    with pytest.raises(mcx.McxError, match="ARG"):
        p.xs_lookup(dE, dm, flags=mcx.LOOKUP_LINEAR)
    p.close()


@pytest.mark.parametrize("out32", [False, True])
def test_linear_form_host_path_over_several_chunks(torch_cuda, out32):
    """7,000,003 banded lookups from pinned host buffers through the pipeline
    (several chunks, each binned on its own), invalid lookups among them;
    a sample of 60,000 outputs against the oracle."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(30, 600, 721)
    mats = synth.lookup_materials(30, 722, n_materials=7)
    E, mat = banded_inputs(lib, mats.n_materials, 7_000_003, 723)
    E[[5, 2_097_152, 6_999_999]] = [np.nan, 1e-9, 1e9]
    mat[[7, 4_194_304]] = [-1, mats.n_materials]
    p = _handle(lib, mats, mcx.FP32, 2000)
    flags = mcx.LOOKUP_FAST | mcx.LOOKUP_SORT | mcx.LOOKUP_LINEAR | (mcx.LOOKUP_OUT32 if out32 else 0)
    host = p.xs_lookup_host(torch.as_tensor(E).pin_memory(), torch.as_tensor(mat).pin_memory(),
                            flags=flags).numpy().astype(np.float64)
    idx = np.unique(np.concatenate([np.random.default_rng(7).choice(len(E), 60_000, replace=False),
                                    [7, 2_097_152, 4_194_304, 6_999_999]]))
    idx = idx[idx != 5]   # a NaN energy: the oracle's output is NaN, the fast forms' is not defined
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E[idx], mat[idx], n_threads=8)
    _check(host[idx], ref)
    p.close()


@pytest.mark.parametrize("n", [777, 1_000_003, 4_194_304 + 4_321])
def test_sort_inputs_and_lookups_from_binned_inputs(torch_cuda, n):
    """mcx_xs_sort_inputs hands over E[perm] exactly and mat[perm] (-1 for an
    id out of range; one-level batches gather them, two-level ones carry the
    energies through both passes and take the material from the bin),
    and a lookup reading them in the processing order gives the results of
    the same lookup through the permutation bit for bit, in every form."""
    from paper_2402_09222_b300 import mcx
    from test_gpu_lookup import _assert_binned
    torch = torch_cuda
    lib = synth.species_library(30, 600, 731)
    mats = synth.lookup_materials(30, 732, n_materials=7)
    E, mat = banded_inputs(lib, mats.n_materials, n, 733)
    p = _handle(lib, mats, mcx.FP32, 2000)
    # the order: binned as mcx_xs_sort bins
    perm, Eb, mb = p.xs_sort_inputs(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32))
    _assert_binned(E, mat, perm.cpu().numpy(), lib, mats.n_materials)
    # invalid lookups among them
    E[[3, n // 2]] = [np.nan, 1e12]
    mat[[5, n - 1]] = [-1, mats.n_materials]
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm, Eb, mb = p.xs_sort_inputs(dE, dm, perm, Eb, mb)
    pm = perm.cpu().numpy()
    assert np.array_equal(np.sort(pm), np.arange(n))
    assert np.array_equal(Eb.cpu().numpy().view(np.uint64), E[pm].view(np.uint64))
    valid = (mat[pm] >= 0) & (mat[pm] < mats.n_materials)
    assert np.array_equal(mb.cpu().numpy(), np.where(valid, mat[pm], -1))
    F, L, O = mcx.LOOKUP_FAST, mcx.LOOKUP_LINEAR, mcx.LOOKUP_OUT32
    for flags in (F, F | L, F | L | O):
        a = p.xs_lookup_ordered(dE, dm, perm, flags=flags).cpu().numpy()
        b = p.xs_lookup_ordered(Eb, mb, perm, flags=flags | mcx.LOOKUP_BINNED_INPUTS).cpu().numpy()
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), flags
        assert np.all(np.isnan(b[[5, n - 1]]))
    for bad in (mcx.LOOKUP_BINNED_INPUTS, F | mcx.LOOKUP_STAGED | mcx.LOOKUP_BINNED_INPUTS):
        with pytest.raises(mcx.McxError, match="ARG"):
            p.xs_lookup_ordered(Eb, mb, perm, flags=bad)
    with pytest.raises(mcx.McxError, match="ARG"):
        p.xs_lookup_ordered(Eb, mb, None, flags=F | mcx.LOOKUP_BINNED_INPUTS)
    p.close()


def test_sort_inputs_with_many_coarse_bins(torch_cuda):
    """120 materials x 16,384 buckets (3,840 coarse bins: pass A's staging
    at its largest) handing the inputs over; the round-linear lookup on
    them within the bound."""
    from paper_2402_09222_b300 import mcx
    from test_gpu_lookup import _assert_binned
    torch = torch_cuda
    lib = synth.species_library(60, 300, 741)
    mats = synth.lookup_materials(60, 742, n_materials=120)
    E, mat = banded_inputs(lib, mats.n_materials, 4_300_007, 743)
    p = _handle(lib, mats, mcx.FP32, 1000)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm, Eb, mb = p.xs_sort_inputs(dE, dm)
    pm = perm.cpu().numpy()
    _assert_binned(E, mat, pm, lib, mats.n_materials)
    assert np.array_equal(Eb.cpu().numpy().view(np.uint64), E[pm].view(np.uint64))
    assert np.array_equal(mb.cpu().numpy(), mat[pm])
    out = p.xs_lookup_ordered(Eb, mb, perm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_LINEAR
                              | mcx.LOOKUP_BINNED_INPUTS).cpu().numpy()
    idx = np.random.default_rng(9).choice(len(E), 40_000, replace=False)
    _check(out[idx], oracle.xs_lookup(lib.fp32_rounded(), mats, E[idx], mat[idx], n_threads=8))
    p.close()
