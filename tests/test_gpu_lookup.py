"""GPU parity of the macroscopic cross-section lookup against the CPU oracle.

Exact mode must reproduce the plain FP64 definition bit for bit (indices and
values); fast mode must stay within 1e-6 relative; hash bins and binning must
change nothing.  Sizes span several 256-thread tiles with a ragged tail, and
the full 355-species / 1e8-lookup workload is checked on sampled outputs in
the launch configuration the benchmark times.
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


@pytest.fixture(scope="module")
def small_case():
    lib = synth.species_library(40, 700, 101)
    mats = synth.lookup_materials(40, 102, n_materials=6)
    E, mat = synth.lookup_inputs(50_011, mats.n_materials, 103)
    rng = np.random.default_rng(104)
    E[:300] = lib.energies[rng.integers(0, len(lib.energies), 300)]       # exact grid points
    E[300:310] = [1e-7, 1e-6, 9.99e-6, 1e-5, 2e7, 2.0000001e7, 3e7, 1e9, 5e-6, 1e-5]
    return lib, mats, E, mat


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _handle(lib, mats, precision, H):
    from paper_2402_09222_b300 import mcx
    p = mcx.Problem(None)
    p.load_tables(lib, mats, precision=precision, hash_bins=H)
    return p


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("H", [0, 4000])
def test_exact_lookup_is_bit_identical(torch_cuda, small_case, precision, H):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    prec = mcx.FP64 if precision == "fp64" else mcx.FP32
    ref_lib = lib if precision == "fp64" else lib.fp32_rounded()
    ref = oracle.xs_lookup(ref_lib, mats, E, mat, n_threads=8)
    p = _handle(lib, mats, prec, H)
    out = p.xs_lookup(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)).cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("H", [0, 1, 100, 4000, 100_000])
def test_grid_indices_match_for_every_hash_size(torch_cuda, small_case, H):
    torch = torch_cuda
    lib, mats, E, mat = small_case
    ref = oracle.xs_indices(lib, mats, E, mat)
    p = _handle(lib, mats, 0, H)
    k = p.xs_indices(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)).cpu().numpy()
    assert np.array_equal(k, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fast_lookup_within_tolerance(torch_cuda, small_case, precision):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    prec = mcx.FP64 if precision == "fp64" else mcx.FP32
    ref = oracle.xs_lookup(lib if precision == "fp64" else lib.fp32_rounded(), mats, E, mat, n_threads=8)
    p = _handle(lib, mats, prec, 4000)
    out = p.xs_lookup(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32),
                      flags=mcx.LOOKUP_FAST).cpu().numpy()
    rel = np.abs(out - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.all(np.isfinite(out))
    assert rel.max() <= FAST_RTOL, rel.max()


@pytest.mark.parametrize("flags", [2, 3])
def test_binning_changes_nothing(torch_cuda, small_case, flags):
    torch = torch_cuda
    lib, mats, E, mat = small_case
    p = _handle(lib, mats, 1, 4000)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    a = p.xs_lookup(dE, dm, flags=flags & 1).cpu().numpy()
    b = p.xs_lookup(dE, dm, flags=flags).cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def _assert_binned(E, mat, pm, lib, n_materials):
    """pm is a permutation of 0..n-1 grouped by material and, within a
    material, ordered by log E up to one bucket: max(n / (materials x 128),
    16,384) equal log-energy buckets per material over the library's energy
    range, at most 2^21 bins (energies outside it fall into the end
    buckets)."""
    n = len(E)
    assert np.array_equal(np.sort(pm), np.arange(n))
    m = mat[pm].astype(np.int64)
    assert np.all(np.diff(m) >= 0)
    lo, hi = np.log(lib.energies.min()), np.log(lib.energies.max())
    nb = max(1, min(max(n // (n_materials * 128), 16384), (1 << 21) // n_materials))
    width = (hi - lo) / nb
    x = np.clip(np.log(E[pm]), lo, hi)
    starts = np.flatnonzero(np.r_[True, np.diff(m) != 0])
    for a, b in zip(starts, np.r_[starts[1:], n]):
        drop = np.maximum.accumulate(x[a:b]) - x[a:b]
        assert drop.max() <= width * (1 + 1e-4) + 1e-5, (drop.max(), width)


@pytest.mark.parametrize("n", [1, 777, 1_000_003, 4_194_304, 50_000_017])
def test_binning_orders_by_material_then_log_energy(torch_cuda, n):
    """mcx_xs_sort over 12 materials: up to 25.2e6 lookups the floor of
    16,384 buckets per material (196,608 bins); 5e7 lookups, 32,552 buckets
    per material (390,624 bins).  Below 2^22 lookups the one-level counting
    sort (counters scanned in 192 parts), from 2^22 the two-level one (384
    coarse bins x 256 tiles of 16384 lookups at 2^22; 763 x 3052 at 5e7).  A
    NaN energy takes the first bucket, energies outside the grid the end
    buckets.  (Counting in shared memory, at most 12,288 bins, is the
    static-scratch entry point's, tested with it.)"""
    torch = torch_cuda
    lib = synth.species_library(20, 200, 141)
    mats = synth.lookup_materials(20, 142, n_materials=12)
    E, mat = synth.lookup_inputs(n, mats.n_materials, 143)
    if n >= 3:
        E[:3] = [np.nan, 1e-9, 1e9]
    p = _handle(lib, mats, 1, 1000)
    perm = p.xs_sort(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32))
    Ec = np.where(np.isnan(E), lib.energies.min(), E)
    _assert_binned(Ec, mat, perm.cpu().numpy(), lib, mats.n_materials)
    p.close()


def test_binning_with_many_coarse_bins(torch_cuda):
    """4.2e6 lookups over 120 materials: 16,384 buckets per material, 1.97e6
    bins, 3,840 coarse bins of 512 -- the two-level binning's tile scan then
    covers nearly its 4,096."""
    torch = torch_cuda
    lib = synth.species_library(150, 200, 161)
    mats = synth.lookup_materials(150, 162, n_materials=120)
    n = 4_200_007
    E, mat = synth.lookup_inputs(n, mats.n_materials, 163)
    p = _handle(lib, mats, 1, 1000)
    perm = p.xs_sort(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32))
    _assert_binned(E, mat, perm.cpu().numpy(), lib, mats.n_materials)
    p.close()


@pytest.mark.parametrize("n", [3_000_017, 5_000_011])
@pytest.mark.parametrize("layout", ["one_bin", "sorted", "pairs"])
def test_binning_of_concentrated_and_presorted_batches(torch_cuda, layout, n):
    """Batches whose neighbouring lookups share bins: every lookup in one bin,
    a batch already sorted by energy, and equal neighbours in pairs, over 12
    materials; 3e6 lookups take the one-level sort (its warp-aggregated
    path), 5e6 the two-level one (every lookup of a one-bin batch in one
    coarse bin)."""
    torch = torch_cuda
    lib = synth.species_library(20, 200, 151)
    mats = synth.lookup_materials(20, 152, n_materials=12)
    E, mat = synth.lookup_inputs(n, mats.n_materials, 153)
    if layout == "one_bin":
        E[:] = 1.0
        mat[:] = 5
    elif layout == "sorted":
        o = np.lexsort((E, mat))
        E, mat = E[o], mat[o]
    else:
        E[1::2] = E[:-1:2]
        mat[1::2] = mat[:-1:2]
    p = _handle(lib, mats, 1, 1000)
    pm = p.xs_sort(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)).cpu().numpy()
    _assert_binned(E, mat, pm, lib, mats.n_materials)
    p.close()


def test_degenerate_inputs(torch_cuda, small_case):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    p = _handle(lib, mats, 0, 100)
    # empty and single lookups
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert p.xs_lookup(empty, torch.empty(0, dtype=torch.int32, device="cuda")).shape == (0, 5)
    one = p.xs_lookup(_dev(torch, E[:1], torch.float64), _dev(torch, mat[:1], torch.int32)).cpu().numpy()
    assert np.array_equal(one, oracle.xs_lookup(lib, mats, E[:1], mat[:1]))
    # out-of-range materials and NaN energies
    Eb = np.array([1.0, 2.0, float("nan"), 3.0])
    mb = np.array([-1, mats.n_materials, 0, 1], np.int32)
    for fl in (mcx.LOOKUP_EXACT, mcx.LOOKUP_FAST):
        o = p.xs_lookup(_dev(torch, Eb, torch.float64), _dev(torch, mb, torch.int32), flags=fl).cpu().numpy()
        assert np.all(np.isnan(o[:3])) and np.all(np.isfinite(o[3]))
    # a library whose materials hold one species and whose grids have 2 points
    lib2 = synth.flat_library(3.0, 4.0)
    mats2 = synth.make_materials([[0]], [[0.5]])
    p2 = _handle(lib2, mats2, 0, 7)
    Es = np.array([1e-9, 1e-5, 1.0, 2e7, 1e12])
    o = p2.xs_lookup(_dev(torch, Es, torch.float64), _dev(torch, np.zeros(5, np.int32), torch.int32))
    np.testing.assert_array_equal(o.cpu().numpy(), np.tile([1.5, 2.0], (5, 1)))


def test_wrong_arguments_raise(torch_cuda, small_case):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    p = _handle(lib, mats, 0, 0)
    with pytest.raises(TypeError):
        p.xs_lookup(torch.zeros(4, dtype=torch.float32, device="cuda"), torch.zeros(4, dtype=torch.int32, device="cuda"))
    with pytest.raises(mcx.McxError):
        p.xs_indices(_dev(torch, E[:4], torch.float64), _dev(torch, mat[:4], torch.int32), max_species=1)
    bad = synth.Library(lib.grid_offsets, lib.energies.copy(), lib.sigma, lib.awr)
    bad.energies[5] = bad.energies[4]
    with pytest.raises(mcx.McxError, match="not strictly increasing"):
        mcx.Problem(None).load_tables(bad, mats)
    negs = synth.Library(lib.grid_offsets, lib.energies, lib.sigma.copy(), lib.awr)
    negs.sigma[7, 1] = -1.0
    with pytest.raises(mcx.McxError, match="sigma"):
        mcx.Problem(None).load_tables(negs, mats)


def test_host_path_matches_device_path(torch_cuda, small_case):
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    p = _handle(lib, mats, 1, 4000)
    dev = p.xs_lookup(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32), flags=mcx.LOOKUP_FAST)
    Eh = torch.as_tensor(E).pin_memory()
    mh = torch.as_tensor(mat).pin_memory()
    host = p.xs_lookup_host(Eh, mh, flags=mcx.LOOKUP_FAST)
    assert torch.equal(host, dev.cpu())
    host2 = p.xs_lookup_host(E, mat, flags=mcx.LOOKUP_FAST)
    assert np.array_equal(host2, dev.cpu().numpy())
    host3 = p.xs_lookup_host(Eh, mh, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT)
    assert torch.equal(host3, dev.cpu())


@pytest.mark.parametrize("flags", [1, 3, 9, 11])
def test_host_path_over_several_pipeline_chunks(torch_cuda, flags):
    """7,000,003 lookups from pinned host buffers: four 2M-lookup chunks over
    the three pipeline streams with FP64 outputs (the first stream's staging
    reused, a ragged last chunk), two 4M-lookup chunks with FP32 outputs,
    binned per chunk or not; equal to the device path bit for bit."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(30, 600, 221)
    mats = synth.lookup_materials(30, 222, n_materials=7)
    E, mat = synth.lookup_inputs(7_000_003, mats.n_materials, 223)
    E[[5, 2_097_152, 6_999_999]] = [np.nan, 1e-9, 1e9]
    mat[[7, 4_194_304]] = [-1, mats.n_materials]
    p = _handle(lib, mats, 1, 2000)
    dev = p.xs_lookup(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32), flags=flags).cpu()
    host = p.xs_lookup_host(torch.as_tensor(E).pin_memory(), torch.as_tensor(mat).pin_memory(), flags=flags)
    assert host.dtype == dev.dtype
    assert torch.equal(host.view(torch.uint8), dev.view(torch.uint8))
    p.close()


def test_backward_matches_oracle_adjoint(torch_cuda):
    torch = torch_cuda
    lib = synth.species_library(12, 300, 211)
    mats = synth.lookup_materials(12, 212, n_materials=4)
    E, mat = synth.lookup_inputs(20_003, mats.n_materials, 213)
    G = np.random.default_rng(214).normal(size=(len(E), lib.n_ch))
    gd_ref, gs_ref = oracle.xs_lookup_backward(lib, mats, E, mat, G)
    p = _handle(lib, mats, 0, 4000)
    gd, gs = p.xs_lookup_backward(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32),
                                  _dev(torch, G, torch.float64))
    gd, gs = gd.cpu().numpy(), gs.cpu().numpy()
    np.testing.assert_allclose(gd, gd_ref, rtol=1e-11, atol=1e-11 * np.abs(gd_ref).max())
    np.testing.assert_allclose(gs, gs_ref, rtol=1e-11, atol=1e-11 * np.abs(gs_ref).max())


@pytest.mark.parametrize("precision,n_ch", [("fp64", 5), ("fp32", 5), ("fp32", 2), ("fp64", 1)])
def test_backward_binned_dense_and_edge_cases(torch_cuda, precision, n_ch):
    """The binned, per-warp aggregated adjoint against the oracle's sequential
    adjoint: 1e6 lookups dense enough that most warps sit inside one grid
    interval of every species (the closed form from the warp's totals), plus
    warps that straddle grid points and edge energies: exact grid points,
    below and above every grid (clamped fractions), zero, negative and
    infinite energies, NaN energies and out-of-range materials (which must
    contribute nothing), and a ragged tail."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    full = synth.species_library(40, 700, 221)
    lib = full.channels(list(range(n_ch))) if n_ch != 5 else full
    mats = synth.lookup_materials(40, 222, n_materials=5)
    rng = np.random.default_rng(223)
    n = 1_000_003
    E, mat = synth.lookup_inputs(n, mats.n_materials, 224)
    # half of the lookups crowd into a few narrow energy windows
    centres = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), 64))
    half = n // 2
    E[:half] = centres[rng.integers(0, 64, half)] * (1.0 + 1e-5 * rng.standard_normal(half))
    E[half:half + 2000] = lib.energies[rng.integers(0, len(lib.energies), 2000)]
    E[half + 2000:half + 2010] = [1e-9, 1e-6, 0.0, -1.0, -0.0, 3e7, 1e12, np.inf, 9.99e-6, 2e7]
    E[half + 3000:half + 3005] = np.nan
    mat[half + 4000:half + 4003] = [-1, mats.n_materials, 1 << 20]
    G = rng.normal(size=(n, lib.n_ch))
    ok = ~np.isnan(E) & (mat >= 0) & (mat < mats.n_materials)
    ref_lib = lib if precision == "fp64" else lib.fp32_rounded()
    gd_ref, gs_ref = oracle.xs_lookup_backward(ref_lib, mats, E[ok], mat[ok], G[ok])
    p = _handle(lib, mats, mcx.FP64 if precision == "fp64" else mcx.FP32, 4000)
    gd, gs = p.xs_lookup_backward(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32),
                                  _dev(torch, G, torch.float64))
    gd, gs = gd.cpu().numpy(), gs.cpu().numpy()
    np.testing.assert_allclose(gd, gd_ref, rtol=1e-11, atol=1e-11 * np.abs(gd_ref).max())
    np.testing.assert_allclose(gs, gs_ref, rtol=1e-11, atol=1e-11 * np.abs(gs_ref).max())
    p.close()


def test_config2_full_size_sampled(torch_cuda):
    """355 species x 11,303 points, 12 materials, 1e8 lookups with FP32 tables
    in exactly the launch the benchmark times (its hash-bin count, binning
    into a caller-held permutation with the inputs carried into the binned
    order, then the round-linear fast lookup over it with chunk-claiming
    warps); 20,000 sampled outputs checked against
    the oracle on the FP32-rounded tables, and the exact FP64 full-search
    path on the same sample bit for bit."""
    import bench
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = bench.workload_inputs(0)
    n = len(E)
    assert n == 100_000_000
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    idx = np.random.default_rng(5).choice(n, 20_000, replace=False)
    p32 = _handle(lib, mats, bench.TUNED["precision"], bench.TUNED["hash_bins"])
    out = torch.empty((n, 5), dtype=torch.float64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    perm, Eb, mb = p32.xs_sort_inputs(dE, dm, perm)
    p32.xs_lookup_ordered(Eb, mb, perm, out=out, flags=bench.TUNED["flags"] | mcx.LOOKUP_BINNED_INPUTS)
    del Eb, mb
    got = out[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E[idx], mat[idx], n_threads=8)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.all((ref == 0) <= (got == 0)), "an exactly-zero channel came out non-zero"
    assert rel.max() <= FAST_RTOL, rel.max()
    # the permutation is a permutation, and sorted by (material, energy bucket)
    _assert_binned(E, mat, perm.cpu().numpy(), lib, mats.n_materials)
    del out, perm
    p32.close()
    p64 = _handle(lib, mats, mcx.FP64, 0)
    out64 = p64.xs_lookup(dE, dm)
    got64 = out64[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ref64 = oracle.xs_lookup(lib, mats, E[idx], mat[idx], n_threads=8)
    assert np.array_equal(got64.view(np.uint64), ref64.view(np.uint64))


@pytest.mark.parametrize("n_ch", [1, 2, 3, 5])
@pytest.mark.parametrize("H", [0, 1, 100_000])
def test_fast_path_every_record_width_and_hash_size(torch_cuda, n_ch, H):
    """Point records hold one float4 for n_ch <= 2 and two above; every width
    and hash size must stay within the fast tolerance, binned or not."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    full = synth.species_library(25, 600, 601)
    lib = full.channels(list(range(n_ch)))
    mats = synth.lookup_materials(25, 602, n_materials=5)
    E, mat = synth.lookup_inputs(30_001, mats.n_materials, 603)
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E, mat, n_threads=8)
    p = _handle(lib, mats, mcx.FP32, H)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    for flags in (mcx.LOOKUP_FAST, mcx.LOOKUP_FAST | mcx.LOOKUP_SORT):
        out = p.xs_lookup(dE, dm, flags=flags).cpu().numpy()
        rel = np.abs(out - ref) / np.maximum(np.abs(ref), 1e-300)
        assert out.shape == (len(E), n_ch)
        assert rel.max() <= FAST_RTOL, (flags, rel.max())
    # exact path on the same handle stays bit-identical
    out = p.xs_lookup(dE, dm).cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


def test_zero_and_subnormal_table_entries(torch_cuda):
    """FP32 tables widen to FP64 with integer operations except for zero and
    FP32-subnormal values; both must come out exact."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(6, 200, 611)
    sig = lib.sigma.copy()
    sig[::7, 3] = 0.0
    sig[::11, 1] = 1e-40          # subnormal in FP32
    sig[::13, 2] = 3e-39          # subnormal in FP32
    lib = synth.Library(lib.grid_offsets, lib.energies, sig, lib.awr)
    mats = synth.lookup_materials(6, 612, n_materials=3)
    E, mat = synth.lookup_inputs(20_000, mats.n_materials, 613)
    E[:500] = lib.energies[np.random.default_rng(1).integers(0, len(lib.energies), 500)]
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E, mat)
    p = _handle(lib, mats, mcx.FP32, 300)
    out = p.xs_lookup(_dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)).cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("n_ch,H", [(5, 68_400), (5, 0), (2, 4000), (3, 100)])
def test_staged_lookup_matches_the_direct_form_bit_for_bit(torch_cuda, n_ch, H):
    """The TMA-staged binned lookup evaluates the same per-species terms in the
    same order as the global-memory form: identical outputs, on a binned order
    with chunks that span materials, a ragged tail, NaN energies and invalid
    materials (those chunks take the global-memory form), exact grid points
    and energies outside the grid."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    chans = {5: None, 2: [synth.CH_SCATTER, synth.CH_ABSORB],
             3: [synth.CH_SCATTER, synth.CH_ABSORB, synth.CH_NU_FISSION]}[n_ch]
    lib = synth.species_library(120, 3000, 111)
    if chans:
        lib = lib.channels(chans)
    mats = synth.lookup_materials(120, 112, n_materials=9)
    E, mat = synth.lookup_inputs(300_017, mats.n_materials, 113)
    rng = np.random.default_rng(114)
    E[:500] = lib.energies[rng.integers(0, len(lib.energies), 500)]
    E[500:510] = [1e-7, 1e-6, 9.99e-6, 1e-5, 2e7, 2.0000001e7, 3e7, 1e9, 5e-6, 1e-5]
    E[600] = np.nan
    mat[700] = -1
    mat[701] = mats.n_materials
    p = _handle(lib, mats, mcx.FP32, H)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm = p.xs_sort(dE, dm)
    direct = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST).cpu().numpy()
    staged = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_STAGED).cpu().numpy()
    p.check_device()
    assert np.array_equal(staged.view(np.uint64), direct.view(np.uint64))
    # and against the definition on the FP32-rounded tables
    ok = np.isfinite(E) & (mat >= 0) & (mat < mats.n_materials)
    ref = oracle.xs_lookup(lib.fp32_rounded(), mats, E[ok], mat[ok], n_threads=8)
    rel = np.abs(staged[ok] - ref) / np.maximum(np.abs(ref), 1e-300)
    assert rel.max() <= FAST_RTOL
    assert np.all(np.isnan(staged[~ok]))
    p.close()


def test_staged_lookup_wait_that_runs_out_is_reported(torch_cuda, monkeypatch):
    """The staged lookup's mbarrier waits are bounded.  With the test hook
    MCX_TEST_STAGED_STALL=1 the producers leave their first chunk unstaged
    and unsignalled (no copy is issued for it) and the waits are limited to
    about 0.1 ms, so the consumers' waits run out: mcx_check_device must
    report it, clear the flag, and the handle must compute correctly
    afterwards."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(120, 3000, 111)
    mats = synth.lookup_materials(120, 112, n_materials=9)
    E, mat = synth.lookup_inputs(300_017, mats.n_materials, 113)
    p = _handle(lib, mats, mcx.FP32, 4000)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm = p.xs_sort(dE, dm)
    monkeypatch.setenv("MCX_TEST_STAGED_STALL", "1")
    p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_STAGED)
    with pytest.raises(mcx.McxError, match="TIMEOUT"):
        p.check_device()
    monkeypatch.delenv("MCX_TEST_STAGED_STALL")
    p.check_device()   # the flag was cleared
    staged = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_STAGED)
    p.check_device()
    direct = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST)
    assert torch.equal(staged.view(torch.int64), direct.view(torch.int64))
    p.close()


def test_staged_lookup_on_the_benchmark_tables(torch_cuda):
    """355 species x 11,303 points, materials up to 321 species, 4e6 binned
    lookups: staged and direct forms agree bit for bit."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib = synth.species_library(355, 11_303, 1236)
    mats = synth.lookup_materials(355, 1236)
    E, mat = synth.lookup_inputs(4_000_000, mats.n_materials, 1336)
    p = _handle(lib, mats, mcx.FP32, 68_400)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    perm = p.xs_sort(dE, dm)
    direct = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST)
    staged = p.xs_lookup_ordered(dE, dm, perm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_STAGED)
    p.check_device()
    assert torch.equal(direct.view(torch.int64), staged.view(torch.int64))
    p.close()


def test_fp32_outputs_are_the_fp64_outputs_rounded_once(torch_cuda, small_case):
    """MCX_LOOKUP_OUT32 writes the compensated sum rounded once to FP32: the
    FP64 fast output rounded to FP32, bit for bit, on device and host paths,
    direct and staged; the exact form refuses it."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    lib, mats, E, mat = small_case
    p = _handle(lib, mats, mcx.FP32, 4000)
    dE, dm = _dev(torch, E, torch.float64), _dev(torch, mat, torch.int32)
    ref = p.xs_lookup(dE, dm, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT).float()
    for fl in (mcx.LOOKUP_FAST, mcx.LOOKUP_FAST | mcx.LOOKUP_SORT,
               mcx.LOOKUP_FAST | mcx.LOOKUP_SORT | mcx.LOOKUP_STAGED):
        got = p.xs_lookup(dE, dm, flags=fl | mcx.LOOKUP_OUT32)
        assert got.dtype == torch.float32
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), fl
    host = p.xs_lookup_host(torch.as_tensor(E), torch.as_tensor(mat),
                            flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT | mcx.LOOKUP_OUT32)
    assert host.dtype == torch.float32 and torch.equal(host.view(torch.int32), ref.cpu().view(torch.int32))
    with pytest.raises(mcx.McxError, match="ARG"):
        p.xs_lookup(dE, dm, out=torch.empty((len(E), lib.n_ch), dtype=torch.float32, device="cuda"),
                    flags=mcx.LOOKUP_OUT32)
    p.close()
