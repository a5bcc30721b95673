"""The static-scratch binned lookup (mcx_xs_lookup_binned_static) for callers
that cannot allocate device memory: it must give what the allocating binned
lookup gives, call after call (its shared scratch keeps the previous call's
contents), and refuse batches beyond its fixed capacity.  Collected last so a
failure here cannot hide the rest of the suite."""
import ctypes as C

import numpy as np
import pytest

from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

FAST_RTOL = 1e-6
MAX_LOOKUPS = 1 << 20


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_09222_b300 import mcx
    f = mcx._lib.mcx_xs_lookup_binned_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    return torch, mcx, f


def _call(torch, mcx, f, h, E, mat, flags):
    out = torch.full((E.numel(), h.n_ch), float("nan"), dtype=torch.float64, device="cuda")
    rc = f(h.h, E.numel(), C.c_void_p(E.data_ptr()), C.c_void_p(mat.data_ptr()),
           C.c_void_p(out.data_ptr()), flags, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, mcx._lib.mcx_last_error().decode()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("flags", [0, 1])
def test_static_scratch_matches_the_oracle_and_the_allocating_lookup(env, flags):
    """Against the oracle on the FP32-rounded tables (the exact form bit for
    bit, the fast form within 1e-6 relative) and against the allocating
    binned lookup, on two calls in a row: a full-capacity batch, then a
    smaller one over a different material mix (stale scratch must not leak
    through)."""
    import oracle
    torch, mcx, f = env
    lib = synth.species_library(60, 900, 501)
    mats = synth.lookup_materials(60, 502, n_materials=9)
    h = mcx.Problem(None).load_tables(lib, mats, precision=mcx.FP32, hash_bins=4000)
    lib32 = lib.fp32_rounded()
    for n, seed, n_mat in ((MAX_LOOKUPS, 503, 9), (123_457, 504, 4)):
        E, mat = synth.lookup_inputs(n, n_mat, seed)
        dE = torch.as_tensor(E, device="cuda")
        dm = torch.as_tensor(mat, device="cuda")
        got = _call(torch, mcx, f, h, dE, dm, flags)
        want = oracle.xs_lookup(lib32, mats, E, mat, n_threads=8)
        g = got.cpu().numpy()
        if flags & mcx.LOOKUP_FAST:
            rel = np.abs(g - want) / np.maximum(np.abs(want), 1e-300)
            assert rel.max() <= FAST_RTOL, rel.max()
        else:
            assert np.array_equal(g.view(np.uint64), want.view(np.uint64))
        ref = h.xs_lookup(dE, dm, flags=flags | mcx.LOOKUP_SORT)
        torch.testing.assert_close(got, ref, rtol=FAST_RTOL, atol=0.0)


def test_static_scratch_rejects_oversized_batches(env):
    torch, mcx, f = env
    lib = synth.species_library(5, 50, 511)
    mats = synth.lookup_materials(5, 512, n_materials=2)
    h = mcx.Problem(None).load_tables(lib, mats)
    E = torch.ones(MAX_LOOKUPS + 1, dtype=torch.float64, device="cuda")
    m = torch.zeros(MAX_LOOKUPS + 1, dtype=torch.int32, device="cuda")
    out = torch.empty((MAX_LOOKUPS + 1, h.n_ch), dtype=torch.float64, device="cuda")
    rc = f(h.h, MAX_LOOKUPS + 1, C.c_void_p(E.data_ptr()), C.c_void_p(m.data_ptr()),
           C.c_void_p(out.data_ptr()), 0, None)
    assert rc == mcx.McxError(-1, "").code
    assert "MCX_STATIC_MAX_LOOKUPS" in mcx._lib.mcx_last_error().decode()
