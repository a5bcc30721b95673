"""The transport kernels' Philox4x32-10 stream against the oracle's (an
independent implementation) and against cuRAND's Philox4x32-10 device
function, run on the GPU."""
import ctypes as C
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("seed,problem,hist,first", [(1, 0, 0, 0), (2**40 + 17, 5, 123456789, 7),
                                                      (0xDEADBEEFCAFE, 63, 2**33 + 5, 1001)])
def test_gpu_stream_equals_oracle_stream(torch_cuda, seed, problem, hist, first):
    from paper_2402_09222_b300 import mcx
    g = mcx.debug_uniforms(seed, problem, hist, 4097, first=first).cpu().numpy()
    o = oracle.uniforms(seed, problem, hist, 4097, first=first)
    assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


def test_philox_core_equals_curand(torch_cuda):
    torch = torch_cuda
    from paper_2402_09222_b300 import mcx  # noqa: F401  (library built)
    lib = C.CDLL(os.path.join(HERE, "csrc", "libcurand_pin.so"))
    rng = np.random.default_rng(3)
    n = 2048
    seeds = rng.integers(0, 2**63, n, dtype=np.uint64)
    hists = rng.integers(0, 2**40, n, dtype=np.uint64)
    draws = rng.integers(0, 2**20, n, dtype=np.uint32)
    ctr = np.stack([draws >> 1, hists & 0xFFFFFFFF, hists >> 32, np.zeros(n, np.uint64)], 1).astype(np.uint32)
    key = np.stack([seeds & 0xFFFFFFFF, seeds >> 32], 1).astype(np.uint32)
    dc = torch.as_tensor(ctr.view(np.int32)).cuda()
    dk = torch.as_tensor(key.view(np.int32)).cuda()
    do = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    assert lib.curand_philox_blocks(C.c_void_p(dc.data_ptr()), C.c_void_p(dk.data_ptr()),
                                    C.c_void_p(do.data_ptr()), n) == 0
    w = do.cpu().numpy().view(np.uint32)
    for i in range(0, n, 97):
        a, b = (w[i, 2], w[i, 3]) if draws[i] & 1 else (w[i, 0], w[i, 1])
        k = (int(a >> 6) << 26) | int(b >> 6)
        u = mcx.debug_uniforms(int(seeds[i]), 0, int(hists[i]), 1, first=int(draws[i])).item()
        assert u == (k + 0.5) * 2.0 ** -52
    # and the raw words agree with the oracle's implementation
    for i in range(0, n, 211):
        assert np.array_equal(oracle.philox4x32_10(ctr[i], key[i]), w[i])


def test_flight_length_logarithm(torch_cuda):
    """The transport's table-driven -ln x (Tang 1990) on 1e6 uniforms of a
    history stream and on the ends of its range (2^-53, around 1/2, 1 - 2^-53)
    and at table boundaries: within 3 ulp of max(1, -ln x) of the host's
    logarithm, as the CUDA library's own is within 1 ulp of it."""
    from paper_2402_09222_b300 import mcx
    torch = torch_cuda
    u = mcx.debug_uniforms(7, 0, 123, 1_000_000)
    edge = [2.0**-53, 3 * 2.0**-53, 2.0**-20, 0.25, 0.5 - 2.0**-54, 0.5, 0.5 + 2.0**-53, 0.75,
            1 / 3, 1 - 2.0**-53, 1 - 2.0**-40, (1 + 1 / 256) / 2, (1 + 255 / 256) / 2 - 2.0**-53]
    x = torch.cat([u, torch.tensor(edge, dtype=torch.float64, device=u.device)])
    out = mcx.debug_neg_log(x).cpu().numpy()
    ref = -np.log(x.cpu().numpy())
    scale = np.maximum(1.0, ref) * 2.0**-52
    err_table = np.abs(out[:, 0] - ref) / scale
    err_lib = np.abs(out[:, 1] - ref) / scale
    assert err_lib.max() <= 1.0, err_lib.max()
    assert err_table.max() <= 3.0, err_table.max()
    assert np.all(out[:, 0] > 0)
