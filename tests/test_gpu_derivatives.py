"""Differentiation on the GPU: the adjoint of the lookup behind a
torch.autograd.Function (gradcheck in FP64, FP32 tables against the oracle's
adjoint), and the likelihood-ratio density-derivative tallies of the lattice
against central finite differences with common random numbers."""
import math

import numpy as np
import pytest

import oracle
from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_autograd_gradcheck_fp64(torch_cuda):
    torch = torch_cuda
    from paper_2402_09222_b300 import autograd, mcx
    lib = synth.species_library(4, 24, 401)
    mats = synth.make_materials([[0, 2], [1, 2, 3]], [[0.02, 0.5], [0.3, 0.01, 0.07]])
    E, mat = synth.lookup_inputs(41, 2, 402)
    h = mcx.Problem(None).load_tables(lib, mats, precision=mcx.FP64, hash_bins=16)
    dE = torch.as_tensor(E, device="cuda")
    dm = torch.as_tensor(mat, device="cuda")
    dens = torch.as_tensor(mats.dens, device="cuda").clone().requires_grad_(True)
    sig = torch.as_tensor(lib.sigma, device="cuda").clone().requires_grad_(True)
    # the map is linear in both inputs, so a large step is exact up to rounding;
    # with cross sections up to ~1e4 b a 1e-6 step would leave ~1e-6 relative
    # rounding noise in the central differences
    assert torch.autograd.gradcheck(lambda d, s: autograd.xs_lookup(h, d, s, dE, dm), (dens, sig),
                                    eps=1e-3, atol=1e-9, rtol=1e-7)
    # forward equals the oracle, and the gradient of a weighted sum equals the oracle adjoint
    out = autograd.xs_lookup(h, dens, sig, dE, dm)
    assert np.array_equal(out.detach().cpu().numpy(), oracle.xs_lookup(lib, mats, E, mat))
    G = torch.randn(out.shape, dtype=torch.float64, device="cuda")
    (out * G).sum().backward()
    gd, gs = oracle.xs_lookup_backward(lib, mats, E, mat, G.cpu().numpy())
    np.testing.assert_allclose(dens.grad.cpu().numpy(), gd, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(sig.grad.cpu().numpy(), gs, rtol=1e-12, atol=1e-14)


def test_backward_into_fp32_tables(torch_cuda):
    torch = torch_cuda
    from paper_2402_09222_b300 import mcx
    lib = synth.species_library(30, 800, 411)
    mats = synth.lookup_materials(30, 412, n_materials=5)
    E, mat = synth.lookup_inputs(30_011, mats.n_materials, 413)
    G = np.random.default_rng(414).normal(size=(len(E), lib.n_ch))
    h = mcx.Problem(None).load_tables(lib, mats, precision=mcx.FP32, hash_bins=4000)
    gd, gs = h.xs_lookup_backward(torch.as_tensor(E, device="cuda"), torch.as_tensor(mat, device="cuda"),
                                  torch.as_tensor(G, device="cuda"))
    rd, rs = oracle.xs_lookup_backward(lib.fp32_rounded(), mats, E, mat, G)
    np.testing.assert_allclose(gd.cpu().numpy(), rd, rtol=1e-11, atol=1e-11 * np.abs(rd).max())
    np.testing.assert_allclose(gs.cpu().numpy(), rs, rtol=1e-11, atol=1e-11 * np.abs(rs).max())


def test_lattice_lr_derivatives_match_central_differences(torch_cuda):
    """2e6 histories on the 17x17 lattice: d(absorption in the 289 pin cells)
    / d(density scale of each material), likelihood ratio against central
    differences at s_m = 1 +- 1e-3 with common random numbers; per-batch
    differences agree within 3 standard errors."""
    from paper_2402_09222_b300 import mcx
    n_hist, h, seed = 2_000_000, 1e-3, 41
    prob = synth.config3_problem(n_histories=n_hist)
    pins = slice(0, 289)
    p = mcx.make_problem(prob, flags=mcx.FLAG_DERIVATIVES)
    p.set_tuning(mode=1, sort_period=4, sort_threshold=0)
    p.run(particles_in_flight=1_000_000, seed=seed)
    lr = p.tallies()["dabsorb"][:, pins, :].sum(1)          # [B][3]
    p.close()
    for m in range(3):
        fd = []
        for sgn in (+1, -1):
            scales = [1.0, 1.0, 1.0]
            scales[m] += sgn * h
            pr = synth.config3_problem(n_histories=n_hist, lib=prob.lib)
            pr.mats = prob.mats.scaled(scales)
            q = mcx.make_problem(pr)
            q.set_tuning(mode=1)
            q.run(particles_in_flight=1_000_000, seed=seed)
            fd.append(q.tallies()["absorb"][:, pins].sum(1))
            q.close()
        fdm = (fd[0] - fd[1]) / (2 * h)
        d = lr[:, m] - fdm
        se = d.std(ddof=1) / math.sqrt(len(d))
        assert abs(d.mean()) <= 3 * se, (m, lr[:, m].sum(), fdm.sum(), d.mean(), se)
        assert np.all(np.isfinite(lr[:, m]))
