"""The bounds-checked debug build (libmcx_bounds.so, MCX_BOUNDS_CHECK=1).

The build is chosen when the binding is imported, so each case runs in a
child process with MCX_LIB=bounds and returns its results through a file;
this process computes the same with the release library.

* On valid inputs no check fires (mcx_check_device and the transport runs
  return MCX_OK) and every result equals the release build's: the lookups in
  each form (device and host buffers) bit for bit, the backward and the
  transport tallies to rounding (their atomics add in no fixed order), the
  per-history collision counts of fixed-source, batched and eigenvalue runs
  and the eigenvalue's ordered fission bank exactly.
* A processing order holding indices outside [0, n) -- input that only the
  debug build's own checks make safe, which is why this case runs only
  there -- is reported by mcx_check_device as MCX_ERR_BOUNDS naming the
  site, in the exact, the warp-cooperative and the staged lookup; the valid
  lookups are computed as usual and the two displaced ones are left
  unwritten."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2402_09222_b300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

LOOKUP_FLAGS = {"exact": 0, "fast": 1, "fast_binned": 3, "staged": 7, "fast_binned_out32": 11,
                "fast_binned_linear": 19}
# the round-linear sums depend on which lookups share a round, and the order
# within a bin is not fixed: compared within the fast bound, not bit for bit
NOT_BITWISE = ("lk_fast_binned_linear", "lk_binned_inputs_linear")
MODES = {"queueless": 0, "queued": 1, "queued_fullest": 2}

CASE = r'''
import sys
import numpy as np
import torch
from paper_2402_09222_b300 import mcx, synth

def lookup_case():
    lib = synth.species_library(40, 800, 161)
    mats = synth.lookup_materials(40, 162, n_materials=6)
    E, mat = synth.lookup_inputs(200_003, mats.n_materials, 163)
    p = mcx.Problem(None).load_tables(lib, mats, precision=mcx.FP32, hash_bins=3000)
    return lib, mats, E, mat, p

def transport_case(mode):
    prob = synth.config3_problem(6000, lattice_n=5, n_points=1500)
    p = mcx.make_problem(prob, precision=mcx.FP32, hash_bins=2000,
                         flags=mcx.FLAG_HISTORY_DEBUG | mcx.FLAG_DERIVATIVES)
    p.set_tuning(mode=mode, sort_period=2, sort_threshold=0)
    return prob, p

def run_all(flags_by_name, modes):
    res = {}
    lib, mats, E, mat, p = lookup_case()
    dE, dm = torch.as_tensor(E, device="cuda"), torch.as_tensor(mat, device="cuda")
    for name, fl in flags_by_name.items():
        res["lk_" + name] = p.xs_lookup(dE, dm, flags=fl).double().cpu().numpy()
        p.check_device()
    g = torch.as_tensor(np.random.default_rng(164).normal(size=(len(E), lib.n_ch)), device="cuda")
    gd, gs = p.xs_lookup_backward(dE, dm, g)
    p.check_device()
    res["bw_dens"], res["bw_sigma"] = gd.cpu().numpy(), gs.cpu().numpy()
    p.close()
    # two-level binning handing the inputs over in the binned order (4.3M
    # lookups, invalid material ids among them), and lookups reading them
    blib = synth.species_library(20, 400, 165)
    bmats = synth.lookup_materials(20, 166, n_materials=5)
    bE, bm = synth.lookup_inputs(4_300_001, bmats.n_materials, 167)
    bm[[11, 2_000_000]] = [-1, bmats.n_materials]
    bp = mcx.Problem(None).load_tables(blib, bmats, precision=mcx.FP32, hash_bins=1000)
    perm, Eb, mb = bp.xs_sort_inputs(torch.as_tensor(bE, device="cuda"), torch.as_tensor(bm, device="cuda"))
    bp.check_device()
    for name, fl in (("fast", mcx.LOOKUP_FAST), ("linear", mcx.LOOKUP_FAST | mcx.LOOKUP_LINEAR)):
        res["lk_binned_inputs_" + name] = bp.xs_lookup_ordered(Eb, mb, perm,
                                                               flags=fl | mcx.LOOKUP_BINNED_INPUTS).cpu().numpy()
        bp.check_device()
    bp.close()
    for name, mode in modes.items():
        prob, q = transport_case(mode)
        q.run(particles_in_flight=1500, seed=5)
        q.check_device()
        t = q.tallies()
        for k in ("flux", "absorb", "outcome", "dabsorb"):
            res[f"tr_{name}_{k}"] = t[k]
        res[f"tr_{name}_ncoll"] = q.history_debug(prob.n_histories)
        q.close()
    # the host-buffer lookup (chunked device pipeline, binned per chunk)
    lib, mats, E, mat, p = lookup_case()
    res["lk_host"] = p.xs_lookup_host(E, mat, flags=mcx.LOOKUP_FAST | mcx.LOOKUP_SORT)
    p.check_device()
    p.close()
    # eigenvalue generations (the transport kernels' fission instantiations)
    eig = synth.eigen_problem(3000, lattice_n=9, n_points=2000)
    q = mcx.make_problem(eig, precision=mcx.FP32, hash_bins=2000)
    q.set_tuning(mode=1, sort_period=2, sort_threshold=0)
    r = q.run_eigenvalue(3000, n_generations=3, n_inactive=1, k0=0.04, particles_in_flight=1500, seed=6)
    q.check_device()
    res["eig_sites"] = r["sites"]
    res["eig_k"] = r["k"]
    res["eig_bank"] = q.fission_bank()
    q.close()
    # batched uneven problems sharing one table set
    blib = synth.species_library(30, 900, 171).channels([synth.CH_SCATTER, synth.CH_ABSORB])
    bmats = synth.lookup_materials(30, 172, n_materials=5)
    probs = synth.config5_problems(blib, bmats, n_problems=5, seed=173, hist_lo=100, hist_hi=2000)
    base = mcx.Problem(probs[0], flags=mcx.FLAG_HISTORY_DEBUG).load_tables(blib, bmats, hash_bins=800)
    hs = [base] + [mcx.Problem(pr, flags=mcx.FLAG_HISTORY_DEBUG).share_tables(base) for pr in probs[1:]]
    base.set_tuning(mode=2, sort_period=2, sort_threshold=0)
    mcx.batch_run(hs, [pr.n_histories for pr in probs], particles_in_flight=1500, seed=8)
    for i, (h, pr) in enumerate(zip(hs, probs)):
        h.check_device()
        res[f"batch{i}_ncoll"] = h.history_debug(pr.n_histories)
        res[f"batch{i}_flux"] = h.tallies()["flux"]
    return res

def bad_order_case(flags_by_name):
    lib, mats, E, mat, p = lookup_case()
    n = len(E)
    dE, dm = torch.as_tensor(E, device="cuda"), torch.as_tensor(mat, device="cuda")
    perm = p.xs_sort(dE, dm)
    shown = perm.cpu().numpy()
    lost = shown[[1000, 150_000]].copy()
    perm[1000] = n          # one past the end
    perm[150_000] = -7
    res = {"lost": lost}
    for name, fl in flags_by_name.items():
        out = torch.full((n, lib.n_ch), float("nan"), dtype=torch.float64, device="cuda")
        p.xs_lookup_ordered(dE, dm, perm, out=out, flags=fl & ~mcx.LOOKUP_SORT)
        try:
            p.check_device()
            res["msg_" + name] = np.array("no error")
        except mcx.McxError as e:
            res["msg_" + name] = np.array(f"{e.code} {e}")
        res["out_" + name] = out.cpu().numpy()
        p.check_device()   # the record was cleared by the read
    return res

if __name__ == "__main__":
    import json
    which, path, spec = sys.argv[1], sys.argv[2], json.loads(sys.argv[3])
    if which == "bounds":
        assert mcx.bounds_checked()
    res = run_all(spec["lookup"], spec["modes"]) if sys.argv[4] == "valid" else bad_order_case(spec["lookup"])
    np.savez(path, **res)
'''


def _child(tmp_path, variant, kind, flags):
    import json
    script = tmp_path / "case.py"
    script.write_text(CASE)
    out = tmp_path / f"{variant}_{kind}.npz"
    spec = json.dumps({"lookup": flags, "modes": MODES})
    r = subprocess.run([sys.executable, str(script), variant, str(out), spec, kind], cwd=ROOT,
                       env={**os.environ, "MCX_LIB": variant, "PYTHONPATH": ROOT}, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_bounds_build_matches_release_on_valid_inputs(torch_cuda, tmp_path):
    dbg = _child(tmp_path, "bounds", "valid", LOOKUP_FLAGS)
    rel = _child(tmp_path, "release", "valid", LOOKUP_FLAGS)
    assert set(dbg) == set(rel)
    for k in sorted(rel):
        if k in NOT_BITWISE:
            np.testing.assert_allclose(dbg[k], rel[k], rtol=2e-6, atol=0, err_msg=k)
        elif k.startswith("lk_") or k.endswith("_ncoll") or k in ("eig_sites", "eig_k", "eig_bank"):
            assert np.array_equal(dbg[k].view(np.uint8), rel[k].view(np.uint8)), k
        else:
            scale = max(np.abs(rel[k]).max(), 1e-300)
            np.testing.assert_allclose(dbg[k], rel[k], rtol=1e-10, atol=1e-12 * scale, err_msg=k)


def test_out_of_range_processing_order_is_reported(torch_cuda, tmp_path):
    flags = {k: v for k, v in LOOKUP_FLAGS.items() if k in ("exact", "fast_binned", "staged", "fast_binned_linear")}
    dbg = _child(tmp_path, "bounds", "bad", flags)
    rel = _child(tmp_path, "release", "valid", {k: v for k, v in flags.items()})
    lost = dbg["lost"]
    n = rel["lk_exact"].shape[0]
    keep = np.ones(n, bool)
    keep[lost] = False
    for name in flags:
        msg = str(dbg["msg_" + name])
        assert msg.startswith("-6 ") and "lookup index from the processing order" in msg, (name, msg)
        out = dbg["out_" + name]
        assert np.all(np.isnan(out[lost])), name
        if "lk_" + name in NOT_BITWISE:
            np.testing.assert_allclose(out[keep], rel["lk_" + name][keep], rtol=2e-6, atol=0, err_msg=name)
        else:
            assert np.array_equal(out[keep].view(np.uint64), rel["lk_" + name][keep].view(np.uint64)), name
