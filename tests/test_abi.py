"""C-ABI checks that need no GPU: the library loads, exports every entry point
that include/mcx.h declares, and rejects bad arguments with status codes and
messages (host-side validation runs before any device call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcx_[a-z0-9_]+)\s*\(", text)))


@pytest.mark.parametrize("variant", ["libmcx.so", "libmcx_bounds.so"])
def test_library_exports_every_declared_symbol(variant):
    """The release library and its bounds-checked debug build export the
    same declared ABI; only the debug build says it checks bounds."""
    from paper_2402_09222_b300 import mcx
    lib = C.CDLL(os.path.join(os.path.dirname(mcx.LIB_PATH), variant))
    names = _declared("mcx.h")
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    lib.mcx_bounds_checked.restype = C.c_int
    assert lib.mcx_bounds_checked() == (1 if variant == "libmcx_bounds.so" else 0)


def test_binding_loads_the_bounds_checked_build_on_request():
    import subprocess
    import sys
    code = "from paper_2402_09222_b300 import mcx; print(mcx.bounds_checked(), mcx.LIB_PATH)"
    for var, want in (("bounds", "True"), ("release", "False")):
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                             env={**os.environ, "MCX_LIB": var}, check=True).stdout.split()
        assert out[0] == want and out[1].endswith("libmcx_bounds.so" if var == "bounds" else "libmcx.so")
    bad = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         env={**os.environ, "MCX_LIB": "nope"})
    assert bad.returncode != 0 and "MCX_LIB" in bad.stderr


def test_version_and_default_tuning():
    from paper_2402_09222_b300 import mcx
    assert "sm_103a" in mcx.version()
    t = mcx.default_tuning()
    assert t["mode"] == mcx.QUEUELESS and t["block_size"] == 256 and t["sort_threshold"] == 20000
    assert t["use_graph"] == 1 and t["iters_per_sync"] >= 1


def _desc(**kw):
    from paper_2402_09222_b300 import mcx
    d = mcx.ProblemDesc()
    rm = np.zeros(290, np.int32)
    edges = np.exp(np.linspace(-11, 16, 51))
    d.geometry = 1
    d.lattice_n = 17
    d.pitch, d.radius, d.height = 1.26, 0.41, 100.0
    d.n_regions = 290
    d.region_material = rm.ctypes.data_as(C.POINTER(C.c_int32))
    d.E0, d.E_cut = 2e6, 1e-5
    d.n_ebins = 50
    d.ebin_edges = edges.ctypes.data_as(C.POINTER(C.c_double))
    d.n_batches = 20
    d.n_histories = 1000
    for k, v in kw.items():
        setattr(d, k, v)
    return d, (rm, edges)


@pytest.mark.parametrize("field,value,needle", [
    ("geometry", 9, "geometry"),
    ("E0", -1.0, "E0"),
    ("n_batches", 0, "n_batches"),
    ("n_histories", 0, "n_histories"),
    ("lattice_n", 0, "lattice_n"),
    ("radius", 0.7, "radius"),
    ("n_regions", 17, "regions"),
    ("pitch", float("nan"), "pitch"),
])
def test_bad_descriptions_are_rejected(field, value, needle):
    from paper_2402_09222_b300 import mcx
    d, keep = _desc(**{field: value})
    h = C.c_void_p()
    rc = mcx._lib.mcx_init_problem(C.byref(d), C.byref(h))
    assert rc == -1
    assert needle in mcx._lib.mcx_last_error().decode()
    assert not h.value


def test_null_handles_and_arguments():
    from paper_2402_09222_b300 import mcx
    L = mcx._lib
    assert L.mcx_init_problem(None, None) == -1
    assert L.mcx_set_tuning(None, None) == -1
    assert L.mcx_run_batch(None, 0, 1, 1, 1, None) == -1
    assert L.mcx_xs_lookup(None, 1, None, None, None, 0, None) == -1
    assert L.mcx_read_tallies(None, 0, None, 0) == -1
    assert L.mcx_debug_uniforms(1, 0, 0, 0, -1, None, None) == -1
    assert L.mcx_debug_uniforms(1, 0, 0, 0, 0, None, None) == 0
    L.mcx_destroy(None)
    assert "NULL" in L.mcx_last_error().decode() or L.mcx_last_error() == b""


def test_no_device_is_an_error_not_a_crash():
    """On a machine without a GPU a valid description fails with a CUDA status."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2402_09222_b300 import mcx
    d, keep = _desc()
    h = C.c_void_p()
    rc = mcx._lib.mcx_init_problem(C.byref(d), C.byref(h))
    assert rc in (-2, -1)
    assert mcx._lib.mcx_last_error().decode()


def test_tuning_validation_without_device():
    from paper_2402_09222_b300 import mcx
    t = mcx.Tune()
    mcx._lib.mcx_default_tuning(C.byref(t))
    assert (t.mode, t.block_size) == (0, 256)


def test_kernel_timing_calls_validate_their_arguments():
    import ctypes as C
    from paper_2402_09222_b300 import mcx
    lib = C.CDLL(mcx.LIB_PATH)
    lib.mcx_set_kernel_timing.argtypes = [C.c_void_p, C.c_int32]
    lib.mcx_last_kernel_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.mcx_last_error.restype = C.c_char_p
    assert lib.mcx_set_kernel_timing(None, 1) != 0
    assert lib.mcx_last_kernel_stats(None, None, None) != 0
