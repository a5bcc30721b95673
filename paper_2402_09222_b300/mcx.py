"""Thin Python binding of libmcx (include/mcx.h).

Argument marshalling only: every step of the lookup and of the transport runs
in the library's CUDA kernels.  PyTorch provides device memory (tensors whose
data pointers are handed to the C ABI) and streams.  There is no fallback: if
libmcx.so is missing or cannot be loaded, importing this module raises.
With MCX_LIB=bounds in the environment at import, the bounds-checked debug
build libmcx_bounds.so is loaded instead (same ABI; see bounds_checked()).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_VARIANT = os.environ.get("MCX_LIB", "release")
if LIB_VARIANT not in ("release", "bounds"):
    raise ImportError(f"MCX_LIB={LIB_VARIANT!r}: expected 'release' or 'bounds'")
LIB_PATH = os.path.join(_HERE, "libmcx_bounds.so" if LIB_VARIANT == "bounds" else "libmcx.so")

MCX_OK = 0
ERR_NAMES = {-1: "MCX_ERR_ARG", -2: "MCX_ERR_CUDA", -3: "MCX_ERR_OOM", -4: "MCX_ERR_ITER_LIMIT",
             -5: "MCX_ERR_STATE", -6: "MCX_ERR_BOUNDS", -7: "MCX_ERR_TIMEOUT"}
ERR_ITER_LIMIT, ERR_TIMEOUT = -4, -7
FP64, FP32 = 0, 1
QUEUELESS, QUEUED, QUEUED_FULLEST = 0, 1, 2
LOOKUP_EXACT, LOOKUP_FAST, LOOKUP_SORT, LOOKUP_STAGED, LOOKUP_OUT32, LOOKUP_LINEAR = 0, 1, 2, 4, 8, 16
LOOKUP_BINNED_INPUTS = 32
FLAG_DERIVATIVES, FLAG_HISTORY_DEBUG = 1, 2
TALLY_FLUX, TALLY_ABSORB, TALLY_OUTCOME, TALLY_DFLUX, TALLY_DABSORB, TALLY_DOUTCOME = range(6)
GEOM_NONE = 3
N_OUT = 5


class McxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run "
                      f"python -m paper_2402_09222_b300.build{' --bounds' if LIB_VARIANT == 'bounds' else ''}")
_lib = C.CDLL(LIB_PATH)

_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32


class ProblemDesc(C.Structure):
    _fields_ = [
        ("geometry", C.c_int32), ("lattice_n", C.c_int32),
        ("pitch", C.c_double), ("radius", C.c_double), ("height", C.c_double),
        ("slab_length", C.c_double), ("n_regions", C.c_int32),
        ("region_material", C.POINTER(C.c_int32)), ("E0", C.c_double), ("E_cut", C.c_double),
        ("n_ebins", C.c_int32), ("ebin_edges", C.POINTER(C.c_double)),
        ("n_batches", C.c_int32), ("problem_id", C.c_uint32), ("n_histories", C.c_int64),
        ("flags", C.c_int32), ("device", C.c_int32),
    ]


class Tune(C.Structure):
    _fields_ = [("mode", C.c_int32), ("block_size", C.c_int32), ("sort_period", C.c_int32),
                ("sort_threshold", C.c_int64), ("iters_per_sync", C.c_int32),
                ("max_event_iters", C.c_int64), ("use_graph", C.c_int32),
                ("time_limit_s", C.c_double)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("mcx_last_error", C.c_char_p)
_sig("mcx_version", C.c_char_p)
_sig("mcx_init_problem", C.c_int, C.POINTER(ProblemDesc), C.POINTER(_vp))
_sig("mcx_destroy", None, _vp)
_sig("mcx_load_xs_tables", C.c_int, _vp, _i32, _vp, _vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _i32, _i32)
_sig("mcx_share_xs_tables", C.c_int, _vp, _vp)
_sig("mcx_set_hash_bins", C.c_int, _vp, _i32)
_sig("mcx_set_densities", C.c_int, _vp, _vp, _i64)
_sig("mcx_update_tables_device", C.c_int, _vp, _vp, _vp, _vp)
_sig("mcx_default_tuning", None, C.POINTER(Tune))
_sig("mcx_set_tuning", C.c_int, _vp, C.POINTER(Tune))
_sig("mcx_run_batch", C.c_int, _vp, _i64, _i64, _i64, C.c_uint64, _vp)
_sig("mcx_batch_run", C.c_int, _i32, _vp, _vp, _i64, C.c_uint64, _vp)
_sig("mcx_tally_size", C.c_int, _vp, _i32, C.POINTER(_i64))
_sig("mcx_read_tallies", C.c_int, _vp, _i32, _vp, _i64)
_sig("mcx_zero_tallies", C.c_int, _vp)
_sig("mcx_read_history_debug", C.c_int, _vp, _vp, _i64)
_sig("mcx_last_run_stats", C.c_int, _vp, _vp, _i32)
_sig("mcx_set_kernel_timing", C.c_int, _vp, _i32)
_sig("mcx_last_kernel_stats", C.c_int, _vp, _vp, _vp)
_sig("mcx_run_eigenvalue", C.c_int, _vp, _i64, _i32, _i32, C.c_double, C.c_double, _i64, C.c_uint64,
     _vp, _vp)
_sig("mcx_fission_bank_size", C.c_int, _vp, C.POINTER(_i64))
_sig("mcx_check_device", C.c_int, _vp, _vp)
_sig("mcx_bounds_checked", C.c_int)
_sig("mcx_read_fission_bank", C.c_int, _vp, _vp, _i64)
_sig("mcx_xs_lookup", C.c_int, _vp, _i64, _vp, _vp, _vp, _i32, _vp)
_sig("mcx_xs_sort", C.c_int, _vp, _i64, _vp, _vp, _vp, _vp)
_sig("mcx_xs_sort_inputs", C.c_int, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("mcx_xs_lookup_ordered", C.c_int, _vp, _i64, _vp, _vp, _vp, _vp, _i32, _vp)
_sig("mcx_xs_lookup_host", C.c_int, _vp, _i64, _vp, _vp, _vp, _i32)
_sig("mcx_xs_indices", C.c_int, _vp, _i64, _vp, _vp, _i32, _vp, _vp)
_sig("mcx_xs_lookup_backward", C.c_int, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("mcx_debug_uniforms", C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, _i64, _vp, _vp)
_sig("mcx_debug_neg_log", C.c_int, _vp, _i64, _vp, _vp)
_sig("mcx_debug_transport_xs", C.c_int, _vp, _i64, _vp, _vp, _vp, _vp)


def _check(rc: int):
    if rc != MCX_OK:
        raise McxError(rc, _lib.mcx_last_error().decode())


def version() -> str:
    return _lib.mcx_version().decode()


def bounds_checked() -> bool:
    """True in the bounds-checked debug build (MCX_LIB=bounds)."""
    return bool(_lib.mcx_bounds_checked())


def _np_ptr(a):
    return a.ctypes.data_as(_vp)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev_ptr(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _vp(t.data_ptr())


def default_tuning() -> dict:
    t = Tune()
    _lib.mcx_default_tuning(C.byref(t))
    return {k: getattr(t, k) for k, _ in Tune._fields_}


class Problem:
    """A transport problem (or, with prob=None, a handle holding only tables)."""

    def __init__(self, prob: "synth.Problem | None" = None, device: int = 0, flags: int = 0):
        d = ProblemDesc()
        self._keep = []
        if prob is None:
            d.geometry = GEOM_NONE
        else:
            rm = np.ascontiguousarray(prob.region_material, np.int32)
            edges = np.ascontiguousarray(prob.ebin_edges, np.float64)
            self._keep += [rm, edges]
            d.geometry = prob.geometry
            d.lattice_n = prob.lattice_n
            d.pitch, d.radius, d.height = prob.pitch, prob.radius, prob.height
            d.slab_length = prob.slab_length
            d.n_regions = len(rm)
            d.region_material = rm.ctypes.data_as(C.POINTER(C.c_int32))
            d.E0, d.E_cut = prob.E0, prob.E_cut
            d.n_ebins = max(len(edges) - 1, 0)
            d.ebin_edges = edges.ctypes.data_as(C.POINTER(C.c_double)) if len(edges) else None
            d.n_batches = prob.n_batches
            d.problem_id = prob.problem_id
            d.n_histories = prob.n_histories
        d.flags = flags
        d.device = device
        h = _vp()
        _check(_lib.mcx_init_problem(C.byref(d), C.byref(h)))
        self.h = h
        self.prob = prob
        self.device = device
        self.flags = flags
        self.n_ch = 0
        self.nnz = 0
        self.max_species = 0
        self.n_points = 0

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            _lib.mcx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- tables
    def load_tables(self, lib: "synth.Library", mats: "synth.Materials", precision: int = FP64,
                    hash_bins: int = 4000):
        go = np.ascontiguousarray(lib.grid_offsets, np.int64)
        en = np.ascontiguousarray(lib.energies, np.float64)
        sg = np.ascontiguousarray(lib.sigma, np.float64)
        aw = np.ascontiguousarray(lib.awr, np.float64)
        mo = np.ascontiguousarray(mats.offsets, np.int32)
        ms = np.ascontiguousarray(mats.species, np.int32)
        md = np.ascontiguousarray(mats.dens, np.float64)
        _check(_lib.mcx_load_xs_tables(self.h, lib.n_species, _np_ptr(go), _np_ptr(en), _np_ptr(sg),
                                       lib.n_ch, _np_ptr(aw), mats.n_materials, _np_ptr(mo),
                                       _np_ptr(ms), _np_ptr(md), precision, hash_bins))
        self.n_ch = lib.n_ch
        self.nnz = len(md)
        self.max_species = int(np.max(np.diff(mo)))
        self.n_points = len(en)
        return self

    def share_tables(self, other: "Problem"):
        _check(_lib.mcx_share_xs_tables(self.h, other.h))
        self.n_ch, self.nnz, self.max_species, self.n_points = (other.n_ch, other.nnz,
                                                                other.max_species, other.n_points)
        return self

    def set_hash_bins(self, H: int):
        _check(_lib.mcx_set_hash_bins(self.h, H))

    def set_densities(self, dens):
        d = np.ascontiguousarray(dens, np.float64)
        _check(_lib.mcx_set_densities(self.h, _np_ptr(d), len(d)))

    def update_tables_device(self, dens=None, sigma=None, stream=None):
        """Replace densities [nnz] and/or cross sections [P][n_ch] from FP64 CUDA tensors."""
        import torch
        pd = _vp(0) if dens is None else _dev_ptr(dens, torch.float64, "dens")
        ps = _vp(0) if sigma is None else _dev_ptr(sigma, torch.float64, "sigma")
        if dens is not None and dens.numel() != self.nnz:
            raise ValueError(f"dens must have {self.nnz} entries")
        if sigma is not None and sigma.numel() != self.n_points * self.n_ch:
            raise ValueError(f"sigma must have {self.n_points} x {self.n_ch} entries")
        _check(_lib.mcx_update_tables_device(self.h, pd, ps, _stream_ptr(stream)))

    # -- transport
    def set_tuning(self, **kw):
        t = Tune()
        _lib.mcx_default_tuning(C.byref(t))
        for k, v in kw.items():
            if not hasattr(t, k):
                raise KeyError(k)
            setattr(t, k, float(v) if k == "time_limit_s" else int(v))
        _check(_lib.mcx_set_tuning(self.h, C.byref(t)))
        return self

    def run(self, first: int = 0, count: int | None = None, particles_in_flight: int = 1_000_000,
            seed: int = 1, stream=None):
        count = self.prob.n_histories - first if count is None else count
        _check(_lib.mcx_run_batch(self.h, first, count, particles_in_flight, seed, _stream_ptr(stream)))
        return self

    def tally(self, which: int) -> np.ndarray:
        n = _i64()
        _check(_lib.mcx_tally_size(self.h, which, C.byref(n)))
        out = np.zeros(n.value)
        _check(_lib.mcx_read_tallies(self.h, which, _np_ptr(out), n.value))
        return out

    def tallies(self) -> dict:
        B, nb = self.prob.n_batches, self.prob.n_tally_bins
        res = dict(flux=self.tally(TALLY_FLUX).reshape(B, nb),
                   absorb=self.tally(TALLY_ABSORB).reshape(B, nb),
                   outcome=self.tally(TALLY_OUTCOME).reshape(B, N_OUT))
        if self.flags & FLAG_DERIVATIVES:
            M = self.prob.mats.n_materials
            res.update(dflux=self.tally(TALLY_DFLUX).reshape(B, nb, M),
                       dabsorb=self.tally(TALLY_DABSORB).reshape(B, nb, M),
                       doutcome=self.tally(TALLY_DOUTCOME).reshape(B, N_OUT, M))
        return res

    def zero_tallies(self):
        _check(_lib.mcx_zero_tallies(self.h))

    def history_debug(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.uint32)
        _check(_lib.mcx_read_history_debug(self.h, _np_ptr(out), n))
        return out

    def set_kernel_timing(self, on: bool = True):
        """Later runs launch without graphs and time each event kernel."""
        _check(_lib.mcx_set_kernel_timing(self.h, 1 if on else 0))
        return self

    def kernel_stats(self) -> dict:
        """Device ms of the lookup, flight and collision kernels of the last
        run (kernel timing on) and its event counts (queued mode)."""
        ms = np.zeros(3)
        cnt = np.zeros(4, np.int64)
        _check(_lib.mcx_last_kernel_stats(self.h, _np_ptr(ms), _np_ptr(cnt)))
        return {"ms": dict(lookup=float(ms[0]), flight=float(ms[1]), collision=float(ms[2])),
                "events": dict(lookups=int(cnt[0]), flights=int(cnt[1]), collisions=int(cnt[2]),
                               row_entries=int(cnt[3]))}

    def stats(self) -> dict:
        out = np.zeros(6, np.int64)
        _check(_lib.mcx_last_run_stats(self.h, _np_ptr(out), 6))
        return dict(iterations=int(out[0]), graph_launches=int(out[1]), kernels=int(out[2]),
                    selected=dict(lookup=int(out[3]), flight=int(out[4]), collision=int(out[5])))

    def run_eigenvalue(self, n_per_gen: int, n_generations: int, n_inactive: int, k0: float = 1.0,
                       particles_in_flight: int = 1_000_000, seed: int = 1, stream=None) -> dict:
        """k-eigenvalue power iteration (see mcx_run_eigenvalue): per generation
        k (site count), k_col, k_tl and the number of banked sites."""
        gen = np.zeros((n_generations, 4))
        T = self.prob.T_fission if self.prob is not None else 1.2895e6
        _check(_lib.mcx_run_eigenvalue(self.h, n_per_gen, n_generations, n_inactive, float(k0), float(T),
                                       particles_in_flight, seed, _np_ptr(gen), _stream_ptr(stream)))
        return dict(k=gen[:, 0].copy(), k_col=gen[:, 1].copy(), k_tl=gen[:, 2].copy(),
                    sites=gen[:, 3].astype(np.int64))

    def check_device(self, stream=None):
        """Raise if a staged lookup on this handle gave up on its pipeline."""
        _check(_lib.mcx_check_device(self.h, _stream_ptr(stream)))
        return self

    def fission_bank(self) -> np.ndarray:
        """The last generation's ordered bank, rows (x, y, z, ci, cj, inpin)."""
        n = _i64()
        _check(_lib.mcx_fission_bank_size(self.h, C.byref(n)))
        rows = np.zeros((n.value, 6))
        _check(_lib.mcx_read_fission_bank(self.h, _np_ptr(rows), n.value))
        return rows

    # -- lookups (device tensors)
    def xs_lookup(self, E, mat, out=None, flags: int = LOOKUP_EXACT, stream=None):
        import torch
        n = E.numel()
        odt = torch.float32 if flags & LOOKUP_OUT32 else torch.float64
        if out is None:
            out = torch.empty((n, self.n_ch), dtype=odt, device=E.device)
        _check(_lib.mcx_xs_lookup(self.h, n, _dev_ptr(E, torch.float64, "E"),
                                  _dev_ptr(mat, torch.int32, "mat"),
                                  _dev_ptr(out, odt, "out"), flags, _stream_ptr(stream)))
        return out

    def xs_sort(self, E, mat, perm=None, stream=None):
        """Binning permutation of the lookups by (material, log-energy bucket)."""
        import torch
        if perm is None:
            perm = torch.empty(E.numel(), dtype=torch.int32, device=E.device)
        _check(_lib.mcx_xs_sort(self.h, E.numel(), _dev_ptr(E, torch.float64, "E"),
                                _dev_ptr(mat, torch.int32, "mat"), _dev_ptr(perm, torch.int32, "perm"),
                                _stream_ptr(stream)))
        return perm

    def xs_sort_inputs(self, E, mat, perm=None, E_binned=None, mat_binned=None, stream=None):
        """Binning permutation plus the energies and materials in the binned
        order (for xs_lookup_ordered with LOOKUP_BINNED_INPUTS)."""
        import torch
        n = E.numel()
        if perm is None:
            perm = torch.empty(n, dtype=torch.int32, device=E.device)
        if E_binned is None:
            E_binned = torch.empty(n, dtype=torch.float64, device=E.device)
        if mat_binned is None:
            mat_binned = torch.empty(n, dtype=torch.int32, device=E.device)
        if perm.numel() < n or E_binned.numel() < n or mat_binned.numel() < n or mat.numel() != n:
            raise ValueError("mat, perm, E_binned and mat_binned must hold n = E.numel() entries")
        _check(_lib.mcx_xs_sort_inputs(self.h, n, _dev_ptr(E, torch.float64, "E"),
                                       _dev_ptr(mat, torch.int32, "mat"), _dev_ptr(perm, torch.int32, "perm"),
                                       _dev_ptr(E_binned, torch.float64, "E_binned"),
                                       _dev_ptr(mat_binned, torch.int32, "mat_binned"), _stream_ptr(stream)))
        return perm, E_binned, mat_binned

    def xs_lookup_ordered(self, E, mat, perm, out=None, flags: int = LOOKUP_EXACT, stream=None):
        """Lookup processed in the order `perm` (None: natural order)."""
        import torch
        n = E.numel()
        odt = torch.float32 if flags & LOOKUP_OUT32 else torch.float64
        if out is None:
            out = torch.empty((n, self.n_ch), dtype=odt, device=E.device)
        pp = _vp(0) if perm is None else _dev_ptr(perm, torch.int32, "perm")
        _check(_lib.mcx_xs_lookup_ordered(self.h, n, _dev_ptr(E, torch.float64, "E"),
                                          _dev_ptr(mat, torch.int32, "mat"), pp,
                                          _dev_ptr(out, odt, "out"), flags, _stream_ptr(stream)))
        return out

    def xs_lookup_host(self, E, mat, out=None, flags: int = LOOKUP_EXACT):
        """Lookup from host buffers (numpy arrays or CPU tensors, ideally pinned)."""
        import torch
        out32 = bool(flags & LOOKUP_OUT32)
        if isinstance(E, torch.Tensor):
            n = E.numel()
            if out is None:
                out = torch.empty((n, self.n_ch), dtype=torch.float32 if out32 else torch.float64,
                                  pin_memory=True)
            if out.dtype != (torch.float32 if out32 else torch.float64):
                raise TypeError("out has the wrong dtype for these flags")
            pe, pm, po = _vp(E.data_ptr()), _vp(mat.data_ptr()), _vp(out.data_ptr())
        else:
            E = np.ascontiguousarray(E, np.float64)
            mat = np.ascontiguousarray(mat, np.int32)
            n = len(E)
            if out is None:
                out = np.empty((n, self.n_ch), np.float32 if out32 else np.float64)
            if out.dtype != (np.float32 if out32 else np.float64):
                raise TypeError("out has the wrong dtype for these flags")
            pe, pm, po = _np_ptr(E), _np_ptr(mat), _np_ptr(out)
        _check(_lib.mcx_xs_lookup_host(self.h, n, pe, pm, po, flags))
        return out

    def debug_transport_xs(self, E, mat, stream=None):
        """The transport's macroscopic lookup on device tensors E (FP64) and
        mat (int32): an [n, 3] tensor of Sigma_t, Sigma_a, nuSigma_f."""
        import torch
        out = torch.empty((E.numel(), 3), dtype=torch.float64, device=E.device)
        _check(_lib.mcx_debug_transport_xs(self.h, E.numel(), _dev_ptr(E, torch.float64, "E"),
                                           _dev_ptr(mat, torch.int32, "mat"), _vp(out.data_ptr()),
                                           _stream_ptr(stream)))
        return out

    def xs_indices(self, E, mat, max_species: int | None = None, stream=None):
        import torch
        ms = max_species or self.max_species
        n = E.numel()
        out = torch.empty((n, ms), dtype=torch.int32, device=E.device)
        _check(_lib.mcx_xs_indices(self.h, n, _dev_ptr(E, torch.float64, "E"),
                                   _dev_ptr(mat, torch.int32, "mat"), ms,
                                   _dev_ptr(out, torch.int32, "kout"), _stream_ptr(stream)))
        return out

    def xs_lookup_backward(self, E, mat, grad_out, grad_dens=None, grad_sigma=None, stream=None):
        import torch
        if grad_dens is None:
            grad_dens = torch.zeros(self.nnz, dtype=torch.float64, device=E.device)
        if grad_sigma is None:
            grad_sigma = torch.zeros((self.n_points, self.n_ch), dtype=torch.float64, device=E.device)
        _check(_lib.mcx_xs_lookup_backward(
            self.h, E.numel(), _dev_ptr(E, torch.float64, "E"), _dev_ptr(mat, torch.int32, "mat"),
            _dev_ptr(grad_out, torch.float64, "grad_out"), _dev_ptr(grad_dens, torch.float64, "grad_dens"),
            _dev_ptr(grad_sigma, torch.float64, "grad_sigma"), _stream_ptr(stream)))
        return grad_dens, grad_sigma


def batch_run(problems, n_hist, particles_in_flight: int, seed: int, stream=None):
    arr = (_vp * len(problems))(*[p.h for p in problems])
    nh = np.ascontiguousarray(n_hist, np.int64)
    _check(_lib.mcx_batch_run(len(problems), C.cast(arr, _vp), _np_ptr(nh), particles_in_flight,
                              seed, _stream_ptr(stream)))


def debug_neg_log(x):
    """(-ln x as the transport computes it, as the CUDA library does) for a
    device FP64 tensor x of uniforms in [2^-53, 1); returns an [n, 2] tensor."""
    import torch
    out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
    _check(_lib.mcx_debug_neg_log(_dev_ptr(x, torch.float64, "x"), x.numel(), _vp(out.data_ptr()),
                                  _stream_ptr(None)))
    return out


def debug_uniforms(seed: int, problem_id: int, hist: int, n: int, first: int = 0, device: int = 0):
    import torch
    out = torch.empty(n, dtype=torch.float64, device=f"cuda:{device}")
    _check(_lib.mcx_debug_uniforms(seed, problem_id, hist, first, n, _vp(out.data_ptr()),
                                   _stream_ptr(None)))
    return out


def make_problem(prob: "synth.Problem", precision: int = FP64, hash_bins: int = 4000,
                 flags: int = 0, device: int = 0) -> Problem:
    """A transport problem with its own copy of the problem's tables."""
    p = Problem(prob, device=device, flags=flags)
    p.load_tables(prob.lib, prob.mats, precision=precision, hash_bins=hash_bins)
    return p
