"""CPU FP64 oracle for the macroscopic cross-section lookup and the event-based
transport it sits in (arXiv 2402.09222, Sec. 5.1).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports, links
or runs anything here, and this package imports nothing from it; both sides
read the same seeded inputs from the synthetic-input module.

Every function follows a plain definition (lookup, adjoint) or runs the
transport algorithm history by history in FP64 (see mcx_oracle.c for the
readings taken where the paper is silent).  Parity is pinned in the tests
against closed forms, brute force and published vectors, not against this
code itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

N_OUT = 5
OUT_ABSORBED, OUT_LEAK_XHI, OUT_LEAK_OTHER, OUT_CUTOFF, OUT_COLLISIONS = range(5)


def build(force: bool = False) -> str:
    """Compile mcx_oracle.c into liboracle.so (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=c11", "-Wall", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)


class _Problem(C.Structure):
    _fields_ = [
        ("geometry", C.c_int32), ("lattice_n", C.c_int32),
        ("pitch", C.c_double), ("radius", C.c_double), ("height", C.c_double),
        ("slab_length", C.c_double),
        ("n_regions", C.c_int32), ("region_material", _i32p),
        ("E0", C.c_double), ("E_cut", C.c_double),
        ("n_ebins", C.c_int32), ("ebin_edges", _dp),
        ("n_batches", C.c_int32), ("problem_id", C.c_uint32),
        ("n_histories_total", C.c_int64),
        ("n_species", C.c_int32), ("grid_offsets", _i64p), ("energies", _dp), ("sigma", _dp),
        ("n_ch", C.c_int32), ("ch_scatter", C.c_int32), ("ch_absorb", C.c_int32),
        ("awr", _dp),
        ("n_materials", C.c_int32), ("mat_offsets", _i32p), ("mat_species", _i32p),
        ("mat_dens", _dp),
        ("derivatives", C.c_int32), ("ch_nu_fission", C.c_int32),
    ]


class _Tallies(C.Structure):
    _fields_ = [("flux", _dp), ("absorb", _dp), ("outcome", _dp), ("dflux", _dp),
                ("dabsorb", _dp), ("doutcome", _dp), ("ncoll", _u32p)]


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_int64, _dp]
    L.orc_grid_index.argtypes = [_dp, C.c_int64, C.c_double]
    L.orc_grid_index.restype = C.c_int64
    L.orc_xs_lookup.argtypes = [C.c_int32, _i64p, _dp, _dp, C.c_int32, C.c_int32, _i32p, _i32p,
                                _dp, C.c_int64, _dp, _i32p, _dp, C.c_int]
    L.orc_xs_lookup.restype = C.c_int64
    L.orc_xs_indices.argtypes = [_i64p, _dp, _i32p, _i32p, C.c_int64, _dp, _i32p, C.c_int32, _i32p]
    L.orc_xs_lookup_backward.argtypes = [_i64p, _dp, _dp, C.c_int32, _i32p, _i32p, _dp,
                                         C.c_int64, _dp, _i32p, _dp, _dp, _dp]
    L.orc_transport.argtypes = [C.POINTER(_Problem), C.POINTER(_Tallies), C.c_int64, C.c_int64,
                                C.c_uint64, C.c_int]
    L.orc_transport.restype = C.c_int64
    L.orc_eigenvalue.argtypes = [C.POINTER(_Problem), C.POINTER(_Tallies), C.c_uint64, C.c_int64,
                                 C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int, _dp, _dp,
                                 C.c_int64, _i64p, _dp, _u32p]
    L.orc_eigenvalue.restype = C.c_int
    L.orc_max_threads.restype = C.c_int


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def uniforms(seed: int, problem_id: int, hist: int, count: int, first: int = 0) -> np.ndarray:
    out = np.zeros(count)
    lib().orc_uniforms(seed, problem_id, hist, first, count, _ptr(out, _dp))
    return out


def grid_index(g, E: float) -> int:
    g = _c(g, np.float64)
    return int(lib().orc_grid_index(_ptr(g, _dp), len(g), float(E)))


def xs_lookup(lib_, mats, E, mat, n_threads: int = 1) -> np.ndarray:
    """out[l][r] = sum_i N_i sigma_{r,i}(E_l) over material mat[l]'s species."""
    E = _c(E, np.float64)
    mat = _c(mat, np.int32)
    go, en, sg = _c(lib_.grid_offsets, np.int64), _c(lib_.energies, np.float64), _c(lib_.sigma, np.float64)
    mo, ms, md = _c(mats.offsets, np.int32), _c(mats.species, np.int32), _c(mats.dens, np.float64)
    out = np.zeros((len(E), lib_.n_ch))
    lib().orc_xs_lookup(lib_.n_species, _ptr(go, _i64p), _ptr(en, _dp), _ptr(sg, _dp), lib_.n_ch,
                        mats.n_materials, _ptr(mo, _i32p), _ptr(ms, _i32p), _ptr(md, _dp),
                        len(E), _ptr(E, _dp), _ptr(mat, _i32p), _ptr(out, _dp), n_threads)
    return out


def xs_indices(lib_, mats, E, mat) -> np.ndarray:
    """k[l][i] for the i-th species of material mat[l] (-1 past its species count)."""
    E = _c(E, np.float64)
    mat = _c(mat, np.int32)
    go, en = _c(lib_.grid_offsets, np.int64), _c(lib_.energies, np.float64)
    mo, ms = _c(mats.offsets, np.int32), _c(mats.species, np.int32)
    maxs = int(np.max(np.diff(mo)))
    out = np.zeros((len(E), maxs), np.int32)
    lib().orc_xs_indices(_ptr(go, _i64p), _ptr(en, _dp), _ptr(mo, _i32p), _ptr(ms, _i32p), len(E),
                         _ptr(E, _dp), _ptr(mat, _i32p), maxs, _ptr(out, _i32p))
    return out


def xs_lookup_backward(lib_, mats, E, mat, grad_out):
    """(grad_dens [nnz], grad_sigma [P][n_ch]) for cotangent grad_out [n][n_ch]."""
    E = _c(E, np.float64)
    mat = _c(mat, np.int32)
    go_ = _c(grad_out, np.float64)
    gofs, en, sg = _c(lib_.grid_offsets, np.int64), _c(lib_.energies, np.float64), _c(lib_.sigma, np.float64)
    mo, ms, md = _c(mats.offsets, np.int32), _c(mats.species, np.int32), _c(mats.dens, np.float64)
    gd = np.zeros(len(md))
    gs = np.zeros_like(sg)
    lib().orc_xs_lookup_backward(_ptr(gofs, _i64p), _ptr(en, _dp), _ptr(sg, _dp), lib_.n_ch,
                                 _ptr(mo, _i32p), _ptr(ms, _i32p), _ptr(md, _dp), len(E),
                                 _ptr(E, _dp), _ptr(mat, _i32p), _ptr(go_, _dp), _ptr(gd, _dp),
                                 _ptr(gs, _dp))
    return gd, gs


def max_threads() -> int:
    return int(lib().orc_max_threads())


def transport(prob, seed: int, first: int = 0, count: int | None = None, n_threads: int = 1,
              derivatives: bool = False, history_debug: bool = False) -> dict:
    """Run histories [first, first + count) of a synthetic Problem.

    Returns per-batch sums: flux and absorb [B][bins], outcome [B][5]
    (absorbed, leaked through +x, leaked elsewhere, cut off, collisions), the
    derivative tallies [.., M] when requested, per-history collision counts
    when requested, and 'capped' (histories that hit the event cap)."""
    L = lib()
    count = prob.n_histories - first if count is None else count
    P, keep = _problem(prob, derivatives)
    B, nb, M = prob.n_batches, prob.n_tally_bins, prob.mats.n_materials
    res = dict(flux=np.zeros((B, nb)), absorb=np.zeros((B, nb)), outcome=np.zeros((B, N_OUT)))
    null = _dp()
    T = _Tallies(_ptr(res["flux"], _dp), _ptr(res["absorb"], _dp), _ptr(res["outcome"], _dp),
                 null, null, null, _u32p())
    if derivatives:
        res.update(dflux=np.zeros((B, nb, M)), dabsorb=np.zeros((B, nb, M)),
                   doutcome=np.zeros((B, N_OUT, M)))
        T.dflux, T.dabsorb, T.doutcome = (_ptr(res["dflux"], _dp), _ptr(res["dabsorb"], _dp),
                                          _ptr(res["doutcome"], _dp))
    if history_debug:
        res["ncoll"] = np.zeros(count, np.uint32)
        T.ncoll = _ptr(res["ncoll"], _u32p)
    capped = L.orc_transport(C.byref(P), C.byref(T), first, count, seed, n_threads)
    if capped < 0:
        raise ValueError("oracle transport rejected its arguments")
    res["capped"] = int(capped)
    return res


def transport_histories(prob, seed: int, hist_ids, n_threads: int = 1) -> np.ndarray:
    """Collision counts of the listed histories, each run alone from its own
    Philox stream (exactly what a full run gives for that history: a history
    depends only on the problem, the seed and its id).  Calls run in a
    thread pool (the C call releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    ids = [int(h) for h in np.asarray(hist_ids).ravel()]

    def one(h):
        return int(transport(prob, seed=seed, first=h, count=1, history_debug=True)["ncoll"][0])

    if n_threads <= 1:
        return np.array([one(h) for h in ids], np.uint32)
    with ThreadPoolExecutor(max_workers=n_threads) as ex:
        return np.array(list(ex.map(one, ids, chunksize=64)), np.uint32)


def _channels(lib_):
    """(scatter, absorb, nu-fission) channel indices of a 2-, 3- or 5-channel
    library (2: scatter, absorb; 3: + nu-fission; 5: total, scatter, absorb,
    fission, nu-fission); nu-fission -1 when absent."""
    if lib_.n_ch == 2:
        return 0, 1, -1
    if lib_.n_ch == 3:
        return 0, 1, 2
    if lib_.n_ch == 5:
        return 1, 2, 4
    raise ValueError("transport needs a 2-, 3- or 5-channel library")


def _problem(prob, derivatives=False):
    lib_, mats = prob.lib, prob.mats
    chs, cha, chnf = _channels(lib_)
    keep = dict(
        rm=_c(prob.region_material, np.int32), edges=_c(prob.ebin_edges, np.float64),
        go=_c(lib_.grid_offsets, np.int64), en=_c(lib_.energies, np.float64),
        sg=_c(lib_.sigma, np.float64), awr=_c(lib_.awr, np.float64),
        mo=_c(mats.offsets, np.int32), ms=_c(mats.species, np.int32), md=_c(mats.dens, np.float64))
    if len(keep["edges"]) == 0:
        keep["edges"] = np.zeros(2)
    P = _Problem(prob.geometry, prob.lattice_n, prob.pitch, prob.radius, prob.height,
                 prob.slab_length, len(keep["rm"]), _ptr(keep["rm"], _i32p), prob.E0, prob.E_cut,
                 max(len(prob.ebin_edges) - 1, 0), _ptr(keep["edges"], _dp), prob.n_batches,
                 prob.problem_id, prob.n_histories, lib_.n_species, _ptr(keep["go"], _i64p),
                 _ptr(keep["en"], _dp), _ptr(keep["sg"], _dp), lib_.n_ch, chs, cha,
                 _ptr(keep["awr"], _dp), mats.n_materials, _ptr(keep["mo"], _i32p),
                 _ptr(keep["ms"], _i32p), _ptr(keep["md"], _dp), int(derivatives), chnf)
    return P, keep


EIGEN_ERRORS = {-1: "bad arguments", -2: "a generation banked no fission site",
                -3: "out of memory", -4: "a history hit the event cap"}


def eigenvalue(prob, seed: int, n_per_gen: int, n_generations: int, n_inactive: int,
               k0: float = 1.0, n_threads: int = 1, bank: bool = False,
               history_debug: bool = False) -> dict:
    """k-eigenvalue power iteration of a synthetic Problem (fission spectrum
    temperature prob.T_fission).  Returns per generation k (site count),
    k_col, k_tl and sites; the active generations' tallies (flux, absorb
    [B][bins], outcome [B][5]); with bank=True the last generation's sites as
    rows (x, y, z, ci, cj, inpin) in bank order and the sites it started from
    ('source', N rows, when there are two or more generations); with
    history_debug the last generation's per-history collision counts."""
    L = lib()
    P, keep = _problem(prob)
    if P.ch_nu_fission < 0:
        raise ValueError("an eigenvalue run needs a nu-fission channel")
    B, nb = prob.n_batches, prob.n_tally_bins
    res = dict(flux=np.zeros((B, nb)), absorb=np.zeros((B, nb)), outcome=np.zeros((B, N_OUT)))
    null = _dp()
    T = _Tallies(_ptr(res["flux"], _dp), _ptr(res["absorb"], _dp), _ptr(res["outcome"], _dp),
                 null, null, null, _u32p())
    gen = np.zeros((n_generations, 4))
    cap = 8 * n_per_gen if bank else 0
    rows = np.zeros((max(cap, 1), 6))
    src = np.zeros((n_per_gen, 6)) if bank else None
    bank_n = C.c_int64(0)
    ncoll = np.zeros(n_per_gen, np.uint32) if history_debug else None
    rc = L.orc_eigenvalue(C.byref(P), C.byref(T), seed, n_per_gen, n_generations, n_inactive,
                          float(k0), float(prob.T_fission), n_threads, _ptr(gen, _dp),
                          _ptr(rows, _dp) if bank else _dp(), cap, C.byref(bank_n),
                          _ptr(src, _dp) if bank else _dp(),
                          _ptr(ncoll, _u32p) if history_debug else _u32p())
    if rc != 0:
        raise RuntimeError(f"oracle eigenvalue run failed: {EIGEN_ERRORS.get(rc, rc)}")
    res.update(k=gen[:, 0].copy(), k_col=gen[:, 1].copy(), k_tl=gen[:, 2].copy(),
               sites=gen[:, 3].astype(np.int64))
    if bank:
        if bank_n.value > cap:
            raise RuntimeError("bank larger than the buffer")
        res["bank"] = rows[:bank_n.value].copy()
        if n_generations > 1:
            res["source"] = src
    if history_debug:
        res["ncoll"] = ncoll
    return res


# ---------------------------------------------------------------------------
# single-step helpers (for pins)
# ---------------------------------------------------------------------------
SURF_NONE, SURF_ZTOP, SURF_ZBOT, SURF_CYL, SURF_XLO, SURF_XHI, SURF_YLO, SURF_YHI = range(8)


def scatter_kinematics(A: float, mu: float):
    """(E'/E, laboratory cosine) of elastic scattering at CM cosine mu."""
    out = np.zeros(2)
    L = lib()
    L.orc_scatter_kinematics.argtypes = [C.c_double, C.c_double, _dp]
    L.orc_scatter_kinematics(A, mu, _ptr(out, _dp))
    return out[0], out[1]


def rotate_direction(direction, mu: float, c: float, s: float) -> np.ndarray:
    d = _c(direction, np.float64)
    out = np.zeros(3)
    L = lib()
    L.orc_rotate_direction.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp]
    L.orc_rotate_direction(_ptr(d, _dp), mu, c, s, _ptr(out, _dp))
    return out


class _Bound:
    """A Problem packed for the C side, with its arrays kept alive."""

    def __init__(self, prob, derivatives=False):
        self.P, self.keep = _problem(prob, derivatives)


def source_state(prob, seed: int, h: int) -> np.ndarray:
    """{x, y, z, u, v, w, region, draws used} of history h's source particle."""
    b = _Bound(prob)
    out = np.zeros(8)
    L = lib()
    L.orc_source_state.argtypes = [C.POINTER(_Problem), C.c_uint64, C.c_int64, _dp]
    L.orc_source_state(C.byref(b.P), seed, h, _ptr(out, _dp))
    return out


def site_source_state(prob, seed: int, h: int, site) -> np.ndarray:
    """{x, y, z, u, v, w, E, region, draws used} of history h started from a
    fission site {x, y, z, ci, cj, inpin}."""
    b = _Bound(prob)
    s = _c(site, np.float64)
    out = np.zeros(9)
    L = lib()
    L.orc_site_source_state.argtypes = [C.POINTER(_Problem), C.c_uint64, C.c_int64, _dp, C.c_double, _dp]
    L.orc_site_source_state(C.byref(b.P), seed, h, _ptr(s, _dp), float(prob.T_fission), _ptr(out, _dp))
    return out


def surface_distance(prob, state):
    """(surface id, distance) from state {x, y, z, u, v, w, ci, cj, inpin}."""
    b = _Bound(prob)
    st = _c(state, np.float64)
    d = C.c_double()
    L = lib()
    L.orc_surface_distance.argtypes = [C.POINTER(_Problem), _dp, C.POINTER(C.c_double)]
    L.orc_surface_distance.restype = C.c_int
    s = L.orc_surface_distance(C.byref(b.P), _ptr(st, _dp), C.byref(d))
    return int(s), float(d.value)


def fission_energies(seed: int, problem_id: int, hist: int, T: float, n: int) -> np.ndarray:
    """n successive fission-spectrum energies drawn from one history's stream."""
    out = np.zeros(n)
    L = lib()
    L.orc_fission_energies.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_double, C.c_int64, _dp]
    L.orc_fission_energies(seed, problem_id, hist, T, n, _ptr(out, _dp))
    return out
