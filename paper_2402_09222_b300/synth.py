"""Seeded synthetic inputs for the transport and lookup workloads.

This module only *generates data*: species energy grids and cross-section
tables, material compositions, lattice descriptions and lookup inputs.  It holds
none of the method's arithmetic (no grid search, interpolation, sampling or
tallying), so both the CUDA path and the CPU oracle may consume what it makes.

The paper tunes OpenMC on the Hoogenboom-Martin "large" reactor model
(Sec. 5.1), whose nuclear data is not available here.  The generators below
stand in for it with the shapes of that problem: a library of a few hundred
species with ~1e4-point energy grids, materials of 4 to 321 species, and a
17x17 pin lattice.

Cross-section model per species (all values in barns, energies in eV):
  * grid: log-spaced on [1e-5, 2e7]; each interior point jittered by
    U(-0.4, 0.4) of one log step (endpoints fixed), so every species has its
    own grid and the per-species search is real;
  * absorption  a0 * sqrt(0.0253 / E), a0 ~ logU(0.1, 1e3);
  * scattering  s0 ~ U(2, 20);
  * 20 Lorentzian resonances h (G/2)^2 / ((E - Ek)^2 + (G/2)^2) with
    Ek ~ logU(1, 1e5), G = Ek * U(1e-4, 1e-2), h ~ logU(10, 1e4), split a
    fraction c ~ U(0.2, 0.8) to scattering and 1 - c to absorption;
  * fission = phi * absorption (phi = 0 for 80 % of species, else U(0.1, 0.9)),
    nu-fission = 2.43 * fission, total = scattering + absorption;
  * mass ratio A ~ U(1, 240).

Channel order of the 5-channel tables: total, scatter, absorb, fission,
nu_fission.  2-channel tables hold scatter, absorb.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

E_MIN = 1.0e-5
E_MAX = 2.0e7

CH_TOTAL, CH_SCATTER, CH_ABSORB, CH_FISSION, CH_NU_FISSION = range(5)

GEOM_INFINITE = 0
GEOM_LATTICE = 1
GEOM_SLAB = 2


def _logu(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def log_grid(n_points: int, rng: np.random.Generator | None, jitter: bool = True) -> np.ndarray:
    """Strictly increasing FP64 grid on [E_MIN, E_MAX], log-spaced, optionally jittered."""
    x = np.linspace(math.log(E_MIN), math.log(E_MAX), n_points)
    if jitter and n_points > 2:
        step = x[1] - x[0]
        x[1:-1] += rng.uniform(-0.4, 0.4, n_points - 2) * step
    g = np.exp(x)
    g[0], g[-1] = E_MIN, E_MAX
    assert np.all(np.diff(g) > 0)
    return g


@dataclass
class Library:
    """Species data: concatenated grids plus per-point cross sections."""
    grid_offsets: np.ndarray      # int64 [S+1]
    energies: np.ndarray          # float64 [P]
    sigma: np.ndarray             # float64 [P][n_ch]
    awr: np.ndarray               # float64 [S] (mass ratio A)

    @property
    def n_species(self) -> int:
        return len(self.awr)

    @property
    def n_ch(self) -> int:
        return self.sigma.shape[1]

    def grid(self, s: int) -> np.ndarray:
        return self.energies[self.grid_offsets[s]:self.grid_offsets[s + 1]]

    def table(self, s: int) -> np.ndarray:
        return self.sigma[self.grid_offsets[s]:self.grid_offsets[s + 1]]

    def channels(self, chans) -> "Library":
        """The same library restricted to the given channel columns."""
        return Library(self.grid_offsets, self.energies,
                       np.ascontiguousarray(self.sigma[:, list(chans)]), self.awr)

    def fp32_rounded(self) -> "Library":
        """Cross sections rounded to FP32 and widened back (exactly) to FP64."""
        return Library(self.grid_offsets, self.energies,
                       self.sigma.astype(np.float32).astype(np.float64), self.awr)

    def subset(self, species) -> "Library":
        species = list(species)
        grids = [self.grid(s) for s in species]
        tabs = [self.table(s) for s in species]
        off = np.zeros(len(species) + 1, np.int64)
        off[1:] = np.cumsum([len(g) for g in grids])
        return Library(off, np.concatenate(grids), np.concatenate(tabs), self.awr[species].copy())


def species_library(n_species: int, n_points: int, seed: int, n_res: int = 20,
                    jitter: bool = True) -> Library:
    rng = np.random.default_rng(seed)
    grids, tabs, awr = [], [], []
    for _ in range(n_species):
        g = log_grid(n_points, rng, jitter)
        a0 = _logu(rng, 0.1, 1e3)
        s0 = rng.uniform(2.0, 20.0)
        ek = _logu(rng, 1.0, 1e5, n_res)
        gam = ek * rng.uniform(1e-4, 1e-2, n_res)
        h = _logu(rng, 10.0, 1e4, n_res)
        c = rng.uniform(0.2, 0.8, n_res)
        phi = 0.0 if rng.uniform() < 0.8 else rng.uniform(0.1, 0.9)
        A = rng.uniform(1.0, 240.0)
        half2 = (gam / 2.0) ** 2
        lor = h[None, :] * half2[None, :] / ((g[:, None] - ek[None, :]) ** 2 + half2[None, :])
        sig_s = s0 + lor @ c
        sig_a = a0 * np.sqrt(0.0253 / g) + lor @ (1.0 - c)
        fis = phi * sig_a
        t = np.empty((n_points, 5))
        t[:, CH_TOTAL] = sig_s + sig_a
        t[:, CH_SCATTER] = sig_s
        t[:, CH_ABSORB] = sig_a
        t[:, CH_FISSION] = fis
        t[:, CH_NU_FISSION] = 2.43 * fis
        grids.append(g)
        tabs.append(t)
        awr.append(A)
    off = np.zeros(n_species + 1, np.int64)
    off[1:] = np.cumsum([len(g) for g in grids])
    return Library(off, np.concatenate(grids), np.concatenate(tabs), np.asarray(awr))


@dataclass
class Materials:
    """CSR material compositions: species ids and atom densities (atoms/b-cm)."""
    offsets: np.ndarray   # int32 [M+1]
    species: np.ndarray   # int32 [nnz]
    dens: np.ndarray      # float64 [nnz]

    @property
    def n_materials(self) -> int:
        return len(self.offsets) - 1

    def members(self, m):
        a, b = self.offsets[m], self.offsets[m + 1]
        return self.species[a:b], self.dens[a:b]

    def scaled(self, scales) -> "Materials":
        """Densities of material m multiplied by scales[m] (all species together)."""
        d = self.dens.copy()
        for m, s in enumerate(scales):
            d[self.offsets[m]:self.offsets[m + 1]] *= s
        return Materials(self.offsets, self.species, d)


def make_materials(members, dens) -> Materials:
    off = np.zeros(len(members) + 1, np.int32)
    off[1:] = np.cumsum([len(m) for m in members])
    return Materials(off, np.concatenate([np.asarray(m, np.int32) for m in members]).astype(np.int32),
                     np.concatenate([np.asarray(d, np.float64) for d in dens]))


def config2_material_sizes(n_materials: int = 12, lo: int = 4, hi: int = 321):
    return [int(round(lo * (hi / lo) ** (m / (n_materials - 1)))) for m in range(n_materials)]


def lookup_materials(n_species: int, seed: int, n_materials: int = 12) -> Materials:
    """Materials of 4..321 species (geometric sizes), densities logU(1e-6, 1e-1)."""
    rng = np.random.default_rng(seed)
    members, dens = [], []
    for n_m in config2_material_sizes(n_materials):
        n_m = min(n_m, n_species)
        members.append(np.sort(rng.choice(n_species, n_m, replace=False)))
        dens.append(_logu(rng, 1e-6, 1e-1, n_m))
    return make_materials(members, dens)


def lookup_inputs(n: int, n_materials: int, seed: int):
    """Lookup energies ~ logU[E_MIN, E_MAX] and materials ~ U{0..M-1}."""
    rng = np.random.default_rng(seed)
    E = _logu(rng, E_MIN, E_MAX, n)
    mat = rng.integers(0, n_materials, n).astype(np.int32)
    return E, mat


@dataclass
class Problem:
    """Everything that defines one fixed-source transport problem."""
    geometry: int
    lib: Library
    mats: Materials
    lattice_n: int = 0
    pitch: float = 1.26
    radius: float = 0.41
    height: float = 100.0
    slab_length: float = 0.0
    region_material: np.ndarray = field(default_factory=lambda: np.zeros(1, np.int32))
    E0: float = 2.0e6
    E_cut: float = 1.0e-5
    T_fission: float = 1.2895e6     # Maxwellian temperature of fission neutrons (eV)
    ebin_edges: np.ndarray = field(default_factory=lambda: np.zeros(0))
    n_batches: int = 20
    problem_id: int = 0
    n_histories: int = 0

    @property
    def n_regions(self) -> int:
        return len(self.region_material)

    @property
    def n_tally_bins(self) -> int:
        if self.geometry == GEOM_INFINITE:
            return len(self.ebin_edges) - 1
        return self.n_regions


def lattice_region_material(n: int, m_pin: int = 0, m_mod: int = 1, m_guide: int = 2) -> np.ndarray:
    """Regions 0..n^2-1 are pins (i*n + j), region n^2 the moderator.
    Pins with i % 3 == 2 and j % 3 == 2 are guide tubes."""
    rm = np.full(n * n + 1, m_pin, np.int32)
    for i in range(n):
        for j in range(n):
            if i % 3 == 2 and j % 3 == 2:
                rm[i * n + j] = m_guide
    rm[n * n] = m_mod
    return rm


def energy_bin_edges(n_bins: int = 50) -> np.ndarray:
    return np.exp(np.linspace(math.log(E_MIN), math.log(E_MAX), n_bins + 1))


def config1_problem(n_histories: int = 10_000, seed: int = 1235) -> Problem:
    """Infinite homogeneous medium of 8 species x 2000 points, FP64."""
    lib = species_library(8, 2000, seed).channels([CH_SCATTER, CH_ABSORB])
    rng = np.random.default_rng(seed + 100)
    mats = make_materials([np.arange(8)], [_logu(rng, 1e-6, 1e-1, 8)])
    return Problem(GEOM_INFINITE, lib, mats, ebin_edges=energy_bin_edges(50),
                   n_histories=n_histories)


def config3_library(n_points: int = 11_303, seed: int = 1237) -> Library:
    return species_library(47, n_points, seed).channels([CH_SCATTER, CH_ABSORB])


def config3_materials(seed: int = 1237) -> Materials:
    """Fuel (species 0-39), moderator (40-43) and guide-tube (44-46) materials."""
    rng = np.random.default_rng(seed + 100)
    return make_materials([np.arange(0, 40), np.arange(40, 44), np.arange(44, 47)],
                          [_logu(rng, 1e-5, 1e-2, 40), _logu(rng, 1e-3, 1e-1, 4),
                           _logu(rng, 1e-3, 1e-1, 3)])


def config3_problem(n_histories: int = 10_000_000, lattice_n: int = 17, n_points: int = 11_303,
                    seed: int = 1237, lib: Library | None = None) -> Problem:
    """17x17 lattice of cylinders (r 0.41, pitch 1.26), height 100, vacuum x/y faces,
    reflective top and bottom, 3 materials of 40/4/3 species."""
    lib = lib if lib is not None else config3_library(n_points, seed)
    return Problem(GEOM_LATTICE, lib, config3_materials(seed), lattice_n=lattice_n,
                   region_material=lattice_region_material(lattice_n), n_histories=n_histories)


def config5_problems(lib: Library, mats: Materials, n_problems: int = 64, seed: int = 1239,
                     hist_lo: float = 1e4, hist_hi: float = 2e6):
    """Independent lattices of uneven size sharing one library and material set.

    Each problem draws n ~ U{3..17}, histories ~ logU[hist_lo, hist_hi] and three
    distinct materials (pin, moderator, guide) from the material set.
    """
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(n_problems):
        n = int(rng.integers(3, 18))
        nh = int(round(_logu(rng, hist_lo, hist_hi)))
        m3 = rng.choice(mats.n_materials, 3, replace=False)
        probs.append(Problem(GEOM_LATTICE, lib, mats, lattice_n=n,
                             region_material=lattice_region_material(n, *[int(x) for x in m3]),
                             problem_id=p, n_histories=nh))
    return probs


# ---------------------------------------------------------------------------
# Special tables for closed-form checks
# ---------------------------------------------------------------------------

def flat_library(sig_s: float, sig_a: float, A: float = 1.0) -> Library:
    """One species whose 2-channel cross sections are constant in energy."""
    g = np.array([E_MIN, E_MAX])
    return Library(np.array([0, 2], np.int64), g, np.array([[sig_s, sig_a], [sig_s, sig_a]]),
                   np.array([A]))


def flat_fission_library(sig_s: float, sig_a: float, nu_sig_f: float, A: float = 1.0) -> Library:
    """One species with constant 3-channel cross sections (scatter, absorb,
    nu-fission): an infinite medium of it has k = nu_sig_f / sig_a."""
    g = np.array([E_MIN, E_MAX])
    row = [sig_s, sig_a, nu_sig_f]
    return Library(np.array([0, 2], np.int64), g, np.array([row, row]), np.array([A]))


def eigen_library(n_points: int = 11_303, seed: int = 1237) -> Library:
    """The lattice library with scatter, absorb and nu-fission channels.
    Only fuel species (0-39) keep their fission data; the moderator and
    guide-tube species (40-46) are made non-fissile."""
    lib = species_library(47, n_points, seed).channels([CH_SCATTER, CH_ABSORB, CH_NU_FISSION])
    lib.sigma[lib.grid_offsets[40]:, 2] = 0.0
    return lib


def eigen_problem(n_per_gen: int, lattice_n: int = 17, n_points: int = 11_303, seed: int = 1237,
                  lib: Library | None = None, n_batches: int = 20) -> Problem:
    """The 17x17 lattice as a k-eigenvalue problem (fission channels kept)."""
    lib = lib if lib is not None else eigen_library(n_points, seed)
    return Problem(GEOM_LATTICE, lib, config3_materials(seed), lattice_n=lattice_n,
                   region_material=lattice_region_material(lattice_n), n_histories=n_per_gen,
                   n_batches=n_batches)


def linear_library(n_species: int, n_points: int, seed: int, n_ch: int = 5,
                   shared_grid: bool = False) -> Library:
    """Cross sections that are exactly linear in E (sigma = a + b E), so
    piecewise-linear interpolation reproduces them up to rounding."""
    rng = np.random.default_rng(seed)
    grids, tabs = [], []
    base = log_grid(n_points, rng, jitter=True)
    for _ in range(n_species):
        g = base.copy() if shared_grid else log_grid(n_points, rng, jitter=True)
        a = rng.uniform(1.0, 10.0, n_ch)
        b = rng.uniform(1e-7, 1e-6, n_ch)
        grids.append(g)
        tabs.append(a[None, :] + b[None, :] * g[:, None])
    off = np.zeros(n_species + 1, np.int64)
    off[1:] = np.cumsum([len(g) for g in grids])
    return Library(off, np.concatenate(grids), np.concatenate(tabs),
                   rng.uniform(1.0, 240.0, n_species))


def infinite_problem(lib: Library, mats: Materials, n_histories: int, E0: float = 2.0e6,
                     E_cut: float = 1.0e-5, n_ebins: int = 50, problem_id: int = 0) -> Problem:
    return Problem(GEOM_INFINITE, lib, mats, ebin_edges=energy_bin_edges(n_ebins), E0=E0,
                   E_cut=E_cut, n_histories=n_histories, problem_id=problem_id)


def slab_problem(lib: Library, mats: Materials, length: float, n_histories: int) -> Problem:
    """Pencil beam along +x entering a box x in [0, length] of material 0."""
    return Problem(GEOM_SLAB, lib, mats, slab_length=length, n_histories=n_histories)
