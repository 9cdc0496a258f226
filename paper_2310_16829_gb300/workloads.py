"""Seeded synthetic workloads for the Lattice Multislice Algorithm (LMA) hot path.

This module only places atoms and states parameters. It holds none of the
method's arithmetic: no potentials, waves, transforms or coefficients. Both the
FP64 oracle (through the tests) and the CUDA library (through the binding and
``bench.py``) consume the same objects built here.

Physical parameters follow the STEM setting of the paper (Sec. 3.1, eqs.
probe_wave_function / aberration_function / aperture_function): wavelength in
Angstrom, interaction constant in rad/(V*Angstrom), projected potentials in
V*Angstrom per slice, angles in rad. The relativistic wavelength and
interaction constant at 300 kV are stored as literals; a CPU test checks them
against the oracle's formulas (the paper quotes lambda(200 kV) = 0.0250793 A in
the captions of Sec. 4.2.3).

The specimens stand in for the paper's M1 workload (Sec. 4.2.5 / 4.2.6), which
is not available: a 1024^2 grid of about 80 A, probe lattices of 10^4-10^5
positions, 100-slice thickness, frozen-phonon averaging.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import List, Tuple

import numpy as np

# Wavelength / interaction constant literals (Angstrom, rad/(V*Angstrom)).
LAMBDA_300KV = 0.019687489006848795
SIGMA_300KV = 0.0006526161421721631
# The simple-cubic toy workload states its constants directly (200 kV, rounded).
LAMBDA_CFG0 = 0.02508
SIGMA_CFG0 = 7.29e-4

# Basis kinds and store precisions (mirror LMA_BASIS_* / LMA_PREC_* in include/lma.h).
BASIS_GAUSS = 0
BASIS_PROBE = 1
BASIS_TRIG = 2
BASIS_TRIG_RADIAL = 3
PREC_C64 = 0
PREC_FP16_STORE = 1
PREC_MIXED = 2


@dataclass
class Grid:
    nx: int
    ny: int
    lx: float          # Angstrom
    ly: float          # Angstrom
    slice_dz: float    # Angstrom
    n_slices: int
    lam: float         # Angstrom
    sigma: float       # rad / (V * Angstrom)
    bandlimit_frac: float = 2.0 / 3.0

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny


@dataclass
class Potential:
    """Gaussian-sum projected potential per atom and slice (V*Angstrom)."""
    peak: Tuple[float, ...]                 # per species
    term_frac: Tuple[float, ...] = (0.7, 0.3)
    term_width: Tuple[float, ...] = (0.15, 0.5)
    r_cut: float = 3.0


@dataclass
class Atoms:
    """One frozen-phonon configuration (structure of arrays)."""
    x: np.ndarray        # float64, Angstrom
    y: np.ndarray        # float64, Angstrom
    slice: np.ndarray    # int32
    species: np.ndarray  # int16

    def __len__(self) -> int:
        return int(self.x.shape[0])


@dataclass
class Probe:
    alpha_max: float          # rad
    cs: float = 0.0           # Angstrom
    defocus: float = 0.0      # Angstrom


@dataclass
class BasisDesc:
    kind: int = BASIS_GAUSS
    gauss_sigma: float = 0.0                 # Angstrom; 0 selects lambda / (2 alpha_max)
    in_spacing_px: Tuple[int, int] = (4, 4)  # input-wave lattice spacing (x, y)
    in_offset_px: Tuple[int, int] = (2, 2)   # input-wave lattice offset (x, y)
    f: int = 1
    L: int = 32
    window: int = 128
    det_window: int = 128
    precision: int = PREC_C64
    phonon_batch: int = 0                    # configurations per launch; 0 = by free memory
    trig_degree: int = 0                     # BASIS_TRIG*: degree of phi_n; 0 = alpha_max l_x / lambda
    coef_mode: int = 0                       # 0: least squares; 1: closed-form trigonometric (BASIS_TRIG)


@dataclass
class Detector:
    r1: float   # rad, inclusive
    r2: float   # rad, exclusive


@dataclass
class Region:
    px0: int
    py0: int
    npx: int
    npy: int
    spacing_px: Tuple[int, int]


@dataclass
class Workload:
    name: str
    grid: Grid
    potential: Potential
    phonons: List[Atoms]
    probe: Probe
    basis: BasisDesc
    detectors: List[Detector]
    region: Region
    notes: str = ""

    @property
    def n_pixels(self) -> int:
        return self.region.npx * self.region.npy

    def with_region(self, region: Region) -> "Workload":
        return replace(self, region=region)

    def with_phonons(self, n: int) -> "Workload":
        return replace(self, phonons=self.phonons[:n])


# ----------------------------------------------------------------------------
# crystal builders
# ----------------------------------------------------------------------------

def _layered_crystal(a: float, ncx: int, ncy: int, n_slices: int,
                     layers: List[List[Tuple[float, float, int]]],
                     rms: float, seed: int | None) -> Atoms:
    """Tile a rectangular cell; slice s uses ``layers[s % len(layers)]``.

    Each layer entry is (fractional x, fractional y, species). A Gaussian
    lateral displacement of standard deviation ``rms`` (Angstrom) is drawn
    independently for x and y of every atom when ``seed`` is given.
    """
    # atom order: slice, layer entry, row j, column i (i fastest)
    ii = np.tile(np.arange(ncx, dtype=np.float64), ncy)
    jj = np.repeat(np.arange(ncy, dtype=np.float64), ncx)
    xs, ys, ss, sp = [], [], [], []
    for s in range(n_slices):
        for (fx, fy, spc) in layers[s % len(layers)]:
            xs.append((ii + fx) * a)
            ys.append((jj + fy) * a)
            ss.append(np.full(ii.shape, s, dtype=np.int32))
            sp.append(np.full(ii.shape, spc, dtype=np.int16))
    x = np.concatenate(xs) if xs else np.zeros(0)
    y = np.concatenate(ys) if ys else np.zeros(0)
    if seed is not None and rms > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.normal(0.0, rms, size=(2, x.shape[0]))
        x = x + d[0]
        y = y + d[1]
    return Atoms(x=x, y=y, slice=np.concatenate(ss) if ss else np.zeros(0, np.int32),
                 species=np.concatenate(sp) if sp else np.zeros(0, np.int16))


# ABO3 perovskite projected along [001]: AO and BO2 layers alternate.
_ABO3_LAYERS = [
    [(0.0, 0.0, 0), (0.5, 0.5, 2)],                   # AO : A at (0,0), O at (1/2,1/2)
    [(0.5, 0.5, 1), (0.5, 0.0, 2), (0.0, 0.5, 2)],    # BO2: B at (1/2,1/2), O at (1/2,0),(0,1/2)
]
ABO3_A = 3.905
ABO3_PEAKS = (600.0, 400.0, 120.0)


def simple_cubic_workload() -> Workload:
    """Simple-cubic toy crystal, 4x4 cells of 4 A, one atom per column per slice.

    128^2 grid (0.125 A), 10 slices of 2 A, 200 kV, 20 mrad aberration-free
    probe, HAADF 60-200 mrad, 16x16 probes every 8 px, no phonons.
    """
    grid = Grid(nx=128, ny=128, lx=16.0, ly=16.0, slice_dz=2.0, n_slices=10,
                lam=LAMBDA_CFG0, sigma=SIGMA_CFG0)
    atoms = _layered_crystal(4.0, 4, 4, 10, [[(0.0, 0.0, 0)]], 0.0, None)
    return Workload(
        name="sc4x4_128sq_10sl",
        grid=grid,
        potential=Potential(peak=(300.0,)),
        phonons=[atoms],
        probe=Probe(alpha_max=0.020),
        basis=BasisDesc(window=128, det_window=128),
        detectors=[Detector(0.060, 0.200)],
        region=Region(0, 0, 16, 16, (8, 8)),
        notes="simple cubic a=4 A, 4x4 cells, W=D=X (periodic window)",
    )


def perovskite_workload(cells: int = 10, nx: int = 512, n_slices: int = 50,
                        n_phonons: int = 8, seed_base: int = 1000,
                        probes: int | None = None, rms: float = 0.08) -> Workload:
    """ABO3 (a = 3.905 A) slab, 300 kV, 25 mrad probe, HAADF 70-200 mrad.

    Defaults are the 10x10-cell, 512^2, 50-slice (100 A) specimen with 8
    frozen-phonon configurations (seed ``seed_base + phi``) and 128x128 probes
    every 4 px.
    """
    l = cells * ABO3_A
    grid = Grid(nx=nx, ny=nx, lx=l, ly=l, slice_dz=2.0, n_slices=n_slices,
                lam=LAMBDA_300KV, sigma=SIGMA_300KV)
    phonons = [_layered_crystal(ABO3_A, cells, cells, n_slices, _ABO3_LAYERS, rms,
                                seed_base + p) for p in range(n_phonons)]
    if probes is None:
        probes = nx // 4
    spacing = nx // probes
    return Workload(
        name=f"abo3_{cells}x{cells}_{nx}sq_{n_slices}sl_{n_phonons}ph",
        grid=grid,
        potential=Potential(peak=ABO3_PEAKS),
        phonons=phonons,
        probe=Probe(alpha_max=0.025),
        basis=BasisDesc(window=128, det_window=128),
        detectors=[Detector(0.070, 0.200)],
        region=Region(0, 0, probes, probes, (spacing, spacing)),
        notes="ABO3 perovskite, frozen phonons RMS 0.08 A",
    )


def batch_workloads(n_phonons: int = 32) -> List[Workload]:
    """Three specimens of uneven size (256^2/40 A, 512^2/100 A, 1024^2/200 A)."""
    out = []
    for k, (cells, nx, ns) in enumerate(((5, 256, 20), (10, 512, 50), (20, 1024, 100))):
        out.append(perovskite_workload(cells=cells, nx=nx, n_slices=ns, n_phonons=n_phonons,
                                       seed_base=2000 + 100 * k))
    return out


def small_batch_workloads(n_phonons: int = 2, f: int = 1) -> List[Workload]:
    """Many small specimens: 16 ABO3 slabs of 2x2 cells on 128^2 (10 slices) and 8 of 5x5
    cells on 256^2 (20 slices), probes every 4 px, input waves every 4 px thinned to the
    sub-lattice I_f (Sec. 4.2.1, reduction (i)). With f = 1 each specimen's slice launch
    is 7 or 27 waves of CTAs deep; with f = 4 it has 64 or 256 translates, fewer than or
    under two waves of the GPU's SMs."""
    out = []
    for k in range(24):
        cells, nx, ns = (2, 128, 10) if k < 16 else (5, 256, 20)
        w = perovskite_workload(cells=cells, nx=nx, n_slices=ns, n_phonons=n_phonons,
                                seed_base=4000 + 100 * k)
        out.append(replace(w, basis=replace(w.basis, f=f)))
    return out


def serving_workload() -> Workload:
    """Resident 20x20-cell ABO3 specimen, 1024^2 grid, 200 A thick, one configuration."""
    w = perovskite_workload(cells=20, nx=1024, n_slices=100, n_phonons=1, seed_base=3000,
                            probes=256)
    return replace(w, name="abo3_20x20_1024sq_100sl_serving")


def column_sites(cells: int) -> np.ndarray:
    """Undisplaced projected column positions of the ABO3 slab, (n, 2) in Angstrom."""
    pts = []
    for j in range(cells):
        for i in range(cells):
            for fx, fy in ((0.0, 0.0), (0.5, 0.5), (0.5, 0.0), (0.0, 0.5)):
                pts.append(((i + fx) * ABO3_A, (j + fy) * ABO3_A))
    return np.asarray(pts, dtype=np.float64)


def edit_request(cells: int, req: int, seed_base: int = 3000) -> Tuple[float, float, int, int]:
    """Seeded single-column edit: (cx, cy, op, new_species); op 0 = remove, 1 = set species."""
    rng = np.random.default_rng(seed_base + req)
    sites = column_sites(cells)
    k = int(rng.integers(0, sites.shape[0]))
    op = int(rng.integers(0, 2))
    spc = int(rng.integers(0, 3))
    return float(sites[k, 0]), float(sites[k, 1]), op, spc


def sample_probes(region: Region, n: int, seed: int) -> np.ndarray:
    """Seeded sample of probe lattice indices (a, b) inside a region, corners included."""
    rng = np.random.default_rng(seed)
    corners = [(0, 0), (region.npx - 1, region.npy - 1), (region.npx - 1, 0), (0, region.npy - 1)]
    pts = set(corners[: min(n, 4)])
    while len(pts) < n:
        pts.add((int(rng.integers(0, region.npx)), int(rng.integers(0, region.npy))))
    return np.asarray(sorted(pts), dtype=np.int64)


# The probe-approximation geometry of Sec. 4.2.3's error-versus-L figures: 62.416 A at
# 0.1219 A per pixel (512^2; the 128-pixel window then spans 15.6 A, the probe's extent),
# 200 kV (lambda = 0.0250793 A), focus Z = 100 A, C_s = -2000 A, alpha_max = 26 mrad, probes
# every 2 px and input waves at I = P + p/2.
LAMBDA_200KV_FIG = 0.0250793


def probe_approximation_workload(kind: int, f: int = 1, L: int = 32, gauss_sigma: float = 0.0,
                                 coef_mode: int = 0, window: int = 128) -> Workload:
    """Probe approximation (coefficients only; one atom, one slice as a placeholder specimen)."""
    grid = Grid(nx=512, ny=512, lx=62.416, ly=62.416, slice_dz=2.0, n_slices=1,
                lam=LAMBDA_200KV_FIG, sigma=SIGMA_CFG0)
    atoms = Atoms(np.array([0.0]), np.array([0.0]), np.array([0], np.int32), np.array([0], np.int16))
    return Workload(
        name=f"probe_approx_512sq_kind{kind}_f{f}_W{window}",
        grid=grid,
        potential=Potential(peak=(300.0,)),
        phonons=[atoms],
        probe=Probe(alpha_max=0.026, cs=-2000.0, defocus=100.0),
        basis=BasisDesc(kind=kind, gauss_sigma=gauss_sigma, in_spacing_px=(2, 2), in_offset_px=(1, 1),
                        f=f, L=L, coef_mode=coef_mode, window=window),
        detectors=[Detector(0.07, 0.2)],
        region=Region(0, 0, 1, 1, (2, 2)),
        notes="probe approximation error versus L and f (no image)",
    )
