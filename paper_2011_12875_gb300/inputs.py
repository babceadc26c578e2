"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module only makes positions, boxes and coefficients; it contains none of
the SNAP arithmetic.  The workloads stand in for the paper's tungsten
benchmark (Sec. II-C: 2000 atoms, 26 neighbours each, 2J = 8 and 14), whose
potential file and LAMMPS input are not available: a BCC lattice with
a = 3.1803 A, n^3 cubic cells (2 n^3 atoms), periodic orthorhombic box,
independent uniform displacements per Cartesian component, an optional
diagonal strain of each box axis, and linear coefficients drawn uniformly.
All draws use numpy's PCG64 with fixed seeds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LATTICE_A = 3.1803       # BCC lattice constant (A)
RCUT = 4.73442           # cutoff radius (A): shells 1-3 (26 neighbours) inside
RFAC0 = 0.99363
RMIN0 = 0.0
SEED_LATTICE = 1234
SEED_BETA = 5678
SEED_BATCH = 42


def ncoeff(twojmax: int) -> int:
    """Number of bispectrum components for 0 <= 2j2 <= 2j1 <= 2j <= 2J."""
    n = 0
    for t1 in range(twojmax + 1):
        for t2 in range(t1 + 1):
            for t in range(t1 - t2, min(twojmax, t1 + t2) + 1, 2):
                if t >= t1:
                    n += 1
    return n


@dataclass
class Config:
    """One atomic configuration: positions (n, 3) and box lengths (3,)."""
    pos: np.ndarray
    box: np.ndarray
    name: str = ""

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])


def bcc(ncell: int, disp: float = 0.1, strain: float = 0.0, seed: int = SEED_LATTICE,
        a: float = LATTICE_A) -> Config:
    """BCC lattice of ncell^3 cells with uniform displacements in [-disp, disp]
    per component and each box axis scaled by 1 + U(-strain, strain)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = np.ones(3)
    if strain > 0:
        scale = 1.0 + rng.uniform(-strain, strain, size=3)
    g = np.arange(ncell, dtype=np.float64)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    corner = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    # interleave so atom 2c is the corner of cell c and 2c+1 its body centre
    frac = np.stack([corner, corner + 0.5], axis=1).reshape(-1, 3)
    pos = frac * a * scale[None, :]
    if disp > 0:
        pos = pos + rng.uniform(-disp, disp, size=pos.shape)
    box = ncell * a * scale
    return Config(pos=np.ascontiguousarray(pos), box=np.ascontiguousarray(box),
                  name=f"bcc{ncell}")


def beta(twojmax: int, scale: float | None = None, seed: int = SEED_BETA) -> np.ndarray:
    """beta_0 followed by the ncoeff linear coefficients, U(-scale, scale).
    Default scale: 1 for 2J <= 8 and 0.1 above (the high-order workload)."""
    if scale is None:
        scale = 1.0 if twojmax <= 8 else 0.1
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=ncoeff(twojmax) + 1)


BATCH_SIZES = (3, 4, 5, 6, 7, 8, 10)   # cells per edge -> 54 ... 2000 atoms


def batch(nconf: int = 64, disp: float = 0.1, strain: float = 0.02,
          seed: int = SEED_BATCH) -> list[Config]:
    """Independent configurations with atom counts drawn uniformly from
    {54, 128, 250, 432, 686, 1024, 2000}, each with its own strain and
    displacements (seed + c for configuration c)."""
    pick = np.random.Generator(np.random.PCG64(seed))
    cells = pick.choice(np.array(BATCH_SIZES), size=nconf)
    out = []
    for c, nc in enumerate(cells):
        cfg = bcc(int(nc), disp=disp, strain=strain, seed=seed + c)
        cfg.name = f"batch{c}_bcc{nc}"
        out.append(cfg)
    return out


FIT_SIZES = (4, 5, 6, 7, 8)   # 128 ... 1024 atoms


def fitting_set(nconf: int = 32, disp: float = 0.2, seed: int = SEED_BATCH + 1000) -> list[Config]:
    """Configurations of 128-1024 atoms with larger displacements (+-0.2 A)."""
    pick = np.random.Generator(np.random.PCG64(seed))
    cells = pick.choice(np.array(FIT_SIZES), size=nconf)
    return [bcc(int(nc), disp=disp, seed=seed + c) for c, nc in enumerate(cells)]


@dataclass
class Workload:
    """A named benchmark/parity workload."""
    name: str
    ncell: int
    twojmax: int
    disp: float = 0.1
    beta_scale: float | None = None
    extra: dict = field(default_factory=dict)

    def config(self) -> Config:
        return bcc(self.ncell, disp=self.disp)

    def beta(self) -> np.ndarray:
        return beta(self.twojmax, self.beta_scale)


WORKLOADS = {
    # parity: 128 atoms, 2J = 8, beta in [-1, 1]
    "bcc4_2j8": Workload("bcc4_2j8", 4, 8),
    # paper-shaped benchmark: 2000 atoms, 2J = 8
    "bcc10_2j8": Workload("bcc10_2j8", 10, 8),
    # high order: 2000 and 16000 atoms, 2J = 14, beta in [-0.1, 0.1]
    "bcc10_2j14": Workload("bcc10_2j14", 10, 14),
    "bcc20_2j14": Workload("bcc20_2j14", 20, 14),
}
