"""Seeded synthetic inputs for the Chebyshev-filtered plane-wave H-apply.

This module only draws random numbers and lays out the inputs of a problem
(cell, atoms, local-potential grid, projector coupling matrices, starting
blocks).  It holds none of the method's arithmetic: the plane-wave sphere, the
projector matrix, the Hamiltonian application, the filter and Rayleigh-Ritz
are computed independently by the CUDA library and by the oracle.  Both of
them take their inputs from here.

The paper's workloads (a 255-atom Ti interface, 320-atom Ga2O3, with PAW
datasets; Sec. 5.1) are not available; these seeded cells stand in for their
shapes: Kohn-Sham problem H psi = lambda S psi of Sec. 3.1 with N plane waves,
M bands and N_projs projectors (Sec. 3.4).

Recipe (all from one ``numpy.random.default_rng(seed)`` stream per problem):
  * atoms uniform in the cell, pairs closer than 1.5 bohr rejected;
  * V_loc(r) = -depth * sum_atoms sum_{27 images} exp(-|r-R-L|^2 / (2 w^2))
    on the FFT grid (depth 2 Ha, w 1 bohr).  For orthorhombic cells the
    27-image sum factorises per axis, which is how it is evaluated here;
  * D: per-atom symmetric blocks, entries uniform [-0.5, 0.5] Ha (or one
    dense symmetric block over all projectors for the tiny problem);
  * Q: per-atom blocks U diag(u) U^T, U from the QR of a Gaussian matrix,
    u uniform [0.05, 0.3], so that S = I + P Q P^dagger is SPD;
  * starting block Psi_0: complex normal, Re and Im ~ N(0, 1/2);
  * Lanczos start vector: complex normal;
  * k-point grids: Monkhorst-Pack-like offsets, plus a seeded per-k cut-off
    jitter for the ragged batched form.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """Inputs of one k-point problem (everything the C-ABI descriptor takes)."""
    name: str
    lattice: np.ndarray          # 3x3, rows a1, a2, a3 (bohr)
    kpt: np.ndarray              # reduced coordinates (3,)
    ecut: float                  # Ha
    box: tuple                   # (n1, n2, n3)
    tau: np.ndarray              # natom x 3 cartesian (bohr)
    sigmas: np.ndarray           # Gaussian widths of the s+p projector channels
    vloc: np.ndarray             # n1 x n2 x n3 real, C order (z fastest)
    D: np.ndarray                # nproj x nproj real symmetric
    Q: Optional[np.ndarray]      # nproj x nproj real symmetric or None (S = I)
    nband: int
    degree: int
    cycles: int
    lanczos_steps: int
    seed: int

    @property
    def natom(self) -> int:
        return int(self.tau.shape[0])

    @property
    def nproj(self) -> int:
        return int(self.tau.shape[0] * 4 * len(self.sigmas))


def _atoms(rng, lattice, natom, min_dist=1.5):
    lat = np.asarray(lattice, dtype=np.float64)
    pos: List[np.ndarray] = []
    tries = 0
    while len(pos) < natom:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place atoms")
        frac = rng.random(3)
        r = frac @ lat
        ok = True
        for q in pos:
            d = r - q
            # minimum image for orthorhombic cells
            f = np.linalg.solve(lat.T, d)
            f -= np.round(f)
            if np.linalg.norm(f @ lat) < min_dist:
                ok = False
                break
        if ok:
            pos.append(r)
    return np.array(pos)


def gaussian_vloc(lattice, box, tau, depth=2.0, width=1.0):
    """V(r) on the n1 x n2 x n3 grid of an orthorhombic cell (C order).

    The 27-image sum is a product of three 1-D three-image sums because the
    cell is orthorhombic, so it is evaluated exactly as outer products."""
    lat = np.asarray(lattice, dtype=np.float64)
    if np.abs(lat - np.diag(np.diag(lat))).max() > 0:
        raise ValueError("synthetic V_loc assumes an orthorhombic cell")
    L = np.diag(lat)
    n = box
    V = np.zeros(n, dtype=np.float64)
    axes = [np.arange(n[i]) * (L[i] / n[i]) for i in range(3)]
    for R in tau:
        f = []
        for i in range(3):
            x = axes[i]
            s = np.zeros_like(x)
            for img in (-1, 0, 1):
                d = x - R[i] - img * L[i]
                s += np.exp(-d * d / (2.0 * width * width))
            f.append(s)
        V -= depth * np.einsum("i,j,k->ijk", f[0], f[1], f[2])
    return V


def _block_sym(rng, nproj, block, lo=-0.5, hi=0.5):
    D = np.zeros((nproj, nproj))
    for s in range(0, nproj, max(block, 1)):
        B = rng.uniform(lo, hi, size=(block, block))
        D[s:s + block, s:s + block] = 0.5 * (B + B.T)
    return D


def _block_q(rng, nproj, block, umin=0.05, umax=0.3):
    Q = np.zeros((nproj, nproj))
    for s in range(0, nproj, max(block, 1)):
        U, _ = np.linalg.qr(rng.standard_normal((block, block)))
        u = rng.uniform(umin, umax, size=block)
        Q[s:s + block, s:s + block] = (U * u) @ U.T
    return Q


CONFIG_NAMES = ("tiny_gamma_fp64", "fp64_at_scale", "paw_precision",
                "batched_kpoints", "differentiation")
SEEDS = {"tiny_gamma_fp64": 1001, "fp64_at_scale": 1002, "paw_precision": 1003,
         "batched_kpoints": 1004, "differentiation": 1005}


def make_problem(name: str, *, box=None, natom=None, ecut=None, nband=None,
                 seed=None, with_q=None, kpt=None) -> Problem:
    """Seeded problem for one of the five named workloads.

    Keyword overrides shrink a workload for tests (smaller box/cut-off/bands),
    keeping its structure."""
    if name == "tiny_gamma_fp64":
        a, b0, ec, na, sig, M, m, cyc, q = 10.0, (24, 24, 24), 7.6, 2, (1.0,), 16, 8, 5, False
        lat = np.diag([a, a, a])
    elif name == "fp64_at_scale":
        a, b0, ec, na, sig, M, m, cyc, q = 24.0, (96, 96, 96), 19.1, 64, (0.7, 1.1), 256, 10, 1, False
        lat = np.diag([a, a, a])
    elif name == "paw_precision":
        a, b0, ec, na, sig, M, m, cyc, q = 30.0, (120, 120, 120), 18.2, 108, (0.7, 1.1), 512, 12, 1, True
        lat = np.diag([a, a, a])
    elif name == "batched_kpoints":
        b0, ec, na, sig, M, m, cyc, q = (72, 72, 90), 19.5, 32, (0.7, 1.1), 128, 10, 1, False
        lat = np.diag([16.0, 16.0, 20.0])
    elif name == "differentiation":
        a, b0, ec, na, sig, M, m, cyc, q = 14.0, (64, 64, 64), 20.3, 16, (0.7, 1.1), 128, 10, 3, False
        lat = np.diag([a, a, a])
    else:
        raise KeyError(name)
    seed = SEEDS[name] if seed is None else seed
    rng = np.random.default_rng(seed)
    box = tuple(box) if box is not None else b0
    na = natom if natom is not None else na
    ec = ecut if ecut is not None else ec
    M = nband if nband is not None else M
    q = with_q if with_q is not None else q
    tau = _atoms(rng, lat, na)
    vloc = gaussian_vloc(lat, box, tau)
    nproj = na * 4 * len(sig)
    if name == "tiny_gamma_fp64":
        D = _block_sym(rng, nproj, nproj)       # one dense symmetric block
    else:
        D = _block_sym(rng, nproj, 4 * len(sig))
    Q = _block_q(rng, nproj, 4 * len(sig)) if q else None
    return Problem(name=name, lattice=lat, kpt=np.zeros(3) if kpt is None else np.asarray(kpt, float),
                   ecut=float(ec), box=box, tau=tau, sigmas=np.array(sig, dtype=np.float64),
                   vloc=vloc, D=D, Q=Q, nband=M, degree=m, cycles=cyc, lanczos_steps=10, seed=seed)


def psi0(seed: int, npw: int, nband: int, dtype=np.complex128) -> np.ndarray:
    """Starting block, column-major N x M as an (M, N) C-order array (band rows)."""
    rng = np.random.default_rng(seed + 7919)
    x = (rng.standard_normal((nband, npw)) + 1j * rng.standard_normal((nband, npw))) * math.sqrt(0.5)
    return x.astype(dtype)


def lanczos_v0(seed: int, npw: int) -> np.ndarray:
    rng = np.random.default_rng(seed + 104729)
    return (rng.standard_normal(npw) + 1j * rng.standard_normal(npw)) * math.sqrt(0.5)


def random_block(seed: int, npw: int, nband: int, dtype=np.complex128) -> np.ndarray:
    """Generic complex-normal test block (band rows), for parity tests."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((nband, npw)) + 1j * rng.standard_normal((nband, npw))) * math.sqrt(0.5)
    return x.astype(dtype)


def mp_kpoints(grid=(4, 4, 2)) -> np.ndarray:
    """Monkhorst-Pack-like reduced k-points ((2i - n - 1) / (2 n) per axis)."""
    ks = []
    for i in range(grid[0]):
        for j in range(grid[1]):
            for l in range(grid[2]):
                ks.append([(2 * i - grid[0] + 1) / (2 * grid[0]),
                           (2 * j - grid[1] + 1) / (2 * grid[1]),
                           (2 * l - grid[2] + 1) / (2 * grid[2])])
    return np.array(ks)


def ecut_jitter(seed: int, nk: int, base: float, lo=0.86, hi=1.10) -> np.ndarray:
    """Per-k cut-off factors that spread the sphere sizes (ragged batches)."""
    rng = np.random.default_rng(seed + 31337)
    return base * rng.uniform(lo, hi, size=nk)


def smooth_field(seed: int, lattice, box, ncenters=6, width=2.0) -> np.ndarray:
    """Seeded smooth Gaussian-sum field in [0, 1]-ish on the grid (target density shape)."""
    rng = np.random.default_rng(seed + 2718)
    lat = np.asarray(lattice, float)
    centers = rng.random((ncenters, 3)) @ lat
    f = -gaussian_vloc(lat, box, centers, depth=1.0, width=width)
    return f / max(1e-300, f.max())
