"""Pins of the oracle's self-consistent field loop (oracle/pw_scf.py, Alg. 3 closed with a
Hartree + Dirac-exchange model), against what physics and mathematics fix:

  * the Hartree potential of a periodic Gaussian charge equals its closed-form Fourier sum;
  * the exchange potential is the derivative of the exchange energy (central differences),
    and the exchange energy per electron of the uniform gas at r_s = 1 is -0.458165 Ha;
  * a free-electron cell with closed shells keeps a uniform density, so its self-consistent
    eigenvalues are the free-electron ones shifted by v_x(N/Omega) exactly and the total
    energy is the kinetic sum plus the exchange energy of the uniform gas;
  * the converged loop is self-consistent (V_out = V_in) and reproduces the electron count.
"""
import math

import numpy as np
import pytest

from oracle import pw_oracle as O
from oracle import pw_scf as F
from paper_2604_11139_gb300 import workloads as W


def cell(natom=2, ecut=3.0, box=(16, 16, 16), nband=8):
    return W.make_problem("tiny_gamma_fp64", box=box, ecut=ecut, natom=natom, nband=nband)


def test_hartree_of_a_gaussian_charge_matches_its_fourier_sum():
    p = cell()
    lat, box = p.lattice, p.box
    omega = abs(np.linalg.det(lat))
    R = np.array([3.1, 4.7, 5.3])
    s, Z = 1.3, 2.0
    # periodic normalised Gaussian on the grid (27 images; tails beyond are < 1e-30)
    axes = [np.arange(box[i]) * lat[i, i] / box[i] for i in range(3)]
    f = []
    for i in range(3):
        d = axes[i][:, None] - R[i] - lat[i, i] * np.array([-1, 0, 1])[None, :]
        f.append(np.exp(-d * d / (2 * s * s)).sum(axis=1))
    rho = Z * np.einsum("i,j,k->ijk", *f) / (2 * math.pi * s * s) ** 1.5
    vh = F.hartree_potential(rho, lat, p.ecut)
    # closed form: V_H(r) = sum_{G != 0, G in the density sphere} (4 pi / G^2) (Z / Omega)
    #              exp(-G^2 s^2 / 2) cos(G.(r - R))
    m, g2 = F.density_sphere(lat, p.ecut, box)
    B = O.reciprocal(lat)
    G = m @ B
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    nz = g2 > 0
    amp = 4 * math.pi / g2[nz] * (Z / omega) * np.exp(-g2[nz] * s * s / 2)
    ref = (np.cos((grid - R) @ G[nz].T) * amp[None, :]).sum(axis=1).reshape(box)
    # the grid Gaussian's own components beyond the density sphere are below 1e-9 of its peak
    np.testing.assert_allclose(vh, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_exchange_potential_is_the_derivative_of_the_energy():
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.01, 0.5, size=32)
    h = 1e-6 * rho
    d = (F.exchange_energy_density(rho + h) - F.exchange_energy_density(rho - h)) / (2 * h)
    np.testing.assert_allclose(F.exchange_potential(rho), d, rtol=1e-8)
    rs = 1.0
    rho0 = 3.0 / (4 * math.pi * rs ** 3)
    assert abs(F.exchange_energy_density(np.array([rho0]))[0] / rho0 - (-0.458165293)) < 1e-8


def test_free_electron_closed_shells_stay_uniform():
    # no atoms: V_ion = 0, no projectors; 7 states (|G|^2 <= (2pi/a)^2) doubly occupied
    p = cell(natom=0, nband=8)
    p.vloc[...] = 0.0
    p.D = np.zeros((0, 0))
    omega = abs(np.linalg.det(p.lattice))
    out = F.scf(p, nocc=7, beta=0.5, tol=1e-11, max_iter=50, v_start=np.zeros(p.box))
    assert out["converged"]
    rho0 = 14.0 / omega
    np.testing.assert_allclose(out["rho"], rho0, rtol=1e-10)
    unit = 0.5 * (2 * math.pi / p.lattice[0, 0]) ** 2
    vx = F.exchange_potential(np.array([rho0]))[0]
    np.testing.assert_allclose(out["eig"][:7], vx + unit * np.array([0, 1, 1, 1, 1, 1, 1]), atol=1e-10)
    e_ref = 2 * 6 * unit + omega * F.exchange_energy_density(np.array([rho0]))[0]
    assert abs(out["energies"]["total"] - e_ref) < 1e-9


def test_scf_loop_converges_to_a_self_consistent_density():
    p = cell(natom=2, nband=8)
    omega = abs(np.linalg.det(p.lattice))
    out = F.scf(p, nocc=4, beta=0.3, tol=1e-10, max_iter=200)
    assert out["converged"]
    assert abs((omega / out["rho"].size) * out["rho"].sum() - 8.0) < 1e-10
    # V_in = V_ion + V_H[rho] + v_x[rho] at convergence
    vh = F.hartree_potential(out["rho"], p.lattice, p.ecut)
    v_out = p.vloc + vh + F.exchange_potential(out["rho"])
    assert np.abs(v_out - out["v"]).max() < 1e-9
    dv = np.array([h[1] for h in out["history"]])
    assert dv[-1] < 1e-10 and np.all(dv[5:] < dv[:-5])   # geometric decrease of the residual
