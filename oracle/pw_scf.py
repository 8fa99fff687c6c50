"""Plain FP64 CPU oracle of the self-consistent field loop around the filter (Alg. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module; the CUDA library never
calls it and shares no code with it.

The paper's Alg. 3 repeats: solve H Psi = Lambda S Psi at the current Hamiltonian, compute
occupations from Lambda, accumulate the electronic density from the occupations and Psi,
stop once self-consistent.  It does not say how the density fixes the next Hamiltonian (the
paper's production code uses PAW datasets and XC functionals it does not list).  This oracle
closes the loop with the smallest published model that makes the density feed back:

  * occupations: the lowest ``nocc`` states hold 2 electrons each (insulating filling);
  * density rho(r_j) = (1/Omega) sum_i f_i |psi_i(r_j)|^2, psi_i(r) = sum_G c_iG e^{iG.r}
    with unit-norm coefficients, so (Omega/n) sum_j rho(r_j) = N_electrons;
  * Hartree potential from Poisson's equation in reciprocal space,
    V_H(G) = 4 pi rho(G) / |G|^2 for G != 0 and 0 at G = 0 (neutralising background),
    rho(G) = (1/n) sum_j rho(r_j) e^{-iG.r_j}, G over the density sphere |G|^2/2 <= 4 E_cut
    (every component a product of two orbitals of the E_cut sphere can have);
  * exchange in the local-density approximation of Dirac (1930) for the spin-unpolarised
    gas, e_x(rho) = -(3/4) (3/pi)^{1/3} rho^{1/3} per electron, v_x = d(rho e_x)/d rho =
    -(3 rho / pi)^{1/3}; correlation is left out;
  * V_in of the next iteration by linear mixing of the potential,
    V_{k+1} = V_k + beta (V_ion + V_H[rho_k] + v_x[rho_k] - V_k);
  * energy of the Kohn-Sham functional at the input potential,
    E = sum_i f_i lambda_i - (Omega/n) sum_j (V_in - V_ion)(r_j) rho(r_j) + E_H + E_x,
    E_H = (Omega / 2n) sum_j V_H(r_j) rho(r_j), E_x = (Omega/n) sum_j rho e_x(rho).

The eigenproblem of each iteration is solved by dense diagonalisation of the oracle's
Hamiltonian (small problems only).  Pins: tests/test_oracle_scf.py.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import scipy.linalg

from . import pw_oracle as O

CX = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0)     # e_x = CX rho^(1/3)


def exchange_energy_density(rho: np.ndarray) -> np.ndarray:
    """rho * e_x(rho) (Dirac exchange, spin-unpolarised), Ha / bohr^3."""
    r = np.maximum(rho, 0.0)
    return CX * r ** (4.0 / 3.0)


def exchange_potential(rho: np.ndarray) -> np.ndarray:
    """v_x = d(rho e_x)/d rho = -(3 rho / pi)^(1/3)."""
    r = np.maximum(rho, 0.0)
    return -(3.0 * r / math.pi) ** (1.0 / 3.0)


def density_sphere(lattice, ecut, box):
    """Miller indices of the density sphere |G|^2/2 <= 4 ecut (Gamma) and |G|^2."""
    m, kin = O.g_sphere(lattice, [0.0, 0.0, 0.0], 4.0 * ecut, box)
    return m, 2.0 * kin


def hartree_potential(rho: np.ndarray, lattice, ecut) -> np.ndarray:
    """V_H on the grid from rho on the grid, through the components of the density sphere."""
    box = rho.shape
    m, g2 = density_sphere(lattice, ecut, box)
    rho_g = O.from_box(O.forward_dft_direct(rho[None].astype(complex)), m, box)[0]
    vg = np.zeros_like(rho_g)
    nz = g2 > 0
    vg[nz] = 4.0 * math.pi * rho_g[nz] / g2[nz]
    return np.real(O.inverse_dft_direct(vg[None], m, box)[0])


def density(C: np.ndarray, occ: np.ndarray, miller, box, omega) -> np.ndarray:
    """rho(r_j) = (1/Omega) sum_i f_i |psi_i(r_j)|^2."""
    return O.density_grad(C, None, np.asarray(occ, float) / omega, miller, box)


def energies(lam, occ, rho, v_in, v_ion, v_h, omega):
    n = rho.size
    w = omega / n
    eb = float(np.dot(occ, lam))
    dc = w * float(np.sum((v_in - v_ion) * rho))
    eh = 0.5 * w * float(np.sum(v_h * rho))
    ex = w * float(np.sum(exchange_energy_density(rho)))
    return {"band": eb, "double_counting": dc, "hartree": eh, "exchange": ex, "total": eb - dc + eh + ex}


def scf(prob, nocc: int, beta: float = 0.3, tol: float = 1e-9, max_iter: int = 200,
        v_start: Optional[np.ndarray] = None):
    """The loop of the module docstring with dense diagonalisation.  Returns a dict with the
    converged eigenvalues, potential, density, energies and the per-iteration history of
    (total energy, max |V_out - V_in|)."""
    omega = abs(float(np.linalg.det(prob.lattice)))
    v_ion = np.asarray(prob.vloc, float)
    v_in = v_ion.copy() if v_start is None else np.asarray(v_start, float).copy()
    occ = np.zeros(prob.nband)
    occ[:nocc] = 2.0
    hist = []
    for it in range(max_iter):
        ham = O.Hamiltonian(prob.lattice, prob.kpt, prob.ecut, prob.box, v_in, prob.tau, prob.sigmas, prob.D,
                            prob.Q)
        H, S = ham.dense()
        lam, X = scipy.linalg.eigh(H, S)
        lam = lam[:prob.nband]
        C = X[:, :prob.nband].T                    # band rows, unit S-norm
        # unit 2-norm coefficients for the density (S = I here: the same thing)
        C = C / np.linalg.norm(C, axis=1, keepdims=True)
        rho = density(C, occ, ham.miller, prob.box, omega)
        v_h = hartree_potential(rho, prob.lattice, prob.ecut)
        v_out = v_ion + v_h + exchange_potential(rho)
        e = energies(lam, occ, rho, v_in, v_ion, v_h, omega)
        dv = float(np.abs(v_out - v_in).max())
        hist.append((e["total"], dv))
        if dv < tol:
            return dict(eig=lam, v=v_in, rho=rho, energies=e, history=hist, iterations=it + 1, converged=True)
        v_in = v_in + beta * (v_out - v_in)
    return dict(eig=lam, v=v_in, rho=rho, energies=e, history=hist, iterations=max_iter, converged=False)
