"""Planted mistakes in the FP64 oracle, each caught by one of its pins.

Every case replaces one piece of the oracle (on the CPU, through monkeypatch) by a
plausible wrong version -- a dropped term, a wrong sign, a missing conjugate, a wrong
coefficient -- and runs the pin that must fail.  A pin that still passed would mean the
oracle could carry that mistake unnoticed.
"""
import numpy as np
import pytest
import scipy.linalg

import tests.test_oracle_lobpcg as lpins
import tests.test_oracle_pins as pins
import tests.test_oracle_slicing as spins
from oracle import pw_lobpcg as L
from oracle import pw_oracle as O
from oracle import pw_slicing as SL


def _apply_h_without_kinetic(self, C):
    C = np.atleast_2d(C)
    return O.apply_local(self.vloc, self.miller, C) + (self.project(C) @ self.D.T) @ self.P.T


def _project_without_conjugate(self, C):
    return C @ self.P


def _sinv_wrong_sign(self, C):
    C = np.atleast_2d(C)
    if self.Q is None:
        return C.copy()
    return C + (self.project(C) @ self.woodbury_k().T) @ self.P.T


def _filter_first_coefficient_everywhere(apply_a, Y0, degree, a, b):
    c, e = 0.5 * (b + a), 0.5 * (b - a)
    Yprev, Y = Y0, (apply_a(Y0) - c * Y0) / e
    for _ in range(1, degree):
        Yprev, Y = Y, (1.0 / e) * (apply_a(Y) - c * Y) - Yprev
    return Y


def _rr_back_transform_without_conjugate(Y, HY, SY):
    Hs = Y.conj() @ HY.T
    Ss = Y.conj() @ SY.T
    Hs = 0.5 * (Hs + Hs.conj().T)
    Ss = 0.5 * (Ss + Ss.conj().T)
    L = np.linalg.cholesky(Ss)
    Li = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    lam, U = np.linalg.eigh(0.5 * ((Li @ Hs @ Li.conj().T) + (Li @ Hs @ Li.conj().T).conj().T))
    X = Li.T @ U
    return lam, X.T @ Y, X.T @ HY, X.T @ SY, X


def _rq_over_plain_norm(C, HC, SC):
    num = np.real(np.einsum("ij,ij->i", C.conj(), HC))
    return num / np.real(np.einsum("ij,ij->i", C.conj(), C))


def _rq_without_conjugate(C, HC, SC):
    num = np.real(np.einsum("ij,ij->i", C, HC))
    den = np.real(np.einsum("ij,ij->i", C.conj(), SC))
    return num / den


_RES_PSI = [None]


def _rr_recording_psi(rr):
    def wrapped(Y, HY, SY):
        out = rr(Y, HY, SY)
        _RES_PSI[0] = out[1]
        return out
    return wrapped


def _residual_with_psi_for_s_psi(lam, HY, SY):
    # the S-less residual || H psi - lambda psi ||: psi (recorded from the last
    # Rayleigh-Ritz call) in place of S psi
    return np.linalg.norm(HY - lam[:, None] * _RES_PSI[0], axis=1)


def _residual_zeros(lam, HY, SY):
    return np.zeros(HY.shape[0])


def _plant(monkeypatch, what):
    if what == "kinetic term dropped from H psi":
        monkeypatch.setattr(O.Hamiltonian, "apply_h", _apply_h_without_kinetic)
    elif what == "forward DFT with the inverse sign":
        fwd = O.forward_dft_direct
        monkeypatch.setattr(O, "forward_dft_direct", lambda F: np.conj(fwd(np.conj(F))))
    elif what == "projection without the conjugate":
        monkeypatch.setattr(O.Hamiltonian, "project", _project_without_conjugate)
    elif what == "Woodbury correction with the wrong sign":
        monkeypatch.setattr(O.Hamiltonian, "apply_sinv", _sinv_wrong_sign)
    elif what == "recurrence coefficient 1/e instead of 2/e":
        monkeypatch.setattr(O, "chebyshev_filter", _filter_first_coefficient_everywhere)
    elif what == "Rayleigh-Ritz back-transform not conjugated":
        monkeypatch.setattr(O, "rayleigh_ritz", _rr_back_transform_without_conjugate)
    elif what == "potential Fourier component at G' - G":
        vt = O.vtilde
        monkeypatch.setattr(O, "vtilde", lambda v, g: vt(v, -np.asarray(g)))
    elif what == "Rayleigh quotient over |psi|^2 instead of psi^dagger S psi":
        monkeypatch.setattr(O, "rayleigh_quotients", _rq_over_plain_norm)
    elif what == "Rayleigh quotient numerator without the conjugate":
        monkeypatch.setattr(O, "rayleigh_quotients", _rq_without_conjugate)
    elif what == "residual returning zeros":
        monkeypatch.setattr(O, "residual_norms", _residual_zeros)
    elif what == "residual with psi in place of S psi":
        monkeypatch.setattr(O, "rayleigh_ritz", _rr_recording_psi(O.rayleigh_ritz))
        monkeypatch.setattr(O, "residual_norms", _residual_with_psi_for_s_psi)
    elif what == "S-Deflate with psi0 in place of S psi0":
        sd = L.s_deflate
        monkeypatch.setattr(L, "s_deflate", lambda X, Y0, SY0: sd(X, Y0, Y0))
    elif what == "LOBPCG residual with the wrong sign":
        monkeypatch.setattr(L, "residuals", lambda lam, HX, SX: HX + lam[:, None] * SX)
    elif what == "preconditioner inverted":
        tpa = L.tpa_preconditioner
        monkeypatch.setattr(L, "tpa_preconditioner", lambda kin, e: 1.0 / tpa(kin, e))
    elif what == "S-Ortho applied to psi only":
        so = L.s_ortho3
        monkeypatch.setattr(L, "s_ortho3", lambda X, HX, SX: (so(X, HX, SX)[0], HX, SX))
    elif what == "window coefficients without the factor 2":
        ic = SL.indicator_coefficients

        def half(degree, ta, tb):
            mu = ic(degree, ta, tb)
            mu[1:] *= 0.5
            return mu
        monkeypatch.setattr(SL, "indicator_coefficients", half)
    elif what == "Jackson damping left out":
        monkeypatch.setattr(SL, "jackson_damping", lambda degree: np.ones(degree + 1))
    elif what == "first Chebyshev step with 2/e":
        def sum2(apply_a, X, coef, lo, hi):
            c, e = 0.5 * (hi + lo), 0.5 * (hi - lo)
            T0, T1 = X, 2.0 * (apply_a(X) - c * X) / e
            acc = coef[0] * T0 + coef[1] * T1
            for j in range(2, len(coef)):
                T0, T1 = T1, 2.0 * (apply_a(T1) - c * T1) / e - T0
                acc = acc + coef[j] * T1
            return acc
        monkeypatch.setattr(SL, "chebyshev_sum", sum2)
    else:  # pragma: no cover
        raise KeyError(what)


CASES = [
    ("kinetic term dropped from H psi", lambda: pins.test_dense_equals_matrix_free(False)),
    ("forward DFT with the inverse sign", pins.test_local_matches_numpy_fft),
    ("projection without the conjugate", lambda: pins.test_hermiticity(False)),
    ("Woodbury correction with the wrong sign", pins.test_woodbury_inverse),
    ("recurrence coefficient 1/e instead of 2/e", lambda: pins.test_chebyshev_scaling_of_eigenvectors(False)),
    ("Rayleigh-Ritz back-transform not conjugated", pins.test_rayleigh_ritz_matches_generalized_eigh),
    ("potential Fourier component at G' - G", lambda: pins.test_dense_equals_matrix_free(False)),
    ("Rayleigh quotient over |psi|^2 instead of psi^dagger S psi",
     lambda: pins.test_rayleigh_quotients_of_exact_and_mixed_vectors(True)),
    ("Rayleigh quotient numerator without the conjugate",
     lambda: pins.test_rayleigh_quotients_of_exact_and_mixed_vectors(False)),
    ("residual returning zeros", lambda: pins.test_residual_norms_of_exact_and_perturbed_pairs(False)),
    ("residual with psi in place of S psi", lambda: pins.test_chebfi_residuals_match_dense_pencil(True)),
    ("S-Deflate with psi0 in place of S psi0", lambda: lpins.test_s_deflate_is_the_s_orthogonal_projection(True)),
    ("LOBPCG residual with the wrong sign",
     lambda: lpins.test_lobpcg_converges_to_the_dense_eigenpairs(True, 4, 2, 1e-12)),
    ("preconditioner inverted", lpins.test_tpa_preconditioner_values),
    ("S-Ortho applied to psi only", lambda: lpins.test_s_ortho_is_s_orthonormal_with_the_same_span(False)),
    ("window coefficients without the factor 2", lambda: spins.test_indicator_coefficients_match_quadrature(-0.3, 0.45)),
    ("Jackson damping left out", lambda: spins.test_damped_window_is_bounded_and_approaches_the_indicator(40)),
    ("first Chebyshev step with 2/e", spins.test_recurrence_sum_on_exact_eigenvectors),
]


@pytest.mark.parametrize("what,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pin(monkeypatch, what, pin):
    pin()                         # the pin passes on the oracle as it stands
    _plant(monkeypatch, what)
    with pytest.raises(AssertionError):
        pin()
