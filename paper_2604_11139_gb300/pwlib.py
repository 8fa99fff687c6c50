"""Thin ctypes binding of libpwcheb (include/pw.h).

Argument marshalling only: every step runs in the CUDA library.  Wave-function
blocks are torch CUDA tensors of shape (M, ld), complex128 (PW_FP64) or
complex64 (PW_MIXED), C-contiguous rows, i.e. the column-major N x M block of
the C ABI with band j at row j.  Importing this module never falls back to any
other implementation: if the library cannot be built or loaded, it raises.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional

import numpy as np

from . import build as _build

PW_FP64 = 0
PW_MIXED = 1

STATUS = {0: "PW_OK", -1: "PW_EINVAL", -2: "PW_ENOMEM", -3: "PW_ECUDA", -4: "PW_ENOTSPD",
          -5: "PW_ETIMEDOUT", -6: "PW_ENOTCONV", -7: "PW_EUNSUPPORTED"}

# every function declared in include/pw.h
EXPORTS = ("pw_ctx_create", "pw_ctx_destroy", "pw_ctx_set_stream", "pw_ctx_info", "pw_ctx_gvectors",
           "pw_ctx_projectors", "pw_hamiltonian_apply", "pw_spectrum_bounds", "pw_chebyshev_filter",
           "pw_rayleigh_ritz", "pw_chebfi_solve", "pw_density_grad", "pw_profile_enable", "pw_profile_read",
           "pw_kernel_launches", "pw_hamiltonian_apply_noalloc", "pw_autotune", "pw_batch_create",
           "pw_batch_destroy", "pw_batch_filter", "pw_batch_chebfi_solve", "pw_ctx_set_vloc", "pw_ctx_set_D",
           "pw_local_apply", "pw_diff_create", "pw_diff_destroy", "pw_diff_tape_bytes", "pw_diff_forward",
           "pw_diff_backward", "pw_fft_config", "pw_tc_config", "pw_fp64_config", "pw_ctx_sync",
           "pw_ctx_test_wait_expiry", "pw_diag_fp64_fma_rate", "pw_scf_potential", "pw_scf_run", "pw_slice_filter", "pw_spectrum_slice",
           "pw_lobpcg_solve", "pw_gamma_symmetrize",
           "pw_gamma_pack", "pw_gamma_unpack", "pw_strerror", "pw_last_error")

PROF_CLASSES = ("plane_inv", "xline", "plane_fwd", "gemm_proj", "gemm_back", "small", "rr")


class PWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("kpt", ctypes.c_double * 3), ("ecut", ctypes.c_double),
                ("box", ctypes.c_int * 3), ("vloc", ctypes.POINTER(ctypes.c_double)), ("natom", ctypes.c_int),
                ("tau", ctypes.POINTER(ctypes.c_double)), ("nchan", ctypes.c_int),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("D", ctypes.POINTER(ctypes.c_double)),
                ("Q", ctypes.POINTER(ctypes.c_double)), ("nproj", ctypes.c_int), ("proj", ctypes.c_void_p)]


_LIB = None


def load(path: Optional[str] = None):
    """Loads (building first if needed) the in-tree library; raises if impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = _build.lib_path()
        if not os.path.exists(path) or os.environ.get("PW_REBUILD"):
            path = _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    lib.pw_ctx_create.argtypes = [ctypes.POINTER(_Desc), vp, ctypes.POINTER(vp)]
    lib.pw_ctx_destroy.argtypes = [vp]
    lib.pw_ctx_set_stream.argtypes = [vp, vp]
    lib.pw_ctx_info.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.pw_ctx_gvectors.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), pd]
    lib.pw_ctx_projectors.argtypes = [vp, vp]
    lib.pw_hamiltonian_apply.argtypes = [vp, vp, i64, ci, vp, vp, i64, ci]
    lib.pw_spectrum_bounds.argtypes = [vp, vp, i64, ci, ci, vp, pd, pd, pd]
    lib.pw_chebyshev_filter.argtypes = [vp, vp, i64, ci, ci, cd, cd, ci]
    lib.pw_rayleigh_ritz.argtypes = [vp, vp, i64, ci, vp, pd, pd]
    lib.pw_chebfi_solve.argtypes = [vp, vp, i64, ci, ci, ci, ci, vp, ci, pd, pd, pd]
    lib.pw_density_grad.argtypes = [vp, vp, vp, i64, ci, pd, vp, ci]
    lib.pw_hamiltonian_apply_noalloc.argtypes = [vp, vp, i64, ci, vp, i64]
    lib.pw_autotune.argtypes = [vp, ci, ci, pd]
    lib.pw_fft_config.argtypes = [vp, ci, i64, ci, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ci)]
    lib.pw_tc_config.argtypes = [vp, ci, ctypes.POINTER(ci)]
    lib.pw_fp64_config.argtypes = [vp, ci, ctypes.POINTER(ci)]
    lib.pw_ctx_sync.argtypes = [vp]
    lib.pw_diag_fp64_fma_rate.argtypes = [vp, pd, pd]
    lib.pw_scf_potential.argtypes = [vp, vp, vp, vp, cd, vp, pd]
    lib.pw_slice_filter.argtypes = [vp, vp, i64, ci, ci, ci, cd, cd, pd, ci]
    lib.pw_spectrum_slice.argtypes = [vp, vp, i64, ci, ci, ci, cd, cd, pd, ci, pd, pd]
    lib.pw_lobpcg_solve.argtypes = [vp, vp, i64, ci, ci, ci, cd, pd, pd, ctypes.POINTER(ctypes.c_int)]
    lib.pw_gamma_symmetrize.argtypes = [vp, vp, i64, ci, ci]
    lib.pw_gamma_pack.argtypes = [vp, vp, i64, ci, vp, i64, ci]
    lib.pw_gamma_unpack.argtypes = [vp, vp, i64, ci, vp, i64, ci]
    lib.pw_scf_run.argtypes = [vp, vp, vp, i64, ci, ci, ci, ci, ci, cd, cd, vp, vp, ci, pd, pd, ctypes.POINTER(ci)]
    lib.pw_ctx_test_wait_expiry.argtypes = [vp]
    pvp = ctypes.POINTER(vp)
    pi64 = ctypes.POINTER(ctypes.c_int64)
    lib.pw_batch_create.argtypes = [pvp, ci, vp, pvp]
    lib.pw_batch_destroy.argtypes = [vp]
    lib.pw_batch_filter.argtypes = [vp, pvp, pi64, ci, ci, pd, pd, ci]
    lib.pw_batch_chebfi_solve.argtypes = [vp, pvp, pi64, ci, ci, ci, ci, pvp, ci, pd, pd]
    lib.pw_ctx_set_vloc.argtypes = [vp, vp]
    lib.pw_ctx_set_D.argtypes = [vp, vp]
    lib.pw_local_apply.argtypes = [vp, vp, cd, vp, i64, ci, vp, i64, ci]
    lib.pw_diff_create.argtypes = [vp, ci, ci, ci, ci, ci, pvp]
    lib.pw_diff_destroy.argtypes = [vp]
    lib.pw_diff_tape_bytes.argtypes = [vp, pi64]
    lib.pw_diff_forward.argtypes = [vp, vp, i64, ci, vp, pd, pd, pd]
    lib.pw_diff_backward.argtypes = [vp, pd, vp, i64, ci, vp, vp, ci]
    lib.pw_profile_enable.argtypes = [vp, ci]
    lib.pw_profile_read.argtypes = [vp, pd, ctypes.POINTER(ctypes.c_int64)]
    lib.pw_kernel_launches.restype = ctypes.c_uint64
    lib.pw_kernel_launches.argtypes = []
    lib.pw_strerror.restype = ctypes.c_char_p
    lib.pw_strerror.argtypes = [ci]
    lib.pw_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("pw_strerror", "pw_last_error", "pw_kernel_launches"):
            getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def fp64_fma_rate(stream=None):
    """Measured FP64 FMA rate of the current GPU in TFLOP/s (pw_diag_fp64_fma_rate)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    t, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().pw_diag_fp64_fma_rate(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(t), ctypes.byref(ms)))
    return t.value


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().pw_kernel_launches())


def _check(status: int):
    if status != 0:
        raise PWError(status, load().pw_last_error().decode(errors="replace"))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _block(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.dim() == 1:
        t = t.unsqueeze(0)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name}: expected a (bands, ld) tensor with unit stride along plane waves")
    return t, t.shape[0], t.stride(0) if t.shape[0] > 1 else t.shape[1]


def _dtype(precision):
    import torch
    return torch.complex128 if precision == PW_FP64 else torch.complex64


class Context:
    """One k-point problem (pw_ctx): sphere, FFT plans, projectors, Woodbury matrices."""

    def __init__(self, lattice, kpt, ecut, box, vloc, tau, sigmas, D, Q=None, stream=None, P=None):
        """P (optional): explicit projector matrix, npw x nproj complex128 in the canonical
        plane-wave order (numpy array); None generates the Gaussian s/p projectors from
        tau and sigmas."""
        import torch
        lib = load()
        self._keep = []
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
        d = _Desc()
        d.lattice[:] = list(lat)
        d.kpt[:] = list(np.asarray(kpt, dtype=np.float64).reshape(3))
        d.ecut = float(ecut)
        d.box[:] = [int(b) for b in box]
        vloc = np.ascontiguousarray(np.asarray(vloc, dtype=np.float64))
        if vloc.size != int(np.prod(box)):
            raise ValueError("vloc size does not match the box")
        tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64).reshape(-1, 3))
        sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64).reshape(-1))
        D = np.asfortranarray(np.asarray(D, dtype=np.float64))
        self._keep += [vloc, tau, sig, D]
        d.vloc = _dptr(vloc)
        d.natom = tau.shape[0]
        d.tau = _dptr(tau)
        d.nchan = sig.shape[0]
        d.sigma = _dptr(sig)
        d.D = _dptr(D)
        if P is not None:
            Pa = np.asfortranarray(np.asarray(P, dtype=np.complex128))
            if Pa.ndim != 2 or D.shape != (Pa.shape[1], Pa.shape[1]):
                raise ValueError("P must be npw x nproj with D nproj x nproj")
            self._keep.append(Pa)
            d.nproj = Pa.shape[1]
            d.proj = ctypes.c_void_p(Pa.ctypes.data)
        if Q is not None:
            Qa = np.asfortranarray(np.asarray(Q, dtype=np.float64))
            self._keep.append(Qa)
            d.Q = _dptr(Qa)
        else:
            d.Q = ctypes.POINTER(ctypes.c_double)()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.pw_ctx_create(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        npw, nproj = ctypes.c_int(), ctypes.c_int()
        _check(lib.pw_ctx_info(h, ctypes.byref(npw), ctypes.byref(nproj)))
        self.npw, self.nproj = npw.value, nproj.value
        self.box = tuple(int(b) for b in box)
        self.has_q = Q is not None
        self._dependents = weakref.WeakSet()   # handles that borrow this context

    @classmethod
    def from_problem(cls, prob, kpt=None, ecut=None, stream=None, P=None):
        return cls(prob.lattice, prob.kpt if kpt is None else kpt, prob.ecut if ecut is None else ecut, prob.box,
                   prob.vloc, prob.tau, prob.sigmas, prob.D, prob.Q, stream=stream, P=P)

    def close(self):
        for d in list(getattr(self, "_dependents", ())):
            d.close()
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pw_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _sync_stream(self):
        import torch
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    # -- tuning / diagnostics -------------------------------------------------------
    def autotune(self, nband, precision=PW_MIXED):
        """Picks the FFT band-batch size for `nband` bands; returns the best apply time (ms)."""
        ms = ctypes.c_double(0.0)
        _check(load().pw_autotune(self._h, int(nband), precision, ctypes.byref(ms)))
        return ms.value

    def fft_config(self, precision=PW_MIXED, batch_bytes=None, variant=None):
        """Returns (batch_bytes, variant) of the FFT passes for `precision`, after setting
        the given fields (None leaves a field unchanged)."""
        bb, v = ctypes.c_int64(0), ctypes.c_int(0)
        _check(load().pw_fft_config(self._h, precision, -1 if batch_bytes is None else int(batch_bytes),
                                    -1 if variant is None else int(variant), ctypes.byref(bb), ctypes.byref(v)))
        out_b = bb.value if batch_bytes is None else int(batch_bytes)
        out_v = v.value if variant is None else int(variant)
        return out_b, out_v

    def tc_config(self, pieces=None):
        """bf16 pieces per operand of the mixed projector GEMMs (2 or 3); sets it if given."""
        v = ctypes.c_int(0)
        _check(load().pw_tc_config(self._h, -1 if pieces is None else int(pieces), ctypes.byref(v)))
        return v.value if pieces is None else int(pieces)

    def sync(self):
        """Waits for the context's queued work; raises PWError (PW_ETIMEDOUT) if a bounded
        device wait expired."""
        _check(load().pw_ctx_sync(self._h))

    def test_wait_expiry(self):
        """Arms the failure-detection test hook (the next tensor-core GEMM's first wait expires)."""
        _check(load().pw_ctx_test_wait_expiry(self._h))

    def fp64_config(self, mode=None):
        """FP64 GEMM mode: 1 digit-sliced tensor-core GEMMs, 0 DFMA; sets it if given."""
        v = ctypes.c_int(0)
        _check(load().pw_fp64_config(self._h, -1 if mode is None else int(mode), ctypes.byref(v)))
        return v.value if mode is None else int(mode)

    def profile(self, on=True):
        _check(load().pw_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{class: (milliseconds, launches)} accumulated since the last read."""
        ms = np.zeros(len(PROF_CLASSES))
        n = np.zeros(len(PROF_CLASSES), dtype=np.int64)
        _check(load().pw_profile_read(self._h, _dptr(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return {c: (float(ms[i]), int(n[i])) for i, c in enumerate(PROF_CLASSES)}

    # -- queries --------------------------------------------------------------------
    def gvectors(self):
        miller = np.zeros((self.npw, 3), dtype=np.int32)
        kin = np.zeros(self.npw, dtype=np.float64)
        _check(load().pw_ctx_gvectors(self._h, miller.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(kin)))
        return miller, kin

    def projectors(self):
        import torch
        P = torch.empty((self.nproj, self.npw), dtype=torch.complex128, device="cuda")
        _check(load().pw_ctx_projectors(self._h, ctypes.c_void_p(P.data_ptr())))
        torch.cuda.synchronize()
        return P  # row i = projector column i

    # -- the path -------------------------------------------------------------------
    def hamiltonian_apply(self, psi, hpsi, spsi=None, precision=PW_FP64):
        dt = _dtype(precision)
        psi, m, ld = _block(psi, dt, "psi")
        hpsi, m2, ldo = _block(hpsi, dt, "hpsi")
        sp = None
        if spsi is not None:
            spsi, m3, lds = _block(spsi, dt, "spsi")
            if lds != ldo or m3 < m:
                raise ValueError("spsi must match hpsi's layout")
            sp = ctypes.c_void_p(spsi.data_ptr())
        if m2 < m:
            raise ValueError("hpsi has fewer bands than psi")
        self._sync_stream()
        _check(load().pw_hamiltonian_apply(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m,
                                           ctypes.c_void_p(hpsi.data_ptr()), sp, ldo, precision))

    def hamiltonian_apply_noalloc(self, psi, hpsi):
        """H psi (FP64) using only the library's static scratch: no device allocation."""
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        hpsi, m2, ldo = _block(hpsi, torch.complex128, "hpsi")
        if m2 < m:
            raise ValueError("hpsi has fewer bands than psi")
        self._sync_stream()
        _check(load().pw_hamiltonian_apply_noalloc(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m,
                                                   ctypes.c_void_p(hpsi.data_ptr()), ldo))

    def spectrum_bounds(self, psi=None, lanczos_steps=10, v0=None):
        import torch
        m, ld, p = 0, self.npw, None
        if psi is not None:
            psi, m, ld = _block(psi, torch.complex128, "psi")
            p = ctypes.c_void_p(psi.data_ptr())
        vp = None
        if lanczos_steps > 0:
            v0, _, _ = _block(v0, torch.complex128, "v0")
            vp = ctypes.c_void_p(v0.data_ptr())
        lo, hi, up = ctypes.c_double(np.nan), ctypes.c_double(np.nan), ctypes.c_double(np.nan)
        self._sync_stream()
        _check(load().pw_spectrum_bounds(self._h, p, ld, m, lanczos_steps, vp, ctypes.byref(lo), ctypes.byref(hi),
                                         ctypes.byref(up)))
        return lo.value, hi.value, up.value

    def chebyshev_filter(self, psi, degree, a, b, precision=PW_FP64):
        psi, m, ld = _block(psi, _dtype(precision), "psi")
        self._sync_stream()
        _check(load().pw_chebyshev_filter(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m, int(degree), float(a),
                                          float(b), precision))

    def rayleigh_ritz(self, psi, hpsi=None):
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        hp = None
        if hpsi is not None:
            hpsi, _, ldh = _block(hpsi, torch.complex128, "hpsi")
            if ldh != ld:
                raise ValueError("hpsi must have psi's leading dimension")
            hp = ctypes.c_void_p(hpsi.data_ptr())
        eig = np.zeros(m)
        res = np.zeros(m)
        self._sync_stream()
        _check(load().pw_rayleigh_ritz(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m, hp, _dptr(eig), _dptr(res)))
        return eig, res

    def chebfi_solve(self, psi, degree, cycles, v0, lanczos_steps=10, precision=PW_FP64):
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        v0, _, _ = _block(v0, torch.complex128, "v0")
        eig = np.zeros(m)
        res = np.zeros(m)
        bnd = np.zeros(2)
        self._sync_stream()
        _check(load().pw_chebfi_solve(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m, int(degree), int(cycles),
                                      int(lanczos_steps), ctypes.c_void_p(v0.data_ptr()), precision, _dptr(eig),
                                      _dptr(res), _dptr(bnd)))
        return eig, res, bnd

    def density_grad(self, a, w, b=None, out=None, accumulate=False):
        import torch
        a, m, ld = _block(a, torch.complex128, "a")
        bp = None
        if b is not None:
            b, mb, ldb = _block(b, torch.complex128, "b")
            if ldb != ld or mb < m:
                raise ValueError("b must match a's layout")
            bp = ctypes.c_void_p(b.data_ptr())
        if out is None:
            out = torch.zeros(self.box, dtype=torch.float64, device="cuda")
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        if w.shape[0] < m:
            raise ValueError("need one weight per band")
        self._sync_stream()
        _check(load().pw_density_grad(self._h, ctypes.c_void_p(a.data_ptr()), bp, ld, m, _dptr(w),
                                      ctypes.c_void_p(out.data_ptr()), 1 if accumulate else 0))
        return out

    # -- spectrum slicing ------------------------------------------------------------------
    def slice_filter(self, psi, nslice, degree, lo, hi, cuts, precision=PW_FP64):
        """Each of the nslice band blocks of psi through its slice's window, in place."""
        psi, m, ld = _block(psi, _dtype(precision), "psi")
        if m % nslice:
            raise ValueError("the band count must be a multiple of nslice")
        c = np.ascontiguousarray(cuts, dtype=np.float64)
        if c.size != nslice + 1:
            raise ValueError("cuts needs nslice + 1 values")
        self._sync_stream()
        _check(load().pw_slice_filter(self._h, ctypes.c_void_p(psi.data_ptr()), ld, int(nslice), m // nslice,
                                      int(degree), float(lo), float(hi), _dptr(c), precision))
        return psi

    def spectrum_slice(self, psi, nslice, degree, lo, hi, cuts, precision=PW_FP64):
        """Window filter + per-slice FP64 Rayleigh-Ritz on psi (complex128, in place); returns
        the Ritz values and residual norms as (nslice, nper) arrays."""
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        if m % nslice:
            raise ValueError("the band count must be a multiple of nslice")
        c = np.ascontiguousarray(cuts, dtype=np.float64)
        if c.size != nslice + 1:
            raise ValueError("cuts needs nslice + 1 values")
        eig = np.zeros(m)
        res = np.zeros(m)
        self._sync_stream()
        _check(load().pw_spectrum_slice(self._h, ctypes.c_void_p(psi.data_ptr()), ld, int(nslice), m // nslice,
                                        int(degree), float(lo), float(hi), _dptr(c), precision, _dptr(eig),
                                        _dptr(res)))
        return eig.reshape(nslice, -1), res.reshape(nslice, -1)

    # -- LOBPCG (Alg. 11) -----------------------------------------------------------------
    def lobpcg_solve(self, psi, nblocks, nline, tol=0.0):
        """FP64 LOBPCG in place on psi (complex128); returns (eig, resid, line minimisations
        per block)."""
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        eig = np.zeros(m)
        res = np.zeros(m)
        its = (ctypes.c_int * max(int(nblocks), 1))()
        self._sync_stream()
        _check(load().pw_lobpcg_solve(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m, int(nblocks), int(nline),
                                      float(tol), _dptr(eig), _dptr(res), its))
        return eig, res, list(its)[:int(nblocks)]

    # -- Gamma-point pairing -------------------------------------------------------------
    def gamma_symmetrize(self, psi, precision=PW_FP64):
        """psi <- its r-space-real part (k = 0 contexts), in place."""
        psi, m, ld = _block(psi, _dtype(precision), "psi")
        self._sync_stream()
        _check(load().pw_gamma_symmetrize(self._h, ctypes.c_void_p(psi.data_ptr()), ld, m, precision))
        return psi

    def gamma_pack(self, a, precision=PW_FP64, out=None):
        """Packs 2m r-space-real bands into m complex bands c_j = a_2j + i a_2j+1."""
        import torch
        a, m, ld = _block(a, _dtype(precision), "a")
        if out is None:
            out = torch.empty((m // 2, self.npw), dtype=_dtype(precision), device="cuda")
        out, _, ldo = _block(out, _dtype(precision), "out")
        self._sync_stream()
        _check(load().pw_gamma_pack(self._h, ctypes.c_void_p(a.data_ptr()), ld, m, ctypes.c_void_p(out.data_ptr()),
                                    ldo, precision))
        return out

    def gamma_unpack(self, c, precision=PW_FP64, out=None):
        """Unpacks m complex bands into the 2m r-space-real bands they carry."""
        import torch
        c, m, ld = _block(c, _dtype(precision), "c")
        if out is None:
            out = torch.empty((2 * m, self.npw), dtype=_dtype(precision), device="cuda")
        out, _, ldo = _block(out, _dtype(precision), "out")
        self._sync_stream()
        _check(load().pw_gamma_unpack(self._h, ctypes.c_void_p(c.data_ptr()), ld, 2 * m,
                                      ctypes.c_void_p(out.data_ptr()), ldo, precision))
        return out

    # -- self-consistent field loop (Alg. 3) -------------------------------------------
    @classmethod
    def density_context(cls, lattice, ecut, box, stream=None):
        """The density context of a wave-function problem (cell, E_cut, box): Gamma point,
        no projectors, sphere |G|^2/2 <= 4 E_cut (pw_scf_potential)."""
        return cls(lattice, [0.0, 0.0, 0.0], 4.0 * ecut, box, np.zeros(tuple(box)), np.zeros((0, 3)), [],
                   np.zeros((0, 0)), stream=stream)

    def scf_potential(self, rho, vion, vin, beta):
        """V_new and (dc, E_H, E_x, max|V_out - V_in|, electrons) for a density context."""
        import torch
        out = np.zeros(5)
        vnew = torch.empty_like(vin)
        for t in (rho, vion, vin):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise TypeError("grids must be contiguous float64 CUDA tensors")
        self._sync_stream()
        _check(load().pw_scf_potential(self._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(vion.data_ptr()),
                                       ctypes.c_void_p(vin.data_ptr()), float(beta),
                                       ctypes.c_void_p(vnew.data_ptr()), _dptr(out)))
        return vnew, out

    def scf_run(self, dctx, psi, nocc, degree, cycles, v0, vion, max_iter=100, beta=0.3, tol=1e-8,
                precision=PW_FP64):
        """The SCF loop of pw_scf_run; returns (eigenvalues, history (iterations x 2), iterations)."""
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        v0, _, _ = _block(v0, torch.complex128, "v0")
        vi = np.ascontiguousarray(np.asarray(vion, dtype=np.float64))
        eig = np.zeros(m)
        hist = np.zeros(2 * max_iter)
        its = ctypes.c_int(0)
        self._sync_stream()
        st = load().pw_scf_run(self._h, dctx._h, ctypes.c_void_p(psi.data_ptr()), ld, m, int(nocc), int(degree),
                               int(cycles), int(max_iter), float(beta), float(tol), ctypes.c_void_p(v0.data_ptr()),
                               ctypes.c_void_p(vi.ctypes.data), precision, _dptr(eig), _dptr(hist),
                               ctypes.byref(its))
        _check(st)
        return eig, hist[:2 * its.value].reshape(-1, 2), its.value

    # -- differentiation form ---------------------------------------------------------
    def set_vloc(self, vloc):
        """Replaces V_loc(r) (n1 x n2 x n3 float64, host array or CUDA tensor)."""
        import torch
        if isinstance(vloc, torch.Tensor):
            v = vloc.detach().to(torch.float64).contiguous()
            size, ptr = v.numel(), v.data_ptr()
        else:
            v = np.ascontiguousarray(np.asarray(vloc, dtype=np.float64))
            size, ptr = v.size, v.ctypes.data
        if size != int(np.prod(self.box)):
            raise ValueError("vloc size does not match the box")
        self._sync_stream()
        _check(load().pw_ctx_set_vloc(self._h, ctypes.c_void_p(ptr)))

    def set_D(self, D):
        """Replaces D (nproj x nproj float64, host array or CUDA tensor; S = I contexts)."""
        import torch
        if isinstance(D, torch.Tensor):
            Dc = D.detach().to(torch.float64).t().contiguous()   # column-major view of D
            self._sync_stream()
            _check(load().pw_ctx_set_D(self._h, ctypes.c_void_p(Dc.data_ptr())))
        else:
            Dc = np.asfortranarray(np.asarray(D, dtype=np.float64))
            _check(load().pw_ctx_set_D(self._h, ctypes.c_void_p(Dc.ctypes.data)))

    def local_apply(self, v, psi, out=None, alpha=1.0, precision=PW_FP64):
        """out = alpha V psi for a real potential v (n1 x n2 x n3 float64 CUDA tensor)."""
        import torch
        dt = _dtype(precision)
        psi, m, ld = _block(psi, dt, "psi")
        if out is None:
            out = torch.empty((m, self.npw), dtype=dt, device="cuda")
        out, m2, ldo = _block(out, dt, "out")
        if m2 < m:
            raise ValueError("out has fewer bands than psi")
        v = v.detach().to(torch.float64).contiguous()
        if v.numel() != int(np.prod(self.box)) or not v.is_cuda:
            raise ValueError("v must be a CUDA tensor with n1*n2*n3 entries")
        self._sync_stream()
        _check(load().pw_local_apply(self._h, ctypes.c_void_p(v.data_ptr()), float(alpha),
                                     ctypes.c_void_p(psi.data_ptr()), ld, m, ctypes.c_void_p(out.data_ptr()), ldo,
                                     precision))
        return out


class Diff:
    """Differentiation handle (pw_diff): taped ChebFi forward and its reverse-mode adjoint."""

    def __init__(self, context, nband, degree, cycles, ckpt=2, precision=PW_FP64):
        self.context = context
        self.nband, self.degree, self.cycles, self.precision = int(nband), int(degree), int(cycles), precision
        h = ctypes.c_void_p()
        _check(load().pw_diff_create(context._h, self.nband, self.degree, self.cycles, int(ckpt), precision,
                                     ctypes.byref(h)))
        self._h = h
        context._dependents.add(self)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pw_diff_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tape_bytes(self):
        b = ctypes.c_int64(0)
        _check(load().pw_diff_tape_bytes(self._h, ctypes.byref(b)))
        return b.value

    def forward(self, psi, v0=None, lanczos_steps=10, bounds=None):
        """psi (complex128 CUDA block) is overwritten with the Ritz vectors; returns
        (eigenvalues, bounds = [upper, cut of every cycle])."""
        import torch
        psi, m, ld = _block(psi, torch.complex128, "psi")
        if m != self.nband:
            raise ValueError("psi must have nband bands")
        vp = None
        if v0 is not None:
            v0, _, _ = _block(v0, torch.complex128, "v0")
            vp = ctypes.c_void_p(v0.data_ptr())
        bin_ = None
        if bounds is not None:
            # [upper, a_1, ..., a_cycles] or (upper, [a_1, ..., a_cycles])
            bin_ = np.ascontiguousarray(np.concatenate([np.atleast_1d(np.asarray(x, dtype=np.float64)).ravel()
                                                        for x in bounds]))
            if bin_.shape[0] != 1 + self.cycles:
                raise ValueError("bounds needs 1 + cycles values")
        eig = np.zeros(m)
        bout = np.zeros(1 + self.cycles)
        self.context._sync_stream()
        _check(load().pw_diff_forward(self._h, ctypes.c_void_p(psi.data_ptr()), ld, int(lanczos_steps), vp,
                                      None if bin_ is None else _dptr(bin_), _dptr(eig), _dptr(bout)))
        return eig, bout

    def backward(self, eig_bar=None, psi_bar=None, split=-1):
        """Returns (dL/dV_loc as an n1 x n2 x n3 float64 CUDA tensor, dL/dD as nproj x nproj)."""
        import torch
        ctx = self.context
        eb = None
        if eig_bar is not None:
            eb = np.ascontiguousarray(np.asarray(eig_bar, dtype=np.float64).reshape(-1))
        pp, ld = None, ctx.npw
        if psi_bar is not None:
            psi_bar, m, ld = _block(psi_bar, torch.complex128, "psi_bar")
            pp = ctypes.c_void_p(psi_bar.data_ptr())
        dV = torch.empty(ctx.box, dtype=torch.float64, device="cuda")
        dDc = torch.empty((max(ctx.nproj, 1), max(ctx.nproj, 1)), dtype=torch.float64, device="cuda")
        ctx._sync_stream()
        _check(load().pw_diff_backward(self._h, None if eb is None else _dptr(eb), pp, ld, int(split),
                                       ctypes.c_void_p(dV.data_ptr()), ctypes.c_void_p(dDc.data_ptr()), 0))
        return dV, dDc.t()[:ctx.nproj, :ctx.nproj]


class Batch:
    """k-point batch (pw_batch): every context's filter in one captured CUDA graph."""

    def __init__(self, contexts, stream=None):
        import torch
        lib = load()
        self.contexts = list(contexts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(lib.pw_batch_create(arr, len(self.contexts), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().pw_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _blocks(self, psis, dtype):
        ptrs, lds, m = [], [], None
        for ctx, p in zip(self.contexts, psis):
            p, mm, ld = _block(p, dtype, "psi")
            if m is None:
                m = mm
            elif mm != m:
                raise ValueError("every k-point needs the same number of bands")
            ptrs.append(p.data_ptr())
            lds.append(ld)
        return (ctypes.c_void_p * len(ptrs))(*ptrs), (ctypes.c_int64 * len(lds))(*lds), m

    def filter(self, psis, degree, a, b, precision=PW_FP64):
        pa, pl, m = self._blocks(psis, _dtype(precision))
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
        _check(load().pw_batch_filter(self._h, pa, pl, m, int(degree), _dptr(a), _dptr(b), precision))

    def chebfi_solve(self, psis, degree, cycles, v0s, lanczos_steps=10, precision=PW_FP64):
        import torch
        pa, pl, m = self._blocks(psis, torch.complex128)
        vptr = (ctypes.c_void_p * len(v0s))(*[_block(v, torch.complex128, "v0")[0].data_ptr() for v in v0s])
        nk = len(self.contexts)
        eig = np.zeros((nk, m))
        res = np.zeros((nk, m))
        _check(load().pw_batch_chebfi_solve(self._h, pa, pl, m, int(degree), int(cycles), int(lanczos_steps), vptr,
                                            precision, _dptr(eig), _dptr(res)))
        return eig, res
