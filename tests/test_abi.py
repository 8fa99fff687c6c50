"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function include/pw.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

from paper_2604_11139_gb300 import build as B
from paper_2604_11139_gb300 import pwlib

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared():
    names = set()
    for f in os.listdir(HDR):
        if f.endswith(".h"):
            txt = open(os.path.join(HDR, f)).read()
            names |= set(re.findall(r"PW_API\s+[\w\s\*]+?\b(pw_\w+)\s*\(", txt))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared()
    assert {"pw_ctx_create", "pw_hamiltonian_apply", "pw_chebyshev_filter", "pw_rayleigh_ritz",
            "pw_density_grad"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(pwlib.EXPORTS)


def test_status_strings_without_gpu():
    lib = pwlib.load()
    assert lib.pw_strerror(0) == b"ok"
    assert lib.pw_strerror(-4) == b"matrix not positive definite"
    # a NULL descriptor is rejected on the host before any CUDA call
    h = ctypes.c_void_p()
    assert lib.pw_ctx_create(None, None, ctypes.byref(h)) == -1
    assert b"NULL" in lib.pw_last_error()


def test_no_cpu_fallback_without_a_gpu():
    """The product path has no CPU fallback: without a usable GPU, creating a context fails
    with PW_ECUDA from the library (the descriptor itself is valid)."""
    import types

    import pytest

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_11139_gb300 import workloads as W

    prob = W.make_problem("tiny_gamma_fp64", box=(16, 16, 16), ecut=3.0, nband=4)
    with pytest.raises(pwlib.PWError) as e:
        pwlib.Context.from_problem(prob, stream=types.SimpleNamespace(cuda_stream=0))
    assert e.value.status == -3


def test_explicit_projector_descriptor_checked_on_the_host():
    """Explicit projectors with nproj < 1 or without D are rejected before any CUDA call."""
    lib = pwlib.load()
    d = pwlib._Desc()
    d.ecut = 1.0
    d.box[:] = [8, 8, 8]
    v = (ctypes.c_double * 512)()
    d.vloc = ctypes.cast(v, ctypes.POINTER(ctypes.c_double))
    buf = (ctypes.c_double * 4)()
    d.proj = ctypes.cast(buf, ctypes.c_void_p)
    d.nproj = 0
    h = ctypes.c_void_p()
    assert lib.pw_ctx_create(ctypes.byref(d), None, ctypes.byref(h)) == -1
    assert b"nproj" in lib.pw_last_error()
    d.nproj = 2
    assert lib.pw_ctx_create(ctypes.byref(d), None, ctypes.byref(h)) == -1
    assert b"need D" in lib.pw_last_error()


def _zero(t):
    if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64):
        return 0
    if t is ctypes.c_double:
        return 0.0
    return None  # pointers and handles


def test_every_entry_point_rejects_a_null_handle_without_a_gpu():
    # every call whose first argument is a context, batch or differentiation handle (or the
    # descriptor / context array that makes one) returns PW_EINVAL for NULL and touches no
    # device; destroy(NULL) is a no-op; the FMA-rate diagnostic takes a stream, not a handle
    lib = pwlib.load()
    skip = {"pw_strerror", "pw_last_error", "pw_kernel_launches", "pw_diag_fp64_fma_rate"}
    destroy = {"pw_ctx_destroy", "pw_batch_destroy", "pw_diff_destroy"}
    for name in sorted(set(pwlib.EXPORTS) - skip):
        fn = getattr(lib, name)
        args = [_zero(t) for t in fn.argtypes]
        st = fn(*args)
        if name in destroy:
            assert st == 0, name
        else:
            assert st == -1, (name, st, lib.pw_last_error())
            assert lib.pw_last_error(), name
