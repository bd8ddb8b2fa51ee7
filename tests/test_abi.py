"""The C-ABI library loads on the CPU machine, exports every symbol that
include/fdfd.h declares, and validates arguments on the host (no GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "fdfd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2509_03622_gb300 import build as B
    if not os.path.exists(B.OUT):
        B.build()
    from paper_2509_03622_gb300 import fdfd
    return fdfd


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["fdfd_create", "schwarz_setup", "fdfd_solve", "fdfd_solve_adjoint", "fdfd_destroy",
                 "fdfd_apply_A", "fdfd_precond_apply", "fdfd_nno_solve", "fdfd_trace_extract",
                 "fdfd_grad_eps", "fdfd_solve_host"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = C.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_host_side_validation(lib):
    h = C.c_void_p()
    assert lib.lib.fdfd_create(None, C.byref(h)) == lib.EINVAL
    d = lib.Desc()
    d.nx, d.ny, d.dx, d.wavelength = 100, 128, 1e-7, 1.55e-6   # nx not a multiple of 64
    d.npml = (C.c_int * 4)(20, 20, 20, 20)
    d.pml_m, d.pml_lnR = 3.0, -30.0
    d.eps = 1  # never dereferenced: validation fails first
    assert lib.lib.fdfd_create(C.byref(d), C.byref(h)) == lib.EINVAL
    d.nx = 128
    d.npml = (C.c_int * 4)(64, 20, 20, 20)  # PML >= half the grid
    assert lib.lib.fdfd_create(C.byref(d), C.byref(h)) == lib.EINVAL
    d.npml = (C.c_int * 4)(20, 20, 20, 20)
    d.wavelength = -1.0
    assert lib.lib.fdfd_create(C.byref(d), C.byref(h)) == lib.EINVAL
    assert not h.value
    assert lib.status_string(lib.ENUMERIC).startswith("NaN")
    assert lib.lib.fdfd_solve(None, None, None, None, None) == lib.EINVAL
    # figure-of-merit entry points: arguments are checked before any launch
    # (the fake pointers below are never dereferenced)
    fake, c = C.c_void_p(16), C.c_void_p(32)
    assert lib.lib.fdfd_mode_overlap(None, 128, 128, fake, 8, 5, 0, 1e-8, c, None) == lib.EINVAL
    assert lib.lib.fdfd_mode_overlap(fake, 128, 128, fake, 8, 128, 0, 1e-8, c, None) == lib.EINVAL  # port_x = nx
    assert lib.lib.fdfd_mode_overlap(fake, 128, 128, fake, 8, 5, 121, 1e-8, c, None) == lib.EINVAL  # y0 + nm > ny
    assert lib.lib.fdfd_mode_overlap(fake, 128, 128, fake, 0, 5, 0, 1e-8, c, None) == lib.EINVAL   # nm = 0
    assert lib.lib.fdfd_mode_overlap(fake, 128, 128, fake, 8, 5, 0, 0.0, c, None) == lib.EINVAL    # dx = 0
    assert lib.lib.fdfd_mode_overlap_grad(128, 128, fake, 8, -1, 0, 1e-8, 1.0, 0.0, c, 0, None) == lib.EINVAL
    assert lib.lib.fdfd_mode_overlap_grad(128, 128, None, 8, 5, 0, 1e-8, 1.0, 0.0, c, 0, None) == lib.EINVAL
    assert lib.lib.fdfd_adjoint_rhs(None, fake, c) == lib.EINVAL


def test_no_oracle_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2509_03622_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_host_side_validation_of_the_extensions(lib):
    """Algorithm 3's stationary solver, the Ritz export and the inverse-design
    entry points refuse a missing handle or out-of-range arguments before any
    device work."""
    L = lib.lib
    assert L.fdfd_schwarz_stationary(None, None, None, 5, 1e-6, 0.5, None, None) == lib.EINVAL
    assert L.fdfd_coarse_ritz(None, None, None) == lib.EINVAL
    d = lib.DesignDesc(0, 0, 8, 8, 2.0, 8.0, 0.5, 2.1, 12.25)
    assert L.fdfd_design_eps(None, C.byref(d), None, None, None) == lib.EINVAL
    assert L.fdfd_design_grad(None, C.byref(d), None, None, None, None) == lib.EINVAL
    a = lib.AdamDesc(0.01, 0.9, 0.999, 1e-8)
    assert L.fdfd_adam_step(None, C.byref(a), 1, 1.0, None, None, None, None, 4) == lib.EINVAL


def test_overlap_binding_rejects_wrong_dtypes(lib):
    """The figure-of-merit bindings check dtypes before passing pointers (the
    library reads complex64 fields and a two-double result)."""
    import torch
    c = torch.zeros(2, dtype=torch.float64)
    with pytest.raises(TypeError):
        lib.mode_overlap(torch.zeros((64, 64), dtype=torch.complex128), torch.zeros(4, dtype=torch.complex64),
                         1, 0, 1e-8, c)
    with pytest.raises(TypeError):
        lib.mode_overlap(torch.zeros((64, 64), dtype=torch.complex64), torch.zeros(4, dtype=torch.complex64),
                         1, 0, 1e-8, torch.zeros(2, dtype=torch.float32))
    with pytest.raises(TypeError):
        lib.mode_overlap_grad((64, 64), torch.zeros(4, dtype=torch.complex64), 1, 0, 1e-8, 1.0,
                              torch.zeros((32, 64), dtype=torch.complex64))
