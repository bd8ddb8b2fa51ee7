"""The coarse space's batched eigen solver (csrc/eig.cuh: Hessenberg
reduction, shifted complex QR, back substitution; used for the Rayleigh-Ritz
step of Algorithm 3's set-up) built as host code with g++ and checked
against numpy.linalg.eig, on the CPU."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2509_03622_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = r"""
#include "eig.cuh"
#include <cstring>
#include <vector>
extern "C" int eig_batch(int n, int k, const double* H, double* eta, double* U) {
  std::vector<ecd> A(k * k), Z(k * k), e(k), u(k * k);
  int bad = 0;
  for (int b = 0; b < n; ++b) {
    std::memcpy(A.data(), H + (size_t)b * k * k * 2, sizeof(ecd) * k * k);
    if (!eig_small(A.data(), Z.data(), e.data(), u.data(), k)) ++bad;
    std::memcpy(eta + (size_t)b * k * 2, e.data(), sizeof(ecd) * k);
    std::memcpy(U + (size_t)b * k * k * 2, u.data(), sizeof(ecd) * k * k);
  }
  return bad;
}
"""


@pytest.fixture(scope="module")
def eig(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("eig")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libeig.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2509_03622_gb300", "csrc"), str(src), "-o", str(so)], check=True)
    lib = C.CDLL(str(so))

    def run(H):
        n, k, _ = H.shape
        Hc = np.ascontiguousarray(H, dtype=np.complex128)
        eta = np.zeros((n, k), np.complex128)
        U = np.zeros((n, k, k), np.complex128)
        bad = lib.eig_batch(n, k, Hc.ctypes.data_as(C.c_void_p), eta.ctypes.data_as(C.c_void_p),
                            U.ctypes.data_as(C.c_void_p))
        return bad, eta, U
    return run


def _check(run, H, tol=1e-12):
    bad, eta, U = run(H)
    assert bad == 0
    for b in range(H.shape[0]):
        scale = max(np.linalg.norm(H[b], 2), 1e-300)
        # every pair is an eigenpair with a unit vector ...
        res = np.linalg.norm(H[b] @ U[b] - U[b] * eta[b][None, :], axis=0)
        assert np.all(res <= tol * scale)
        nz = np.linalg.norm(U[b], axis=0)
        assert np.allclose(nz, 1.0)
        # ... and the eigenvalues are numpy's, as a multiset
        ref = list(np.linalg.eigvals(H[b]))
        for e in eta[b]:
            j = int(np.argmin([abs(e - r) for r in ref]))
            assert abs(e - ref.pop(j)) <= 100 * tol * scale


@pytest.mark.parametrize("k", [1, 2, 3, 8, 36, 64])
def test_random_complex_matrices(eig, k):
    g = wl.rng(20 + k)
    H = g.standard_normal((6, k, k)) + 1j * g.standard_normal((6, k, k))
    _check(eig, H)


def test_structured_matrices(eig):
    """Zero rows and columns (trials dropped by Gram-Schmidt), the zero
    matrix, a diagonal matrix and a Jordan-type (defective) block."""
    g = wl.rng(30)
    H = g.standard_normal((4, 8, 8)) + 1j * g.standard_normal((4, 8, 8))
    H[:, 3, :] = 0
    H[:, :, 3] = 0
    _check(eig, H)
    bad, eta, _ = eig(np.zeros((2, 5, 5), complex))
    assert bad == 0 and not np.any(eta)
    _check(eig, np.stack([np.diag(np.arange(6) + 1j)]).astype(complex))
    J = (2.0 * np.eye(6) + np.eye(6, k=1)).astype(complex)[None]
    bad, eta, _ = eig(J)
    assert bad == 0 and np.allclose(eta, 2.0)


def test_out_of_range_size_is_refused(eig):
    bad, _, _ = eig(np.zeros((1, 65, 65), complex))
    assert bad == 1
