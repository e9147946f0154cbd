"""Host dense linear algebra of the LOBPCG Rayleigh-Ritz step (CPU).

The routines are compiled from the library's own source (dense.cpp) with a C
harness and checked against LAPACK (numpy.linalg.eigh) and against the defining
identities: A V = V diag(w), V^T V = I; A X = B X diag(w), X^T B X = I;
L L^T = B; L^T R = I.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1403_7561_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    out = str(tmp_path_factory.mktemp("dense") / "libdense.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "dense_harness.cpp"), os.path.join(CSRC, "dense.cpp"), "-o", out],
                   check=True, capture_output=True)
    L = C.CDLL(out)
    P = C.POINTER(C.c_double)
    L.h_sym_eig.argtypes = [C.c_int, P, P, P]
    L.h_gen_eig.argtypes = [C.c_int, P, P, P, P]
    L.h_gen_eig.restype = C.c_int
    L.h_cholesky.argtypes = [C.c_int, P]
    L.h_cholesky.restype = C.c_int
    L.h_inv_lt.argtypes = [C.c_int, P, P]
    return L


def ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def sym_eig(lib, A):
    n = A.shape[0]
    a = np.asfortranarray(A.copy())
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    lib.h_sym_eig(n, ptr(a), ptr(w), ptr(V))
    return w, V


def matrices():
    rng = np.random.default_rng(11)
    out = []
    for n in (1, 2, 3, 7, 24, 36, 60):
        M = rng.standard_normal((n, n))
        out.append(("random%d" % n, 0.5 * (M + M.T)))
    out.append(("identity12", np.eye(12)))
    out.append(("diag_graded", np.diag(10.0 ** np.linspace(-8, 8, 20))))
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    out.append(("clustered", Q @ np.diag([1.0] * 10 + [1.0 + 1e-9] * 10 + list(np.linspace(2, 3, 10))) @ Q.T))
    T = np.diag(np.full(16, 2.0)) - np.diag(np.ones(15), 1) - np.diag(np.ones(15), -1)
    out.append(("laplacian16", T))
    return out


@pytest.mark.parametrize("name,A", matrices(), ids=[m[0] for m in matrices()])
def test_symmetric_eigenproblem(lib, name, A):
    n = A.shape[0]
    w, V = sym_eig(lib, A)
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - ref)) <= 1e-12 * scale * max(1, n)
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-12 * max(1, n)
    assert np.max(np.abs(A @ V - V * w)) <= 1e-12 * scale * max(1, n)


def test_laplacian_closed_form(lib):
    # eigenvalues of the 1D Dirichlet Laplacian stencil: 2 - 2 cos(k pi / (n + 1))
    n = 16
    T = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    w, _ = sym_eig(lib, T)
    k = np.arange(1, n + 1)
    assert np.max(np.abs(w - (2 - 2 * np.cos(k * np.pi / (n + 1))))) <= 1e-13


@pytest.mark.parametrize("n", [3, 12, 36])
def test_generalized_eigenproblem(lib, n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = 0.5 * (M + M.T)
    Bm = rng.standard_normal((n, n))
    B = Bm @ Bm.T + n * np.eye(n)
    w = np.zeros(n)
    X = np.zeros((n, n), order="F")
    assert lib.h_gen_eig(n, ptr(np.asfortranarray(A)), ptr(np.asfortranarray(B)), ptr(w), ptr(X)) == 1
    Lb = np.linalg.cholesky(B)
    ref = np.linalg.eigvalsh(np.linalg.solve(Lb, np.linalg.solve(Lb, A).T).T)
    assert np.max(np.abs(w - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(X.T @ B @ X - np.eye(n))) <= 1e-11
    assert np.max(np.abs(A @ X - B @ X * w)) <= 1e-10 * max(1.0, np.max(np.abs(w)))


def test_cholesky_and_inverse_transpose(lib):
    rng = np.random.default_rng(4)
    n = 20
    M = rng.standard_normal((n, n))
    B = M @ M.T + n * np.eye(n)
    L = np.asfortranarray(B.copy())
    assert lib.h_cholesky(n, ptr(L)) == 1
    assert np.max(np.abs(np.triu(L, 1))) == 0.0
    assert np.max(np.abs(L @ L.T - B)) <= 1e-12 * np.max(np.abs(B))
    R = np.zeros((n, n), order="F")
    lib.h_inv_lt(n, ptr(L), ptr(R))
    assert np.max(np.abs(L.T @ R - np.eye(n))) <= 1e-12
    # not positive definite
    Bad = np.asfortranarray(np.diag([1.0, -1.0, 2.0]))
    assert lib.h_cholesky(3, ptr(Bad)) == 0
