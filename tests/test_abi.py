"""The C-ABI library builds, loads without a GPU and exports every entry point its header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcad.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qcad_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    import importlib.util
    spec = importlib.util.spec_from_file_location("qcad_build", os.path.join(ROOT, "paper_1403_7561_gb300", "build.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    path, _ = B.build()
    return path


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("qcad_mesh_create", "qcad_poisson_solve", "qcad_schrodinger_eigs", "qcad_capacitance",
              "qcad_adjoint", "qcad_poisson_solve_batch", "qcad_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib_path):
    import paper_1403_7561_gb300 as q
    for s in declared_symbols():
        assert s in q.EXPORTED, s


def test_invalid_mesh_is_rejected_without_gpu_work(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.qcad_mesh_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.qcad_mesh_create.restype = ctypes.c_int
    lib.qcad_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    assert lib.qcad_mesh_create(None, None, ctypes.byref(out)) == 1  # QCAD_ERR_INVALID_ARG
    assert b"null" in lib.qcad_last_error()


def test_binding_rejects_surface_terms_it_does_not_solve(lib_path):
    # charged gates and surface charges exist in the oracle only: the library must not ignore them
    import copy

    import paper_1403_7561_gb300 as q
    import workloads as W
    dev = W.five_gate_device(n=(8, 8, 6))
    d1 = copy.deepcopy(dev)
    d1["gates"][1]["robin"] = dict(sigma=1e-3, d=10.0)
    with pytest.raises(NotImplementedError, match="P1"):
        q.Mesh(d1)
    d2 = copy.deepcopy(dev)
    d2["surface_charges"] = [dict(z=90.0, x0=0.0, x1=200.0, y0=0.0, y1=200.0, sigma=1e-3)]
    with pytest.raises(NotImplementedError):
        q.Mesh(d2)
    if not q.torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="CUDA"):       # an ordinary device passes the check
            q.Mesh(dev)
