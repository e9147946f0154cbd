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


def test_binding_passes_surface_terms(lib_path):
    # charged gates (a gate's "robin" entry) and surface charges reach the C description
    import copy

    import paper_1403_7561_gb300 as q
    import workloads as W
    dev = W.five_gate_device(n=(8, 8, 6))
    dev["gates"][3]["robin"] = dict(sigma=5e-4, d=10.0)
    dev["surface_charges"] = [dict(z=90.0, x0=0.0, x1=200.0, y0=25.0, y1=175.0, sigma=-1e-3)]
    d, keep = q._device_struct(dev)
    assert d.n_charged_gates == 1 and d.charged_gates[0].gate == 3
    assert (d.charged_gates[0].sigma, d.charged_gates[0].d) == (5e-4, 10.0)
    assert d.n_surface_charges == 1
    S = d.surface_charges[0]
    assert (S.z, S.x0, S.x1, S.y0, S.y1, S.sigma) == (90.0, 0.0, 200.0, 25.0, 175.0, -1e-3)
    d0, _ = q._device_struct(copy.deepcopy(W.five_gate_device(n=(8, 8, 6))))
    assert d0.n_charged_gates == 0 and d0.n_surface_charges == 0


def test_binding_structs_match_the_header(lib_path, tmp_path):
    # every field of the ctypes mirrors sits at the offset the C compiler gives it
    import shutil
    import subprocess

    import paper_1403_7561_gb300 as q
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"qcad_device": q.Device, "qcad_charged_gate": q.ChargedGate,
               "qcad_surface_charge": q.SurfaceCharge, "qcad_material": q.Material, "qcad_bias": q.Bias,
               "qcad_solver_opts": q.SolverOpts, "qcad_solve_report": q.SolveReport}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qcad.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def _noalloc_call(dev):
    """Calls the allocation-free residual's C entry point directly with placeholder phi and R
    pointers (never dereferenced: every case below is rejected by host-side checks, before the
    entry point touches a device); returns (status, message)."""
    import paper_1403_7561_gb300 as q
    d, keep = q._device_struct(dev)
    b = q.make_bias(dev["bias"])
    fake = ctypes.c_void_p(1 << 20)
    code = q._lib.qcad_poisson_residual_noalloc(ctypes.byref(d), ctypes.byref(b), None, None, fake, fake, None)
    return code, q._lib.qcad_last_error().decode()


@pytest.mark.parametrize("case", ["index_limit", "layers", "two_semiconductors", "permittivity", "charged_gate",
                                  "scratch"])
def test_noalloc_rejects_what_mesh_create_rejects(lib_path, case):
    # the allocation-free residual checks a description with qcad_mesh_create's own host function
    # (the kernels index nodes with 32-bit integers) before the scratch limit and before any device
    # call; a description that passes these checks is never handed to a kernel here
    import workloads as W
    dev = W.five_gate_device(n=(16, 16, 8), T=4.0, with_subdomain=False)
    expect = {"index_limit": "32-bit", "layers": "too many element layers",
              "two_semiconductors": "one semiconductor", "permittivity": "permittivity",
              "charged_gate": "charged gates", "scratch": "scratch"}[case]
    if case == "index_limit":      # about 2.2e9 nodes: fits the 2 MiB scratch, overflows int indices
        dev.update(nx=1000, ny=1000)
        dev["layers"] = [dict(material=0, thickness=90.0, n=2190), dict(material=1, thickness=10.0, n=10)]
    elif case == "layers":
        dev.update(nx=1, ny=1)
        dev["layers"] = [dict(material=0, thickness=90.0, n=70000), dict(material=1, thickness=10.0, n=10)]
    elif case == "two_semiconductors":
        other = dict(dev["materials"][0], N_A=2e-6)
        dev["materials"].append(other)
        dev["layers"][0]["material"] = 2
        dev["layers"].insert(0, dict(material=0, thickness=10.0, n=2))
    elif case == "permittivity":
        dev["materials"][1]["eps_r"] = 0.0
    elif case == "charged_gate":
        dev["gates"][1]["robin"] = dict(sigma=1e-4, d=10.0)
    else:                          # the top-plane contact mask alone (2049^2 bytes) exceeds 2 MiB
        dev.update(nx=2048, ny=2048)
    code, msg = _noalloc_call(dev)
    assert code == 1 and expect in msg, (code, msg)
