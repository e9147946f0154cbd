"""Python binding of libqcad (include/qcad.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts device
descriptions (``workloads`` dictionaries) into the C structures, checks the
torch tensors it is given (device, dtype, size, contiguity) and passes their
device pointers. PyTorch provides device memory and streams only.

The library is loaded from this package's directory; if it is missing the
import fails loudly (build it with ``python -m paper_1403_7561_gb300.build``
or ``__graft_entry__.build()``). There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcad.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libqcad.so is not built at %s; run `python -m paper_1403_7561_gb300.build`" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)

QCAD_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "NONFINITE", 6: "TIMEOUT"}
PROF_CLASSES = {"apply32": 0, "apply64": 1, "update32": 2, "update64": 3, "residual": 4, "hm": 5, "mg": 6}


class QcadError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class NotConverged(QcadError):
    pass


class Material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("chi", C.c_double), ("Eg", C.c_double), ("semiconductor", C.c_int),
                ("m_l", C.c_double), ("m_t", C.c_double), ("m_hh", C.c_double), ("m_lh", C.c_double),
                ("N_A", C.c_double), ("N_D", C.c_double), ("E_a", C.c_double), ("E_d", C.c_double),
                ("g_A", C.c_double), ("g_D", C.c_double)]


class Rect(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double)]


class Box(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("z0", C.c_double), ("z1", C.c_double)]


class ChargedGate(C.Structure):
    _fields_ = [("gate", C.c_int), ("sigma", C.c_double), ("d", C.c_double)]


class SurfaceCharge(C.Structure):
    _fields_ = [("z", C.c_double), ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("sigma", C.c_double)]


class Device(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("n_layers", C.c_int), ("layer_n", C.POINTER(C.c_int)),
                ("layer_thickness", C.POINTER(C.c_double)), ("layer_material", C.POINTER(C.c_int)),
                ("n_materials", C.c_int), ("materials", C.POINTER(Material)),
                ("n_gates", C.c_int), ("gates", C.POINTER(Rect)),
                ("gate_work_function_set", C.c_int), ("gate_work_function", C.c_double),
                ("bottom_ohmic", C.c_int), ("n_dots", C.c_int), ("dots", C.POINTER(Box)),
                ("has_subdomain", C.c_int), ("sub", C.c_int * 6),
                ("n_charged_gates", C.c_int), ("charged_gates", C.POINTER(ChargedGate)),
                ("n_surface_charges", C.c_int), ("surface_charges", C.POINTER(SurfaceCharge))]


class Bias(C.Structure):
    _fields_ = [("T", C.c_double), ("n_gates", C.c_int), ("V_gate", C.POINTER(C.c_double)),
                ("V_sub", C.c_double), ("statistics", C.c_int), ("incomplete_ionization", C.c_int)]


class SolverOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("newton_tol_R", C.c_double), ("newton_tol_dphi", C.c_double),
                ("max_newton", C.c_int), ("max_krylov", C.c_int), ("cheb_degree", C.c_int),
                ("warm_start", C.c_int), ("linear", C.c_int)]


class SolveReport(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("krylov_iters_total", C.c_int), ("applies_total", C.c_int),
                ("final_res_inf", C.c_double), ("final_dphi_inf", C.c_double), ("seconds", C.c_double),
                ("status_detail", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SP_HIST = 64


class SpReport(C.Structure):
    _fields_ = [("sp_iters", C.c_int), ("converged", C.c_int), ("dphi_inf", C.c_double), ("n_quantum", C.c_double),
                ("seconds", C.c_double), ("dphi_hist", C.c_double * SP_HIST), ("e1_hist", C.c_double * SP_HIST)]

    def as_dict(self):
        k = min(self.sp_iters, SP_HIST)
        return {"sp_iters": self.sp_iters, "converged": bool(self.converged), "dphi_inf": self.dphi_inf,
                "n_quantum": self.n_quantum, "seconds": self.seconds, "dphi_hist": list(self.dphi_hist)[:k],
                "e1_hist": list(self.e1_hist)[:k]}


CALIB_HIST = 32


class CalibReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("N", C.c_double), ("dN_dsigma", C.c_double),
                ("seconds", C.c_double), ("sigma_hist", C.c_double * CALIB_HIST), ("N_hist", C.c_double * CALIB_HIST)]

    def as_dict(self):
        k = min(self.iters, CALIB_HIST)
        return {"iters": self.iters, "converged": bool(self.converged), "N": self.N, "dN_dsigma": self.dN_dsigma,
                "seconds": self.seconds, "sigma_hist": list(self.sigma_hist)[:k], "N_hist": list(self.N_hist)[:k]}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_sigs = {
    "qcad_mesh_create": [C.POINTER(Device), _P, C.POINTER(_P)],
    "qcad_mesh_destroy": [_P],
    "qcad_mesh_info": [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                       C.POINTER(C.c_int64)],
    "qcad_contact_values": [_P, C.POINTER(Bias), _P, _D, _D],
    "qcad_poisson_residual": [_P, C.POINTER(Bias), _P, _P, _P, _P, _D],
    "qcad_poisson_jv": [_P, C.POINTER(Bias), _P, _P, _P, C.c_int],
    "qcad_poisson_solve": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), _P, _P, C.POINTER(SolveReport)],
    "qcad_electron_counts": [_P, C.POINTER(Bias), _P, _P, _D],
    "qcad_capacitance": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), C.c_int, C.c_double, _P, _P, _D],
    "qcad_adjoint": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), _P, _P, _D, _P],
    "qcad_schrodinger_apply": [_P, C.POINTER(Bias), _P, _D, C.c_int, _P, _P, _P, C.c_int],
    "qcad_schrodinger_eigs": [_P, C.POINTER(Bias), _P, C.c_int, _D, C.c_double, _D, _P, C.POINTER(SolveReport)],
    "qcad_launch_info": [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                         C.POINTER(C.c_int)],
    "qcad_adjoint_eigs": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), _P, _P, _D, _P, C.c_int, _D, C.c_double, _D,
                          _P, C.POINTER(SolveReport)],
    "qcad_poisson_solve_batch": [C.c_int, C.POINTER(_P), C.POINTER(Bias), C.POINTER(SolverOpts), C.POINTER(_P),
                                 C.POINTER(SolveReport)],
    "qcad_adjoint_batch": [C.c_int, C.POINTER(_P), C.POINTER(Bias), C.POINTER(SolverOpts), C.POINTER(_P), _D],
    "qcad_calibrate_sheet_charge": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), C.c_int, C.c_double, _P, C.c_double,
                                    C.c_double, C.c_int, _P, _P, _D, C.POINTER(CalibReport)],
    "qcad_sp_solve": [_P, C.POINTER(Bias), C.POINTER(SolverOpts), C.c_int, _D, C.c_double, C.c_double, C.c_int,
                      C.c_int, _P, _D, C.POINTER(SpReport)],
    "qcad_profile_enable": [_P, C.c_int],
    "qcad_profile_reset": [_P],
    "qcad_profile_read": [_P, C.c_int, C.POINTER(C.c_int64), _D],
    "qcad_set_launch": [_P, C.c_int, C.c_int, C.c_int, C.c_int],
    "qcad_autotune": [_P, C.POINTER(Bias), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                      C.POINTER(C.c_float)],
    "qcad_launch_count": [C.POINTER(C.c_int64)],
    "qcad_alu_peaks": [_D, _D, _D],
    "qcad_poisson_residual_noalloc": [C.POINTER(Device), C.POINTER(Bias), _P, _P, _P, _P, _D],
    "qcad_last_error": [],
}
for _name, _args in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.qcad_mesh_destroy.restype = None
_lib.qcad_last_error.restype = C.c_char_p

EXPORTED = sorted(_sigs)


def _check(code, allow_not_converged=False):
    if code == QCAD_OK:
        return code
    msg = _lib.qcad_last_error().decode(errors="replace")
    if code == 4:
        if allow_not_converged:
            return code
        raise NotConverged(code, msg)
    raise QcadError(code, msg)


def _dptr(t, n=None, dtype=torch.float64, name="tensor", allow_none=False):
    """Device pointer of a contiguous CUDA tensor with at least n elements."""
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), n))
    return C.c_void_p(t.data_ptr())


class Mesh:
    """Owning handle of a qcad mesh built from a device description dictionary."""

    def __init__(self, dev: dict, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libqcad needs a CUDA device")
        self.dev = dev
        d, self._keep = _device_struct(dev)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(_lib.qcad_mesh_create(C.byref(d), C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.handle = h
        nn, ne, ns = C.c_int64(), C.c_int64(), C.c_int64()
        ng, nd = C.c_int(), C.c_int()
        _check(_lib.qcad_mesh_info(h, C.byref(nn), C.byref(ne), C.byref(ng), C.byref(nd), C.byref(ns)))
        self.n_nodes, self.n_elems, self.n_gates, self.n_dots, self.n_sub_dof = \
            nn.value, ne.value, ng.value, nd.value, ns.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.qcad_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_bias(bias: dict):
    V = bias["V_gate"]
    arr = (C.c_double * max(1, len(V)))(*V)
    b = Bias(float(bias["T"]), len(V), arr, float(bias.get("V_sub", 0.0)), int(bias.get("statistics", 1)),
             int(bias.get("incomplete_ionization", 1)))
    b._arr = arr  # keep alive
    return b


def make_opts(precision=0, tol_R=1e-10, tol_dphi=1e-10, max_newton=100, max_krylov=20000, cheb_degree=1,
              warm_start=0, linear=0):
    return SolverOpts(int(precision), float(tol_R), float(tol_dphi), int(max_newton), int(max_krylov),
                      int(cheb_degree), int(warm_start), int(linear))


# ---------------------------------------------------------------------------
# Entry points with the C ABI's names.
def qcad_mesh_create(dev: dict, stream=None) -> Mesh:
    return Mesh(dev, stream)


def qcad_mesh_destroy(mesh: Mesh):
    mesh.close()


def qcad_contact_values(mesh: Mesh, bias: dict, phi=None):
    b = make_bias(bias)
    gv = (C.c_double * max(1, mesh.n_gates))()
    ov = C.c_double()
    _check(_lib.qcad_contact_values(mesh.handle, C.byref(b), _dptr(phi, mesh.n_nodes, name="phi", allow_none=True),
                                    gv, C.byref(ov)))
    return list(gv)[:mesh.n_gates], ov.value


def qcad_poisson_residual(mesh: Mesh, bias: dict, phi, R, diag=None, fixed_charge=None):
    b = make_bias(bias)
    st = (C.c_double * 2)()
    _check(_lib.qcad_poisson_residual(mesh.handle, C.byref(b),
                                      _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True),
                                      _dptr(phi, mesh.n_nodes, name="phi"), _dptr(R, mesh.n_nodes, name="R"),
                                      _dptr(diag, mesh.n_nodes, name="diag", allow_none=True), st))
    return st[0], st[1]


def qcad_poisson_jv(mesh: Mesh, bias: dict, phi, v, y, precision=0):
    b = make_bias(bias)
    _check(_lib.qcad_poisson_jv(mesh.handle, C.byref(b), _dptr(phi, mesh.n_nodes, name="phi"),
                                _dptr(v, mesh.n_nodes, name="v"), _dptr(y, mesh.n_nodes, name="y"), int(precision)))


def qcad_poisson_solve(mesh: Mesh, bias: dict, opts=None, phi=None, fixed_charge=None, allow_not_converged=False):
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    rep = SolveReport()
    code = _check(_lib.qcad_poisson_solve(mesh.handle, C.byref(b), C.byref(o),
                                          _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True),
                                          _dptr(phi, mesh.n_nodes, name="phi"), C.byref(rep)), allow_not_converged)
    d = rep.as_dict()
    d["status"] = STATUS[code]
    return d


def qcad_electron_counts(mesh: Mesh, bias: dict, phi, fixed_charge=None):
    b = make_bias(bias)
    N = (C.c_double * max(1, mesh.n_dots))()
    _check(_lib.qcad_electron_counts(mesh.handle, C.byref(b),
                                     _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True),
                                     _dptr(phi, mesh.n_nodes, name="phi"), N))
    return list(N)[:mesh.n_dots]


def qcad_capacitance(mesh: Mesh, bias: dict, gate: int, dV=0.01, opts=None, phi=None, fixed_charge=None):
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    Cf = (C.c_double * max(1, mesh.n_dots))()
    _check(_lib.qcad_capacitance(mesh.handle, C.byref(b), C.byref(o), int(gate), float(dV),
                                 _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True),
                                 _dptr(phi, mesh.n_nodes, name="phi", allow_none=True), Cf))
    return list(Cf)[:mesh.n_dots]


def qcad_adjoint(mesh: Mesh, bias: dict, phi, opts=None, fixed_charge=None, dN_dq=None):
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    out = (C.c_double * max(1, mesh.n_dots * mesh.n_gates))()
    _check(_lib.qcad_adjoint(mesh.handle, C.byref(b), C.byref(o), _dptr(phi, mesh.n_nodes, name="phi"),
                             _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True), out,
                             _dptr(dN_dq, mesh.n_dots * mesh.n_elems, name="dN_dq", allow_none=True)))
    flat = list(out)
    return [flat[d * mesh.n_gates:(d + 1) * mesh.n_gates] for d in range(mesh.n_dots)]


def qcad_schrodinger_apply(mesh: Mesh, bias: dict, phi, m_eff, X, HX=None, MX=None, precision=0):
    b = make_bias(bias)
    me = (C.c_double * 3)(*m_eff)
    nvec = X.shape[0] if X.dim() == 2 else 1
    n = mesh.n_sub_dof * nvec
    _check(_lib.qcad_schrodinger_apply(mesh.handle, C.byref(b), _dptr(phi, mesh.n_nodes, name="phi"), me, nvec,
                                       _dptr(X, n, name="X"), _dptr(HX, n, name="HX", allow_none=True),
                                       _dptr(MX, n, name="MX", allow_none=True), int(precision)))


def qcad_schrodinger_eigs(mesh: Mesh, bias: dict, phi, nev=10, m_eff=(0.19, 0.19, 0.19), tol=1e-7, evecs=None,
                          allow_not_converged=False):
    b = make_bias(bias)
    me = (C.c_double * 3)(*m_eff)
    ev = (C.c_double * nev)()
    rep = SolveReport()
    code = _check(_lib.qcad_schrodinger_eigs(mesh.handle, C.byref(b), _dptr(phi, mesh.n_nodes, name="phi"), int(nev),
                                             me, float(tol), ev,
                                             _dptr(evecs, mesh.n_sub_dof * nev, name="evecs", allow_none=True),
                                             C.byref(rep)), allow_not_converged)
    d = rep.as_dict()
    d["status"] = STATUS[code]
    return list(ev), d


def qcad_calibrate_sheet_charge(mesh: Mesh, bias: dict, pattern, opts=None, dot=0, target=1.0, sigma0=0.0,
                                tol_N=1e-9, max_iter=30, phi=None, theta=None, allow_not_converged=False):
    """Interface sheet density sigma with N_dot = target; returns (sigma, report, phi, theta)."""
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    if phi is None:
        phi = torch.zeros(mesh.n_nodes, dtype=torch.float64, device="cuda")
    if theta is None:
        theta = torch.zeros(mesh.n_elems, dtype=torch.float64, device="cuda")
    sig = C.c_double()
    rep = CalibReport()
    code = _check(_lib.qcad_calibrate_sheet_charge(mesh.handle, C.byref(b), C.byref(o), int(dot), float(target),
                                                   _dptr(pattern, mesh.n_elems, name="pattern"), float(sigma0),
                                                   float(tol_N), int(max_iter), _dptr(phi, mesh.n_nodes, name="phi"),
                                                   _dptr(theta, mesh.n_elems, name="theta"), C.byref(sig),
                                                   C.byref(rep)), allow_not_converged)
    d = rep.as_dict()
    d["status"] = STATUS[code]
    return sig.value, d, phi, theta


def qcad_sp_solve(mesh: Mesh, bias: dict, phi, opts=None, nev=10, m_eff=(0.19, 0.19, 0.19), eig_tol=1e-9,
                  tol_dphi=1e-5, max_iter=60, use_vxc=True, allow_not_converged=False):
    """Self-consistent Schrodinger-Poisson solve (predictor-corrector); phi is written; returns (evals, report)."""
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    me = (C.c_double * 3)(*m_eff)
    ev = (C.c_double * nev)()
    rep = SpReport()
    code = _check(_lib.qcad_sp_solve(mesh.handle, C.byref(b), C.byref(o), int(nev), me, float(eig_tol),
                                     float(tol_dphi), int(max_iter), int(bool(use_vxc)),
                                     _dptr(phi, mesh.n_nodes, name="phi"), ev, C.byref(rep)), allow_not_converged)
    d = rep.as_dict()
    d["status"] = STATUS[code]
    return list(ev), d


def qcad_adjoint_eigs(mesh: Mesh, bias: dict, phi, opts=None, fixed_charge=None, dN_dq=None, nev=10,
                      m_eff=(0.19, 0.19, 0.19), tol=1e-7, evecs=None, allow_not_converged=False):
    """qcad_adjoint and qcad_schrodinger_eigs at phi, run concurrently; returns (dN_dV, evals, eig_report)."""
    b = make_bias(bias)
    o = opts if opts is not None else make_opts()
    out = (C.c_double * max(1, mesh.n_dots * mesh.n_gates))()
    me = (C.c_double * 3)(*m_eff)
    ev = (C.c_double * nev)()
    rep = SolveReport()
    code = _check(_lib.qcad_adjoint_eigs(mesh.handle, C.byref(b), C.byref(o), _dptr(phi, mesh.n_nodes, name="phi"),
                                         _dptr(fixed_charge, mesh.n_elems, name="fixed_charge", allow_none=True), out,
                                         _dptr(dN_dq, mesh.n_dots * mesh.n_elems, name="dN_dq", allow_none=True),
                                         int(nev), me, float(tol), ev,
                                         _dptr(evecs, mesh.n_sub_dof * nev, name="evecs", allow_none=True),
                                         C.byref(rep)), allow_not_converged)
    flat = list(out)
    d = rep.as_dict()
    d["status"] = STATUS[code]
    return [flat[k * mesh.n_gates:(k + 1) * mesh.n_gates] for k in range(mesh.n_dots)], list(ev), d


def qcad_poisson_solve_batch(meshes, biases, opts, phis, allow_not_converged=False):
    n = len(meshes)
    hs = (C.c_void_p * n)(*[m.handle for m in meshes])
    bs_list = [make_bias(b) for b in biases]
    bs = (Bias * n)(*bs_list)
    ps = (C.c_void_p * n)(*[_dptr(p, m.n_nodes, name="phi").value for p, m in zip(phis, meshes)])
    reps = (SolveReport * n)()
    code = _check(_lib.qcad_poisson_solve_batch(n, hs, bs, C.byref(opts), ps, reps), allow_not_converged)
    return [r.as_dict() for r in reps], STATUS[code]


def qcad_adjoint_batch(meshes, biases, opts, phis):
    """Batched adjoint of several meshes; returns [dN/dV of mesh i as n_dots x n_gates lists]."""
    n = len(meshes)
    hs = (C.c_void_p * n)(*[m.handle for m in meshes])
    bs_list = [make_bias(b) for b in biases]
    bs = (Bias * n)(*bs_list)
    ps = (C.c_void_p * n)(*[_dptr(p, m.n_nodes, name="phi").value for p, m in zip(phis, meshes)])
    tot = sum(m.n_dots * m.n_gates for m in meshes)
    out = (C.c_double * max(1, tot))()
    _check(_lib.qcad_adjoint_batch(n, hs, bs, C.byref(opts), ps, out))
    flat, res, off = list(out), [], 0
    for m in meshes:
        res.append([flat[off + k * m.n_gates: off + (k + 1) * m.n_gates] for k in range(m.n_dots)])
        off += m.n_dots * m.n_gates
    return res


def qcad_alu_peaks():
    """Measured FP64 / FP32 FMA throughput (TFLOP/s) and FP64 exp() evaluations per second of the current device."""
    f64, f32, ex = C.c_double(), C.c_double(), C.c_double()
    _check(_lib.qcad_alu_peaks(C.byref(f64), C.byref(f32), C.byref(ex)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value, "fp64_exp_per_s": ex.value}


def qcad_profile_enable(mesh: Mesh, enable=True):
    _check(_lib.qcad_profile_enable(mesh.handle, int(bool(enable))))


def qcad_profile_reset(mesh: Mesh):
    _check(_lib.qcad_profile_reset(mesh.handle))


def qcad_profile_read(mesh: Mesh, kernel_class):
    cls = PROF_CLASSES.get(kernel_class, kernel_class)
    n, ms = C.c_int64(), C.c_double()
    _check(_lib.qcad_profile_read(mesh.handle, int(cls), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def qcad_set_launch(mesh: Mesh, family: int, variant: int, tile_rows: int, z_chunk: int):
    _check(_lib.qcad_set_launch(mesh.handle, int(family), int(variant), int(tile_rows), int(z_chunk)))


def _device_struct(dev: dict):
    """C device description of a workloads dictionary plus the arrays it points to (keep both alive)."""
    L = dev["layers"]
    mats = dev["materials"]
    gates = dev.get("gates", [])
    dots = dev.get("dots", [])
    keep = [(C.c_int * len(L))(*[l["n"] for l in L]), (C.c_double * len(L))(*[l["thickness"] for l in L]),
            (C.c_int * len(L))(*[l["material"] for l in L]),
            (Material * len(mats))(*[Material(*[float(m[k]) if k != "semiconductor" else int(m[k])
                                                for k, _ in Material._fields_]) for m in mats]),
            (Rect * max(1, len(gates)))(*[Rect(g["x0"], g["x1"], g["y0"], g["y1"]) for g in gates]),
            (Box * max(1, len(dots)))(*[Box(d["x0"], d["x1"], d["y0"], d["y1"], d["z0"], d["z1"]) for d in dots])]
    d = Device()
    d.Lx, d.Ly, d.nx, d.ny = dev["Lx"], dev["Ly"], dev["nx"], dev["ny"]
    d.n_layers, d.layer_n, d.layer_thickness, d.layer_material = len(L), keep[0], keep[1], keep[2]
    d.n_materials, d.materials = len(mats), keep[3]
    d.n_gates, d.gates = len(gates), keep[4]
    wf = dev.get("gate_work_function")
    d.gate_work_function_set = 0 if wf is None else 1
    d.gate_work_function = 0.0 if wf is None else float(wf)
    d.bottom_ohmic = int(dev.get("bottom_ohmic", 1))
    d.n_dots, d.dots = len(dots), keep[5]
    S = dev.get("subdomain")
    d.has_subdomain = 0 if S is None else 1
    if S is not None:
        for q, k in enumerate(("i0", "i1", "j0", "j1", "k0", "k1")):
            d.sub[q] = int(S[k])
    # surface terms: charged gates (a gate's "robin" entry) and surface charges
    charged = [ChargedGate(g, float(G["robin"].get("sigma", 0.0)), float(G["robin"].get("d", 10.0)))
               for g, G in enumerate(gates) if G.get("robin")]
    sheets = [SurfaceCharge(S_["z"], S_["x0"], S_["x1"], S_["y0"], S_["y1"], S_["sigma"])
              for S_ in dev.get("surface_charges", [])]
    keep.append((ChargedGate * max(1, len(charged)))(*charged))
    keep.append((SurfaceCharge * max(1, len(sheets)))(*sheets))
    d.n_charged_gates, d.charged_gates = len(charged), keep[6]
    d.n_surface_charges, d.surface_charges = len(sheets), keep[7]
    return d, keep


def qcad_poisson_residual_noalloc(dev: dict, bias: dict, phi, R, fixed_charge=None, stream=None):
    """Allocation-free residual (no mesh object, no device allocation); returns (max |R_i|, sum R_i^2)."""
    d, keep = _device_struct(dev)
    b = make_bias(bias)
    n_nodes = (dev["nx"] + 1) * (dev["ny"] + 1) * (sum(l["n"] for l in dev["layers"]) + 1)
    n_elems = dev["nx"] * dev["ny"] * sum(l["n"] for l in dev["layers"])
    st = (C.c_double * 2)()
    s = C.c_void_p(stream.cuda_stream) if stream is not None else C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(_lib.qcad_poisson_residual_noalloc(C.byref(d), C.byref(b), s,
                                              _dptr(fixed_charge, n_elems, name="fixed_charge", allow_none=True),
                                              _dptr(phi, n_nodes, name="phi"), _dptr(R, n_nodes, name="R"), st))
    return st[0], st[1]


def qcad_launch_count():
    n = C.c_int64()
    _check(_lib.qcad_launch_count(C.byref(n)))
    return n.value


def qcad_launch_info(mesh: Mesh, family: int):
    """(variant, tile_rows, z_chunk, autotuned Chebyshev degree or 0) of a kernel family."""
    v, r, z, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(_lib.qcad_launch_info(mesh.handle, int(family), C.byref(v), C.byref(r), C.byref(z), C.byref(d)))
    return v.value, r.value, z.value, d.value


def qcad_autotune(mesh: Mesh, bias: dict, precision=1):
    """Returns (variant, tile_rows, z_chunk, ms per apply) of the fastest launch shape."""
    b = make_bias(bias)
    v, r, z, t = C.c_int(), C.c_int(), C.c_int(), C.c_float()
    _check(_lib.qcad_autotune(mesh.handle, C.byref(b), int(precision), C.byref(v), C.byref(r), C.byref(z),
                              C.byref(t)))
    return v.value, r.value, z.value, t.value


class QcadDotCharge(torch.autograd.Function):
    """Dot electron counts as a differentiable function of the gate voltages and the fixed charge.

    ``N = QcadDotCharge.apply(V_gate, fixed_charge, mesh, bias, opts)``: V_gate a 1-D tensor of
    the gate voltages (V), fixed_charge a CUDA FP64 tensor of n_elems volume charges (nm^-3) or
    None. Forward: Newton solve of the nonlinear Poisson problem (qcad_poisson_solve) and the
    dot counts (qcad_electron_counts, Sec. III). Backward: one adjoint solve per dot
    (qcad_adjoint) gives dN/dV (n_dots x n_gates) and dN/dtheta (n_dots x n_elems); the
    incoming gradient is contracted with them. The converged potential of the last forward
    call is kept on ctx for the backward pass.
    """

    @staticmethod
    def forward(ctx, V_gate, fixed_charge, mesh, bias, opts=None):
        o = opts if opts is not None else make_opts(precision=1)
        b = dict(bias, V_gate=[float(v) for v in V_gate.detach().double().cpu().tolist()])
        phi = torch.zeros(mesh.n_nodes, dtype=torch.float64, device="cuda")
        fc = fixed_charge.detach() if fixed_charge is not None else None
        qcad_poisson_solve(mesh, b, o, phi, fixed_charge=fc)
        N = qcad_electron_counts(mesh, b, phi, fixed_charge=fc)
        ctx.mesh, ctx.bias, ctx.opts, ctx.phi, ctx.fc = mesh, b, o, phi, fc
        ctx.has_fc = fixed_charge is not None
        return torch.tensor(N, dtype=torch.float64, device=V_gate.device)

    @staticmethod
    def backward(ctx, gN):
        mesh = ctx.mesh
        want_q = ctx.has_fc and ctx.needs_input_grad[1]
        dq = torch.empty(mesh.n_dots * mesh.n_elems, dtype=torch.float64, device="cuda") if want_q else None
        dNdV = qcad_adjoint(mesh, ctx.bias, ctx.phi, ctx.opts, fixed_charge=ctx.fc, dN_dq=dq)
        g = gN.detach().double()
        JV = torch.tensor(dNdV, dtype=torch.float64, device=g.device)
        gV = g @ JV if ctx.needs_input_grad[0] else None
        gq = None
        if want_q:
            gq = g.to(dq.device) @ dq.view(mesh.n_dots, mesh.n_elems)
        return gV, gq, None, None, None
