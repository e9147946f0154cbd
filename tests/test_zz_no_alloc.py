"""The allocation-free residual entry point agrees with the regular one and with the oracle.

Callers that cannot allocate device memory (inside another framework's
allocator or memory pool, in allocation-free loops) use
qcad_poisson_residual_noalloc; it keeps its scratch in a static device array
shared by all calls. This file is collected last so that a failure here does
not hide the other tests; it passes both alone in a fresh process and after
them.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle.poisson import PoissonProblem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_7561_gb300 as qcad
    return qcad


def _phi(q, dev, seed):
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_contact_values(m, dev["bias"], phi)
    g = torch.Generator(device="cpu").manual_seed(seed)
    phi += 0.05 * torch.randn(m.n_nodes, generator=g, dtype=torch.float64).cuda()
    q.qcad_contact_values(m, dev["bias"], phi)  # Dirichlet entries back to their values
    return m, phi


@pytest.mark.parametrize("with_theta", [False, True], ids=["no_theta", "fixed_charge"])
@pytest.mark.parametrize("dev", [W.five_gate_device(n=(37, 33, 21), T=4.0), W.get("mos_cap_16x16x32")],
                         ids=["dqd_37x33x21", "mos_cap"])
def test_noalloc_residual_matches_regular_twice(q, dev, with_theta):
    m, phi1 = _phi(q, dev, 1)
    _, phi2 = _phi(q, dev, 2)
    theta = None
    if with_theta:  # the per-element fixed charge of the differentiation form, on this mesh
        theta = torch.tensor(W.interface_fixed_charge(dev, seed=5), dtype=torch.float64, device="cuda")
    P = PoissonProblem(dev, fixed_charge=None if theta is None else theta.cpu().numpy())
    for phi in (phi1, phi2):  # two calls in a row: leftover scratch from the first must not leak
        R_ref = torch.empty_like(phi)
        ref = q.qcad_poisson_residual(m, dev["bias"], phi, R_ref, fixed_charge=theta)
        R = torch.full_like(phi, float("nan"))
        st = q.qcad_poisson_residual_noalloc(dev, dev["bias"], phi, R, fixed_charge=theta)
        scale = torch.max(torch.abs(R_ref)).item()
        assert torch.isfinite(R).all()
        assert torch.max(torch.abs(R - R_ref)).item() <= 1e-12 * scale
        assert abs(st[0] - ref[0]) <= 1e-12 * scale
        assert abs(st[1] - ref[1]) <= 1e-10 * ref[1]
        # and the oracle's residual of Eq. PoissonWeakForm at the same potential, node by node
        Ro = P.residual(phi.cpu().numpy())
        assert np.max(np.abs(R.cpu().numpy() - Ro)) <= 1e-12 * np.max(np.abs(Ro))


def test_noalloc_rejects_oversized_mesh(q):
    # the top-plane contact mask alone (2049^2 bytes) exceeds the 2 MiB scratch
    dev = W.five_gate_device(n=(2048, 2048, 4), T=4.0, with_subdomain=False)
    n = W.n_nodes(dev)
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    R = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QcadError) as e:
        q.qcad_poisson_residual_noalloc(dev, dev["bias"], phi, R)
    assert e.value.code == 1 and "scratch" in str(e.value)
    assert torch.all(R == 0)
