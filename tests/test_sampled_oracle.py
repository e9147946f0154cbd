"""The sampled oracle residual (tests/sampled_oracle.py) against the assembled oracle (CPU)."""
import numpy as np
import pytest

import workloads as W
from oracle.poisson import PoissonProblem
from sampled_oracle import SampledPoisson


@pytest.mark.parametrize("make", [lambda: W.five_gate_device(n=(24, 20, 16), T=4.0),
                                  lambda: W.get("mos_cap_16x16x32")], ids=["dqd", "moscap"])
def test_sampled_residual_reproduces_the_oracle(make):
    dev = make()
    theta = np.array(W.interface_fixed_charge(dev, seed=3)) if dev.get("dots") else None
    P = PoissonProblem(dev, fixed_charge=theta)
    S = SampledPoisson(dev, fixed_charge=theta)
    m = P.mesh
    assert np.array_equal(S.is_dirichlet(m.ni, m.nj, m.nk), P.dir)
    rng = np.random.default_rng(1)
    phi = P.initial_guess() + 0.02 * rng.standard_normal(m.n_nodes)
    R = P.residual(phi, full=True)
    ijk = np.stack([m.ni, m.nj, m.nk], axis=1)
    Rs = S.residual_at(phi, ijk)
    assert np.max(np.abs(Rs - R)) <= 1e-12 * np.max(np.abs(R))
    sub = S.sample_nodes(50, seed=2)
    assert not np.any(P.dir[S.node(sub[:, 0], sub[:, 1], sub[:, 2])])
    assert np.max(np.abs(S.residual_at(phi, sub) - R[S.node(sub[:, 0], sub[:, 1], sub[:, 2])])) <= \
        1e-12 * np.max(np.abs(R))


def test_stored_fullsize_oracle_solution_is_a_solution():
    # the oracle's stored 128 x 128 x 96 solution (tests/golden, written by a script that calls
    # only the oracle) zeroes the oracle's residual at sampled free nodes, carries the device's
    # gate voltages and lists its eigenvalues in ascending order
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dqd_128x128x96_4K_oracle.npz")
    ref = np.load(path)
    dev = W.get("dqd_128x128x96_4K")
    assert np.array_equal(ref["V_gate"], np.array(dev["bias"]["V_gate"]))
    S = SampledPoisson(dev)
    phi = ref["phi"]
    assert phi.shape == (S.nxn * S.nyn * S.nzn,)
    ijk = S.sample_nodes(300, seed=31)
    assert np.max(np.abs(S.residual_at(phi, ijk))) < 1e-10
    assert np.all(np.diff(ref["evals"]) > 0) and ref["counts"].shape == (2,) and ref["dN_dV"].shape == (2, 5)
