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
