"""Write the oracle's full-size solution of the 128x128x96 five-gate device at 4 K.

Calls only ``oracle/`` and the seeded inputs of ``workloads/``: the Newton solve
of Sec. II.A.3 to ||R||_inf < 1e-10 V*nm and ||delta phi||_inf < 1e-10 V, the dot
electron counts and the adjoint dN/dV of Sec. III, and the 10 lowest eigenvalues
of Eq. SchrodEqnWeakForm on the 64x64x32-element subdomain (ARPACK shift-invert).

Output: dqd_128x128x96_4K_oracle.npz beside this file (phi as float64, one value
per node in node order i + (nx+1)(j + (ny+1)k)). Runs for about an hour on one
core; the GPU parity tests read the file and never run this script.

    python tests/golden/make_dqd_128x128x96_oracle.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import capacitance as OC  # noqa: E402
from oracle import schrodinger as OS  # noqa: E402
from oracle.poisson import PoissonProblem  # noqa: E402

NAME = "dqd_128x128x96_4K"


def main(out=os.path.join(HERE, NAME + "_oracle.npz")):
    t0 = time.time()
    dev = W.get(NAME)
    P = PoissonProblem(dev)
    print("problem built %.0f s, %d nodes" % (time.time() - t0, P.mesh.n_nodes), flush=True)
    phi, rep = P.solve(verbose=True)
    assert rep["converged"], rep
    print("newton done %.0f s" % (time.time() - t0), flush=True)
    counts = OC.electron_counts(P, phi)
    dN_dV, _ = OC.adjoint(P, phi)
    print("adjoint done %.0f s" % (time.time() - t0), flush=True)
    E, _, _, _, _ = OS.solve_device(P, phi, nev=10)
    print("eigs done %.0f s" % (time.time() - t0), flush=True)
    np.savez_compressed(out, phi=phi, evals=E, counts=counts, dN_dV=dN_dV,
                        newton_iters=rep["newton_iters"], res_inf=rep["res_inf"], dphi_inf=rep["dphi_inf"],
                        V_gate=np.array(dev["bias"]["V_gate"]))
    print("wrote", out, "%.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    main(*sys.argv[1:])
