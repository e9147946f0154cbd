"""FP64 CPU oracle for the QCAD finite-element quantum-dot solver path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or runs
this package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA library; the only
module both sides read is ``workloads`` (seeded input descriptions, which hold
none of the method's arithmetic).

The oracle is deliberately plain: numpy/scipy, FP64, an assembled sparse
matrix and direct (SuperLU) or conjugate-gradient linear solves, written in
the paper's order and notation (Gao et al., "QCAD Simulation and Optimization
of Semiconductor Quantum Dots", arXiv:1403.7561):

- ``physics``      carrier statistics, ionization, reference potential and
                   contact potentials (Sec. II.A, Eqs. 1-16)
- ``mesh``         tensor-product hexahedral mesh, contacts, regions
- ``fem``          Q1 element quadrature and sparse assembly (Eq. 11, Eq. 18)
- ``poisson``      nonlinear Poisson Newton solve (Sec. II.A)
- ``schrodinger``  effective-mass Schrodinger eigenpairs (Sec. II.B, Eq. 26)
- ``boundary``     surface terms: charged gates (Robin) and surface charges
                   (Sec. II.A.4, Eq. NeuBC4fc)
- ``capacitance``  dot electron counts, finite-difference capacitance
                   (Sec. III) and the adjoint sensitivities
- ``sp``           self-consistent Schrodinger-Poisson predictor-corrector
                   loop (Sec. II.C)

Parity status of every function is listed in its docstring ("pinned by ...").
"""
