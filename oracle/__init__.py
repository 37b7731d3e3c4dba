"""CPU FP64 oracle for the polarized-traces Helmholtz solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run anything in this
package.  The product (the CUDA library and its Python binding) never calls
it and shares no code with it; the only shared module is the seeded input
generator ``paper_1801_08655_gb300.workloads``, which holds no arithmetic of
the method.

Contents
--------
``discretization``  the 7-point FD Helmholtz operator with PML by complex
                    coordinate stretching, in a complex-symmetric form
                    (Formulation section, Eqs. 1, 3-5 and the sigma profile).
``direct``          the plain definition of the answer: a global FP64 sparse
                    direct solve (SuperLU on a nested-dissection-ordered
                    matrix) and a dense LAPACK solve for tiny grids.
``polarized``       a slow, step-by-step model of the method itself (layer
                    decomposition, local solves, the SIE matrix, the blocks of
                    the polarized system, the Gauss-Seidel preconditioner,
                    GMRES and the local reconstruction; Algorithms 1-9), and
                    the explicit trace-to-trace blocks, used to pin
                    intermediate quantities.
``multifrontal``    the global solve again, organised as a multifrontal
                    factorization with a generic symbolic phase, for grids too
                    large for SuperLU (96^3 - 160^3).

Pins (what each function is checked against, in ``tests/test_oracle_*.py``):
dense LAPACK solve, an independent Kronecker-product assembly, exact complex
symmetry, discrete reciprocity, residual <= 1e-12, convergence to the free
space Green's function -exp(ikr)/(4 pi r), exactness of the Green's
representation formula (Theorem 1 of the 2D polarized-traces paper, cited
in the SIE section), the exact traces solving the SIE, the reductive case of
exact local Green's functions, reciprocity of the explicit trace blocks, and
the special cases L = 1 and L = 2.
"""
