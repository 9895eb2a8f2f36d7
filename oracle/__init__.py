"""FP64 CPU oracle for MCTDHF on an adaptive finite-element mesh (arXiv 2301.02387).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the GPU library computes, built from assembled sparse
matrices in float64 / complex128 (dense PyTorch CPU maps in ``step_grad``).
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA
library: the two share no code, tables or constants.

Modules and the parts of the paper they follow:

* ``gll``      - Gauss-Lobatto-Legendre nodes/weights and the 1D Lagrange basis
                 (Sec. 3.1, the FEDVR-like tensor-product basis and GLL quadrature).
* ``mesh``     - coarse uniform cubes refined by halving toward the nuclei,
                 2:1 vertex balance, global support points, hanging-node
                 ("bridged" function) constraints (Sec. 3.1).
* ``fem``      - assembled stiffness, lumped mass, pointwise potentials and the
                 one-body Hamiltonian matrix (Sec. 3.1, Eq. discretized_eom).
* ``rows``     - selected rows of the same operators formed cell by cell, for
                 meshes too large to assemble on the host (Sec. 3.1).
* ``poisson``  - pair-density right-hand sides, multipole Dirichlet data and
                 the Poisson solve for the mean fields (Sec. 3.1, Eq. mean-field).
* ``krylov``   - short-iterative Arnoldi propagator (Sec. 3.2).
* ``ci``       - determinant space, excitation operators, RDMs, CI Hamiltonian
                 (Sec. 2, Eqs. ci_eom and the RDM definitions).
* ``mctdhf``   - the packed orbital operator G and one MCTDHF time step
                 (Sec. 3.2, Eq. packed_orb_eom).
* ``adjoint``  - dense one-electron step, its tangent and adjoint (the
                 differentiation form in the one-electron limit; Sec. 3.2).
* ``step_grad`` - the full MCTDHF step as dense PyTorch maps on tiny meshes and
                 the gradient of a dipole functional with respect to the field by
                 automatic differentiation (the differentiation form beyond the
                 one-electron limit; Sec. 2, Sec. 3.2).
* ``rows``     - selected rows of the assembled operators, formed cell by cell
                 (parity at sizes whose assembled matrices would not fit).

Every function that has no independent pin says "parity unpinned" in its
docstring.
"""
