"""CPU FP64 oracle for the statically condensed HDG operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

What it computes is the plain definition of the method (Huismann, Stiller,
Froehlich, "Linearizing the hybridizable discontinuous Galerkin method: a
linearly scaling operator", arXiv:2007.11891):

* ``basis1d``   -- nodes, quadrature and the standard 1D matrices M, D, E, G,
                   B, C, L of Eq. (element_matrices), Sec. 2.2.
* ``element3d`` -- the dense 7x7-block LDG element system of
                   Eq. (ldg_element_operator_threed) built from the tensor
                   products of Tab. (hdg_matrices_threed), Sec. 3.2, and its
                   Schur complement K_e = G_e - R_e^T A_e^{-1} R_e of
                   Eq. (hdg_operator), Sec. 3.3, by dense LU (tier O1) or with
                   q eliminated first via Eq. (element_operator_u_q_3d) /
                   Eq. (hdg_operator_factorized) without the eigenbasis
                   (tier O2).
* ``mesh``      -- the Cartesian mesh, its face-wise trace storage and the
                   gather/scatter Q_e of Eq. (hdg_system).
* ``solver``    -- the global apply sum_e Q_e^T K_e Q_e, the right-hand side
                   and recovery of Alg. (hdg_cg) (signs from block
                   elimination), plain CG, and the discrete adjoint.
* ``lowdim``    -- the same construction in one and two directions: the 1D
                   system of Eq. (ldg_element_operator) and its Schur
                   complement Eq. (hdg_operator_oned), the 2D system from the
                   blocks of Tab. (hdg_matrices_threed) with one direction
                   fewer, global apply and a direct solve.

* ``facebasis`` -- the face eigenbasis that defines the library's
                   transformed trace basis (Eq. (generalized_eigenvalue_
                   decomposition) with the documented parity, order and sign
                   convention), used only to express the dense K in that
                   basis for comparisons: K-hat = T^T K T face by face.

It shares no code with the CUDA path: its operator uses no
eigen-decomposition, no sum factorisation and no fast diagonalisation
(``facebasis`` changes the basis of the dense operator, nothing else).  Every pin it is checked against
lives in ``tests/test_oracle_*.py``.
"""

from . import basis1d, element3d, facebasis, lowdim, mesh, solver  # noqa: F401
