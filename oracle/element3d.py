"""Dense 3D element system and its condensation (test infrastructure only).

Sec. 3.2-3.3 of arXiv:2007.11891.  An element of widths (h1, h2, h3) has the
metric factors d0 = h1 h2 h3 / 8, d_i = d0 (2 / h_i)^2 and the penalty
tau_{i,e} = 2 tau_hat / h_i.  Its unknowns are ordered
(u, q1, q2, q3, ut1, ut2, ut3):

* u, q_i: n^3 nodal values, index i + n j + n^2 k (x1 fastest);
* ut1: shape 2 x n x n (face side s fastest), index s + 2 (j + n k);
* ut2: shape n x 2 x n, index i + n (s + 2 k);
* ut3: shape n x n x 2, index i + n (j + n s);

following Tab. (hdg_matrices_threed), where C (x) B (x) A lets A act on the
fastest index (Eq. (tp_definition)); ``np.kron(B, A)`` is exactly that.
Side s = 0 is the face at the lower coordinate, s = 1 the upper one.
"""

import numpy as np
import scipy.linalg as sla


def kron3(c, b, a):
    """C (x) B (x) A with A acting on the fastest index."""
    return np.kron(c, np.kron(b, a))


def metric(h):
    h1, h2, h3 = (float(v) for v in h)
    d0 = h1 * h2 * h3 / 8.0
    return d0, d0 * (2.0 / h1) ** 2, d0 * (2.0 / h2) ** 2, d0 * (2.0 / h3) ** 2


def element_blocks(m1, h):
    """Tensor-product element matrices of Tab. (hdg_matrices_threed)."""
    M, D, E, G, B, C = m1.M, m1.D, m1.E, m1.G, m1.B, m1.C
    h1, h2, h3 = (float(v) for v in h)
    d0, d1, d2, d3 = metric(h)
    blk = {}
    blk["M"] = d0 * kron3(M, M, M)
    blk["D1"] = h1 / 2 * d1 * kron3(M, M, D)
    blk["D2"] = h2 / 2 * d2 * kron3(M, D, M)
    blk["D3"] = h3 / 2 * d3 * kron3(D, M, M)
    blk["E"] = d1 * kron3(M, M, E) + d2 * kron3(M, E, M) + d3 * kron3(E, M, M)
    blk["G1"] = d1 * kron3(M, M, G)
    blk["G2"] = d2 * kron3(M, G, M)
    blk["G3"] = d3 * kron3(G, M, M)
    blk["B1"] = d1 * kron3(M, M, B)
    blk["B2"] = d2 * kron3(M, B, M)
    blk["B3"] = d3 * kron3(B, M, M)
    blk["C1"] = h1 / 2 * d1 * kron3(M, M, C)
    blk["C2"] = h2 / 2 * d2 * kron3(M, C, M)
    blk["C3"] = h3 / 2 * d3 * kron3(C, M, M)
    return blk


def element_system(m1, h, lam):
    """Dense matrix of Eq. (ldg_element_operator_threed), size 4n^3 + 6n^2."""
    b = element_blocks(m1, h)
    n3 = m1.n ** 3
    f2 = 2 * m1.n ** 2
    N = 4 * n3 + 3 * f2
    A = np.zeros((N, N))
    U, Q = slice(0, n3), [slice((1 + d) * n3, (2 + d) * n3) for d in range(3)]
    T = [slice(4 * n3 + d * f2, 4 * n3 + (d + 1) * f2) for d in range(3)]
    A[U, U] = lam * b["M"] + b["E"]
    for d in range(3):
        Dd, Bd, Cd, Gd = b["D%d" % (d + 1)], b["B%d" % (d + 1)], b["C%d" % (d + 1)], b["G%d" % (d + 1)]
        A[U, Q[d]] = -Dd
        A[Q[d], U] = -Dd.T
        A[Q[d], Q[d]] = -b["M"]
        A[U, T[d]] = Bd
        A[T[d], U] = Bd.T
        A[Q[d], T[d]] = Cd
        A[T[d], Q[d]] = Cd.T
        A[T[d], T[d]] = Gd
    return A


def split(m1, system):
    """(A_e, R_e, G_e) of Eq. (hdg_operator): volume block, coupling, trace block."""
    nv = 4 * m1.n ** 3
    return system[:nv, :nv], system[:nv, nv:], system[nv:, nv:]


def condense_lu(m1, h, lam):
    """Tier O1: K_e = G_e - R_e^T A_e^{-1} R_e by dense LU with pivoting."""
    A, R, G = split(m1, element_system(m1, h, lam))
    lu = sla.lu_factor(A)
    return G - R.T @ sla.lu_solve(lu, R)


def condense_q_eliminated(m1, h, lam):
    """Tier O2: q eliminated first, no eigenbasis.

    Z^{-1} = lam d0 M(x)M(x)M + d1 M(x)M(x)L + d2 M(x)L(x)M + d3 L(x)M(x)M
    (Eq. (element_operator_u_q_3d)); with P_e R_e per direction
    PR_d = B_{d,e} - D_{d,e} M_e^{-1} C_{d,e},
    K_e = G_e + blkdiag(C_d^T M_e^{-1} C_d) - PR^T Z PR
    (Eq. (hdg_operator_factorized) before the fast diagonalisation).
    """
    M, L = m1.M, m1.L
    d0, d1, d2, d3 = metric(h)
    b = element_blocks(m1, h)
    Zinv = (lam * d0 * kron3(M, M, M) + d1 * kron3(M, M, L)
            + d2 * kron3(M, L, M) + d3 * kron3(L, M, M))
    Me = b["M"]
    PR = []
    face = []
    for d in (1, 2, 3):
        Cd = b["C%d" % d]
        MinvC = np.linalg.solve(Me, Cd)
        PR.append(b["B%d" % d] - b["D%d" % d] @ MinvC)
        face.append(b["G%d" % d] + Cd.T @ MinvC)
    PR = np.hstack(PR)
    chol = sla.cho_factor(Zinv)
    K = sla.block_diag(*face) - PR.T @ sla.cho_solve(chol, PR)
    return K


def condense(m1, h, lam, tier=None):
    """K_e for widths h; tier 'O1' (LU) or 'O2' (q eliminated).  Default: O1
    while the volume block is small, O2 above."""
    if tier is None:
        tier = "O1" if m1.n <= 5 else "O2"
    if tier == "O1":
        return condense_lu(m1, h, lam)
    if tier == "O2":
        return condense_q_eliminated(m1, h, lam)
    raise ValueError(tier)


def volume_solve_factors(m1, h, lam):
    """Pieces for right-hand side and recovery: (lu(A_e), R_e, M_e)."""
    A, R, _ = split(m1, element_system(m1, h, lam))
    return sla.lu_factor(A), R, element_blocks(m1, h)["M"]
