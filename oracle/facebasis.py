"""The face eigenbasis that defines the library's transformed trace basis
(test infrastructure only).

The oracle's operator itself uses no eigen-decomposition (``solver`` applies
the dense condensed K).  This module only writes down, from its definition,
the basis in which the library's ``HDG_BASIS_TRANSFORMED`` traces are
expressed, so that the dense K can be compared with the library's K-hat
entry by entry:

* Sec. 4.1, Eq. (generalized_eigenvalue_decomposition): S^T M S = I,
  S^T L S = Lambda with L = E + D M^-1 D^T (Eq. (element_matrices)).
* The GLL points are mirror symmetric, so M and L commute with the reversal
  J of the nodes and every eigenvector can be taken even (J s = s) or odd
  (J s = -s).  The generalised problem is solved on the even and on the odd
  subspace separately (a library eigen-solver on each projected pair), which
  keeps the parity exact even where an even and an odd eigenvalue coincide.
* Order: even modes first, then odd modes, each by increasing eigenvalue.
* Sign: B_S[m][0] > 0 for every mode, with B_S = S^T B - S^T D M^-1 C
  (Eq. (hdg_bs)).
* On a face (n x n nodes, lower axis fastest) the nodal traces are
  ut = (S (x) S) ut-hat, mode (m1, m2) stored at m1 + n m2 (Sec. 4.2), and
  K-hat = (S (x) S)^T K (S (x) S) face block by face block.
"""

import numpy as np
import scipy.linalg as sla


def face_eigenbasis(m1):
    """(S, Lambda, B_S) of a ``Matrices1D`` by the convention above;
    S[i, m] is node i of mode m, B_S is n x 2."""
    n = m1.n
    J = np.eye(n)[::-1]
    I = np.eye(n)
    cols, lams = [], []
    for sgn in (1.0, -1.0):
        # orthonormal basis of the subspace {v : J v = sgn v}
        P, sv, _ = np.linalg.svd(0.5 * (I + sgn * J))
        P = P[:, sv > 0.5]
        if P.shape[1] == 0:
            continue
        lam, W = sla.eigh(P.T @ m1.L @ P, P.T @ m1.M @ P)   # W^T (P^T M P) W = I
        order = np.argsort(lam)
        cols.append(P @ W[:, order])
        lams.append(lam[order])
    S = np.hstack(cols)
    Lam = np.concatenate(lams)
    BS = S.T @ m1.B - S.T @ m1.D @ np.linalg.solve(m1.M, m1.C)
    flip = np.where(BS[:, 0] < 0.0, -1.0, 1.0)
    return S * flip[None, :], Lam, BS * flip[:, None]


def face_transform(m1):
    """T = S (x) S: nodal face values = T @ face-mode coefficients."""
    S, _, _ = face_eigenbasis(m1)
    return np.kron(S, S)


def to_nodal(problem, xhat):
    """Nodal traces of transformed ones (every unknown face, n^2 values each)."""
    T = face_transform(problem.m1)
    n2 = problem.mesh.n2
    return (np.asarray(xhat, dtype=np.float64).reshape(-1, n2) @ T.T).ravel()


def to_transformed(problem, y):
    """T^T y face by face: the transformed image of a nodal residual."""
    T = face_transform(problem.m1)
    n2 = problem.mesh.n2
    return (np.asarray(y, dtype=np.float64).reshape(-1, n2) @ T).ravel()


def apply_transformed(problem, xhat):
    """K-hat x-hat = T^T K T x-hat with the oracle's dense condensed K."""
    return to_transformed(problem, problem.apply(to_nodal(problem, xhat)))


def abs_element_sum(problem, xhat):
    """sum_e Q_e^T |K-hat_e| Q_e |x-hat|: a bound on the sum of the absolute
    values of the (up to two) element contributions to each output entry,
    for error bounds of arithmetic that rounds each contribution.  K-hat_e is
    the element's dense K_e with each of its six faces transformed by
    T = S (x) S."""
    m = problem.mesh
    T = face_transform(problem.m1)
    n2 = m.n2
    ax = np.abs(np.asarray(xhat, dtype=np.float64))
    out = np.zeros(m.n_trace)
    for e in m.elements():
        loc = m.local_trace_map(e)
        faces = {}
        for li, (kind, g) in enumerate(loc):
            faces.setdefault((kind, g // n2), np.zeros(n2, dtype=np.int64))[g % n2] = li
        Tloc = np.zeros((len(loc), len(loc)))
        for pos in faces.values():
            Tloc[np.ix_(pos, pos)] = T
        Khat = np.abs(Tloc.T @ problem.K_e(e) @ Tloc)
        xe = np.zeros(len(loc))
        for (kind, f), pos in faces.items():
            if kind == "u":
                xe[pos] = ax[f * n2:(f + 1) * n2]
        ye = Khat @ xe
        for (kind, f), pos in faces.items():
            if kind == "u":
                out[f * n2:(f + 1) * n2] += ye[pos]
    return out
