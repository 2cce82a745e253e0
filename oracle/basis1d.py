"""1D building blocks of the oracle (test infrastructure only).

Sec. 2.2 of arXiv:2007.11891: a nodal basis {phi_i}_{i=0..p} on the standard
element [-1, 1], the face basis (phi-tilde_1, phi-tilde_2) with
phi-tilde_1(-1) = 1, phi-tilde_1(1) = 0, phi-tilde_2(-1) = 0,
phi-tilde_2(1) = 1 (the printed "phi_1(1) = 1" is a typo for phi-tilde_2), and
the standard matrices of Eq. (element_matrices):

    M_ij = int phi_i phi_j            D_ij = int phi_i d(phi_j)/dxi
    E_ij = +tau_hat [phi_i phi_j]     G_ij = +tau_hat [phit_i phit_j]
    B_ij = -tau_hat [phi_i phit_j]    C_ij = [phi_i phit_j n]
    L    = E + D M^{-1} D^T

where [.] sums over the two end points xi = -1 (outer normal n = -1) and
xi = +1 (n = +1).  The nodal basis is the Lagrange basis on the
Gauss-Lobatto-Legendre (GLL) points.  M is integrated exactly (Gauss rule
with p+2 points) by default; ``mass="gll"`` gives the GLL-lumped diagonal
mass the paper mentions for HDG-TP (Sec. 4.1).
"""

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(q):
    """Gauss-Legendre rule with q points on [-1, 1] (library routine)."""
    x, w = npleg.leggauss(q)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gll_nodes(n):
    """GLL points and weights for n = p+1 >= 2 points.

    The interior points are the roots of P_p'; the weights are
    w_i = 2 / (p (p+1) P_p(x_i)^2).  Roots from the companion matrix are
    polished by Newton steps on P_p'.
    """
    if n < 2:
        raise ValueError("need at least two GLL points")
    p = n - 1
    Pp = npleg.Legendre.basis(p)
    dP = Pp.deriv(1)
    ddP = Pp.deriv(2)
    interior = np.sort(np.real(dP.roots())) if p >= 2 else np.zeros(0)
    for _ in range(4):
        interior = interior - dP(interior) / ddP(interior)
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (p * (p + 1) * Pp(x) ** 2)
    return x, w


def lagrange(nodes, t):
    """Values V[q, i] = phi_i(t_q) and derivatives dV[q, i] = phi_i'(t_q).

    phi_i(t) = prod_{m != i} (t - x_m) / (x_i - x_m); its derivative is the
    sum over l != i of 1/(x_i - x_l) times the product over m != i, l.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(t), n))
    dV = np.zeros((len(t), n))
    for i in range(n):
        for m in range(n):
            if m != i:
                V[:, i] *= (t - nodes[m]) / (nodes[i] - nodes[m])
        for l in range(n):
            if l == i:
                continue
            term = np.full(len(t), 1.0 / (nodes[i] - nodes[l]))
            for m in range(n):
                if m != i and m != l:
                    term = term * (t - nodes[m]) / (nodes[i] - nodes[m])
            dV[:, i] += term
    return V, dV


class Matrices1D:
    """Standard-element matrices of Eq. (element_matrices) for degree p.

    Attributes: n, nodes, M, D, E, G, B, C, L, tau_hat, mass.
    B and C are n x 2 (column 0: left face xi=-1, column 1: right face).
    """

    def __init__(self, p, tau_hat, mass="exact"):
        if p < 1:
            raise ValueError("degree p must be >= 1")
        self.p = p
        self.n = n = p + 1
        self.tau_hat = float(tau_hat)
        self.mass = mass
        self.nodes, self.gll_weights = gll_nodes(n)
        tq, wq = gauss_legendre(n + 1)   # exact for degree 2n+1 >= 2p
        V, dV = lagrange(self.nodes, tq)
        if mass == "exact":
            self.M = V.T @ (wq[:, None] * V)
        elif mass == "gll":
            self.M = np.diag(self.gll_weights)
        else:
            raise ValueError("mass must be 'exact' or 'gll'")
        # D_ij = int phi_i phi_j'  (degree 2p-1: exact with n+1 Gauss points)
        self.D = V.T @ (wq[:, None] * dV)
        ends, _ = lagrange(self.nodes, np.array([-1.0, 1.0]))
        phi_m, phi_p = ends[0], ends[1]            # phi_i(-1), phi_i(+1)
        # face basis values: phit_1 = (1 at -1, 0 at +1), phit_2 = (0, 1)
        phit = np.array([[1.0, 0.0], [0.0, 1.0]])  # phit[x_index, j]
        normal = np.array([-1.0, 1.0])
        vol_at = np.stack([phi_m, phi_p])          # vol_at[x_index, i]
        t = self.tau_hat
        self.E = t * (np.outer(phi_m, phi_m) + np.outer(phi_p, phi_p))
        self.G = t * (phit.T @ phit)
        self.B = -t * (vol_at.T @ phit)
        self.C = vol_at.T @ (normal[:, None] * phit)
        self.L = self.E + self.D @ np.linalg.solve(self.M, self.D.T)
