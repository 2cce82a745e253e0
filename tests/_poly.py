"""Exact polynomial fields for the reproduction pins (no method arithmetic).

u = sum_m c_m x^a_m y^b_m z^c_m with every exponent <= p lies in Q_p, as do
grad u and lambda u - laplace u; HDG with exact integration then reproduces
u, q = grad u and the traces exactly.
"""
import numpy as np


class PolyField:
    def __init__(self, p, rng, terms=4):
        self.exps = rng.integers(0, p + 1, size=(terms, 3))
        self.coef = rng.standard_normal(terms)

    def _mono(self, X, e):
        out = np.ones(len(X))
        for d in range(3):
            if e[d] < 0:
                return np.zeros(len(X))
            out = out * X[:, d] ** e[d]
        return out

    def u(self, X):
        return sum(c * self._mono(X, e) for c, e in zip(self.coef, self.exps))

    def grad(self, X):
        g = np.zeros((len(X), 3))
        for c, e in zip(self.coef, self.exps):
            for d in range(3):
                if e[d] > 0:
                    ee = e.copy(); ee[d] -= 1
                    g[:, d] += c * e[d] * self._mono(X, ee)
        return g

    def lap(self, X):
        out = np.zeros(len(X))
        for c, e in zip(self.coef, self.exps):
            for d in range(3):
                if e[d] > 1:
                    ee = e.copy(); ee[d] -= 2
                    out += c * e[d] * (e[d] - 1) * self._mono(X, ee)
        return out


def boundary_data(problem, field):
    """g_D = u on Dirichlet sides, g_N = n . grad u on Neumann sides."""
    m = problem.mesh
    Xb, nrm = m.bdry_coords(problem.m1.nodes)
    out = np.zeros(m.n_bdry)
    for side in range(6):
        lo = m.side_offset[side] * m.n2
        d = side // 2
        a, b = [(1, 2), (0, 2), (0, 1)][d]
        hi = lo + m.ne[a] * m.ne[b] * m.n2
        sl = slice(lo, hi)
        if m.bc[side] == 0:
            out[sl] = field.u(Xb[sl])
        else:
            out[sl] = np.sum(field.grad(Xb[sl]) * nrm[sl], axis=1)
    return out
