"""One- and two-dimensional condensed HDG systems (test infrastructure only).

arXiv:2007.11891, Sec. 2.2: the 1D element system of
Eq. (ldg_element_operator) with the element matrices of
Eq. (element_matrices), its Schur complement K_e = G_e - R_e^T A_e^{-1} R_e
(Eq. (hdg_operator_oned)), and the same construction on rectangles: the
tensor-product blocks of Tab. (hdg_matrices_threed) with one direction
fewer.  For dim directions and widths h_1..h_dim the metric factors are
d0 = prod(h_d / 2) and d_i = d0 (2 / h_i)^2 (in 1D: d0 = h/2, d1 = 2/h, so
M_e = h/2 M, E_e = 2/h E, G_e = 2/h G, B_e = 2/h B, D_e = D, C_e = C, as in
Eq. (element_matrices)).

Element unknowns (u, q_1..q_dim, ut_1..ut_dim): u and q_i have n^dim nodal
values (x1 fastest); ut_i has the face side s in place of the direction-i
node index (2 n^(dim-1) values), which is what the Kronecker products of
the blocks produce.

Global trace layout (the library's documented layout for these meshes):
faces normal to direction d lie on grid planes 0..N_d; a plane is an
unknown unless it is a boundary plane of a Dirichlet side.  Block d holds
the unknown planes lo_d..hi_d in order; in 2D each plane holds N_other
faces (one per element along the other axis) of n nodes; in 1D each plane
is one face of one node.  Blocks are concatenated d = 0, then 1.  Boundary
data: sides (x1-, x1+[, x2-, x2+]), each N_other faces of n^(dim-1) nodes.
"""

import itertools

import numpy as np
import scipy.linalg as sla

from .basis1d import Matrices1D

DIRICHLET = 0
NEUMANN = 1


def kron_dirs(mats):
    """Kronecker product with mats[0] acting on the fastest index (x1)."""
    out = mats[-1]
    for m in reversed(mats[:-1]):
        out = np.kron(out, m)
    return out


def metric(h):
    h = [float(v) for v in h]
    d0 = float(np.prod([v / 2.0 for v in h]))
    return d0, [d0 * (2.0 / v) ** 2 for v in h]


def element_system(m1, h, lam):
    """Dense element matrix for dim = len(h) directions; the blocks are those
    of Eq. (ldg_element_operator) (1D) / Tab. (hdg_matrices_threed) reduced
    to dim directions."""
    dim = len(h)
    M = m1.M
    d0, dd = metric(h)

    def along(i, X):
        return kron_dirs([X if d == i else M for d in range(dim)])

    nv = m1.n ** dim
    nf = 2 * m1.n ** (dim - 1)
    N = (1 + dim) * nv + dim * nf
    A = np.zeros((N, N))
    Me = d0 * kron_dirs([M] * dim)
    U = slice(0, nv)
    A[U, U] = lam * Me + sum(dd[i] * along(i, m1.E) for i in range(dim))
    for i in range(dim):
        Q = slice((1 + i) * nv, (2 + i) * nv)
        T = slice((1 + dim) * nv + i * nf, (1 + dim) * nv + (i + 1) * nf)
        Di = h[i] / 2.0 * dd[i] * along(i, m1.D)
        Bi = dd[i] * along(i, m1.B)
        Ci = h[i] / 2.0 * dd[i] * along(i, m1.C)
        A[U, Q] = -Di
        A[Q, U] = -Di.T
        A[Q, Q] = -Me
        A[U, T] = Bi
        A[T, U] = Bi.T
        A[Q, T] = Ci
        A[T, Q] = Ci.T
        A[T, T] = dd[i] * along(i, m1.G)
    return A, Me


def condense(m1, h, lam):
    """K_e = G_e - R_e^T A_e^{-1} R_e by dense LU with pivoting."""
    S, _ = element_system(m1, h, lam)
    nv = (1 + len(h)) * m1.n ** len(h)
    A, R, G = S[:nv, :nv], S[:nv, nv:], S[nv:, nv:]
    return G - R.T @ sla.lu_solve(sla.lu_factor(A), R)


class LowDimMesh:
    """Cartesian mesh of dim = len(ne) in {1, 2} directions."""

    def __init__(self, ne, grid, bc, p):
        self.dim = len(ne)
        if self.dim not in (1, 2):
            raise ValueError("one or two directions")
        self.ne = tuple(int(v) for v in ne)
        self.grid = [np.asarray(g, dtype=np.float64) for g in grid]
        self.bc = tuple(int(v) for v in bc)
        self.n = p + 1
        self.nf = self.n ** (self.dim - 1)   # nodes per face
        self.lo, self.hi, self.block_offset = [], [], []
        off = 0
        for d in range(self.dim):
            lo = 0 if self.bc[2 * d] == NEUMANN else 1
            hi = self.ne[d] if self.bc[2 * d + 1] == NEUMANN else self.ne[d] - 1
            self.lo.append(lo)
            self.hi.append(hi)
            self.block_offset.append(off)
            off += max(0, hi - lo + 1) * self.n_other(d)
        self.n_faces = off
        self.n_trace = off * self.nf
        self.side_offset = []
        off = 0
        for side in range(2 * self.dim):
            self.side_offset.append(off)
            off += self.n_other(side // 2)
        self.n_bdry = off * self.nf

    def n_other(self, d):
        return self.ne[1 - d] if self.dim == 2 else 1

    def elements(self):
        return itertools.product(*[range(v) for v in reversed(self.ne)]) if self.dim == 1 else \
            ((e1, e2) for e2 in range(self.ne[1]) for e1 in range(self.ne[0]))

    def widths(self, e):
        return tuple(self.grid[d][e[d] + 1] - self.grid[d][e[d]] for d in range(self.dim))

    def elem_index(self, e):
        return e[0] + (self.ne[0] * e[1] if self.dim == 2 else 0)

    def local_trace_map(self, e):
        """(kind, global index) per element-local trace entry: 'u' for the
        trace vector, 'D' for the boundary-data vector."""
        n, out = self.n, []
        for d in range(self.dim):
            other = e[1 - d] if self.dim == 2 else 0
            loc = [None] * (2 * self.nf)
            for s in range(2):
                plane = e[d] + s
                for c in range(self.nf):
                    if self.dim == 1:
                        li = s
                    else:
                        li = s + 2 * c if d == 0 else c + n * s
                    if self.lo[d] <= plane <= self.hi[d]:
                        fid = self.block_offset[d] + (plane - self.lo[d]) * self.n_other(d) + other
                        loc[li] = ("u", fid * self.nf + c)
                    else:
                        bf = self.side_offset[2 * d + s] + other
                        loc[li] = ("D", bf * self.nf + c)
            out.extend(loc)
        return out

    def volume_coords(self, nodes):
        """(n_elem n^dim, dim) physical coordinates of the volume nodes."""
        pts = []
        for e in sorted(self.elements(), key=self.elem_index):
            xs = [self.grid[d][e[d]] + (nodes + 1.0) * self.widths(e)[d] / 2.0 for d in range(self.dim)]
            if self.dim == 1:
                pts.append(xs[0][:, None])
            else:
                X1, X2 = np.meshgrid(xs[0], xs[1], indexing="xy")
                pts.append(np.stack([X1.ravel(), X2.ravel()], axis=1))
        return np.concatenate(pts)

    def bdry_coords(self, nodes):
        """(n_bdry, dim) coordinates of the boundary-data nodes."""
        out = np.zeros((self.n_bdry, self.dim))
        for side in range(2 * self.dim):
            d, s = side // 2, side % 2
            xd = self.grid[d][0 if s == 0 else self.ne[d]]
            for o in range(self.n_other(d)):
                b = (self.side_offset[side] + o) * self.nf
                if self.dim == 1:
                    out[b, 0] = xd
                else:
                    a = 1 - d
                    ha = self.grid[a][o + 1] - self.grid[a][o]
                    out[b:b + self.nf, d] = xd
                    out[b:b + self.nf, a] = self.grid[a][o] + (nodes + 1.0) * ha / 2.0
        return out


class LowDimProblem:
    """Global condensed system on a 1D or 2D mesh (Eq. (hdg_system))."""

    def __init__(self, ne, grid, bc, p, tau_hat, lam, mass="exact"):
        self.mesh = LowDimMesh(ne, grid, bc, p)
        self.m1 = Matrices1D(p, tau_hat, mass)
        self.lam = float(lam)
        self._K = {}

    def K_e(self, e):
        k = tuple(float(v) for v in self.mesh.widths(e))
        if k not in self._K:
            self._K[k] = condense(self.m1, k, self.lam)
        return self._K[k]

    def _map(self, e):
        loc = self.mesh.local_trace_map(e)
        return np.array([k == "u" for k, _ in loc]), np.array([g for _, g in loc], dtype=np.int64)

    def apply(self, x):
        """y = sum_e Q_e^T K_e Q_e x with homogeneous Dirichlet data."""
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros(self.mesh.n_trace)
        for e in self.mesh.elements():
            isu, idx = self._map(e)
            xe = np.where(isu, x[np.where(isu, idx, 0)], 0.0)
            np.add.at(y, idx[isu], (self.K_e(e) @ xe)[isu])
        return y

    def solve(self, f, bdry):
        """Direct solve with volume load f (nodal, per element) and boundary
        data (g_D on Dirichlet sides, g_N = n . grad u on Neumann sides);
        returns (ut, u).  F_e = g_N - R_e^T A_e^{-1} (M_e f_e, 0), Dirichlet
        lift - K_e[., D] g_D, recovery (u, q)_e = A_e^{-1}(b_e - R_e ut_e)."""
        m, n = self.mesh, self.mesh.n
        nv = n ** m.dim
        K = np.zeros((m.n_trace, m.n_trace))
        F = np.zeros(m.n_trace)
        data = {}
        for e in m.elements():
            h = m.widths(e)
            S, Me = element_system(self.m1, h, self.lam)
            nvol = (1 + m.dim) * nv
            A, R = S[:nvol, :nvol], S[:nvol, nvol:]
            lu = sla.lu_factor(A)
            ie = m.elem_index(e)
            b = np.zeros(nvol)
            b[:nv] = Me @ f[ie * nv:(ie + 1) * nv]
            isu, idx = self._map(e)
            gD = np.where(~isu, np.asarray(bdry)[np.where(~isu, idx, 0)], 0.0)
            Ke = self.K_e(e)
            Fe = -R.T @ sla.lu_solve(lu, b) - Ke @ gD
            np.add.at(F, idx[isu], Fe[isu])
            ui = np.nonzero(isu)[0]
            K[np.ix_(idx[ui], idx[ui])] += Ke[np.ix_(ui, ui)]
            data[e] = (lu, R, b, isu, idx, gD)
        # Neumann load: int mu g_N over the Neumann-side faces
        for side in range(2 * m.dim):
            if m.bc[side] != NEUMANN:
                continue
            d, s = side // 2, side % 2
            plane = 0 if s == 0 else m.ne[d]
            for o in range(m.n_other(d)):
                g = np.asarray(bdry)[(m.side_offset[side] + o) * m.nf:(m.side_offset[side] + o + 1) * m.nf]
                if m.dim == 1:
                    w = g
                else:
                    a = 1 - d
                    ha = m.grid[a][o + 1] - m.grid[a][o]
                    w = ha / 2.0 * (self.m1.M @ g)
                fid = m.block_offset[d] + (plane - m.lo[d]) * m.n_other(d) + o
                F[fid * m.nf:(fid + 1) * m.nf] += w
        ut = np.linalg.solve(K, F) if m.n_trace else np.zeros(0)
        u = np.zeros(sum(1 for _ in m.elements()) * nv)
        for e, (lu, R, b, isu, idx, gD) in data.items():
            ute = np.where(isu, ut[np.where(isu, idx, 0)], 0.0) + gD
            sol = sla.lu_solve(lu, b - R @ ute)
            ie = m.elem_index(e)
            u[ie * nv:(ie + 1) * nv] = sol[:nv]
        return ut, u
