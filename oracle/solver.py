"""Global condensed system, solve, recovery and adjoint (test infrastructure only).

arXiv:2007.11891, Eq. (hdg_system): sum_e Q_e^T K_e Q_e ut = sum_e Q_e^T F_e.

* The element right-hand side comes from block elimination of
  Eq. (ldg_element_operator_threed) with volume load b_e = (M_e f_e, 0, 0, 0):
  F_e = g_{N,e} - R_e^T A_e^{-1} b_e, and the volume recovery is
  (u, q)_e = A_e^{-1} (b_e - R_e ut_e).  Alg. (hdg_cg) prints both with the
  opposite sign in front of R_e; that equals this with R_e -> -R_e, which
  leaves K_e unchanged, and only these signs reproduce polynomial solutions.
* Dirichlet faces carry ut = g_D and are not unknowns: the unknown block is
  K_II ut_I = F_I - K_IB g_D.  Neumann faces are unknowns whose transmission
  row gets int mu g_N (Eq. (transmission_condition)).
* Plain CG (no preconditioner, no basis change) on K_II.
* Adjoint of L = sum (u - u_t)^2 over volume nodal values: the element system
  is symmetric, so the adjoint solve is the same solve with the volume load
  b_e = 2 (u_e - u_t,e); then dL/df_e = M_e z_{u,e} and
  dL/dlambda = - sum_e z_{u,e}^T M_e u_e.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis1d import Matrices1D
from .element3d import condense, element_blocks, element_system, split
from .mesh import DIRICHLET, NEUMANN, OTHER_AXES, Mesh


class Problem:
    """One mesh + degree + penalty + lambda, with per-width caches."""

    def __init__(self, ne, grid, bc, p, tau_hat, lam, mass="exact", tier=None):
        self.mesh = Mesh(ne, grid, bc, p)
        self.m1 = Matrices1D(p, tau_hat, mass)
        self.lam = float(lam)
        self.tier = tier
        self._K = {}
        self._vol = {}
        self._maps = {}

    # -- per element -------------------------------------------------------
    def _key(self, e):
        return tuple(float(v) for v in self.mesh.widths(e))

    def K_e(self, e):
        k = self._key(e)
        if k not in self._K:
            self._K[k] = condense(self.m1, k, self.lam, self.tier)
        return self._K[k]

    def volume_factors(self, e):
        k = self._key(e)
        if k not in self._vol:
            A, R, _ = split(self.m1, element_system(self.m1, k, self.lam))
            Me = element_blocks(self.m1, k)["M"]
            self._vol[k] = (sla.lu_factor(A), R, Me)
        return self._vol[k]

    def local_map(self, e):
        if e not in self._maps:
            loc = self.mesh.local_trace_map(e)
            kinds = np.array([k == "u" for k, _ in loc])
            idx = np.array([g for _, g in loc], dtype=np.int64)
            self._maps[e] = (kinds, idx)
        return self._maps[e]

    # -- global operator -----------------------------------------------------
    def assemble(self):
        """Sparse (K_II, K_IB): unknown x unknown and unknown x Dirichlet data."""
        m = self.mesh
        rows, cols, vals = [], [], []
        brows, bcols, bvals = [], [], []
        for e in m.elements():
            Ke = self.K_e(e)
            isu, idx = self.local_map(e)
            ui = np.nonzero(isu)[0]
            di = np.nonzero(~isu)[0]
            r, c = np.meshgrid(idx[ui], idx[ui], indexing="ij")
            rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Ke[np.ix_(ui, ui)].ravel())
            if len(di):
                r, c = np.meshgrid(idx[ui], idx[di], indexing="ij")
                brows.append(r.ravel()); bcols.append(c.ravel())
                bvals.append(Ke[np.ix_(ui, di)].ravel())
        nt, nb = m.n_trace, m.n_bdry
        cat = lambda L: np.concatenate(L) if L else np.zeros(0)
        K = sp.coo_matrix((cat(vals), (cat(rows).astype(np.int64), cat(cols).astype(np.int64))),
                          shape=(nt, nt)).tocsr()
        KB = sp.coo_matrix((cat(bvals), (cat(brows).astype(np.int64), cat(bcols).astype(np.int64))),
                           shape=(nt, nb)).tocsr()
        return K, KB

    def apply(self, x):
        """y = sum_e Q_e^T K_e Q_e x with homogeneous Dirichlet data (the
        operator the CG iterates on), element by element."""
        m = self.mesh
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros(m.n_trace)
        for e in m.elements():
            isu, idx = self.local_map(e)
            xe = _take(x, isu, idx)
            ye = self.K_e(e) @ xe
            np.add.at(y, idx[isu], ye[isu])
        return y

    def apply_rows(self, x, dofs):
        """Selected entries of K_II x, from the one or two elements touching
        each selected face only (sampled parity at full size)."""
        m = self.mesh
        x = np.asarray(x, dtype=np.float64)
        want = {}
        for g in np.asarray(dofs, dtype=np.int64):
            want.setdefault(int(g) // m.n2, []).append(int(g))
        out = {}
        for fid, gs in want.items():
            for e in self.face_elements(fid):
                isu, idx = self.local_map(e)
                xe = _take(x, isu, idx)
                ye = self.K_e(e) @ xe
                for g in gs:
                    hit = np.nonzero(isu & (idx == g))[0]
                    out[g] = out.get(g, 0.0) + float(ye[hit].sum())
        return np.array([out[int(g)] for g in np.asarray(dofs, dtype=np.int64)])

    def face_elements(self, fid):
        """Elements adjacent to unknown face ``fid``."""
        m = self.mesh
        d = max(k for k in range(3) if m.block_offset[k] <= fid and
                (k == 2 or fid < m.block_offset[k + 1]))
        r = fid - m.block_offset[d]
        Na, Nb = m.nab[d]
        plane = m.lo[d] + r // (Na * Nb)
        ab = r % (Na * Nb)
        a_ax, b_ax = OTHER_AXES[d]
        els = []
        for s, ed in ((1, plane - 1), (0, plane)):
            if 0 <= ed < m.ne[d]:
                e = [0, 0, 0]
                e[d] = ed
                e[a_ax] = ab % Na
                e[b_ax] = ab // Na
                els.append(tuple(e))
        return els

    # -- right-hand side, solve, recovery --------------------------------------
    def _volume_load(self, f=None, b=None):
        """Per element the u-row load b_e: M_e f_e, or b given directly."""
        m = self.mesh
        n3 = m.n ** 3
        loads = {}
        for e in m.elements():
            ie = m.elem_index(e)
            if b is not None:
                loads[e] = np.asarray(b[ie * n3:(ie + 1) * n3], dtype=np.float64)
            else:
                _, _, Me = self.volume_factors(e)
                loads[e] = Me @ np.asarray(f[ie * n3:(ie + 1) * n3], dtype=np.float64)
        return loads

    def neumann_load(self, bdry):
        """int mu g_N on the Neumann-side unknown faces, from g_N nodal values:
        the face mass (h_a h_b / 4) M (x) M times the values."""
        m = self.mesh
        M = self.m1.M
        Mf = np.kron(M, M)
        F = np.zeros(m.n_trace)
        for side in range(6):
            if m.bc[side] != NEUMANN:
                continue
            d, s = side // 2, side % 2
            a, b = OTHER_AXES[d]
            plane = 0 if s == 0 else m.ne[d]
            for eb in range(m.ne[b]):
                for ea in range(m.ne[a]):
                    e = [0, 0, 0]
                    e[a], e[b] = ea, eb
                    e[d] = 0 if s == 0 else m.ne[d] - 1
                    ha = m.grid[a][ea + 1] - m.grid[a][ea]
                    hb = m.grid[b][eb + 1] - m.grid[b][eb]
                    bf = m.bdry_face(d, s, e)
                    uf = m.unknown_face(d, plane, e)
                    g = bdry[bf * m.n2:(bf + 1) * m.n2]
                    F[uf * m.n2:(uf + 1) * m.n2] += ha * hb / 4.0 * (Mf @ g)
        return F

    def rhs(self, f=None, bdry=None, b=None):
        """F_I = sum_e Q_e^T (-R_e^T A_e^{-1} b_e) + g_N - K_IB g_D."""
        m = self.mesh
        bdry = np.zeros(m.n_bdry) if bdry is None else np.asarray(bdry, dtype=np.float64)
        loads = self._volume_load(f=f, b=b)
        F = np.zeros(m.n_trace)
        gD = np.where(self._dirichlet_mask(), bdry, 0.0)
        for e in m.elements():
            lu, R, _ = self.volume_factors(e)
            nv = R.shape[0]
            rhs = np.zeros(nv)
            rhs[:m.n ** 3] = loads[e]
            Fe = -R.T @ sla.lu_solve(lu, rhs)
            isu, idx = self.local_map(e)
            # Dirichlet lift: - K_e[u, D] g_D
            Ke = self.K_e(e)
            xD = _take(gD, ~isu, idx)
            Fe = Fe - Ke @ xD
            np.add.at(F, idx[isu], Fe[isu])
        F += self.neumann_load(bdry)
        return F

    def _dirichlet_mask(self):
        m = self.mesh
        mask = np.zeros(m.n_bdry, dtype=bool)
        for side in range(6):
            if m.bc[side] == DIRICHLET:
                d = side // 2
                a, b = OTHER_AXES[d]
                lo = m.side_offset[side] * m.n2
                mask[lo:lo + m.ne[a] * m.ne[b] * m.n2] = True
        return mask

    def recover(self, ut, f=None, bdry=None, b=None):
        """(u, q)_e = A_e^{-1} (b_e - R_e ut_e); returns u (n_elem*n^3) and
        q (n_elem*n^3, 3)."""
        m = self.mesh
        n3 = m.n ** 3
        bdry = np.zeros(m.n_bdry) if bdry is None else np.asarray(bdry, dtype=np.float64)
        gD = np.where(self._dirichlet_mask(), bdry, 0.0)
        loads = self._volume_load(f=f, b=b)
        u = np.zeros(m.n_elem * n3)
        q = np.zeros((m.n_elem * n3, 3))
        for e in m.elements():
            lu, R, _ = self.volume_factors(e)
            isu, idx = self.local_map(e)
            ute = _take(ut, isu, idx) + _take(gD, ~isu, idx)
            rhs = -R @ ute
            rhs[:n3] += loads[e]
            sol = sla.lu_solve(lu, rhs)
            ie = m.elem_index(e)
            u[ie * n3:(ie + 1) * n3] = sol[:n3]
            for d in range(3):
                q[ie * n3:(ie + 1) * n3, d] = sol[(1 + d) * n3:(2 + d) * n3]
        return u, q

    def solve(self, f=None, bdry=None, b=None, tol=1e-12, method="cg", x0=None, max_iter=None):
        """Condensed solve; returns (ut, u, q, info)."""
        F = self.rhs(f=f, bdry=bdry, b=b)
        K, _ = self.assemble()
        if method == "direct":
            import scipy.sparse.linalg as spla
            ut = spla.spsolve(K.tocsc(), F) if K.shape[0] else np.zeros(0)
            info = {"iters": 0}
        else:
            ut, info = cg(lambda v: K @ v, F, tol=tol, x0=x0, max_iter=max_iter)
        u, q = self.recover(ut, f=f, bdry=bdry, b=b)
        info["rel_residual"] = rel_residual(K, F, ut)
        return ut, u, q, info

    # -- adjoint -----------------------------------------------------------------
    def adjoint(self, f, u_target, tol=1e-12, method="cg"):
        """Loss L = sum (u - u_t)^2 with homogeneous Dirichlet data.
        Returns (L, dL/df, dL/dlambda, u)."""
        m = self.mesh
        n3 = m.n ** 3
        _, u, _, _ = self.solve(f=f, tol=tol, method=method)
        r = 2.0 * (u - u_target)
        _, z, _, _ = self.solve(b=r, tol=tol, method=method)
        dLdf = np.zeros_like(u)
        dLdlam = 0.0
        for e in m.elements():
            ie = m.elem_index(e)
            sl = slice(ie * n3, (ie + 1) * n3)
            _, _, Me = self.volume_factors(e)
            dLdf[sl] = Me @ z[sl]
            dLdlam -= z[sl] @ (Me @ u[sl])
        L = float(np.sum((u - u_target) ** 2))
        return L, dLdf, dLdlam, u


def _take(v, mask, idx):
    """Entries v[idx] where mask holds, zero elsewhere."""
    out = np.zeros(len(idx))
    out[mask] = np.asarray(v)[idx[mask]]
    return out


def cg(A, b, tol=1e-12, x0=None, max_iter=None):
    """Plain conjugate gradients (Hestenes-Stiefel), stop at ||r|| <= tol ||b||."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A(x)
    p = r.copy()
    rr = r @ r
    nb = np.linalg.norm(b)
    max_iter = 10 * len(b) + 100 if max_iter is None else max_iter
    it = 0
    while np.sqrt(rr) > tol * nb and it < max_iter:
        Ap = A(p)
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, {"iters": it}


def rel_residual(K, F, ut):
    nF = np.linalg.norm(F)
    return float(np.linalg.norm(F - K @ ut) / nF) if nF > 0 else float(np.linalg.norm(K @ ut))


def uniform_grid(N, length=1.0, origin=0.0):
    return origin + np.linspace(0.0, length, N + 1)
