"""Cartesian mesh and face-wise trace storage (test infrastructure only).

Sec. 3.2 (Cartesian cuboidal elements) and Eq. (hdg_system) of
arXiv:2007.11891: the trace unknowns are stored face-wise and Q_e maps the
global trace vector to the element-local traces ut_{1,e}, ut_{2,e}, ut_{3,e}.

Global trace layout (the library's documented layout, written here
independently):

* Elements (e1, e2, e3), volume index e1 + N1 (e2 + N2 e3); volume nodal
  values n^3 per element, node i + n j + n^2 k.
* Faces normal to direction d lie on grid planes 0..N_d.  A plane is a trace
  unknown unless it is a boundary plane of a Dirichlet side; boundary planes
  of Neumann sides are unknowns.  Unknown planes of direction d run over
  lo_d..hi_d.
* The trace vector is the concatenation of the blocks d = 0, 1, 2.  Block d
  holds (hi_d - lo_d + 1) planes, each with Na x Nb faces (the other two
  element counts in increasing axis order, face a + Na b), each face n x n
  nodes in the order of its two axes, lower axis fastest.
* The boundary-data vector holds, for the six sides 0..5 = (x1-, x1+, x2-,
  x2+, x3-, x3+), Na x Nb faces of n x n nodes each: g_D nodal values on a
  Dirichlet side, g_N = n . grad u nodal values on a Neumann side.
"""

import numpy as np

DIRICHLET = 0
NEUMANN = 1
OTHER_AXES = ((1, 2), (0, 2), (0, 1))


class Mesh:
    def __init__(self, ne, grid, bc, p):
        self.ne = tuple(int(v) for v in ne)
        if any(v < 1 for v in self.ne):
            raise ValueError("each direction needs at least one element")
        self.grid = [np.asarray(g, dtype=np.float64) for g in grid]
        for d in range(3):
            if len(self.grid[d]) != self.ne[d] + 1 or np.any(np.diff(self.grid[d]) <= 0):
                raise ValueError("grid lines must be increasing, N_d + 1 per direction")
        self.bc = tuple(int(v) for v in bc)
        self.p = p
        self.n = n = p + 1
        self.n2 = n * n
        self.n_elem = self.ne[0] * self.ne[1] * self.ne[2]
        self.lo, self.hi, self.nplanes, self.nab = [], [], [], []
        self.block_offset = []
        off = 0
        for d in range(3):
            a, b = OTHER_AXES[d]
            lo = 0 if self.bc[2 * d] == NEUMANN else 1
            hi = self.ne[d] if self.bc[2 * d + 1] == NEUMANN else self.ne[d] - 1
            npl = max(0, hi - lo + 1)
            self.lo.append(lo)
            self.hi.append(hi)
            self.nplanes.append(npl)
            self.nab.append((self.ne[a], self.ne[b]))
            self.block_offset.append(off)
            off += npl * self.ne[a] * self.ne[b]
        self.n_faces = off
        self.n_trace = off * self.n2
        self.side_offset = []
        off = 0
        for side in range(6):
            a, b = OTHER_AXES[side // 2]
            self.side_offset.append(off)
            off += self.ne[a] * self.ne[b]
        self.n_bdry_faces = off
        self.n_bdry = off * self.n2

    # -- element geometry --------------------------------------------------
    def widths(self, e):
        return tuple(self.grid[d][e[d] + 1] - self.grid[d][e[d]] for d in range(3))

    def elements(self):
        for e3 in range(self.ne[2]):
            for e2 in range(self.ne[1]):
                for e1 in range(self.ne[0]):
                    yield (e1, e2, e3)

    def elem_index(self, e):
        return e[0] + self.ne[0] * (e[1] + self.ne[1] * e[2])

    # -- faces ---------------------------------------------------------------
    def face_ab(self, d, e):
        a, b = OTHER_AXES[d]
        return e[a], e[b]

    def unknown_face(self, d, plane, e):
        """Global face id of the direction-d face on ``plane`` next to e, or
        None when that plane is a Dirichlet boundary."""
        if plane < self.lo[d] or plane > self.hi[d]:
            return None
        a, b = self.face_ab(d, e)
        Na, _ = self.nab[d]
        return self.block_offset[d] + (plane - self.lo[d]) * Na * self.nab[d][1] + a + Na * b

    def bdry_face(self, d, s, e):
        a, b = self.face_ab(d, e)
        Na, _ = self.nab[d]
        return self.side_offset[2 * d + s] + a + Na * b

    def local_trace_map(self, e):
        """For element e: list over the 6n^2 element-local trace entries (in
        the element3d ordering) of (kind, global index): kind 'u' indexes the
        trace vector (interior or Neumann-side face), kind 'D' indexes the
        boundary-data vector (Dirichlet-side face)."""
        n = self.n
        out = []
        for d in range(3):
            loc = [None] * (2 * n * n)
            for s in range(2):
                plane = e[d] + s
                on_bdry = (plane == 0 and s == 0) or (plane == self.ne[d] and s == 1)
                fid = self.unknown_face(d, plane, e)
                for c1 in range(n):          # fastest face axis
                    for c2 in range(n):      # slower face axis
                        node = c1 + n * c2
                        if d == 0:
                            li = s + 2 * (c1 + n * c2)
                        elif d == 1:
                            li = c1 + n * (s + 2 * c2)
                        else:
                            li = c1 + n * (c2 + n * s)
                        if fid is not None:
                            loc[li] = ("u", fid * self.n2 + node)
                        elif on_bdry:
                            loc[li] = ("D", self.bdry_face(d, s, e) * self.n2 + node)
                        else:
                            raise AssertionError("interior plane must be an unknown")
            out.extend(loc)
        return out

    # -- node coordinates ------------------------------------------------------
    def volume_coords(self, nodes):
        """(n_elem*n^3, 3) physical coordinates of the volume nodes."""
        n = self.n
        X = np.zeros((self.n_elem, n, n, n, 3))
        for e in self.elements():
            lo = [self.grid[d][e[d]] for d in range(3)]
            h = self.widths(e)
            xs = [lo[d] + (nodes + 1.0) * h[d] / 2.0 for d in range(3)]
            ie = self.elem_index(e)
            X[ie, :, :, :, 0] = xs[0][None, None, :]
            X[ie, :, :, :, 1] = xs[1][None, :, None]
            X[ie, :, :, :, 2] = xs[2][:, None, None]
        return X.reshape(-1, 3)

    def _face_coords(self, d, plane_coord, e, nodes):
        a, b = OTHER_AXES[d]
        n = self.n
        ha = self.grid[a][e[a] + 1] - self.grid[a][e[a]]
        hb = self.grid[b][e[b] + 1] - self.grid[b][e[b]]
        xa = self.grid[a][e[a]] + (nodes + 1.0) * ha / 2.0
        xb = self.grid[b][e[b]] + (nodes + 1.0) * hb / 2.0
        P = np.zeros((n, n, 3))
        P[:, :, d] = plane_coord
        P[:, :, a] = xa[None, :]
        P[:, :, b] = xb[:, None]
        return P.reshape(-1, 3)

    def trace_coords(self, nodes):
        """(n_trace, 3) coordinates of the unknown trace nodes."""
        out = np.zeros((self.n_trace, 3))
        for d in range(3):
            a, b = OTHER_AXES[d]
            for plane in range(self.lo[d], self.hi[d] + 1):
                for eb in range(self.ne[b]):
                    for ea in range(self.ne[a]):
                        e = [0, 0, 0]
                        e[a], e[b] = ea, eb
                        fid = self.unknown_face(d, plane, e)
                        out[fid * self.n2:(fid + 1) * self.n2] = self._face_coords(
                            d, self.grid[d][plane], e, nodes)
        return out

    def bdry_coords(self, nodes):
        """(n_bdry, 3) coordinates of the boundary-data nodes, and the outer
        normal direction (d, sign) per entry."""
        out = np.zeros((self.n_bdry, 3))
        nrm = np.zeros((self.n_bdry, 3))
        for side in range(6):
            d, s = side // 2, side % 2
            a, b = OTHER_AXES[d]
            plane = 0 if s == 0 else self.ne[d]
            for eb in range(self.ne[b]):
                for ea in range(self.ne[a]):
                    e = [0, 0, 0]
                    e[a], e[b] = ea, eb
                    fid = self.bdry_face(d, s, e)
                    sl = slice(fid * self.n2, (fid + 1) * self.n2)
                    out[sl] = self._face_coords(d, self.grid[d][plane], e, nodes)
                    nrm[sl, d] = -1.0 if s == 0 else 1.0
        return out, nrm
