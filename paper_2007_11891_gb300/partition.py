"""Slab partition of the mesh across ranks: x3-slabs with one face-layer
exchange per operator application.

The condensed operator is a sum of element contributions,
K = sum_e Q_e^T K_e Q_e (Eq. (hdg_system)), so elements can be split across
ranks: rank r owns the elements with e3 in its slab [z0_r, z1_r) and applies
the operator of its own sub-mesh.  The x3-plane between two slabs is an
interior plane of the whole mesh, but on each of the two sub-meshes it is a
boundary side; declaring that side Neumann makes its faces unknowns that
receive the one element contribution of that sub-mesh (the Neumann data
only enter the right-hand side, not K).  Summing the two partial values of
each interface face -- one exchange of n_e1 x n_e2 x n^2 values per
interface and apply -- gives exactly the rows of K x of the whole mesh:
x1- and x2-faces never cross a slab boundary.

This module is bookkeeping and communication only: the sub-meshes, the map
of local trace entries to the global trace layout of include/hdg.h, which
rank owns an interface plane (for inner products), the exchange, done as an
all-reduce (sum) over the two ranks that share the plane, so that the
collective library adds the two partial values (both ranks receive the same
sum, bitwise), and the partitioned CG, whose inner products add the ranks'
owned shares in one all-reduce per iteration.  The local operator is
whatever the caller passes: the library's apply on each rank's own GPU.
"""
import numpy as np

DIRICHLET, NEUMANN = 0, 1


def slab_bounds(n3, world):
    """[z0, z1) of every rank: contiguous, sizes differing by at most one."""
    if n3 < world:
        raise ValueError("need at least one x3 element layer per rank")
    base, extra = divmod(n3, world)
    out, z = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((z, z + size))
        z += size
    return out


def _layout(ne, bc):
    """Unknown planes (lo, hi) and block offsets (in faces) of the trace layout."""
    lo, hi, blk, off = [], [], [], 0
    for d in range(3):
        a, b = [ax for ax in range(3) if ax != d]
        lo.append(0 if bc[2 * d] == NEUMANN else 1)
        hi.append(ne[d] if bc[2 * d + 1] == NEUMANN else ne[d] - 1)
        blk.append(off)
        off += max(0, hi[d] - lo[d] + 1) * ne[a] * ne[b]
    return lo, hi, blk, off


class SlabPartition:
    """Rank `rank` of `world`: its x3-slab of the mesh (ne, grid, bc) at
    degree p.

    Attributes: local_ne, local_grid, local_bc (the sub-mesh, to build the
    rank's own operator context); local_trace_size, global_trace_size;
    global_index (global trace entry of every local entry, int64);
    bottom, top (slices of the local trace vector holding the interface
    planes shared with rank - 1 and rank + 1, or None); owned (bool mask:
    the bottom interface plane belongs to rank - 1 in inner products).
    """

    def __init__(self, ne, grid, bc, p, world, rank):
        self.ne = tuple(int(v) for v in ne)
        self.bc = tuple(int(v) for v in bc)
        self.n = n = int(p) + 1
        self.world, self.rank = int(world), int(rank)
        self.bounds = slab_bounds(self.ne[2], self.world)
        z0, z1 = self.bounds[self.rank]
        self.z0, self.z1 = z0, z1
        self.local_ne = (self.ne[0], self.ne[1], z1 - z0)
        g = [np.asarray(v, dtype=np.float64) for v in grid]
        self.local_grid = [g[0], g[1], g[2][z0:z1 + 1]]
        lb = list(self.bc)
        if self.rank > 0:
            lb[4] = NEUMANN
        if self.rank < self.world - 1:
            lb[5] = NEUMANN
        self.local_bc = tuple(lb)
        glo, ghi, gblk, gfaces = _layout(self.ne, self.bc)
        llo, lhi, lblk, lfaces = _layout(self.local_ne, self.local_bc)
        n2 = n * n
        self.global_trace_size = gfaces * n2
        self.local_trace_size = lfaces * n2
        N1, N2, N3 = self.ne
        n3 = self.local_ne[2]
        gface = np.empty(lfaces, dtype=np.int64)
        # x1 faces: plane e1, face (e2, e3); x2 faces: plane e2, face (e1, e3)
        for d, (na, nb_loc, nb_glob) in ((0, (N2, n3, N3)), (1, (N1, n3, N3))):
            planes = np.arange(llo[d], lhi[d] + 1)
            if len(planes) == 0:
                continue
            P, B, A = np.meshgrid(planes, np.arange(nb_loc), np.arange(na), indexing="ij")
            loc = lblk[d] + (P - llo[d]) * na * nb_loc + A + na * B
            glob = gblk[d] + (P - glo[d]) * na * nb_glob + A + na * (B + z0)
            gface[loc.ravel()] = glob.ravel()
        # x3 faces: plane e3 (shifted by z0), face (e1, e2)
        planes = np.arange(llo[2], lhi[2] + 1)
        if len(planes):
            P, B, A = np.meshgrid(planes, np.arange(N2), np.arange(N1), indexing="ij")
            loc = lblk[2] + (P - llo[2]) * N1 * N2 + A + N1 * B
            glob = gblk[2] + (P + z0 - glo[2]) * N1 * N2 + A + N1 * B
            gface[loc.ravel()] = glob.ravel()
        self.global_index = (gface[:, None] * n2 + np.arange(n2)[None, :]).ravel()
        plane = N1 * N2 * n2
        self.bottom = None
        self.top = None
        if self.rank > 0:
            start = (lblk[2] + (0 - llo[2]) * N1 * N2) * n2
            self.bottom = slice(start, start + plane)
        if self.rank < self.world - 1:
            start = (lblk[2] + (n3 - llo[2]) * N1 * N2) * n2
            self.top = slice(start, start + plane)
        self.owned = np.ones(self.local_trace_size, dtype=bool)
        if self.bottom is not None:
            self.owned[self.bottom] = False
        self._groups = None

    # -- communication ------------------------------------------------------------
    def init_groups(self):
        """Create the process groups of the interfaces (rank r with r + 1);
        every rank must call this, in the same order, after
        torch.distributed.init_process_group."""
        import torch.distributed as dist
        self._groups = [dist.new_group([r, r + 1]) for r in range(self.world - 1)]
        return self

    def exchange(self, y):
        """Sum the partial values of the interface planes of the local trace
        vector y (torch tensor, local layout) with the neighbouring ranks, in
        place: afterwards both ranks hold the complete rows of K x there."""
        import torch.distributed as dist
        if self.world == 1:
            return y
        if self._groups is None:
            raise RuntimeError("call init_groups() first")
        # lower interface first on every rank: rank r's top exchange pairs
        # with rank r + 1's bottom one, in the same order on both sides
        if self.bottom is not None:
            dist.all_reduce(y[self.bottom], op=dist.ReduceOp.SUM, group=self._groups[self.rank - 1])
        if self.top is not None:
            dist.all_reduce(y[self.top], op=dist.ReduceOp.SUM, group=self._groups[self.rank])
        return y

    def apply(self, local_apply, x_local):
        """y = K x on the local slab: the rank's own operator, then the
        interface exchange."""
        return self.exchange(local_apply(x_local))

    def dots(self, pairs):
        """Global inner products of pairs of local vectors (torch tensors):
        each rank sums its owned entries (an interface value is owned by the
        rank below it), and one all-reduce of the whole list of scalars adds
        the ranks' shares.  Returns a float64 tensor of len(pairs)."""
        import torch
        import torch.distributed as dist
        own = torch.as_tensor(self.owned, device=pairs[0][0].device)
        vals = torch.stack([(a[own].double() * b[own].double()).sum() for a, b in pairs])
        if self.world > 1:
            dist.all_reduce(vals, op=dist.ReduceOp.SUM)
        return vals

    def cg(self, local_apply, b_local, tol=1e-10, max_iter=1000, w_local=None):
        """Solve K x = b on the partitioned operator with the single-reduction
        preconditioned CG (Chronopoulos-Gear; the iterates of the textbook
        preconditioned CG in exact arithmetic): per iteration one operator
        application (the rank's own apply and the interface exchange) and one
        all-reduce of three scalars (r . u, w . u, r . r).  w_local: the
        diagonal preconditioner on the local entries, or None.  Every rank
        takes the same decisions (the scalars are identical after the
        all-reduce).  Returns (x_local, iterations, relative residual
        ||b - K x|| / ||b|| as tracked by the recurrence)."""
        import torch
        W = (lambda v: v) if w_local is None else (lambda v: w_local * v)
        x = torch.zeros_like(b_local)
        r = b_local.clone()
        u = W(r)
        w = self.apply(local_apply, u)
        gam, dlt, rr = [float(v) for v in self.dots([(r, u), (w, u), (r, r)])]
        bb = rr
        if bb == 0.0:
            return x, 0, 0.0
        p, s = u.clone(), w.clone()
        alpha = gam / dlt
        it = 0
        while it < max_iter:
            x += alpha * p
            r -= alpha * s
            it += 1
            u = W(r)
            w = self.apply(local_apply, u)
            gam_new, dlt, rr = [float(v) for v in self.dots([(r, u), (w, u), (r, r)])]
            if rr <= tol * tol * bb:
                break
            beta = gam_new / gam
            alpha = gam_new / (dlt - beta * gam_new / alpha)
            p = u + beta * p
            s = w + beta * s
            gam = gam_new
        return x, it, (rr / bb) ** 0.5

    # -- layout helpers -------------------------------------------------------------
    def scatter(self, x_global):
        """The local entries of a global trace vector (numpy or torch)."""
        try:
            import torch
            if isinstance(x_global, torch.Tensor):
                return x_global[torch.as_tensor(self.global_index, device=x_global.device)]
        except ImportError:
            pass
        return np.asarray(x_global)[self.global_index]
