"""Torch-facing wrapper of the C ABI (device memory and streams from torch).

Every operation runs in the CUDA library; this module only checks shapes and
dtypes, passes ``data_ptr()`` values and the current torch stream, and
raises on a non-OK status.
"""
import ctypes
import json
import os

import numpy as np
import torch

from . import _capi


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _lams(lam, nrhs):
    if isinstance(lam, torch.Tensor):
        lam = lam.detach().cpu().reshape(-1).tolist()
    elif np.isscalar(lam):
        lam = [float(lam)] * nrhs
    lam = [float(v) for v in lam]
    if len(lam) != nrhs:
        raise ValueError("need one lambda per right-hand side")
    return _capi.doubles(lam)


class HDG:
    """One Cartesian mesh + degree + penalty on the current CUDA device.

    ne: elements per direction; grid: three increasing coordinate arrays of
    length ne[d] + 1; bc: six sides (x1-, x1+, x2-, x2+, x3-, x3+), 0 for
    Dirichlet and 1 for Neumann; p: degree 1..16; tau_hat: penalty
    (tau_{i,e} = 2 tau_hat / h_{i,e}).
    """

    def __init__(self, ne, grid, bc=(0, 0, 0, 0, 0, 0), p=4, tau_hat=25.0, mass_lumped=False):
        L = _capi.lib()
        torch.cuda.init()
        self.ne = tuple(int(v) for v in ne)
        self.p, self.n = int(p), int(p) + 1
        self.bc = tuple(int(v) for v in bc)
        self._grid = [(ctypes.c_double * (self.ne[d] + 1))(*[float(v) for v in grid[d]]) for d in range(3)]
        m = _capi.HdgMesh()
        for d in range(3):
            m.ne[d] = self.ne[d]
            m.h_grid[d] = ctypes.cast(self._grid[d], ctypes.POINTER(ctypes.c_double))
        for s in range(6):
            m.bc[s] = self.bc[s]
        o = _capi.HdgOptions(float(tau_hat), int(bool(mass_lumped)))
        h = ctypes.c_void_p()
        _capi.check(L.hdg_setup(ctypes.byref(m), self.p, ctypes.byref(o), ctypes.byref(h)), "hdg_setup")
        self._h = h
        self.trace_size = int(L.hdg_trace_size(h))
        self.volume_size = int(L.hdg_volume_size(h))
        self.boundary_size = int(L.hdg_boundary_size(h))
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _capi.lib().hdg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_x1_segment(self, elements):
        """Operator-kernel tuning: x1-segment length (0 = automatic)."""
        _capi.check(_capi.lib().hdg_set_x1_segment(self._h, int(elements)), "hdg_set_x1_segment")

    def set_slots_per_cta(self, slots):
        """Operator-kernel tuning: x1-pencil segments per CTA (0 = automatic)."""
        _capi.check(_capi.lib().hdg_set_slots_per_cta(self._h, int(slots)), "hdg_set_slots_per_cta")

    def autotune(self, precision="fp32", nrhs=1, lam=1.0, cache=None):
        """Time the operator kernel over its tile candidates (x1-segment
        length, slots per CTA) and keep the fastest.  With `cache` (a JSON
        path) results are looked up and stored per GPU, degree, precision,
        right-hand-side count and mesh.  Returns (segment, slots, us)."""
        key = "|".join([torch.cuda.get_device_name(), "p%d" % self.p, precision, "nrhs%d" % nrhs,
                        "ne%dx%dx%d" % self.ne, "bc" + "".join(map(str, self.bc))])
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if key in table:
            seg, slots, us = table[key]
            self.set_x1_segment(seg)
            self.set_slots_per_cta(slots)
            return seg, slots, us
        seg, slots, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = _capi.lib().hdg_autotune(self._h, nrhs, _lams(lam, nrhs), _capi.PRECISION[precision],
                                      ctypes.byref(seg), ctypes.byref(slots), ctypes.byref(us), _stream())
        _capi.check(st, "hdg_autotune")
        if cache:
            table[key] = [seg.value, slots.value, us.value]
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return seg.value, slots.value, us.value

    def set_dz_mode(self, mode):
        """FP32 operator tuning: D_Z^-1 from 'auto', 'table' or 'kernel'."""
        code = {"auto": 0, "table": 1, "kernel": 2}[mode]
        _capi.check(_capi.lib().hdg_set_dz_mode(self._h, code), "hdg_set_dz_mode")

    def set_operator_variant(self, variant):
        """Operator kernel: 'auto' (the measured fastest per precision,
        degree and batch size), 'tiles' (element tiles), 'runs' (one thread
        per x1-line in element runs) or 'generic' (the runtime-degree kernel
        that degrees above 16 use, any degree)."""
        code = {"auto": 0, "runs": 1, "tiles": 2, "generic": 3}[variant]
        _capi.check(_capi.lib().hdg_set_operator_variant(self._h, code), "hdg_set_operator_variant")

    def set_cg_variant(self, variant):
        """Inner CG iteration: 'auto' (the default: two kernels), 'persistent'
        (the whole inner CG in one cooperative launch of the tile kernel),
        'fused' (one tile-kernel launch per iteration) or 'two_kernel'
        (operator, then the vector update)."""
        code = {"persistent": 0, "fused": 2, "two_kernel": 1, "auto": 3}[variant]
        _capi.check(_capi.lib().hdg_set_cg_variant(self._h, code), "hdg_set_cg_variant")

    def set_nodal_variant(self, variant):
        """FP64 nodal-basis apply: 'facewise' (transform every face once around
        the transformed operator, three launches) or 'fused' (Alg. hdg_op_3d,
        each element transforms its own faces, one launch, no workspace)."""
        code = {"facewise": 0, "fused": 1}[variant]
        _capi.check(_capi.lib().hdg_set_nodal_variant(self._h, code), "hdg_set_nodal_variant")

    # -- measurement -------------------------------------------------------------
    KERNEL_CLASSES = {"op_fp32": 0, "op_fp64": 1, "face": 2, "volume": 3, "rhs_recover": 4, "vector": 5}

    def profile(self, enable):
        """Start (reset) or stop per-launch event timing inside the library."""
        _capi.check(_capi.lib().hdg_profile(self._h, int(bool(enable))), "hdg_profile")

    def profile_read(self, kernel_class):
        """(total ms, launches) of one kernel class; "all" gives (0, launches
        of every class since profile(True))."""
        cls = -1 if kernel_class == "all" else self.KERNEL_CLASSES[kernel_class]
        ms, cnt = ctypes.c_double(), ctypes.c_longlong()
        _capi.check(_capi.lib().hdg_profile_read(self._h, cls, ctypes.byref(ms), ctypes.byref(cnt)),
                    "hdg_profile_read")
        return ms.value, cnt.value

    def nodes(self):
        out = (ctypes.c_double * self.n)()
        _capi.check(_capi.lib().hdg_get_nodes(self._h, out), "hdg_get_nodes")
        return np.array(out[:])

    # -- node coordinates of the data layouts (host-side bookkeeping) ----------
    def _lines(self, nodes):
        # per direction: (ne[d], n) physical node coordinates of each element
        g = [np.asarray(self._grid[d][:], dtype=np.float64) for d in range(3)]
        return [g[d][:-1, None] + (nodes[None, :] + 1.0) * 0.5 * np.diff(g[d])[:, None] for d in range(3)], g

    def volume_coords(self):
        """(volume_size, 3) coordinates of the volume nodes in the volume layout
        (element e1 + N1 (e2 + N2 e3), node i + n j + n^2 k)."""
        x, _ = self._lines(self.nodes())
        n, (N1, N2, N3) = self.n, self.ne
        X = np.empty((N3, N2, N1, n, n, n, 3))
        X[..., 0] = x[0][None, None, :, None, None, :]
        X[..., 1] = x[1][None, :, None, None, :, None]
        X[..., 2] = x[2][:, None, None, :, None, None]
        return X.reshape(-1, 3)

    def boundary_coords(self):
        """(boundary_size, 3) coordinates of the boundary-data nodes and the
        (boundary_size, 3) outer unit normals, in the boundary layout (sides
        x1-, x1+, x2-, x2+, x3-, x3+; faces a + Na b; nodes lower axis fastest)."""
        x, g = self._lines(self.nodes())
        n = self.n
        P, Nrm = [], []
        for side in range(6):
            d, s = divmod(side, 2)
            a, b = [ax for ax in range(3) if ax != d]
            na, nb = self.ne[a], self.ne[b]
            F = np.empty((nb, na, n, n, 3))
            F[..., d] = g[d][-1] if s else g[d][0]
            F[..., a] = x[a][None, :, None, :]
            F[..., b] = x[b][:, None, :, None]
            P.append(F.reshape(-1, 3))
            nrm = np.zeros((nb * na * n * n, 3))
            nrm[:, d] = 1.0 if s else -1.0
            Nrm.append(nrm)
        return np.concatenate(P), np.concatenate(Nrm)

    # -- operator ------------------------------------------------------------
    def apply(self, x, lam, basis="nodal", out=None):
        """y = K x (homogeneous Dirichlet data).  x: (T,) or (nrhs, T) CUDA
        tensor, float64 or float32 (the precision of the application)."""
        x2 = x.reshape(-1, self.trace_size)
        if not x2.is_cuda or not x2.is_contiguous():
            raise ValueError("x must be a contiguous CUDA tensor")
        prec = {torch.float64: "fp64", torch.float32: "fp32", torch.bfloat16: "bf16"}[x2.dtype]
        y = torch.empty_like(x2) if out is None else out.reshape(-1, self.trace_size)
        nrhs = x2.shape[0]
        st = _capi.lib().hdg_apply(self._h, nrhs, _lams(lam, nrhs), _capi.PRECISION[prec],
                                   _capi.BASIS[basis], ctypes.c_void_p(x2.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), _stream())
        _capi.check(st, "hdg_apply")
        return y.reshape(x.shape)

    # -- solve -----------------------------------------------------------------
    def _opts(self, tol, inner, max_iter, max_outer, inner_tol, precond=True):
        return _capi.HdgSolveOpts(float(tol), int(max_iter), int(max_outer), _capi.PRECISION[inner],
                                  float(inner_tol), int(bool(precond)))

    def solve(self, f, lam, bdry=None, x0=None, tol=1e-10, inner="fp32", max_iter=50000,
              max_outer=40, inner_tol=0.0, return_u=True, check=True, precond=True):
        """Solve K ut = F for nodal loads f ((V,) or (nrhs, V), float64).
        precond: face-block Jacobi preconditioner (Sec. 5.1) in the inner CG.
        Returns (traces, u or None, list of info dicts)."""
        f2 = f.reshape(-1, self.volume_size).contiguous()
        nrhs = f2.shape[0]
        if f2.dtype != torch.float64 or not f2.is_cuda:
            raise ValueError("f must be a float64 CUDA tensor")
        tr = torch.empty((nrhs, self.trace_size), dtype=torch.float64, device=f2.device)
        u = torch.empty_like(f2) if return_u else None
        b = None if bdry is None else bdry.reshape(nrhs, self.boundary_size).contiguous()
        x = None if x0 is None else x0.reshape(nrhs, self.trace_size).contiguous()
        info = (_capi.HdgSolveInfo * nrhs)()
        opts = self._opts(tol, inner, max_iter, max_outer, inner_tol, precond)
        st = _capi.lib().hdg_solve(self._h, nrhs, _lams(lam, nrhs), ctypes.c_void_p(f2.data_ptr()),
                                   ctypes.c_void_p(b.data_ptr() if b is not None else 0),
                                   ctypes.c_void_p(x.data_ptr() if x is not None else 0),
                                   ctypes.c_void_p(tr.data_ptr()),
                                   ctypes.c_void_p(u.data_ptr() if u is not None else 0),
                                   ctypes.byref(opts), info, _stream())
        infos = [info[i].as_dict() for i in range(nrhs)]
        if check:
            _capi.check(st, "hdg_solve")
        shape_t = (self.trace_size,) if f.dim() == 1 else (nrhs, self.trace_size)
        return tr.reshape(shape_t), (u.reshape(f.shape) if u is not None else None), infos

    def solve_adjoint(self, u, grad_u, lam, tol=1e-10, inner="fp32", max_iter=50000, max_outer=40,
                      inner_tol=0.0):
        """dL/df and dL/dlambda for dL/du = grad_u at the forward solution u
        (homogeneous boundary data)."""
        u2 = u.reshape(-1, self.volume_size).contiguous()
        g2 = grad_u.reshape(-1, self.volume_size).contiguous().to(torch.float64)
        nrhs = u2.shape[0]
        gf = torch.empty_like(u2)
        gl = torch.empty(nrhs, dtype=torch.float64, device=u2.device)
        info = (_capi.HdgSolveInfo * nrhs)()
        opts = self._opts(tol, inner, max_iter, max_outer, inner_tol)
        st = _capi.lib().hdg_solve_adjoint(self._h, nrhs, _lams(lam, nrhs), ctypes.c_void_p(u2.data_ptr()),
                                           ctypes.c_void_p(g2.data_ptr()), ctypes.c_void_p(gf.data_ptr()),
                                           ctypes.c_void_p(gl.data_ptr()), ctypes.byref(opts), info, _stream())
        _capi.check(st, "hdg_solve_adjoint")
        return gf.reshape(u.shape), gl, [info[i].as_dict() for i in range(nrhs)]


def measure_fma_peak(precision="fp64"):
    """Fused multiply-add rate of the current device in TFLOP/s (a register
    FMA loop on every SM, CUDA events): the measured denominator of the
    FP64 and FP32 pipe rooflines."""
    out = ctypes.c_double()
    st = _capi.lib().hdg_measure_fma_peak(_capi.PRECISION[precision], ctypes.byref(out), _stream())
    _capi.check(st, "hdg_measure_fma_peak")
    return out.value


class HDGLowDim:
    """The condensed operator on a 1D or 2D Cartesian mesh (apply only).

    ne: one or two element counts; grid: that many increasing coordinate
    arrays of length ne[d] + 1; bc: two or four sides (x1-, x1+[, x2-,
    x2+]), 0 Dirichlet, 1 Neumann; p: degree 1..16.
    """

    def __init__(self, ne, grid, bc=None, p=4, tau_hat=25.0, mass_lumped=False):
        L = _capi.lib()
        torch.cuda.init()
        self.ne = tuple(int(v) for v in ne)
        self.dim = len(self.ne)
        self.p, self.n = int(p), int(p) + 1
        bc = (0,) * (2 * self.dim) if bc is None else tuple(int(v) for v in bc)
        self._grid = [(ctypes.c_double * (self.ne[d] + 1))(*[float(v) for v in grid[d]]) for d in range(self.dim)]
        m = _capi.HdgLowDimMesh()
        m.dim = self.dim
        for d in range(self.dim):
            m.ne[d] = self.ne[d]
            m.h_grid[d] = ctypes.cast(self._grid[d], ctypes.POINTER(ctypes.c_double))
        for s_ in range(2 * self.dim):
            m.bc[s_] = bc[s_]
        o = _capi.HdgOptions(float(tau_hat), int(bool(mass_lumped)))
        h = ctypes.c_void_p()
        _capi.check(L.hdg_lowdim_setup(ctypes.byref(m), self.p, ctypes.byref(o), ctypes.byref(h)),
                    "hdg_lowdim_setup")
        self._h = h
        self.trace_size = int(L.hdg_lowdim_trace_size(h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _capi.lib().hdg_lowdim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, lam, basis="nodal", out=None):
        """y = K x (homogeneous Dirichlet data); x: (T,) or (nrhs, T) float64 CUDA tensor."""
        x2 = x.reshape(-1, self.trace_size)
        if not x2.is_cuda or not x2.is_contiguous() or x2.dtype != torch.float64:
            raise ValueError("x must be a contiguous float64 CUDA tensor")
        y = torch.empty_like(x2) if out is None else out.reshape(-1, self.trace_size)
        nrhs = x2.shape[0]
        st = _capi.lib().hdg_lowdim_apply(self._h, nrhs, _lams(lam, nrhs), _capi.BASIS[basis],
                                          ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y.data_ptr()), _stream())
        _capi.check(st, "hdg_lowdim_apply")
        return y.reshape(x.shape)


class HDGSolve(torch.autograd.Function):
    """u = solve(f, lambda) with homogeneous boundary data; backward runs the
    hand-written adjoint solve (dL/df = M z_u, dL/dlambda = -z_u^T M u)."""

    @staticmethod
    def forward(ctx, f, lam, hdg, tol=1e-10, inner="fp32"):
        lam_list = lam.detach().reshape(-1).tolist()
        _, u, _ = hdg.solve(f.detach(), lam_list, tol=tol, inner=inner)
        ctx.hdg, ctx.tol, ctx.inner, ctx.lam = hdg, tol, inner, lam_list
        ctx.save_for_backward(u)
        ctx.lam_shape = lam.shape
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        gf, gl, _ = ctx.hdg.solve_adjoint(u, grad_u.contiguous(), ctx.lam, tol=ctx.tol, inner=ctx.inner)
        return gf, gl.reshape(ctx.lam_shape), None, None, None
