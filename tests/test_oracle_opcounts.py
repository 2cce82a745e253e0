"""The paper's operation counts (tests/golden/paper_operation_counts.txt)
pinned by counting evaluators, on the CPU.

Two small evaluators restate, loop by loop, the element operator of
Alg. (hdg_op_3d_transformed) (transformed basis: expand the six faces into
the element eigenspace, scale by D_Z^-1, contract back, add the face term)
and Alg. (hdg_op_3d) (nodal basis: the same core between per-face basis
changes S^T M (x) S^T M and M S (x) M S, each as two n x n matrix products).
They count every multiply-add as two flops and every access to the trace
vectors and to the stored D_Z^-1 as one load or store (y += counts as a load
and a store).  Each evaluator must reproduce the oracle's dense element
operator, and its counts must have the leading terms the paper prints.
"""
import os
import re

import numpy as np
import pytest

from oracle.basis1d import Matrices1D
from oracle.element3d import condense, metric
from oracle.facebasis import face_eigenbasis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_operation_counts.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, expr = re.split(r"\s{2,}", line.strip(), maxsplit=1)
        out[name] = expr.replace("^", "**")
    return out


def _local_index(d, s, c1, c2, n):
    # element-local trace ordering of oracle/element3d.py: blocks ut1 | ut2 | ut3
    if d == 0:
        return s + 2 * (c1 + n * c2)
    if d == 1:
        return 2 * n * n + c1 + n * (s + 2 * c2)
    return 4 * n * n + c1 + n * (c2 + n * s)


class Counter:
    def __init__(self):
        self.flops = 0
        self.mem = 0


def tpt_element(m1, h, lam, xf, cnt):
    """Alg. (hdg_op_3d_transformed) on one element.  xf[d][s] is the n x n
    face array (axes: the two other directions in increasing order).
    Returns yf with the same layout."""
    n = m1.n
    S, Lam, BS = face_eigenbasis(m1)
    H = m1.G + m1.C.T @ np.linalg.solve(m1.M, m1.C)
    d0, d1, d2, d3 = metric(h)
    dd = (d1, d2, d3)
    # D_Z^-1 stored per point
    Dinv = np.empty((n, n, n))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                Dinv[i, j, k] = 1.0 / (lam * d0 + d1 * Lam[i] + d2 * Lam[j] + d3 * Lam[k])
    x = [[np.empty((n, n)) for _ in range(2)] for _ in range(3)]
    for d in range(3):
        for s in range(2):
            for a in range(n):
                for b in range(n):
                    x[d][s][a, b] = xf[d][s][a, b]
                    cnt.mem += 1
    u = np.zeros((n, n, n))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                F = 0.0
                for s in range(2):
                    F += BS[i, s] * d1 * x[0][s][j, k]
                    F += BS[j, s] * d2 * x[1][s][i, k]
                    F += BS[k, s] * d3 * x[2][s][i, j]
                    cnt.flops += 3 * 2
                u[i, j, k] = F * Dinv[i, j, k]
                cnt.flops += 1
                cnt.mem += 1
    y = [[np.zeros((n, n)) for _ in range(2)] for _ in range(3)]
    for d in range(3):
        for s in range(2):
            for a in range(n):
                for b in range(n):
                    acc = 0.0
                    for t in range(2):
                        acc += dd[d] * H[s, t] * x[d][t][a, b]
                        cnt.flops += 2
                    y[d][s][a, b] = acc
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for s in range(2):
                    y[0][s][j, k] -= dd[0] * BS[i, s] * u[i, j, k]
                    y[1][s][i, k] -= dd[1] * BS[j, s] * u[i, j, k]
                    y[2][s][i, j] -= dd[2] * BS[k, s] * u[i, j, k]
                    cnt.flops += 3 * 2
    for d in range(3):
        for s in range(2):
            cnt.mem += 2 * n * n   # y += : load and store
    return y


def face_basis_change(A, x, cnt):
    """(A (x) A) applied to an n x n face array as two matrix products."""
    n = A.shape[0]
    t = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            for m in range(n):
                t[a, b] += A[a, m] * x[m, b]
                cnt.flops += 2
    out = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            for m in range(n):
                out[a, b] += t[a, m] * A[b, m]
                cnt.flops += 2
    return out


def tp_element(m1, h, lam, xf, cnt):
    """Alg. (hdg_op_3d): face basis changes around the transformed core."""
    S, _, _ = face_eigenbasis(m1)
    StM, MS = S.T @ m1.M, m1.M @ S
    xh = [[face_basis_change(StM, xf[d][s], cnt) for s in range(2)] for d in range(3)]
    yh = tpt_element(m1, h, lam, xh, cnt)
    return [[face_basis_change(MS, yh[d][s], cnt) for s in range(2)] for d in range(3)]


def _faces_from_local(v, n):
    # face array [a, b]: a = faster face axis, b = slower one
    return [[np.array([[v[_local_index(d, s, a, b, n)] for b in range(n)] for a in range(n)])
             for s in range(2)] for d in range(3)]


def _local_from_faces(f, n):
    v = np.zeros(6 * n * n)
    for d in range(3):
        for s in range(2):
            for a in range(n):
                for b in range(n):
                    v[_local_index(d, s, a, b, n)] = f[d][s][a, b]
    return v


@pytest.mark.parametrize("p", [1, 2, 3])
def test_counting_evaluators_reproduce_the_oracle(p):
    m1 = Matrices1D(p, 25.0)
    n = m1.n
    h, lam = (0.6, 1.1, 0.9), 2.5
    K = condense(m1, h, lam, tier="O1")
    S, _, _ = face_eigenbasis(m1)
    T = np.kron(S, S)
    Tloc = np.zeros((6 * n * n, 6 * n * n))
    for d in range(3):
        for s in range(2):
            pos = [_local_index(d, s, a, b, n) for b in range(n) for a in range(n)]
            Tloc[np.ix_(pos, pos)] = T
    x = np.random.default_rng(p).uniform(-1.0, 1.0, 6 * n * n)
    # nodal: Alg. (hdg_op_3d) == dense K_e
    y = _local_from_faces(tp_element(m1, h, lam, _faces_from_local(x, n), Counter()), n)
    assert np.abs(y - K @ x).max() <= 1e-11 * np.abs(K @ x).max()
    # transformed: Alg. (hdg_op_3d_transformed) == T^T K_e T
    yt = _local_from_faces(tpt_element(m1, h, lam, _faces_from_local(x, n), Counter()), n)
    ref = Tloc.T @ K @ Tloc @ x
    assert np.abs(yt - ref).max() <= 1e-11 * np.abs(ref).max()


def test_counts_match_the_paper():
    g = _golden()
    counts = {}
    for n in (2, 3, 4, 5):
        m1 = Matrices1D(n - 1, 25.0)
        xf = _faces_from_local(np.ones(6 * n * n), n)
        c_tpt, c_tp = Counter(), Counter()
        tpt_element(m1, (1.0, 1.0, 1.0), 1.0, xf, c_tpt)
        tp_element(m1, (1.0, 1.0, 1.0), 1.0, xf, c_tp)
        counts[n] = (c_tpt.flops, c_tp.flops, c_tpt.mem)
    for n, (f_tpt, f_tp, mem) in counts.items():
        lead_tpt = eval(g["HDG-TPT flops"], {"n": n})
        lead_tp = eval(g["HDG-TP flops"], {"n": n})
        # leading n^3 terms as printed; the rest is the face term, O(n^2)
        assert (f_tpt - lead_tpt) == 24 * n * n, (n, f_tpt)
        assert (f_tp - lead_tp) == 24 * n * n, (n, f_tp)
        assert mem == eval(g["loads/stores"], {"n": n})
