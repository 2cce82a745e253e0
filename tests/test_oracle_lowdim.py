"""Pins of the 1D/2D oracle (oracle/lowdim.py), CPU only.

* constant patch: lambda = 0, ut = 1 gives (u, q) = (1, 0), so K_e 1 = 0;
* K_e symmetric, positive definite for lambda > 0;
* the 1D system of Eq. (ldg_element_operator) is the dim = 1 case of the
  generic construction, entry by entry against the element matrices of
  Eq. (element_matrices) written out;
* polynomial reproduction (exact mass): u = x^a (1D) and x^a y^b (2D) with
  a, b <= p are reproduced at the nodes to round-off, with Dirichlet and
  Neumann sides;
* convergence: sin solutions converge at order about p + 1 (Sec. 2.1);
* agreement with the separately pinned 3D oracle: on a mesh one element
  thick in x3 with Neumann x3-sides, x3-independent data give the 2D
  solution at every node of every x3-layer.
"""
import numpy as np
import pytest

from oracle.basis1d import Matrices1D
from oracle.lowdim import DIRICHLET, NEUMANN, LowDimProblem, condense, element_system


@pytest.mark.parametrize("h", [(0.7,), (0.4, 1.3)])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_constant_patch_symmetry_definiteness(h, p):
    m1 = Matrices1D(p, 25.0)
    K0 = condense(m1, h, 0.0)
    assert np.abs(K0 @ np.ones(K0.shape[0])).max() < 1e-10 * np.abs(K0).max()
    K = condense(m1, h, 2.0)
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > 0


def test_one_dimensional_system_is_eq_ldg_element_operator():
    p, h, lam = 4, 0.37, 1.7
    m1 = Matrices1D(p, 3.0)
    S, Me = element_system(m1, (h,), lam)
    n = p + 1
    Mh, Dh, Eh, Gh, Bh, Ch = h / 2 * m1.M, m1.D, 2 / h * m1.E, 2 / h * m1.G, 2 / h * m1.B, m1.C
    ref = np.block([[lam * Mh + Eh, -Dh, Bh], [-Dh.T, -Mh, Ch], [Bh.T, Ch.T, Gh]])
    assert S.shape == (2 * n + 2, 2 * n + 2)
    assert np.abs(S - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(Me - Mh).max() < 1e-15


def _grid(ne, seed, length=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for v in ne:
        w = rng.uniform(0.5, 2.0, v)
        out.append(np.concatenate([[0.0], np.cumsum(w)]) / w.sum() * length + 0.2)
    return out


def _boundary_data(pr, u, grad):
    """g_D = u on Dirichlet sides, g_N = n . grad u on Neumann sides."""
    m = pr.mesh
    X = m.bdry_coords(pr.m1.nodes)
    g = np.zeros(m.n_bdry)
    for side in range(2 * m.dim):
        d, s = side // 2, side % 2
        sl = slice(m.side_offset[side] * m.nf, (m.side_offset[side] + m.n_other(d)) * m.nf)
        g[sl] = u(X[sl]) if m.bc[side] == DIRICHLET else (1.0 if s else -1.0) * grad(X[sl])[:, d]
    return g


@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (0, 1)])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_polynomial_reproduction_1d(p, bc):
    a, lam = p, 0.8
    pr = LowDimProblem((4,), _grid((4,), 1), bc, p, 25.0, lam)
    X = pr.mesh.volume_coords(pr.m1.nodes)[:, 0]
    u = lambda x: x[..., 0] ** a if x.ndim > 1 else x ** a
    f = lam * X ** a - a * (a - 1) * X ** max(a - 2, 0)
    grad = lambda x: (a * x[:, 0] ** (a - 1))[:, None]
    _, uh = pr.solve(f, _boundary_data(pr, lambda x: x[:, 0] ** a, grad))
    assert np.abs(uh - X ** a).max() < 1e-10


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 0, 0, 1), (0, 1, 1, 0)])
@pytest.mark.parametrize("p", [1, 3])
def test_polynomial_reproduction_2d(p, bc):
    a, b, lam = p, max(p - 1, 1), 0.0
    pr = LowDimProblem((3, 2), _grid((3, 2), 2), bc, p, 10.0, lam)
    X = pr.mesh.volume_coords(pr.m1.nodes)
    uex = lambda x: x[:, 0] ** a * x[:, 1] ** b
    lap = a * (a - 1) * X[:, 0] ** max(a - 2, 0) * X[:, 1] ** b + b * (b - 1) * X[:, 0] ** a * X[:, 1] ** max(b - 2, 0)
    grad = lambda x: np.stack([a * x[:, 0] ** (a - 1) * x[:, 1] ** b, b * x[:, 0] ** a * x[:, 1] ** (b - 1)], axis=1)
    _, uh = pr.solve(lam * uex(X) - lap, _boundary_data(pr, uex, grad))
    assert np.abs(uh - uex(X)).max() < 1e-10


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_order_1d(p):
    errs = []
    for ne in (4, 8):
        pr = LowDimProblem((ne,), [np.linspace(0.0, 1.0, ne + 1)], (0, 0), p, 1.0, 1.0)
        X = pr.mesh.volume_coords(pr.m1.nodes)[:, 0]
        f = (1.0 + np.pi ** 2) * np.sin(np.pi * X)
        _, uh = pr.solve(f, np.zeros(pr.mesh.n_bdry))
        errs.append(np.abs(uh - np.sin(np.pi * X)).max())
    assert np.log2(errs[0] / errs[1]) > p + 0.6


def test_two_dimensional_matches_three_dimensional_layer():
    """x3-independent data on a 3D mesh of one element layer with Neumann
    x3-sides: the 3D oracle's solution is the 2D oracle's, node by node."""
    from oracle.solver import Problem
    p, lam, tau = 2, 1.5, 5.0
    g2 = _grid((3, 2), 7)
    g3 = g2 + [np.array([0.0, 0.9])]
    bc2 = (0, 1, 0, 0)
    pr2 = LowDimProblem((3, 2), g2, bc2, p, tau, lam)
    pr3 = Problem((3, 2, 1), g3, bc2 + (1, 1), p, tau, lam)
    uex = lambda x: np.cos(1.3 * x[:, 0]) * (1.0 + x[:, 1] ** 2)
    grad = lambda x: np.stack([-1.3 * np.sin(1.3 * x[:, 0]) * (1.0 + x[:, 1] ** 2),
                               np.cos(1.3 * x[:, 0]) * 2.0 * x[:, 1], 0.0 * x[:, 0]], axis=1)
    X2 = pr2.mesh.volume_coords(pr2.m1.nodes)
    f2 = lam * uex(X2) + (1.69 * np.cos(1.3 * X2[:, 0]) * (1.0 + X2[:, 1] ** 2) - 2.0 * np.cos(1.3 * X2[:, 0]))
    _, u2 = pr2.solve(f2, _boundary_data(pr2, uex, lambda x: grad(x)[:, :2]))
    X3 = pr3.mesh.volume_coords(pr3.m1.nodes)
    f3 = lam * uex(X3) + (1.69 * np.cos(1.3 * X3[:, 0]) * (1.0 + X3[:, 1] ** 2) - 2.0 * np.cos(1.3 * X3[:, 0]))
    B3, nrm = pr3.mesh.bdry_coords(pr3.m1.nodes)
    bd3 = np.zeros(pr3.mesh.n_bdry)
    for side in range(6):
        lo = pr3.mesh.side_offset[side] * pr3.mesh.n2
        cnt = [2 * 1, 2 * 1, 3 * 1, 3 * 1, 3 * 2, 3 * 2][side] * pr3.mesh.n2
        sl = slice(lo, lo + cnt)
        if pr3.mesh.bc[side] == 0:
            bd3[sl] = uex(B3[sl])
        else:
            bd3[sl] = np.sum(nrm[sl] * grad(B3[sl]), axis=1)
    _, u3, _, _ = pr3.solve(f=f3, bdry=bd3, method="direct")
    n = p + 1
    u3 = u3.reshape(-1, n, n * n)   # (element, k, j i)
    for k in range(n):
        assert np.abs(u3[:, k, :].ravel() - u2).max() < 1e-11
