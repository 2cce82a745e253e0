"""Pins for the oracle's 3D element system and its condensation.

* The tensor-product table (Tab. hdg_matrices_threed, metric factors of
  Sec. 3.2) is rebuilt here by direct 3D/face quadrature of the weak form of
  Eq. (ldg_discretization) on a random cuboid, with the penalty
  tau_i = 2 tau_hat / h_i (Eq. penalty_parameter_oned and its 3D form).
* K_e = G_e - R_e^T A_e^{-1} R_e (Eq. hdg_operator) must be symmetric, have
  the constants as null vector at lambda = 0 (u = 1, q = 0 solves every
  element system then) and be positive definite for lambda > 0.
* The two condensation tiers (dense LU; q eliminated first) must agree.
"""
import numpy as np
import pytest

from oracle.basis1d import Matrices1D, gauss_legendre, lagrange
from oracle.element3d import (condense_lu, condense_q_eliminated, element_blocks,
                              element_system)


def _direct_blocks(p, tau_hat, h):
    n = p + 1
    m1 = Matrices1D(p, tau_hat)
    tq, wq = gauss_legendre(n + 1)
    V, dV = lagrange(m1.nodes, tq)             # (q, n)
    ends, _ = lagrange(m1.nodes, np.array([-1.0, 1.0]))
    h = np.asarray(h, dtype=np.float64)
    jac = np.prod(h) / 8.0
    nq = len(tq)
    # volume basis at the tensor quadrature grid: Phi[q3, q2, q1, I]
    n3 = n ** 3
    Phi = np.zeros((nq, nq, nq, n3))
    dPhi = np.zeros((3, nq, nq, nq, n3))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                I = i + n * j + n * n * k
                Phi[:, :, :, I] = V[:, k][:, None, None] * V[:, j][None, :, None] * V[:, i][None, None, :]
                dPhi[0, :, :, :, I] = (2 / h[0]) * V[:, k][:, None, None] * V[:, j][None, :, None] * dV[:, i][None, None, :]
                dPhi[1, :, :, :, I] = (2 / h[1]) * V[:, k][:, None, None] * dV[:, j][None, :, None] * V[:, i][None, None, :]
                dPhi[2, :, :, :, I] = (2 / h[2]) * dV[:, k][:, None, None] * V[:, j][None, :, None] * V[:, i][None, None, :]
    W = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * jac
    Pf = Phi.reshape(-1, n3)
    Wf = W.reshape(-1)
    out = {"M": Pf.T @ (Wf[:, None] * Pf)}
    for d in range(3):
        out["D%d" % (d + 1)] = Pf.T @ (Wf[:, None] * dPhi[d].reshape(-1, n3))
    out["E"] = np.zeros((n3, n3))
    axes = [(1, 2), (0, 2), (0, 1)]
    for d in range(3):
        a, b = axes[d]
        tau = 2.0 * tau_hat / h[d]
        f2 = 2 * n * n
        G = np.zeros((f2, f2))
        B = np.zeros((n3, f2))
        C = np.zeros((n3, f2))
        for s in range(2):
            normal = -1.0 if s == 0 else 1.0
            # volume basis on face (d, s): Phi restricted, sampled on the face grid (qb, qa)
            PhiF = np.zeros((nq, nq, n3))
            for k in range(n):
                for j in range(n):
                    for i in range(n):
                        I = i + n * j + n * n * k
                        idx = [i, j, k]
                        fa = V[:, idx[a]]
                        fb = V[:, idx[b]]
                        PhiF[:, :, I] = ends[s, idx[d]] * fb[:, None] * fa[None, :]
            wF = (wq[:, None] * wq[None, :]) * (h[a] * h[b] / 4.0)
            PFf = PhiF.reshape(-1, n3)
            wFf = wF.reshape(-1)
            out["E"] += tau * PFf.T @ (wFf[:, None] * PFf)
            # trace basis mu_(c1, c2) on face (d, s), c1 along axis a (fastest)
            mu = np.zeros((nq, nq, n * n))
            for c2 in range(n):
                for c1 in range(n):
                    mu[:, :, c1 + n * c2] = V[:, c2][:, None] * V[:, c1][None, :]
            muf = mu.reshape(-1, n * n)
            for c2 in range(n):
                for c1 in range(n):
                    if d == 0:
                        li = s + 2 * (c1 + n * c2)
                    elif d == 1:
                        li = c1 + n * (s + 2 * c2)
                    else:
                        li = c1 + n * (c2 + n * s)
                    col = muf[:, c1 + n * c2]
                    B[:, li] = -tau * PFf.T @ (wFf * col)
                    C[:, li] = normal * PFf.T @ (wFf * col)
                    for e2 in range(n):
                        for e1 in range(n):
                            if d == 0:
                                lj = s + 2 * (e1 + n * e2)
                            elif d == 1:
                                lj = e1 + n * (s + 2 * e2)
                            else:
                                lj = e1 + n * (e2 + n * s)
                            G[li, lj] = tau * np.sum(wFf * col * muf[:, e1 + n * e2])
        out["G%d" % (d + 1)] = G
        out["B%d" % (d + 1)] = B
        out["C%d" % (d + 1)] = C
    return out


@pytest.mark.parametrize("p,tau_hat", [(1, 1.0), (2, 25.0), (3, 4.0)])
def test_tensor_table_matches_direct_quadrature(p, tau_hat):
    rng = np.random.default_rng(7 + p)
    h = rng.uniform(0.3, 2.5, 3)
    m1 = Matrices1D(p, tau_hat)
    table = element_blocks(m1, h)
    direct = _direct_blocks(p, tau_hat, h)
    for key, ref in direct.items():
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(table[key] - ref).max() < 1e-12 * scale, key


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_condensed_element_invariants(p):
    rng = np.random.default_rng(100 + p)
    m1 = Matrices1D(p, tau_hat=rng.uniform(0.5, 30.0))
    h = rng.uniform(0.2, 3.0, 3)
    sysm = element_system(m1, h, 0.8)
    np.testing.assert_allclose(sysm, sysm.T, atol=1e-12 * np.abs(sysm).max())
    K0 = condense_lu(m1, h, 0.0)
    np.testing.assert_allclose(K0, K0.T, atol=1e-11 * np.abs(K0).max())
    ones = np.ones(K0.shape[0])
    assert np.abs(K0 @ ones).max() < 1e-11 * np.abs(K0).max()
    ev0 = np.linalg.eigvalsh(0.5 * (K0 + K0.T))
    assert ev0[0] > -1e-10 * ev0[-1] and ev0[1] > 1e-8 * ev0[-1]   # one-dimensional null space
    K1 = condense_lu(m1, h, 2.5)
    assert np.linalg.eigvalsh(0.5 * (K1 + K1.T))[0] > 0


@pytest.mark.parametrize("p,lam", [(1, 0.0), (2, 1.3), (3, 0.0), (4, 7.0)])
def test_condensation_tiers_agree(p, lam):
    rng = np.random.default_rng(200 + p)
    m1 = Matrices1D(p, tau_hat=rng.uniform(0.5, 30.0))
    h = rng.uniform(0.2, 3.0, 3)
    K1 = condense_lu(m1, h, lam)
    K2 = condense_q_eliminated(m1, h, lam)
    assert np.abs(K1 - K2).max() < 1e-12 * np.abs(K1).max()
