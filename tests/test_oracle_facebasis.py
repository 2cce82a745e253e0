"""Pins of the face eigenbasis that defines the library's transformed trace
basis (oracle/facebasis.py), on the CPU.

The basis is fixed by Eq. (generalized_eigenvalue_decomposition) plus a
documented parity, order and sign convention (include/hdg.h).  These tests
check each property from its definition, and that the dense oracle K
expressed in the basis has the factorised structure of
Eq. (hdg_operator_factorized) built with the same S; a wrong order, sign or
transpose anywhere in the construction fails one of them.
"""
import numpy as np
import pytest

from oracle.basis1d import Matrices1D
from oracle.element3d import condense, kron3, metric
from oracle.facebasis import abs_element_sum, apply_transformed, face_eigenbasis, to_nodal, to_transformed
from oracle.solver import Problem


@pytest.mark.parametrize("mass", ["exact", "gll"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 8, 12, 16])
def test_identities_parity_order_sign(p, mass):
    m1 = Matrices1D(p, 25.0, mass)
    S, Lam, BS = face_eigenbasis(m1)
    n = m1.n
    ne = (n + 1) // 2
    assert np.abs(S.T @ m1.M @ S - np.eye(n)).max() <= 1e-13
    assert np.abs(S.T @ m1.L @ S - np.diag(Lam)).max() <= 1e-13 * np.abs(Lam).max()
    J = np.eye(n)[::-1]
    for m in range(n):
        sig = 1.0 if m < ne else -1.0
        assert np.abs(J @ S[:, m] - sig * S[:, m]).max() <= 1e-12 * np.abs(S[:, m]).max()
        assert BS[m, 0] > 0.5
        assert abs(BS[m, 1] - sig * BS[m, 0]) <= 1e-12 * BS[m, 0]
    assert np.all(np.diff(Lam[:ne]) > 0) and np.all(np.diff(Lam[ne:]) > 0)
    # every eigenvalue of the pencil appears once
    ref = np.sort(np.linalg.eigvals(np.linalg.solve(m1.M, m1.L)).real)
    assert np.abs(np.sort(Lam) - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("p,h,lam", [(2, (0.7, 1.3, 0.4), 0.0), (4, (0.5, 0.9, 2.0), 3.0)])
def test_dense_operator_in_the_basis_has_the_factorised_form(p, h, lam):
    # T^T K_e T with T = S (x) S on each face equals blkdiag(d_i H) - E^T D_Z^-1 E
    m1 = Matrices1D(p, 25.0)
    S, Lam, BS = face_eigenbasis(m1)
    n = m1.n
    K = condense(m1, h, lam, tier="O1")
    I, I2 = np.eye(n), np.eye(2)
    T = np.block([[kron3(S, S, I2), np.zeros((2 * n * n, 4 * n * n))],
                  [np.zeros((2 * n * n, 2 * n * n)), kron3(S, I2, S), np.zeros((2 * n * n, 2 * n * n))],
                  [np.zeros((2 * n * n, 4 * n * n)), kron3(I2, S, S)]])
    Khat = T.T @ K @ T
    d0, d1, d2, d3 = metric(h)
    H = m1.G + m1.C.T @ np.linalg.solve(m1.M, m1.C)
    E = np.hstack([d1 * kron3(I, I, BS), d2 * kron3(I, BS, I), d3 * kron3(BS, I, I)])
    li, lj, lk = np.arange(n ** 3) % n, (np.arange(n ** 3) // n) % n, np.arange(n ** 3) // (n * n)
    DZ = lam * d0 + d1 * Lam[li] + d2 * Lam[lj] + d3 * Lam[lk]
    face = np.block([[d1 * kron3(I, I, H), np.zeros((2 * n * n, 4 * n * n))],
                     [np.zeros((2 * n * n, 2 * n * n)), d2 * kron3(I, H, I), np.zeros((2 * n * n, 2 * n * n))],
                     [np.zeros((2 * n * n, 4 * n * n)), d3 * kron3(H, I, I)]])
    ref = face - E.T @ (E / DZ[:, None])
    assert np.abs(Khat - ref).max() <= 1e-11 * np.abs(ref).max()


def test_global_transformed_apply_and_bound():
    ne = (3, 2, 2)
    rng = np.random.default_rng(0)
    grid = [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, v))]) for v in ne]
    pr = Problem(ne, grid, (0, 1, 0, 0, 1, 0), 3, 25.0, 1.3)
    x = rng.uniform(-1.0, 1.0, pr.mesh.n_trace)
    z = rng.uniform(-1.0, 1.0, pr.mesh.n_trace)
    y = apply_transformed(pr, x)
    # K-hat = T^T K T is symmetric, and each entry is bounded by the sum of
    # the absolute element contributions
    assert abs(z @ y - x @ apply_transformed(pr, z)) <= 1e-12 * np.abs(y).max() * len(y)
    A = abs_element_sum(pr, x)
    assert np.all(np.abs(y) <= A * (1.0 + 1e-12))
    # the input transform (S^T M per face) inverts the nodal map (S per face)
    m1 = pr.m1
    S, _, _ = face_eigenbasis(m1)
    StM = np.kron(S.T @ m1.M, S.T @ m1.M)
    xn = to_nodal(pr, x)
    back = (xn.reshape(-1, pr.mesh.n2) @ StM.T).ravel()
    assert np.abs(back - x).max() <= 1e-12
    # K-hat x-hat is the transformed image of K applied to the nodal traces
    assert np.abs(to_transformed(pr, pr.apply(xn)) - y).max() == 0.0
