"""The method's algebra against the plain definition, on the CPU.

The GPU path evaluates the element operator in its factorised, transformed
form: with the generalised eigenpairs S^T M S = I, S^T L S = Lambda
(Eq. (generalized_eigenvalue_decomposition)),
B_S = S^T B - S^T D M^-1 C (Eq. (hdgbs)), H = G + C^T M^-1 C and
D_Z = lambda d0 + d1 Lambda_i + d2 Lambda_j + d3 Lambda_k,

    K-hat_e = blkdiag(d_i H along direction i) - E^T D_Z^-1 E,
    E = [d1 (I (x) I (x) B_S), d2 (I (x) B_S (x) I), d3 (B_S (x) I (x) I)]

(Eq. (hdg_operator_factorized) transformed as in Sec. 4.3,
Alg. (hdg_op_3d_transformed)), and K_e = T^-T K-hat_e T^-1 with T = S (x) S
on every face.  This test builds that form from an independent
eigen-decomposition (scipy) and checks it against the oracle's dense
Schur complement K_e = G_e - R_e^T A_e^-1 R_e, for the exact and the
lumped mass, on stretched elements, lambda = 0 and lambda > 0.  It pins the
operator the kernels compute, not the kernels.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.basis1d import Matrices1D
from oracle.element3d import condense, metric


def _factorised(m1, h, lam):
    n = m1.n
    M, D, B, C, L, G = m1.M, m1.D, m1.B, m1.C, m1.L, m1.G
    Lam, S = sla.eigh(L, M)                       # S^T M S = I, S^T L S = diag(Lam)
    Minv = np.linalg.inv(M)
    BS = S.T @ B - S.T @ D @ Minv @ C             # n x 2
    H = G + C.T @ Minv @ C                        # 2 x 2
    d0, d1, d2, d3 = metric(h)
    I = np.eye(n)
    kron3 = lambda c, b, a: np.kron(c, np.kron(b, a))
    E = np.hstack([d1 * kron3(I, I, BS), d2 * kron3(I, BS, I), d3 * kron3(BS, I, I)])
    li = np.arange(n ** 3) % n
    lj = (np.arange(n ** 3) // n) % n
    lk = np.arange(n ** 3) // (n * n)
    DZ = lam * d0 + d1 * Lam[li] + d2 * Lam[lj] + d3 * Lam[lk]
    face = sla.block_diag(d1 * kron3(I, I, H), d2 * kron3(I, H, I), d3 * kron3(H, I, I))
    Khat = face - E.T @ (E / DZ[:, None])
    # face transforms: ut_nodal = T ut_hat, T = S (x) S on the two face axes
    I2 = np.eye(2)
    T = sla.block_diag(kron3(S, S, I2), kron3(S, I2, S), kron3(I2, S, S))
    Tinv = np.linalg.inv(T)
    return Tinv.T @ Khat @ Tinv, Khat, S


@pytest.mark.parametrize("mass", ["exact", "gll"])
@pytest.mark.parametrize("p,h,lam", [(1, (0.7, 1.3, 0.4), 0.0), (3, (0.5, 0.9, 2.0), 1.5), (5, (1.1, 0.3, 0.8), 10.0)])
def test_factorised_transformed_operator_equals_dense_condensation(p, h, lam, mass):
    m1 = Matrices1D(p, 25.0, mass)
    K_dense = condense(m1, h, lam, tier="O1")
    K_fact, Khat, S = _factorised(m1, h, lam)
    scale = np.abs(K_dense).max()
    assert np.abs(K_fact - K_dense).max() <= 1e-11 * scale
    # the transformed operator is symmetric
    assert np.abs(Khat - Khat.T).max() <= 1e-11 * np.abs(Khat).max()


def test_mode_parity_of_bs_on_gll_points():
    """The GLL points are mirror symmetric, so every eigenvector is even or
    odd and B_S[m] = c_m (1, sigma_m): the property the kernels' sum /
    difference split uses (S = x_lo + x_hi reaches even modes only)."""
    m1 = Matrices1D(6, 25.0)
    Lam, S = sla.eigh(m1.L, m1.M)
    BS = S.T @ m1.B - S.T @ m1.D @ np.linalg.inv(m1.M) @ m1.C
    R = np.eye(m1.n)[::-1]
    for m in range(m1.n):
        sig = 1.0 if np.allclose(R @ S[:, m], S[:, m], atol=1e-10) else -1.0
        assert np.allclose(R @ S[:, m], sig * S[:, m], atol=1e-10)
        assert abs(BS[m, 1] - sig * BS[m, 0]) <= 1e-10 * max(1.0, abs(BS[m, 0]))
