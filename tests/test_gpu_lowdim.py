"""GPU parity of the 1D (Alg. hdg_op_1d) and 2D condensed operators
(hdg_lowdim_apply) against the CPU oracle (oracle/lowdim.py).

Nodal basis: element by element against the oracle's dense-condensed
global apply, 1e-12 relative (max-norm).  Transformed basis (2D): the
operator K-hat = T^T K T with T = S per edge and S^T M S = I is similar to
K M_f^-1 (T T^T = M_f^-1), so its eigenvalues must equal those of the
oracle's K M_f^-1; it must also be symmetric.  In 1D the faces are points
and both bases give K.  Meshes span several CTAs with ragged tails,
stretched grids, Dirichlet/Neumann sides, single elements and p = 1..16.
"""
import numpy as np
import pytest
import torch

import hdg_inputs
from oracle.lowdim import LowDimProblem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2007_11891_gb300 import build
    build.build(verbose=False)


def _grid(ne, seed):
    rng = np.random.default_rng(seed)
    return [0.1 + np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, v))]) / v for v in ne]


CASES = [
    # name, ne, bc, p, lam, tau_hat
    ("1d_single_neumann", (1,), (1, 1), 2, 0.5, 25.0),
    ("1d_ragged_p3", (7,), (0, 0), 3, 1.3, 25.0),
    ("1d_many_p8", (1000,), (1, 0), 8, 10.0, 25.0),
    ("1d_p16_poisson", (5,), (0, 1), 16, 0.0, 1.0),
    ("2d_single_neumann", (1, 1), (1, 1, 1, 1), 2, 0.7, 25.0),
    ("2d_mixed_p4", (5, 3), (0, 1, 0, 0), 4, 2.0, 10.0),
    ("2d_p1", (4, 6), (0, 0, 0, 0), 1, 0.0, 25.0),
    ("2d_many_p7", (40, 33), (1, 0, 0, 1), 7, 1.0, 25.0),
    ("2d_p16", (3, 2), (0, 0, 1, 0), 16, 1.0, 25.0),
]


@pytest.mark.parametrize("name,ne,bc,p,lam,tau", CASES, ids=[c[0] for c in CASES])
def test_lowdim_nodal_apply_matches_oracle(name, ne, bc, p, lam, tau):
    from paper_2007_11891_gb300 import HDGLowDim
    grid = _grid(ne, 3)
    h = HDGLowDim(ne, grid, bc, p, tau)
    pr = LowDimProblem(ne, grid, bc, p, tau, lam)
    assert h.trace_size == pr.mesh.n_trace
    x = hdg_inputs.uniform_pm1(h.trace_size, 17)
    y = h.apply(torch.tensor(x, device="cuda"), lam).cpu().numpy()
    ref = pr.apply(x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    if len(ne) == 1:   # faces are points: the basis does not matter
        yt = h.apply(torch.tensor(x, device="cuda"), lam, basis="transformed").cpu().numpy()
        assert np.array_equal(y, yt)
    h.close()


@pytest.mark.parametrize("ne,bc,p", [((3, 2), (0, 1, 0, 0), 3), ((2, 2), (1, 1, 1, 1), 5)])
def test_lowdim_transformed_basis_spectrum(ne, bc, p):
    from paper_2007_11891_gb300 import HDGLowDim
    lam, tau = 1.7, 25.0
    grid = _grid(ne, 5)
    h = HDGLowDim(ne, grid, bc, p, tau)
    pr = LowDimProblem(ne, grid, bc, p, tau, lam)
    T = h.trace_size
    eye = torch.eye(T, dtype=torch.float64, device="cuda")
    Kh = h.apply(eye, [lam] * T, basis="transformed").cpu().numpy()   # row r = K-hat e_r
    K = np.stack([pr.apply(e) for e in np.eye(T)], axis=1)
    assert np.abs(Kh - Kh.T).max() <= 1e-12 * np.abs(Kh).max()
    Minv = np.linalg.inv(pr.m1.M)
    Mf_inv = np.kron(np.eye(T // (p + 1)), Minv)
    ev_ref = np.sort(np.linalg.eigvals(K @ Mf_inv).real)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Kh + Kh.T)))
    assert np.abs(ev - ev_ref).max() <= 1e-10 * np.abs(ev_ref).max()
    h.close()


def test_lowdim_batched_deterministic():
    from paper_2007_11891_gb300 import HDGLowDim
    ne, bc, p = (13, 9), (0, 0, 1, 0), 6
    grid = _grid(ne, 8)
    h = HDGLowDim(ne, grid, bc, p, 25.0)
    lams = [0.1, 1.0, 100.0, 0.0]
    X = torch.tensor(np.stack([hdg_inputs.uniform_pm1(h.trace_size, 60 + r) for r in range(4)]), device="cuda")
    for basis in ("nodal", "transformed"):
        Y1 = h.apply(X, lams, basis=basis)
        assert torch.equal(Y1, h.apply(X, lams, basis=basis))
    Y = h.apply(X, lams).cpu().numpy()
    for r, lam in enumerate(lams):
        ref = LowDimProblem(ne, grid, bc, p, 25.0, lam).apply(X[r].cpu().numpy())
        assert np.abs(Y[r] - ref).max() <= 1e-12 * np.abs(ref).max()
    h.close()
