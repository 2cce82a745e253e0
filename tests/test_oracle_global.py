"""Pins for the oracle's global condensed system, solve, recovery and adjoint.

* Polynomial reproduction: for u in Q_p, exact integration makes
  (u, grad u, u|faces) an exact solution of Eq. (ldg_element_operator_threed)
  (the penalty terms vanish since u - ut = 0), so the solve must return it to
  round-off.  This fixes every sign and scale of the right-hand side, the
  Dirichlet lift, the Neumann load and the recovery (Alg. hdg_cg).
* Convergence of order p + 1 (Sec. 1) on u = sin(pi x) sin(pi y) sin(pi z).
* The global K (Eq. hdg_system) is symmetric, positive definite with a
  Dirichlet side, and has the constants as null vector for lambda = 0 with
  Neumann data everywhere.
* Central finite differences pin the adjoint gradients.
* Planted mistakes in the oracle make a pin fail.
"""
import numpy as np
import pytest

import hdg_inputs
from oracle import basis1d
from oracle.solver import Problem, cg, uniform_grid
from tests._poly import PolyField, boundary_data


def _stretched(ne, rng):
    return [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, ne[d]))]) for d in range(3)]


CASES = [
    # (ne, bc, p, stretched, lam, tau_hat)
    ((1, 1, 1), (0, 0, 0, 0, 0, 0), 2, False, 1.0, 25.0),
    ((2, 3, 2), (0, 0, 0, 0, 0, 0), 3, True, 0.0, 3.0),
    ((2, 2, 3), (1, 0, 0, 1, 0, 0), 2, True, 0.7, 25.0),
    ((3, 2, 2), (1, 1, 0, 1, 1, 0), 4, True, 2.0, 1.0),
    ((2, 2, 2), (0, 1, 1, 0, 0, 1), 1, False, 0.5, 10.0),
]


@pytest.mark.parametrize("ne,bc,p,stretched,lam,tau", CASES)
def test_polynomial_reproduction(ne, bc, p, stretched, lam, tau):
    rng = np.random.default_rng(sum(ne) * 10 + p)
    grid = _stretched(ne, rng) if stretched else [uniform_grid(ne[d], 1.7) for d in range(3)]
    pr = Problem(ne, grid, bc, p, tau, lam)
    fld = PolyField(p, rng)
    nodes = pr.m1.nodes
    Xv = pr.mesh.volume_coords(nodes)
    f = lam * fld.u(Xv) - fld.lap(Xv)
    bd = boundary_data(pr, fld)
    ut, u, q, info = pr.solve(f=f, bdry=bd, method="direct")
    scale = max(1.0, np.abs(fld.u(Xv)).max())
    assert np.abs(u - fld.u(Xv)).max() < 1e-10 * scale
    if len(ut):
        assert np.abs(ut - fld.u(pr.mesh.trace_coords(nodes))).max() < 1e-10 * scale
    assert np.abs(q - fld.grad(Xv)).max() < 1e-8 * scale


def test_polynomial_reproduction_with_lumped_mass():
    # With the GLL-lumped mass every integral is a GLL-point sum, so the scheme
    # is collocation at the GLL points and a Q_p solution still satisfies
    # every nodal equation: u and the traces are reproduced as well.
    rng = np.random.default_rng(5)
    ne, p = (2, 3, 2), 3
    pr = Problem(ne, _stretched(ne, rng), (0, 1, 0, 0, 1, 0), p, 25.0, 1.0, mass="gll")
    fld = PolyField(p, rng)
    fld.exps[0] = [p, p, p]
    Xv = pr.mesh.volume_coords(pr.m1.nodes)
    ut, u, _, _ = pr.solve(f=pr.lam * fld.u(Xv) - fld.lap(Xv), bdry=boundary_data(pr, fld), method="direct")
    scale = np.abs(fld.u(Xv)).max()
    assert np.abs(u - fld.u(Xv)).max() < 1e-10 * scale
    assert np.abs(ut - fld.u(pr.mesh.trace_coords(pr.m1.nodes))).max() < 1e-10 * scale


def _l2_error(pr, u):
    # quadrature-free nodal RMS error weighted by element volume
    Xv = pr.mesh.volume_coords(pr.m1.nodes)
    err = u - hdg_inputs.sinsinsin(Xv)
    return np.sqrt(np.mean(err ** 2))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_order(p):
    errs = []
    for N in (2, 4):
        pr = Problem((N, N, N), [uniform_grid(N) for _ in range(3)], (0,) * 6, p, 25.0, 1.0)
        Xv = pr.mesh.volume_coords(pr.m1.nodes)
        f = hdg_inputs.sinsinsin_load(Xv, 1.0)
        _, u, _, _ = pr.solve(f=f, method="direct")
        errs.append(_l2_error(pr, u))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 1 - 0.5, (errs, rate)


def test_global_operator_structure():
    rng = np.random.default_rng(3)
    ne = (3, 2, 2)
    grid = _stretched(ne, rng)
    pr = Problem(ne, grid, (0, 1, 0, 0, 1, 0), 2, 25.0, 0.0)
    K, _ = pr.assemble()
    Kd = K.toarray()
    np.testing.assert_allclose(Kd, Kd.T, atol=1e-11 * np.abs(Kd).max())
    assert np.linalg.eigvalsh(Kd)[0] > 0            # Dirichlet side present
    x = rng.standard_normal(K.shape[0])
    np.testing.assert_allclose(pr.apply(x), K @ x, atol=1e-11 * np.abs(K @ x).max())
    dofs = rng.choice(K.shape[0], 25, replace=False)
    np.testing.assert_allclose(pr.apply_rows(x, dofs), (K @ x)[dofs], atol=1e-11 * np.abs(K @ x).max())
    # all-Neumann, lambda = 0: constants are the null vector
    prn = Problem(ne, grid, (1,) * 6, 2, 25.0, 0.0)
    Kn, _ = prn.assemble()
    assert np.abs(Kn @ np.ones(Kn.shape[0])).max() < 1e-10 * abs(Kn).max()


def test_cg_matches_direct():
    rng = np.random.default_rng(4)
    ne = (3, 3, 2)
    pr = Problem(ne, _stretched(ne, rng), (0,) * 6, 3, 25.0, 10.0)
    f = rng.standard_normal(pr.mesh.n_elem * 64)
    ut_d, u_d, _, _ = pr.solve(f=f, method="direct")
    ut_c, u_c, _, info = pr.solve(f=f, tol=1e-13)
    assert info["rel_residual"] < 1e-12
    np.testing.assert_allclose(ut_c, ut_d, atol=1e-10 * np.abs(ut_d).max())
    np.testing.assert_allclose(u_c, u_d, atol=1e-10 * np.abs(u_d).max())


@pytest.mark.parametrize("ne,p", [((2, 2, 2), 2), ((4, 4, 4), 3)])
def test_adjoint_matches_central_differences(ne, p):
    rng = np.random.default_rng(11)
    grid = [uniform_grid(ne[d]) for d in range(3)]
    lam = 5.0
    pr = Problem(ne, grid, (0,) * 6, p, 25.0, lam)
    Xv = pr.mesh.volume_coords(pr.m1.nodes)
    f = rng.standard_normal(len(Xv))
    ut = hdg_inputs.smooth_target(Xv, hdg_inputs.smooth_target_coeffs())
    L, dLdf, dLdlam, _ = pr.adjoint(f, ut, method="direct")

    def loss(fv, lv):
        q = Problem(ne, grid, (0,) * 6, p, 25.0, lv)
        _, u, _, _ = q.solve(f=fv, method="direct")
        return np.sum((u - ut) ** 2)

    # L is exactly quadratic in f, so a central difference has no truncation
    # error and a large step only shrinks the round-off (eps * L / step)
    for idx in rng.choice(len(f), 4, replace=False):
        step = 1e-1 * max(1.0, abs(f[idx]))
        fp, fm = f.copy(), f.copy()
        fp[idx] += step
        fm[idx] -= step
        fd = (loss(fp, lam) - loss(fm, lam)) / (2 * step)
        assert abs(fd - dLdf[idx]) <= 1e-6 * abs(dLdf).max()
    # in lambda the truncation error is O(step^2): step 1e-4 lambda keeps it
    # and the round-off (eps * L / step) below 1e-7 relative
    step = 1e-4 * lam
    fd = (loss(f, lam + step) - loss(f, lam - step)) / (2 * step)
    assert abs(fd - dLdlam) <= 1e-6 * max(1e-3, abs(dLdlam))


# -- planted mistakes: each must make a pin above fail ---------------------------

def _reproduction_error(monkeypatch, mutate):
    orig = basis1d.Matrices1D.__init__

    def patched(self, *a, **k):
        orig(self, *a, **k)
        mutate(self)

    monkeypatch.setattr(basis1d.Matrices1D, "__init__", patched)
    rng = np.random.default_rng(9)
    ne, p = (2, 2, 1), 2
    pr = Problem(ne, _stretched(ne, rng), (0,) * 6, p, 5.0, 1.0)
    fld = PolyField(p, rng)
    fld.exps[0] = [2, 1, 2]
    Xv = pr.mesh.volume_coords(pr.m1.nodes)
    _, u, _, _ = pr.solve(f=pr.lam * fld.u(Xv) - fld.lap(Xv), bdry=boundary_data(pr, fld), method="direct")
    return np.abs(u - fld.u(Xv)).max() / max(1.0, np.abs(fld.u(Xv)).max())


@pytest.mark.parametrize("name,mutate", [
    ("B sign", lambda m: setattr(m, "B", -m.B)),
    ("D transposed", lambda m: setattr(m, "D", m.D.T.copy())),
    ("C sign", lambda m: setattr(m, "C", -m.C)),
    ("G dropped", lambda m: setattr(m, "G", 0.0 * m.G)),
    ("E halved", lambda m: setattr(m, "E", 0.5 * m.E)),
])
def test_planted_mistake_is_caught(monkeypatch, name, mutate):
    assert _reproduction_error(monkeypatch, mutate) > 1e-6, name
