"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no arithmetic of the HDG method: it only draws grid
widths, loads, trace vectors, lambda values and the coefficients of a smooth
target field, and evaluates closed-form fields at coordinates it is given.
Both the CUDA path and the CPU oracle consume what it returns.

Workloads (all synthetic; the paper's own runs use n_e = 8^3 Cartesian meshes
and a manufactured solution, Sec. 4.3 and Sec. 5.3):

* ``unit_cube_p4``   4x4x4 uniform, p = 4, lambda = 1, tau_hat = 25,
                     Dirichlet, u = sin(pi x) sin(pi y) sin(pi z),
                     f = (lambda + 3 pi^2) u.
* ``stretched_p8``   16^3, per-direction widths ~ U[0.5, 2] (seeds 11892,
                     11893, 11894), normalised to the unit cube, p = 8,
                     lambda = 10, f ~ N(0, 1) per volume node (seed 11890).
* ``uniform32``      32^3 uniform, lambda = 1, p in {2, 4, 8, 12, 16},
                     trace vectors ~ U[-1, 1] (seed 11893).
* ``batched24_p7``   24^3 uniform, p = 7, 64 right-hand sides f ~ N(0, 1)
                     (seed 11894), lambda_r from {0.1, 1, 100} (seed 11895).
* ``adjoint32_p6``   32^3 uniform, p = 6, lambda = 5, f ~ N(0, 1)
                     (seed 11897), target u_t = sum of 8 sinusoids
                     (seed 11896); finite-difference copy at 4^3, p = 3.
* ``paper_case``     the paper's own solver test (Sec. 5.3): 8^3 uniform
                     elements on (0, 2 pi)^3, lambda = 0, tau_hat = 25,
                     inhomogeneous Dirichlet data and load from the
                     manufactured solution u_ex with stiffness k = 5.
"""

import numpy as np

TAU_HAT = 25.0   # penalty "tau = 25" of Sec. 5.4 read as tau_hat (tau_e = 2 tau_hat / h)

WORKLOADS = {
    "unit_cube_p4": dict(ne=(4, 4, 4), p=4, lam=1.0, stretched=False),
    "stretched_p8": dict(ne=(16, 16, 16), p=8, lam=10.0, stretched=True),
    "uniform32": dict(ne=(32, 32, 32), p=8, lam=1.0, stretched=False),
    "batched24_p7": dict(ne=(24, 24, 24), p=7, lam=None, stretched=False, nrhs=64),
    "adjoint32_p6": dict(ne=(32, 32, 32), p=6, lam=5.0, stretched=False),
    "paper_case": dict(ne=(8, 8, 8), p=8, lam=0.0, stretched=False, length=2.0 * np.pi),
}


def grid_lines(ne, stretched=False, seeds=(11892, 11893, 11894), length=1.0):
    """Grid-line coordinates per direction on [0, length]: uniform, or widths
    drawn uniform in [0.5, 2] with one seed per direction and normalised."""
    out = []
    for d in range(3):
        if stretched:
            w = np.random.default_rng(seeds[d]).uniform(0.5, 2.0, ne[d])
        else:
            w = np.ones(ne[d])
        x = np.concatenate([[0.0], np.cumsum(w)])
        out.append(length * x / x[-1])
    return out


def gaussian(count, seed):
    """count values ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(count)


def uniform_pm1(count, seed):
    """count values ~ U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, count)


def batch_lambdas(nrhs, seed=11895, choices=(0.1, 1.0, 100.0)):
    """lambda_r drawn uniformly from ``choices``."""
    idx = np.random.default_rng(seed).integers(0, len(choices), nrhs)
    return np.asarray(choices, dtype=np.float64)[idx]


def sinsinsin(X):
    """u = sin(pi x) sin(pi y) sin(pi z) at coordinates X (m, 3)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])


def sinsinsin_load(X, lam):
    """f = lambda u - laplace u = (lambda + 3 pi^2) u for u = sinsinsin."""
    return (lam + 3.0 * np.pi ** 2) * sinsinsin(X)


def smooth_target_coeffs(seed=11896, modes=8):
    """Amplitudes a_m ~ N(0,1), wave vectors k_m in {1,2,3}^3, phases
    phi_m ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(modes)
    k = rng.integers(1, 4, size=(modes, 3)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, modes)
    return a, k, phi


def smooth_target(X, coeffs):
    """u_t(x) = sum_m a_m sin(2 pi k_m . x + phi_m) at coordinates X (m, 3)."""
    a, k, phi = coeffs
    X = np.asarray(X, dtype=np.float64)
    return np.sin(2.0 * np.pi * X @ k.T + phi[None, :]) @ a


# ---- manufactured solution of the paper's solver test (Sec. 5.3) ---------------
# u_ex = cos(k (x1 - 3 x2 + 2 x3)) sin(k (1 + x1)) sin(k (1 - x2))
#        sin(k (2 x1 + x2)) sin(k (3 x1 - 2 x2 + 2 x3))
# is a product of factors g_m = trig_m(theta_m), theta_m = k (a_m . x + c_m).
# With g_m' the derivative of trig_m: grad g_m = k a_m g_m' and
# laplace g_m = -k^2 |a_m|^2 g_m, so
# laplace u = -k^2 sum_m |a_m|^2 u + 2 k^2 sum_{m<l} (a_m . a_l) g_m' g_l' prod_{others} g.
_PAPER_FACTORS = (  # (a_m, c_m, is_cos)
    ((1.0, -3.0, 2.0), 0.0, True),
    ((1.0, 0.0, 0.0), 1.0, False),
    ((0.0, -1.0, 0.0), 1.0, False),
    ((2.0, 1.0, 0.0), 0.0, False),
    ((3.0, -2.0, 2.0), 0.0, False),
)


def _paper_case_parts(X, k):
    X = np.asarray(X, dtype=np.float64)
    g, dg, a = [], [], []
    for av, c, is_cos in _PAPER_FACTORS:
        av = np.asarray(av)
        th = k * (X @ av + c)
        g.append(np.cos(th) if is_cos else np.sin(th))
        dg.append(-np.sin(th) if is_cos else np.cos(th))
        a.append(av)
    return g, dg, a


def paper_case_u(X, k=5.0):
    """u_ex at coordinates X (m, 3)."""
    g, _, _ = _paper_case_parts(X, k)
    return np.prod(g, axis=0)


def paper_case_load(X, lam=0.0, k=5.0):
    """f = lambda u_ex - laplace u_ex at coordinates X (m, 3)."""
    g, dg, a = _paper_case_parts(X, k)
    u = np.prod(g, axis=0)
    lap = -k * k * sum(a_m @ a_m for a_m in a) * u
    nf = len(g)
    for m in range(nf):
        for l in range(m + 1, nf):
            rest = np.ones_like(u)
            for o in range(nf):
                if o != m and o != l:
                    rest = rest * g[o]
            lap = lap + 2.0 * k * k * (a[m] @ a[l]) * dg[m] * dg[l] * rest
    return lam * u - lap
