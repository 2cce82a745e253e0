"""Checks of the synthetic input module (no method arithmetic involved)."""
import numpy as np

import hdg_inputs


def test_paper_case_load_is_the_laplacian():
    # f = -laplace u_ex (lambda = 0) against a fourth-order central difference
    rng = np.random.default_rng(0)
    X = rng.uniform(0.0, 2 * np.pi, (40, 3))
    h = 1e-3
    lap = np.zeros(len(X))
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        u = hdg_inputs.paper_case_u
        lap += (-u(X + 2 * e) + 16 * u(X + e) - 30 * u(X) + 16 * u(X - e) - u(X - 2 * e)) / (12 * h * h)
    f = hdg_inputs.paper_case_load(X)
    assert np.abs(f + lap).max() <= 1e-5 * np.abs(lap).max()
    np.testing.assert_allclose(hdg_inputs.paper_case_load(X, lam=2.0), f + 2.0 * hdg_inputs.paper_case_u(X))


def test_seeded_generators_are_reproducible():
    assert np.array_equal(hdg_inputs.gaussian(10, 3), hdg_inputs.gaussian(10, 3))
    lams = hdg_inputs.batch_lambdas(64)
    assert set(np.unique(lams)) <= {0.1, 1.0, 100.0}
    g = hdg_inputs.grid_lines((4, 5, 6), stretched=True, length=2.0)
    assert all(abs(x[-1] - 2.0) < 1e-14 and x[0] == 0.0 and np.all(np.diff(x) > 0) for x in g)
