"""Failure reporting of the solve, made on the host (no GPU fault involved).

* An iteration limit below what the tolerance needs ends the device-driven
  CG loop (conditional CUDA graph: the CG flags stop the updates and the
  loop's trip cap bounds the graph) and is reported as NOT_CONVERGED.
* A non-finite load (NaN in the host data copied to the device) is reported
  as BREAKDOWN for its right-hand side.
* In a batch, one bad right-hand side is reported while the others converge
  to the tolerance, which the oracle re-evaluates.
"""
import numpy as np
import pytest
import torch

import hdg_inputs
from oracle.solver import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2007_11891_gb300 import build
    build.build(verbose=False)


def _problem(ne=(4, 3, 3), p=3, lam=2.0, seed=7):
    from paper_2007_11891_gb300 import HDG
    rng = np.random.default_rng(seed)
    grid = [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, ne[d]))]) for d in range(3)]
    return HDG(ne, grid, (0,) * 6, p, 25.0), Problem(ne, grid, (0,) * 6, p, 25.0, lam), lam


@pytest.mark.parametrize("inner", ["fp32", "fp64"])
def test_iteration_limit_reports_not_converged(inner):
    from paper_2007_11891_gb300 import _capi
    h, _, lam = _problem(ne=(8, 6, 5), p=4, lam=0.5)
    f = torch.tensor(hdg_inputs.gaussian(h.volume_size, 3), device="cuda")
    _, _, ok = h.solve(f, lam, tol=1e-10, inner=inner, return_u=False)
    need = ok[0]["iterations"]
    assert ok[0]["status"] == "OK" and need >= 60
    # 7: inside the eagerly launched first chunk of 16 iterations; need / 2:
    # inside the conditional-graph loop that runs the rest of an inner solve
    for cap in (7, need // 2):
        h.profile(True)    # resets the launch counter ...
        h.profile(False)   # ... and leaves recording off, so the graph path runs
        tr, _, info = h.solve(f, lam, tol=1e-10, inner=inner, max_iter=cap, return_u=False, check=False)
        _, launches = h.profile_read("all")
        assert info[0]["status"] == "NOT_CONVERGED", cap
        assert info[0]["iterations"] == cap
        assert info[0]["rel_residual"] > 1e-10 and np.isfinite(info[0]["rel_residual"])
        assert torch.isfinite(tr).all()
        # the loop ended at the cap: about two kernels per allowed iteration
        # (plus one 16-iteration eager chunk per inner solve, loop-control
        # kernels and the set-up and refinement launches), not a runaway loop
        assert launches <= 2 * cap + 40 * 8 + 100, (cap, launches)
    with pytest.raises(_capi.HdgError) as ei:
        h.solve(f, lam, tol=1e-10, inner=inner, max_iter=7, return_u=False)
    assert ei.value.status == 5


@pytest.mark.parametrize("inner", ["fp32", "fp64"])
def test_nan_load_reports_breakdown(inner):
    from paper_2007_11891_gb300 import _capi
    h, _, lam = _problem()
    f_host = hdg_inputs.gaussian(h.volume_size, 4)
    f_host[h.volume_size // 2] = np.nan
    f = torch.tensor(f_host, device="cuda")
    _, _, info = h.solve(f, lam, tol=1e-10, inner=inner, check=False)
    assert info[0]["status"] == "BREAKDOWN"
    with pytest.raises(_capi.HdgError) as ei:
        h.solve(f, lam, tol=1e-10, inner=inner)
    assert ei.value.status == 6


def test_one_bad_rhs_in_a_batch():
    h, pr, lam = _problem()
    lams = [lam, 0.5, 7.0]
    F = np.stack([hdg_inputs.gaussian(h.volume_size, 40 + r) for r in range(3)])
    F[1, 5] = np.inf
    tr, u, info = h.solve(torch.tensor(F, device="cuda"), lams, tol=1e-10, inner="fp32", check=False)
    assert [i["status"] for i in info] == ["OK", "BREAKDOWN", "OK"]
    for r in (0, 2):
        prr = Problem(pr.mesh.ne, pr.mesh.grid, (0,) * 6, 3, 25.0, lams[r])
        K, _ = prr.assemble()
        Fr = prr.rhs(f=F[r])
        res = np.linalg.norm(Fr - K @ tr[r].cpu().numpy()) / np.linalg.norm(Fr)
        assert res <= 1e-10, (r, res)
        assert torch.isfinite(u[r]).all()
