"""hdg_apply_static: the allocation-free nodal FP64 operator application.

Some callers cannot allocate device memory (code running during CUDA graph
capture, real-time loops, programs whose memory belongs to a pooling
allocator); for them hdg_apply_static keeps its temporaries in a static
device array.  It must give the same product as hdg_apply, call after call,
and reject requests larger than that array.  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import hdg_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2007_11891_gb300 import build
    build.build(verbose=False)


def _call_static(h, x, lams):
    from paper_2007_11891_gb300 import _capi
    y = torch.full_like(x, float("nan"))
    st = _capi.lib().hdg_apply_static(h._h, x.shape[0], _capi.doubles(lams), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, y


def test_static_apply_matches_apply_on_consecutive_calls():
    from paper_2007_11891_gb300 import HDG
    ne, p = (4, 3, 5), 3
    rng = np.random.default_rng(3)
    grid = [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, ne[d]))]) for d in range(3)]
    h = HDG(ne, grid, (0, 1, 0, 0, 1, 0), p, hdg_inputs.TAU_HAT)
    lams = [0.5, 3.0]
    for call in range(2):
        x = torch.tensor(np.stack([hdg_inputs.uniform_pm1(h.trace_size, 10 * call + r) for r in range(2)]),
                         device="cuda")
        ref = h.apply(x, lams)
        st, y = _call_static(h, x, lams)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        err = float((y - ref).abs().max()) / float(ref.abs().max())
        assert err <= 1e-12, (call, err)


def test_static_apply_rejects_oversized_requests():
    from paper_2007_11891_gb300 import HDG, _capi
    ne = (20, 20, 20)
    h = HDG(ne, hdg_inputs.grid_lines(ne), (0,) * 6, 8, hdg_inputs.TAU_HAT)
    x = torch.zeros((1, h.trace_size), dtype=torch.float64, device="cuda")
    st, _ = _call_static(h, x, [1.0])
    assert st == 1
    assert b"maximum" in _capi.lib().hdg_last_error()
