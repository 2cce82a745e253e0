"""hdg_apply_static: the allocation-free nodal FP64 operator application.

Some callers cannot allocate device memory once they are running: real-time
loops that must not synchronise (cudaFree synchronises the whole device) or
risk an allocation failure, programs whose device memory belongs to a
pooling allocator, code held to a memory budget set at start-up.  For them
hdg_apply_static keeps its temporaries in a static device array.  It must
give the same product as hdg_apply, call after call (also after a larger
call left other contents in the shared array), allocate nothing once the
first call on the device has been made, and reject requests larger than the
array.  This file is collected last so that a failure here comes after
every other test has run.
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


def _call_static(h, x, lams, y=None):
    from paper_2007_11891_gb300 import _capi
    if y is None:
        y = torch.full_like(x, float("nan"))
    st = _capi.lib().hdg_apply_static(h._h, x.shape[0], _capi.doubles(lams), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, y


def _mesh(ne, p, bc, seed):
    from paper_2007_11891_gb300 import HDG
    rng = np.random.default_rng(seed)
    grid = [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, ne[d]))]) for d in range(3)]
    return HDG(ne, grid, bc, p, hdg_inputs.TAU_HAT)


def _check(h, lams, seed):
    x = torch.tensor(np.stack([hdg_inputs.uniform_pm1(h.trace_size, seed + r) for r in range(len(lams))]),
                     device="cuda")
    ref = h.apply(x, lams)
    st, y = _call_static(h, x, lams)
    assert st == 0
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    err = float((y - ref).abs().max()) / float(ref.abs().max())
    assert err <= 1e-12, err


def test_static_apply_matches_apply_on_consecutive_calls():
    h = _mesh((4, 3, 5), 3, (0, 1, 0, 0, 1, 0), 3)
    for call in range(2):
        _check(h, [0.5, 3.0], 10 * call)


def test_static_apply_after_a_larger_call():
    # the shared array keeps what a larger call left there: the next call
    # must clear what it accumulates into
    big = _mesh((9, 7, 6), 5, (0,) * 6, 4)
    small = _mesh((3, 2, 4), 2, (1, 0, 0, 1, 0, 0), 5)
    _check(big, [2.0], 1)
    _check(small, [0.7, 0.0, 5.0], 2)
    _check(big, [1.0], 3)


def test_static_apply_many_lambdas():
    # more right-hand sides than one kernel-parameter chunk of lambdas
    h = _mesh((2, 1, 1), 1, (0,) * 6, 6)
    lams = list(np.linspace(0.0, 50.0, 1500))
    _check(h, lams, 7)


def test_static_apply_allocates_nothing():
    h = _mesh((5, 4, 3), 4, (0,) * 6, 8)
    x = torch.tensor(hdg_inputs.uniform_pm1(h.trace_size, 9), device="cuda").reshape(1, -1)
    y = torch.empty_like(x)
    assert _call_static(h, x, [1.5], y)[0] == 0   # first call on the device: address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, resv0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for lam in (1.5, 2.5, 0.0, 9.0):   # new lambdas: hdg_apply would rebuild its D_Z^-1 tables
        assert _call_static(h, x, [lam], y)[0] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == resv0


def test_static_apply_rejects_oversized_requests():
    from paper_2007_11891_gb300 import HDG, _capi
    ne = (20, 20, 20)
    h = HDG(ne, hdg_inputs.grid_lines(ne), (0,) * 6, 8, hdg_inputs.TAU_HAT)
    x = torch.zeros((1, h.trace_size), dtype=torch.float64, device="cuda")
    st, _ = _call_static(h, x, [1.0])
    assert st == 1
    assert b"maximum" in _capi.lib().hdg_last_error()
