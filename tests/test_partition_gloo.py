"""Slab partition of the operator across ranks, on CPU (gloo).

Each rank owns an x3-slab of elements, applies the operator of its own
sub-mesh (the interface sides declared Neumann) and sums the interface
planes with its neighbours (one all-reduce per interface and apply).  Here
the per-rank operator is the oracle's dense condensed apply of the sub-mesh;
on GPUs it is the library's.  The assembled result must equal the oracle's
apply of the whole mesh entry by entry, the two copies of every interface
value must agree bitwise, and inner products over owned entries must add up
to the global one.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2007_11891_gb300.partition import SlabPartition, slab_bounds  # noqa: E402

MESH = dict(ne=(3, 2, 5), bc=(0, 1, 0, 0, 1, 0), p=2, lam=1.7, tau=25.0)


def _grid(ne, seed=3):
    rng = np.random.default_rng(seed)
    return [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 2.0, v))]) for v in ne]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle.solver import Problem
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ne, bc, p = MESH["ne"], MESH["bc"], MESH["p"]
    grid = _grid(ne)
    part = SlabPartition(ne, grid, bc, p, world, rank).init_groups()
    x = np.random.default_rng(11).uniform(-1.0, 1.0, part.global_trace_size)
    xl = torch.tensor(part.scatter(x))
    local = Problem(part.local_ne, part.local_grid, part.local_bc, p, MESH["tau"], MESH["lam"])
    assert local.mesh.n_trace == part.local_trace_size
    y = part.apply(lambda v: torch.tensor(local.apply(v.numpy())), xl)
    z = torch.tensor(part.scatter(np.random.default_rng(12).uniform(-1.0, 1.0, part.global_trace_size)))
    owned = torch.tensor(part.owned)
    dot = torch.tensor([float((y[owned] * z[owned]).sum())], dtype=torch.float64)
    dist.all_reduce(dot)
    q.put((rank, part.global_index, y.numpy(), float(dot[0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_partition_apply_equals_whole_mesh(world):
    import torch.multiprocessing as mp
    from oracle.solver import Problem
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ne, bc, p = MESH["ne"], MESH["bc"], MESH["p"]
    whole = Problem(ne, _grid(ne), bc, p, MESH["tau"], MESH["lam"])
    x = np.random.default_rng(11).uniform(-1.0, 1.0, whole.mesh.n_trace)
    ref = whole.apply(x)
    y = np.full(whole.mesh.n_trace, np.nan)
    seen = np.zeros(whole.mesh.n_trace, dtype=int)
    for _, gi, yl, _ in out:
        dup = seen[gi] > 0
        # an interface value held by two ranks: the same sum on both, bitwise
        assert np.array_equal(y[gi[dup]], yl[dup])
        y[gi] = yl
        seen[gi] += 1
    assert np.all(seen >= 1)                                   # every global entry is held somewhere
    assert np.count_nonzero(seen == 2) == (world - 1) * ne[0] * ne[1] * (p + 1) ** 2
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    z = np.random.default_rng(12).uniform(-1.0, 1.0, whole.mesh.n_trace)
    for _, _, _, d in out:
        assert d == pytest.approx(float(ref @ z), rel=1e-12)


def _cg_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle.solver import Problem
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ne, bc, p = MESH["ne"], MESH["bc"], MESH["p"]
    grid = _grid(ne)
    part = SlabPartition(ne, grid, bc, p, world, rank).init_groups()
    local = Problem(part.local_ne, part.local_grid, part.local_bc, p, MESH["tau"], MESH["lam"])
    # b = K x* of the whole mesh, computed by the oracle on every rank
    whole = Problem(ne, grid, bc, p, MESH["tau"], MESH["lam"])
    xs = np.random.default_rng(21).uniform(-1.0, 1.0, whole.mesh.n_trace)
    b = torch.tensor(part.scatter(whole.apply(xs)))
    x, it, rel = part.cg(lambda v: torch.tensor(local.apply(v.numpy())), b, tol=1e-12, max_iter=500)
    q.put((rank, part.global_index, x.numpy(), it, rel))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_partition_cg_solves_the_whole_mesh_system(world):
    # the partitioned CG (local applies + interface exchange, one all-reduce
    # of the inner products per iteration) recovers x* from b = K x* of the
    # whole mesh; every rank takes the same number of iterations, and the
    # two copies of an interface value agree bitwise
    import torch.multiprocessing as mp
    from oracle.solver import Problem
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_cg_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ne, bc, p = MESH["ne"], MESH["bc"], MESH["p"]
    whole = Problem(ne, _grid(ne), bc, p, MESH["tau"], MESH["lam"])
    xs = np.random.default_rng(21).uniform(-1.0, 1.0, whole.mesh.n_trace)
    x = np.full(whole.mesh.n_trace, np.nan)
    for _, gi, xl, it, rel in out:
        held = ~np.isnan(x[gi])
        assert np.array_equal(x[gi[held]], xl[held])
        x[gi] = xl
        assert it == out[0][3] and rel <= 1e-12
    assert not np.any(np.isnan(x))
    assert np.abs(x - xs).max() <= 1e-9 * np.abs(xs).max()


def test_slab_bounds_and_local_layout():
    assert slab_bounds(5, 2) == [(0, 3), (3, 5)]
    assert slab_bounds(7, 3) == [(0, 3), (3, 5), (5, 7)]
    with pytest.raises(ValueError):
        slab_bounds(2, 3)
    ne, bc, p = (2, 3, 4), (1, 0, 0, 1, 0, 1), 1
    parts = [SlabPartition(ne, _grid(ne), bc, p, 2, r) for r in range(2)]
    # the interface sides become Neumann, the global x3 sides stay as given
    assert parts[0].local_bc == (1, 0, 0, 1, 0, 1) and parts[1].local_bc == (1, 0, 0, 1, 1, 1)
    assert parts[0].top is not None and parts[0].bottom is None
    assert parts[1].bottom is not None and parts[1].top is None
    # the shared plane maps to the same global entries from both sides
    assert np.array_equal(parts[0].global_index[parts[0].top], parts[1].global_index[parts[1].bottom])
    # every global entry is reached, and only the interface plane twice
    allidx = np.concatenate([pt.global_index for pt in parts])
    assert np.unique(allidx).size == parts[0].global_trace_size
    assert allidx.size - np.unique(allidx).size == ne[0] * ne[1] * (p + 1) ** 2
    # owned entries partition the global vector
    owned = np.concatenate([pt.global_index[pt.owned] for pt in parts])
    assert np.array_equal(np.sort(owned), np.arange(parts[0].global_trace_size))
