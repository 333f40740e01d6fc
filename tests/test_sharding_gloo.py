"""Sharding of independent instances across ranks, on CPU.

The batched and served workloads are independent problems: every rank
computes the same split from the library's cost estimate and partitioner
(host code, no GPU needed) and solves its share; results go to rank 0 only
to be reported.  Two gloo ranks solve a set of small cubic instances with the
FP64 oracle standing in for the device solver, and rank 0 checks that the
gathered results are exactly those of one process solving everything.  Also:
the partitioner's guarantees (every item once, the longest-processing-time
bound against brute force, determinism) and its argument checks.
"""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1810_11111_gb300 import sgkiif, sharding, workloads  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_1810_11111_gb300 import build
    if not os.path.exists(sgkiif.LIB_PATH):
        build.build()
    return sgkiif.load()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_instances():
    rng = np.random.default_rng(21)
    out = []
    for i in range(7):
        n = int(rng.integers(2, 4))
        c = float(rng.uniform(1.0, 100.0))
        amp, wavenum, kind = workloads.fourier_modes(rng, 2)
        out.append(dict(name="small%d" % i, d=2, n=n, k=1, kappas=[list(rng.uniform(0.05, 1.0, 2))],
                        reaction=workloads.reaction_terms(workloads.CUBIC, c), M=8, dt=0.005, steps=2,
                        init=[dict(amp=amp, wavenum=wavenum, kind=kind, const=0.0)]))
    return out


def _solve(cfg):
    from oracle.iif import IIF2Solver
    from oracle.index_set import IndexSet
    from oracle.operator import sipg_1d
    from oracle.projection import project_separable
    idx = IndexSet(cfg["d"], cfg["n"], cfg["k"])
    init = cfg["init"][0]
    U0 = project_separable(idx, init["amp"], init["wavenum"], init["kind"], init["const"])
    sol = IIF2Solver(idx, sipg_1d(cfg["n"], cfg["k"]), cfg["kappas"], cfg["reaction"], cfg["dt"], cfg["M"])
    return sol.run([U0], cfg["steps"])[0]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfgs = _small_instances()
        mine = sharding.my_share(cfgs, rank, world)
        local = {i: _solve(cfgs[i]) for i in mine}
        got = sharding.gather_to_root(local, dist, world)
        if rank == 0:
            out["parts"] = [sorted(g) for g in got]
            merged = {}
            for g in got:
                merged.update(g)
            out["merged"] = merged
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_their_shares_and_gather_the_whole_batch(lib):
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    cfgs = _small_instances()
    parts = res["parts"]
    assert sorted(parts[0] + parts[1]) == list(range(len(cfgs)))  # every instance exactly once
    assert parts[0] and parts[1]                                   # both ranks have work
    for i, cfg in enumerate(cfgs):
        assert np.array_equal(res["merged"][i], _solve(cfg))


def test_partition_bound_and_determinism(lib):
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(1, 4))
        cost = rng.uniform(0.0, 10.0, n)
        part = sharding.partition(cost, m)
        assert part == sharding.partition(cost, m)
        assert all(0 <= p < m for p in part)
        loads = np.bincount(part, weights=cost, minlength=m)
        best = min(max(np.bincount(a, weights=cost, minlength=m)) for a in itertools.product(range(m), repeat=n))
        assert loads.max() <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-12


def test_partition_rejects_bad_arguments(lib):
    c = np.array([1.0, np.nan])
    cp = c.ctypes.data_as(sgkiif._c_double_p)
    outa = (sgkiif.ctypes.c_int * 2)()
    assert sgkiif.sgk_partition(2, cp, 2, outa) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_partition(2, cp, 0, outa) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_partition(-1, cp, 2, outa) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_partition(0, None, 2, None) == sgkiif.SGK_OK


def test_work_estimate_orders_shapes(lib):
    est = sgkiif.sgk_estimate_work
    assert est(0, 3, 1, 1, 30, 1) < 0 and est(3, 3, 4, 1, 30, 1) < 0
    assert est(3, 6, 2, 1, 30, 1) > est(3, 5, 2, 1, 30, 1) > est(2, 5, 2, 1, 30, 1)
    assert est(3, 6, 2, 1, 30, 1) > est(3, 6, 2, 1, 30, 0) > est(3, 6, 2, 1, 20, 0)
    assert est(2, 8, 2, 2, 40, 1) == pytest.approx(2 * est(2, 8, 2, 1, 40, 1))


def test_interpolation_form_costs_less_to_shard():
    # the partitioner's cost of an instance follows its reaction form: the
    # interpolation form has no finest-grid passes
    from paper_1810_11111_gb300 import sharding, workloads
    cfg = workloads.cubic3d()
    quad = sharding.instance_cost(cfg)
    interp = sharding.instance_cost(dict(cfg, reaction_form="interp"))
    none = sharding.instance_cost(dict(cfg, reaction=[[]]))
    assert none < interp < quad
