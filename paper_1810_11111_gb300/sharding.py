"""Sharding of independent instances across ranks (one GPU per rank).

Batched instances and served requests are independent problems, so they
shard with no data-path collective: every rank computes the same split from
the library's cost estimate (sgk_estimate_work, sgk_partition: longest
processing time first), solves its own share, and the results are gathered
to rank 0 only to report them.  Marshalling only; the split itself is the
library's host code.
"""
import ctypes

import numpy as np

from . import sgkiif


def instance_cost(cfg, steps=None):
    """Estimated work of a workload dict (as workloads.batch_instances /
    served_requests): per-step estimate times its steps."""
    sgkiif.load()
    # 0: no reaction, 1: the paper's finest-grid form, 2: the interpolation form
    has_rx = int(any(len(t) for t in cfg["reaction"]))
    if has_rx and cfg.get("reaction_form", "quadrature") == "interp":
        has_rx = 2
    w = sgkiif.sgk_estimate_work(cfg["d"], cfg["n"], cfg["k"], len(cfg["kappas"]), cfg["M"], has_rx)
    if w < 0:
        raise sgkiif.SgkError(sgkiif.SGK_EINVAL, "sgk_estimate_work: invalid shape")
    return w * (steps if steps is not None else cfg.get("steps", 1))


def partition(costs, nparts):
    """Part (rank) of every item, from the library's partitioner."""
    sgkiif.load()
    c = np.ascontiguousarray(costs, dtype=np.float64)
    out = (ctypes.c_int * max(1, len(c)))()
    rc = sgkiif.sgk_partition(len(c), c.ctypes.data_as(sgkiif._c_double_p), int(nparts), out)
    if rc != sgkiif.SGK_OK:
        raise sgkiif.SgkError(rc, "sgk_partition")
    return [int(out[i]) for i in range(len(c))]


def my_share(cfgs, rank, world, steps=None):
    """Indices of the instances this rank solves."""
    parts = partition([instance_cost(c, steps) for c in cfgs], world)
    return [i for i, p in enumerate(parts) if p == rank]


def gather_to_root(local, dist, world):
    """Rank 0 receives every rank's local result object (a list by rank);
    other ranks get None.  dist is torch.distributed or None (one rank)."""
    if dist is None or world == 1:
        return [local]
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(local, out, dst=0)
    return out
