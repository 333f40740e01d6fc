"""Batched stepping (sgk_batch_*): many independent problems of uneven size.

On the GPU: every instance of a mixed batch (2D/3D/4D cubic reaction in
FP64 and mixed precision, pure diffusion, a two-species system that takes
the host-driven path) matches the same problem solved alone through the
solver API within the parity tolerance of its precision (1e-10 FP64, 1e-6
mixed; the persistent Arnoldi grid differs, so sums run in another order);
the batch's results do not depend on its stream count (bitwise); the
batched Arnoldi launches (one persistent cooperative launch per kernel
class, CTAs walking (instance, slice) work lists) give bitwise the results
of every instance's own whole-step graph, also when many instances of one
class must share the CTAs in turn.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1810_11111_gb300 import sgkiif, workloads  # noqa: E402
from paper_1810_11111_gb300.runner import Problem  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cubic(d, n, k, seed, c=100.0):
    rng = np.random.default_rng(seed)
    amp, wn, kind = workloads.fourier_modes(rng, d)
    kap = list(rng.uniform(0.05, 1.0, d))
    return dict(d=d, n=n, k=k, kappas=[kap], reaction=workloads.reaction_terms(workloads.CUBIC, c),
                M=30, dt=0.005, steps=3, init=[dict(amp=amp, wavenum=wn, kind=kind, const=0.0)])


INSTANCES = [
    (cubic(3, 5, 2, 41), sgkiif.SGK_MIXED),
    (cubic(2, 7, 1, 42, 37.0), sgkiif.SGK_FP64),
    (cubic(4, 3, 1, 43, 5.0), sgkiif.SGK_MIXED),
    (dict(cubic(3, 4, 2, 44), reaction=[[]]), sgkiif.SGK_FP64),
    (workloads.schnak2d(n=5, k=1, steps=3, seed=45), sgkiif.SGK_MIXED),
    (cubic(2, 5, 2, 46), sgkiif.SGK_FP64),
]


def run_batch(streams, steps, fused=True, instances=INSTANCES, with_est=False):
    b = sgkiif.Batch(0, streams=streams, fused=fused)
    for cfg, prec in instances:
        b.add(cfg, prec)
    rc, st = b.step(steps)
    assert rc == sgkiif.SGK_OK and all(s == sgkiif.SGK_OK for s in st)
    out = [np.concatenate(b.state(i)) for i in range(len(instances))]
    est = [b.stats(i)["max_krylov_err_est"] for i in range(len(instances))]
    assert (b.launches() > 0) == fused
    b.close()
    return (out, est) if with_est else out


def test_batch_matches_instances_alone():
    got = run_batch(4, 3)
    for (cfg, prec), g in zip(INSTANCES, got):
        p = Problem(cfg, prec)
        p.reset()
        p.solver.step(3)
        want = np.concatenate(p.state())
        p.close()
        assert rel(g, want) <= (1e-10 if prec == sgkiif.SGK_FP64 else 1e-6)


def test_batch_independent_of_stream_count():
    a = run_batch(1, 2)
    b = run_batch(5, 2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_batched_launch_equals_whole_step_graphs():
    a, ea = run_batch(3, 2, fused=True, with_est=True)
    b, eb = run_batch(3, 2, fused=False, with_est=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # the a-posteriori Krylov estimates come out of the same projections
    assert ea == eb and all(np.isfinite(e) and e >= 0.0 for e in ea)


def test_batched_launch_with_more_instances_than_sms():
    # 60 small 2D instances (1024 coefficients, 3 CTAs each: 180 CTAs, more
    # than the SMs): CTAs take several instances in turn from their work lists
    many = [(cubic(2, 6, 1, 100 + i, 10.0 + i), sgkiif.SGK_MIXED) for i in range(60)]
    a = run_batch(8, 2, fused=True, instances=many)
    b = run_batch(8, 2, fused=False, instances=many)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_batch_accuracy_guard_matches_guarded_solver():
    # instances with the Krylov accuracy guard (M = 10, tolerance 1e-9, at
    # most 32 sub-projections): a step the guard rolls back is taken again
    # in a later tick, every instance still takes its 3 steps, and each
    # equals the same problem stepped alone with the guard, having settled
    # on the same sub-projection count
    insts = [(dict(cubic(2, 6, 1, 60 + i, 20.0 + 10 * i), M=10, krylov_tol=1e-9, krylov_max_substeps=32), prec)
             for i, prec in enumerate([sgkiif.SGK_MIXED, sgkiif.SGK_FP64, sgkiif.SGK_MIXED])]
    insts.append((cubic(3, 4, 2, 63), sgkiif.SGK_MIXED))  # no guard: stays in the batched Arnoldi launch
    b = sgkiif.Batch(0, streams=3)
    for cfg, prec in insts:
        b.add(cfg, prec)
    rc, st = b.step(3)
    assert rc == sgkiif.SGK_OK and all(x == sgkiif.SGK_OK for x in st)
    got = [np.concatenate(b.state(i)) for i in range(len(insts))]
    bst = [b.stats(i) for i in range(len(insts))]
    b.close()
    for (cfg, prec), g, sb in zip(insts, got, bst):
        p = Problem(cfg, prec)
        if cfg.get("krylov_tol"):
            p.solver.set_krylov_tolerance(cfg["krylov_tol"], cfg["krylov_max_substeps"])
        p.reset()
        p.solver.step(3)
        want = np.concatenate(p.state())
        ps = p.solver.stats()
        p.close()
        assert sb["steps"] == ps["steps"] == 3
        assert sb["krylov_substeps"] == ps["krylov_substeps"]
        assert (sb["krylov_substeps"] > 1) == bool(cfg.get("krylov_tol"))
        assert rel(g, want) <= (1e-10 if prec == sgkiif.SGK_FP64 else 1e-6)
