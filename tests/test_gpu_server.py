"""The request loop (sgk_server_*): continuous batching of whole IIF2 solves.

Checks, on the GPU:
  * a request's result is the same alone and in a mix of concurrent requests
    on a server with the same worker count (bitwise: every kernel sums in a
    fixed order and the persistent Arnoldi grid depends only on the worker
    count), and matches the direct solver path within the parity tolerance
    of its precision (1e-10 FP64, 1e-6 mixed);
  * requests overlap (more than one runs at once) when the budget allows;
  * the memory admission serialises requests when only one fits, and
    rejects a request larger than the whole budget;
  * the engine (iteration-level continuous batching of the single-species
    requests on the batched Arnoldi launches) runs several requests at once,
    reports them as engine requests, gives each the same coefficients alone
    and in a mix, and matches the worker path and the direct solver path
    within the parity tolerance; requests that arrive while others are
    stepping join the running batch.
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


def cubic(d, n, k, steps, seed):
    cfg = workloads.cubic3d(n=n, k=k, steps=steps, seed=seed)
    if d != 3:
        rng = np.random.default_rng(seed)
        amp, wn, kind = workloads.fourier_modes(rng, d)
        cfg.update(d=d, kappas=[[1.0, 0.5, 0.1, 0.7][:d]], init=[dict(amp=amp, wavenum=wn, kind=kind, const=0.0)])
    return cfg


MIX = [
    (cubic(3, 5, 2, 6, 21), sgkiif.SGK_MIXED),
    (workloads.schnak2d(n=6, k=1, steps=5, seed=22), sgkiif.SGK_MIXED),
    (cubic(2, 7, 1, 8, 23), sgkiif.SGK_FP64),
    (cubic(3, 4, 3, 4, 24), sgkiif.SGK_FP64),
    (cubic(4, 3, 1, 5, 25), sgkiif.SGK_MIXED),
]


def direct(cfg, prec):
    p = Problem(cfg, prec)
    p.reset()
    p.solver.step(cfg["steps"])
    out = np.concatenate(p.state())
    p.close()
    return out


@pytest.mark.parametrize("engine", [True, False])
def test_same_alone_and_in_mix(engine):
    srv = sgkiif.Server(0, workers=3, engine=engine)
    alone = []
    for cfg, prec in MIX:
        t = srv.submit(cfg, prec)
        out, info = srv.wait(t, cap=4 * sgkiif.dof_of(cfg["d"], cfg["n"], cfg["k"]))
        assert info["status"] == sgkiif.SGK_OK and info["steps"] == cfg["steps"]
        alone.append(out)
    tickets = [srv.submit(cfg, prec) for cfg, prec in MIX for _ in range(2)]
    mixed = [srv.wait(t, cap=4 * sgkiif.dof_of(cfg["d"], cfg["n"], cfg["k"]))
             for t, (cfg, prec) in zip(tickets, [m for m in MIX for _ in range(2)])]
    st = srv.stats()
    srv.close()
    assert st["max_concurrent"] >= 2
    assert st["failed"] == 0
    for i, (out, info) in enumerate(mixed):
        assert info["status"] == sgkiif.SGK_OK
        assert np.array_equal(out, alone[i // 2])
    for (cfg, prec), a in zip(MIX, alone):
        tol = 1e-10 if prec == sgkiif.SGK_FP64 else 1e-6
        assert rel(a, direct(cfg, prec)) <= tol


def test_admission_by_memory():
    cfg = cubic(3, 5, 2, 3, 31)
    est = int(sgkiif.sgk_estimate_bytes(3, 5, 2, 1, cfg["M"], sgkiif.SGK_MIXED, 1))
    assert est > 0
    # room for one request at a time: four workers but no overlap
    srv = sgkiif.Server(0, workers=4, mem_budget_bytes=int(1.5 * est))
    ts = [srv.submit(cfg, sgkiif.SGK_MIXED) for _ in range(4)]
    infos = [srv.wait(t)[1] for t in ts]
    st = srv.stats()
    assert all(i["status"] == sgkiif.SGK_OK for i in infos)
    assert st["max_concurrent"] == 1 and st["peak_reserved_bytes"] <= int(1.5 * est)
    # larger than the whole budget: rejected at submission
    with pytest.raises(sgkiif.SgkError) as e:
        srv.submit(cubic(3, 7, 3, 1, 32), sgkiif.SGK_MIXED)
    assert e.value.code == sgkiif.SGK_ENOMEM
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_engine_batches_requests_and_matches_workers():
    reqs = [(cubic(3, 5, 2, 6 + i, 40 + i), sgkiif.SGK_MIXED) for i in range(5)] + \
           [(cubic(2, 6, 1, 4 + i, 50 + i), sgkiif.SGK_FP64) for i in range(3)]
    caps = [4 * sgkiif.dof_of(c["d"], c["n"], c["k"]) for c, _ in reqs]
    srv = sgkiif.Server(0, workers=2, engine=True)
    tickets = [srv.submit(c, p) for c, p in reqs]
    eng = [srv.wait(t, cap=cap) for t, cap in zip(tickets, caps)]
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0 and st["max_concurrent"] >= 2
    assert all(info["worker"] == -1 and info["steps"] == c["steps"] for (_, info), (c, _) in zip(eng, reqs))
    srv = sgkiif.Server(0, workers=2, engine=False)
    wrk = [srv.wait(srv.submit(c, p), cap=cap) for (c, p), cap in zip(reqs, caps)]
    srv.close()
    for (c, p), (a, _), (b, _) in zip(reqs, eng, wrk):
        tol = 1e-10 if p == sgkiif.SGK_FP64 else 1e-6
        assert rel(a, b) <= tol and rel(a, direct(c, p)) <= tol


def test_engine_admits_requests_while_stepping():
    import time
    srv = sgkiif.Server(0, workers=1, engine=True)
    long_req = cubic(3, 5, 2, 400, 61)
    s0 = time.perf_counter()
    t0 = srv.submit(long_req, sgkiif.SGK_MIXED)
    time.sleep(0.1)  # the long request is being set up or stepping
    short = [cubic(2, 5, 1, 3, 62 + i) for i in range(3)]
    s1 = time.perf_counter()
    ts = [srv.submit(c, sgkiif.SGK_MIXED) for c in short]
    outs = [srv.wait(t, cap=4 * sgkiif.dof_of(c["d"], c["n"], c["k"])) for t, c in zip(ts, short)]
    out0, info0 = srv.wait(t0, cap=4 * sgkiif.dof_of(3, 5, 2))
    srv.close()
    assert info0["status"] == sgkiif.SGK_OK and info0["steps"] == 400
    done_long = s0 * 1e3 + info0["latency_ms"]
    for (out, info), c in zip(outs, short):
        assert info["status"] == sgkiif.SGK_OK and info["worker"] == -1
        # admitted at once and finished while the long request was still
        # stepping: they joined its batch instead of waiting behind it
        assert info["queue_ms"] < 50.0
        assert s1 * 1e3 + info["latency_ms"] < done_long
        assert rel(out, direct(c, sgkiif.SGK_MIXED)) <= 1e-6


def test_accuracy_guard_through_engine_and_workers():
    # requests that set the Krylov accuracy guard (M = 10, tolerance 1e-9):
    # through the engine (a rolled-back step is taken again in the next tick)
    # and through the workers (synchronous steps), each equals the problem
    # stepped alone with the guard and reports all its steps
    reqs = [(dict(cubic(2, 6, 1, 4 + i, 70 + i), M=10, krylov_tol=1e-9, krylov_max_substeps=32), prec)
            for i, prec in enumerate([sgkiif.SGK_MIXED, sgkiif.SGK_FP64])]

    def guarded(cfg, prec):
        p = Problem(cfg, prec)
        p.solver.set_krylov_tolerance(cfg["krylov_tol"], cfg["krylov_max_substeps"])
        p.reset()
        p.solver.step(cfg["steps"])
        out = np.concatenate(p.state())
        p.close()
        return out

    for engine in (True, False):
        srv = sgkiif.Server(0, workers=2, engine=engine)
        res = [srv.wait(srv.submit(c, p), cap=4 * sgkiif.dof_of(c["d"], c["n"], c["k"])) for c, p in reqs]
        srv.close()
        for (c, p), (out, info) in zip(reqs, res):
            assert info["status"] == sgkiif.SGK_OK and info["steps"] == c["steps"]
            assert (info["worker"] == -1) == engine
            assert rel(out, guarded(c, p)) <= (1e-10 if p == sgkiif.SGK_FP64 else 1e-6)


def test_request_guard_fields_are_validated():
    srv = sgkiif.Server(0, workers=1)
    bad = dict(cubic(2, 4, 1, 2, 80), krylov_tol=1e-6, krylov_max_substeps=0)
    with pytest.raises(sgkiif.SgkError) as e:
        srv.submit(bad, sgkiif.SGK_FP64)
    assert e.value.code == sgkiif.SGK_EINVAL
    srv.close()
