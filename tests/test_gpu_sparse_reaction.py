"""GPU parity of the sparse-grid interpolation form of the reaction term
(SGK_REACTION_INTERP, through the C ABI) against oracle.interp.

The form is a labelled deviation from the paper's finest-grid F, built for
its first stated future direction (Section 5): F_I(U) = C^{-1} f(C U) with C
the collocation matrix of the sparse set, applied direction by direction.
The oracle computes the same definition with dense 1D factors (pinned in
tests/test_oracle_interp.py against the collocation matrix formed entry by
entry); the library builds its factors from local formulas in C++ (checked
against the oracle on the CPU in tests/test_abi.py).

Tolerances (relative 2-norm): F_I and its Jacobian <= 1e-12 in both
precision modes (the transforms and the point kernels are FP64 in both);
IIF steps <= 1e-10 (FP64) and <= 1e-6 (mixed: double-float Krylov matvec);
the GPU solves the implicit stage pointwise at the collocation points to
rounding, the oracle by Newton-GMRES in coefficient space to 1e-12.
Sizes run from one cell to the largest served shape (d = 4, level 9,
degree 3: 6.8 M coefficients), whose finest full grid (1.6e14 quadrature
points) the quadrature form cannot hold.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.iif import IIF2Solver, IIF3Solver  # noqa: E402
from oracle.index_set import IndexSet as OIndex  # noqa: E402
from oracle.interp import InterpReaction  # noqa: E402
from oracle.operator import DIRICHLET0, PERIODIC, sipg_1d  # noqa: E402
from oracle.projection import project_separable  # noqa: E402
from paper_1810_11111_gb300 import sgkiif, workloads  # noqa: E402
from paper_1810_11111_gb300.runner import Problem  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DEV = torch.device("cuda", 0)
CUBIC = workloads.reaction_terms(workloads.CUBIC, 100.0)
SCHNAK = workloads.reaction_terms(workloads.SCHNAKENBERG)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device=DEV).contiguous()


def interp(cfg):
    return dict(cfg, reaction_form="interp")


class _Rig:
    """Context, index set, operators and an interpolation-form solver."""

    def __init__(self, d, n, k, rx, precision=sgkiif.SGK_FP64):
        self.ctx = sgkiif.Context(0, torch.cuda.current_stream().cuda_stream, precision)
        self.idx = sgkiif.IndexSet(self.ctx, d, n, k)
        self.ops = [sgkiif.Operator(self.ctx, self.idx, [1.0] * d) for _ in rx]
        self.sol = sgkiif.Solver(self.ctx, self.ops, rx, 10, 0.01, reaction_form="interp")

    def F(self, U):
        Ud = dev(np.concatenate(U))
        Fd = torch.empty_like(Ud)
        self.sol.reaction_eval(Ud.data_ptr(), Fd.data_ptr())
        torch.cuda.synchronize()
        return Fd.cpu().numpy()

    def J(self, U, W):
        Ud, Wd = dev(np.concatenate(U)), dev(np.concatenate(W))
        Jd = torch.empty_like(Ud)
        self.sol.jacobian_apply(Ud.data_ptr(), Wd.data_ptr(), Jd.data_ptr())
        torch.cuda.synchronize()
        return Jd.cpu().numpy()

    def close(self):
        self.sol.close()
        for o in self.ops:
            o.close()
        self.idx.close()
        self.ctx.close()


def _state(dof, S, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return [(1.0 if s == 0 else 0.9) * (np.arange(dof) == 0) + scale * rng.standard_normal(dof) for s in range(S)]


# one cell, every dimension template 1..6, every degree, ragged lengths
# (none of these DOF counts is a multiple of the 256-thread block), the
# benchmarked 3D shape and a two-species system
RX_CASES = [
    (1, 0, 1, CUBIC), (1, 6, 3, CUBIC), (2, 4, 1, CUBIC), (2, 7, 2, SCHNAK), (3, 4, 2, CUBIC),
    (3, 6, 2, CUBIC), (4, 4, 3, CUBIC), (4, 5, 2, SCHNAK), (5, 3, 1, CUBIC), (6, 2, 1, CUBIC),
]


@pytest.mark.parametrize("precision", [sgkiif.SGK_FP64, sgkiif.SGK_MIXED])
@pytest.mark.parametrize("d,n,k,rx", RX_CASES)
def test_interp_reaction_and_jacobian_match_oracle(d, n, k, rx, precision):
    S = len(rx)
    rig = _Rig(d, n, k, rx, precision)
    U = _state(rig.idx.dof, S, 11)
    W = [np.random.default_rng(12 + s).standard_normal(rig.idx.dof) for s in range(S)]
    ref = InterpReaction(OIndex(d, n, k), rx)
    assert rel(rig.F(U), np.concatenate(ref.F(U))) <= 1e-12
    assert rel(rig.J(U, W), np.concatenate(ref.J(U, W))) <= 1e-12
    rig.close()


@pytest.mark.parametrize("d,n,k", [(4, 9, 3), (3, 9, 3), (4, 8, 2)])
def test_interp_linear_reaction_is_exact_at_the_largest_shapes(d, n, k):
    # f(u) = a u + b lies in the sparse space, so F_I = a U + b e_0 exactly:
    # every pass of C and C^{-1} at full size must be right for this to hold
    rx = [[(-1.7, (1,)), (0.3, (0,))]]
    rig = _Rig(d, n, k, rx)
    U = _state(rig.idx.dof, 1, 13)
    want = -1.7 * U[0]
    want[0] += 0.3
    assert rel(rig.F(U), want) <= 1e-12
    rig.close()


def test_interp_cubic_reaction_at_a_large_shape():
    # d = 4, level 8, degree 2 (850 176 coefficients; the finest full grid
    # would hold 3.5e11 nodal values): the oracle's directional computation
    # of the whole vector
    d, n, k = 4, 8, 2
    rig = _Rig(d, n, k, CUBIC)
    idx = OIndex(d, n, k)
    U = [project_separable(idx, [0.8, -0.5], [[1, 2, 1, 3], [2, 1, 1, 1]], [[0, 1, 0, 1], [1, 1, 0, 0]], 0.2)]
    assert rel(rig.F(U), InterpReaction(idx, CUBIC).F(U)[0]) <= 1e-12
    rig.close()


def _oracle_steps(cfg, U0, nsteps, obc=PERIODIC, sources=None, t0=0.0):
    idx = OIndex(cfg["d"], cfg["n"], cfg["k"])
    cls = IIF3Solver if cfg.get("scheme", sgkiif.SGK_IIF2) == sgkiif.SGK_IIF3 else IIF2Solver
    sol = cls(idx, sipg_1d(cfg["n"], cfg["k"], obc), cfg["kappas"], cfg["reaction"], cfg["dt"], cfg["M"],
              sources=sources, t0=t0, reaction_form="interp")
    return sol.run(U0, nsteps)


STEP_CASES = [
    ("cubic3d_small", workloads.cubic3d(n=3, k=2), 3),
    ("cubic3d_l4", workloads.cubic3d(n=4, k=2), 3),
    ("schnak2d_small", workloads.schnak2d(n=4, k=1), 3),
    ("schnak2d_k2", workloads.schnak2d(n=5, k=2), 2),
    ("cubic2d_k3", dict(workloads.cubic3d(n=4, k=3), d=2, kappas=[[1.0, 0.3]],
                        init=[dict(amp=np.array([0.7, -0.4]), wavenum=np.array([[1, 2], [3, 1]], np.int32),
                                   kind=np.array([[0, 1], [1, 0]], np.int32), const=0.1)]), 2),
]


@pytest.mark.parametrize("name,cfg,nsteps", STEP_CASES)
@pytest.mark.parametrize("precision", [sgkiif.SGK_FP64, sgkiif.SGK_MIXED])
def test_interp_iif2_steps_match_oracle(name, cfg, nsteps, precision):
    # IIF2 with one or two species runs as one device-driven graph per step
    prob = Problem(interp(cfg), precision)
    prob.reset()
    U0 = [u.cpu().numpy() for u in prob.U0]
    prob.solver.step(nsteps)
    got = prob.state()
    want = _oracle_steps(cfg, U0, nsteps)
    tol = 1e-10 if precision == sgkiif.SGK_FP64 else 1e-6
    for s in range(len(want)):
        assert rel(got[s], want[s]) <= tol, (name, s, rel(got[s], want[s]))
    st = prob.solver.stats()
    assert st["steps"] == nsteps and st["inner_iters"] == 0 and st["newton_iters"] >= nsteps
    prob.close()


@pytest.mark.parametrize("scheme", [sgkiif.SGK_IIF2, sgkiif.SGK_IIF3])
@pytest.mark.parametrize("precision", [sgkiif.SGK_FP64, sgkiif.SGK_MIXED])
def test_interp_example3_steps_with_source_match_oracle(scheme, precision):
    # zero Dirichlet, f = u^2 and the source -e^{-2t} prod sin^2(2 pi x_i)
    # (Example 3) from t0 = 0.37: the source enters the pointwise stage as
    # C (W + c S(t^{n+1})); IIF3 is host-driven
    from test_gpu_parity import _example23_cfg, _oracle_sources
    k = 1 if scheme == sgkiif.SGK_IIF2 else 2
    cfg, bc, obc = _example23_cfg(3, 2, k, 4, scheme)
    t0, nsteps = 0.37, 5
    prob = Problem(interp(cfg), precision, bc=bc)
    prob.reset()
    prob.solver.set_time(t0)
    U0 = [u.cpu().numpy() for u in prob.U0]
    prob.solver.step(nsteps)
    got = prob.state()[0]
    idx = OIndex(2, 4, k)
    want = _oracle_steps(cfg, U0, nsteps, obc, _oracle_sources(cfg, idx), t0)[0]
    assert rel(got, want) <= (1e-10 if precision == sgkiif.SGK_FP64 else 1e-6)
    prob.close()


def test_interp_newton_failure_rolls_back():
    # one correction allowed per point: the pointwise solve cannot converge,
    # the step reports SGK_ENEWTON and the state is the one before it
    cfg = dict(interp(workloads.cubic3d(n=3, k=1)), opts={"max_iter": 1})
    prob = Problem(cfg, sgkiif.SGK_FP64)
    prob.reset()
    before = prob.state()[0]
    with pytest.raises(sgkiif.SgkError) as ei:
        prob.solver.step(1)
    assert ei.value.code == sgkiif.SGK_ENEWTON
    assert np.array_equal(prob.state()[0], before)
    assert prob.solver.stats()["steps"] == 0
    prob.close()


@pytest.mark.parametrize("precision,tol", [(sgkiif.SGK_FP64, 1e-10), (sgkiif.SGK_MIXED, 1e-6)])
def test_interp_cubic3d_full_size_20_steps_match_oracle(precision, tol):
    # the benchmarked workload (d = 3, level 6, degree 2, 20 steps) with the
    # interpolation form, against the oracle's stored run
    # (tests/golden/make_full_size.py cubic3d_interp)
    path = os.path.join(GOLDEN, "cubic3d_interp_steps.npz")
    if not os.path.exists(path):
        pytest.skip("golden run not generated")
    g = np.load(path)
    prob = Problem(interp(workloads.cubic3d()), precision)
    assert np.abs(prob.U0[0].cpu().numpy() - g["U0"][0]).max() <= 1e-13
    prob.solver.set_state(0, g["U0"][0])
    done = 0
    for step in (1, 5, 10, 20):
        prob.solver.step(step - done)
        done = step
        assert rel(prob.state()[0], g["U%d" % step][0]) <= tol, (step, rel(prob.state()[0], g["U%d" % step][0]))
    prob.close()


def test_interp_batch_and_server_match_the_solver():
    # instances of the interpolation form (the batched Arnoldi launch and
    # the engine's continuous batching) next to a quadrature-form instance:
    # each equals the same problem stepped alone by the solver
    from test_gpu_batch import cubic as batch_cubic
    insts = [(interp(batch_cubic(3, 5, 2, 61)), sgkiif.SGK_MIXED), (interp(batch_cubic(4, 4, 1, 62)), sgkiif.SGK_FP64),
             (interp(workloads.schnak2d(n=5, k=1, steps=3, seed=63)), sgkiif.SGK_MIXED),
             (batch_cubic(2, 5, 2, 64), sgkiif.SGK_FP64)]
    alone = []
    for cfg, prec in insts:
        p = Problem(cfg, prec)
        p.reset()
        p.solver.step(3)
        alone.append(np.concatenate(p.state()))
        p.close()
    b = sgkiif.Batch(0, streams=4)
    for cfg, prec in insts:
        b.add(cfg, prec)
    rc, st = b.step(3)
    assert rc == sgkiif.SGK_OK and all(s == sgkiif.SGK_OK for s in st)
    for i, (cfg, prec) in enumerate(insts):
        tol = 1e-10 if prec == sgkiif.SGK_FP64 else 1e-6
        assert rel(np.concatenate(b.state(i)), alone[i]) <= tol, i
    b.close()
    srv = sgkiif.Server(0, workers=2, engine=True)
    tickets = [srv.submit(dict(cfg, steps=3), prec) for cfg, prec in insts]
    for t, (cfg, prec), ref in zip(tickets, insts, alone):
        out, info = srv.wait(t, cap=4 * sgkiif.dof_of(cfg["d"], cfg["n"], cfg["k"]))
        assert info["status"] == sgkiif.SGK_OK
        if "reaction_form" in cfg:
            assert info["inner_iters"] == 0
        assert rel(out, ref) <= (1e-10 if prec == sgkiif.SGK_FP64 else 1e-6)
    srv.close()


def test_interp_admits_a_shape_the_quadrature_form_cannot_hold():
    # d = 4, level 9, degree 3: the finest full grid needs ~34 GB per array
    # in FP32 (far more with its work arrays); the interpolation form needs
    # the sparse vectors only.  Two IIF2 steps of a 6.8 M-coefficient cubic
    # problem in mixed precision: finite, decaying, and equal to FP64 within
    # the mixed tolerance.
    cfg = dict(workloads.cubic3d(n=9, k=3), d=4, kappas=[[1.0, 0.5, 0.1, 0.7]], steps=2,
               init=[dict(amp=np.array([0.8, -0.5]), wavenum=np.array([[1, 2, 1, 3], [2, 1, 1, 1]], np.int32),
                          kind=np.array([[0, 1, 0, 1], [1, 1, 0, 0]], np.int32), const=0.2)])
    quad = sgkiif.sgk_estimate_bytes(4, 9, 3, 1, 30, sgkiif.SGK_MIXED, 1)
    sparse = sgkiif.sgk_estimate_bytes(4, 9, 3, 1, 30, sgkiif.SGK_MIXED, 2)
    free, _ = torch.cuda.mem_get_info()
    assert sparse < free < quad
    out = {}
    for prec in (sgkiif.SGK_MIXED, sgkiif.SGK_FP64):
        prob = Problem(interp(cfg), prec)
        prob.reset()
        n0 = np.linalg.norm(prob.U0[0].cpu().numpy())
        prob.solver.step(2)
        out[prec] = prob.state()[0]
        assert np.all(np.isfinite(out[prec])) and np.linalg.norm(out[prec]) < n0
        prob.close()
    assert rel(out[sgkiif.SGK_MIXED], out[sgkiif.SGK_FP64]) <= 1e-6
