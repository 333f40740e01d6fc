"""IIF2 and IIF3 time steps with a Newton implicit stage (oracle; test
infrastructure only).

Eq. krylov5 (IIF2):
    U^{n+1} = exp(dt A) (U^n + dt/2 F(U^n)) + dt/2 F(U^{n+1}).
Eq. krylov6 (IIF3):
    U^{n+1} = exp(dt A) U^n
              + dt (5/12 F(U^{n+1}) + 2/3 exp(dt A) F(U^n) - 1/12 exp(2 dt A) F(U^{n-1})).
Reading for IIF3: the two exp(dt A) terms are one Krylov projection of
U^n + 2/3 dt F(U^n) (as IIF2 projects U^n + dt/2 F(U^n)), and exp(2 dt A)
F(U^{n-1}) is a second projection with time 2 dt; the first step, which has
no F(U^{n-1}), is an IIF2 step.
Eq. krylov3 (r-th order, IIFr):
    U^{n+1} = exp(dt A) U^n + dt (alpha_1 F(U^{n+1})
              + sum_{i=0}^{r-2} alpha_{-i} exp((i+1) dt A) F(U^{n-i})),
with the alphas of eq. krylov4: the integrals over [0, dt] of the Lagrange
basis polynomials on the nodes tau = -k dt, k = -1..r-2.  The same reading:
the i = 0 term joins exp(dt A) U^n in one projection, every other i is a
projection over (i+1) dt, and a step uses the highest order its history of
past F values allows (IIF2, IIF3, ... up to r after a new state).
For a system the diffusion is block diagonal across species, so exp(dt A)
acts per species with that species' operator, one Krylov projection each.

Source terms (Examples 2 and 3): the equation u_t = k Lap u + f(u) + s(x, t)
puts the projection of s(., t) into F, so F(U, t) = P f(u_h) + P s(., t).
Every source used here is a sum of terms e^{lambda t} g(x) with g separable,
so P s(., t) = sum_m e^{lambda_m t} S_m with S_m = P g_m fixed vectors.  In
both schemes every F is taken at the time of its argument: F(U^n) at t^n,
F(U^{n+1}) (the Newton stage) at t^{n+1} = t^n + dt, F(U^{n-1}) at t^{n-1}.

The implicit stage G(U) = U - dt/2 F(U) - W = 0 (W the exponential term) is
solved by Newton's method, as Example 3 and Section 5 state.  Readings where
the paper is silent:
  * initial guess U = W;
  * Newton matrix I - dt/2 J_F(U), J_F(U) w = P(f'(u_h) w_h);
  * inner solver: conjugate gradients for a scalar equation (the matrix is
    symmetric), restarted GMRES(50) with Givens rotations for systems and
    for the interpolation form of F (module interp: J is not symmetric); both
    start from 0 and stop at relative residual INNER_TOL or INNER_MAX steps;
  * outer stop relative to the scale of the stage: ||G(U)||_2 <= NEWTON_TOL
    max(||W||_2, ||G(W)||_2) (the second term only matters when W = 0), at
    most NEWTON_MAX iterations, otherwise NewtonError.  A relative rule fixes
    the implicit stage to NEWTON_TOL of the state's size at every scale; an
    absolute floor (max(1, ||W||)) would leave states that have decayed far
    below 1 fixed only to 1e-12 in absolute terms.
"""
import numpy as np

from .combination import CombinationReaction
from .interp import InterpReaction
from .krylov import BREAKDOWN_TOL, krylov_expv_substeps
from .operator import sparse_matvec
from .reaction import Reaction

NEWTON_TOL = 1e-12
NEWTON_MAX = 50
INNER_TOL = 1e-13
INNER_MAX = 500
GMRES_RESTART = 50


class NewtonError(RuntimeError):
    pass


def cg(apply, b, tol=INNER_TOL, maxit=INNER_MAX):
    """Conjugate gradients from x = 0; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    stop = (tol ** 2) * rr
    it = 0
    while it < maxit and rr > stop:
        q = apply(p)
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def gmres(apply, b, tol=INNER_TOL, maxit=INNER_MAX, restart=GMRES_RESTART):
    """Restarted GMRES from x = 0 with CGS2 Arnoldi and Givens rotations."""
    n = b.size
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0
    it = 0
    while it < maxit:
        r = b - apply(x) if it else b.copy()
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm:
            break
        m = min(restart, maxit - it)
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        used = 0
        for j in range(m):
            w = apply(V[:, j])
            h1 = V[:, : j + 1].T @ w
            w = w - V[:, : j + 1] @ h1
            h2 = V[:, : j + 1].T @ w
            w = w - V[:, : j + 1] @ h2
            H[: j + 1, j] = h1 + h2
            hn = float(np.linalg.norm(w))
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            used = j + 1
            it += 1
            if abs(g[j + 1]) <= tol * bnorm or hn <= BREAKDOWN_TOL * den:
                break
            V[:, j + 1] = w / hn
        y = np.zeros(used)
        for i in range(used - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:used] @ y[i + 1:]) / H[i, i]
        x = x + V[:, :used] @ y
        if abs(g[used]) <= tol * bnorm:
            break
    return x, it


class IIF2Solver:
    """Sparse-grid Krylov IIF2 DG solver (Sections 2-3)."""

    def __init__(self, idx, S, kappas, reaction, dt, M, sources=None, t0=0.0, substeps=1,
                 reaction_form="quadrature"):
        """S: 1D SIPG matrix; kappas: per species, a length-d diagonal;
        sources: per species a list of (lambda, S_m) pairs (the source
        P s(., t) = sum_m e^{lambda t} S_m), or None; t0: the time of the
        state passed to run(); substeps: every exponential as that many
        successive projections (an extension; 1 is the paper's method);
        reaction_form: "quadrature" (the paper's finest-grid F, module
        reaction), "interp" (the sparse-grid interpolation form of module
        interp) or "combination" (the combination-technique form of module
        combination); the last two are deviations from the paper."""
        self.idx, self.S, self.dt, self.M = idx, S, dt, M
        self.substeps = int(substeps)
        self.kappas = [np.asarray(k, dtype=np.float64) for k in kappas]
        self.nspecies = len(self.kappas)
        self.reaction = reaction
        self.has_reaction = any(len(t) for t in reaction)
        rx_cls = {"quadrature": Reaction, "interp": InterpReaction, "combination": CombinationReaction}[reaction_form]
        self.rx = rx_cls(idx, reaction) if self.has_reaction else None
        self.sources = sources if sources is not None else [[] for _ in range(self.nspecies)]
        self.has_source = any(len(t) for t in self.sources)
        self.has_F = self.has_reaction or self.has_source
        self.t = float(t0)
        self.stats = {"newton": [], "inner": [], "m_eff": []}

    def A(self, s):
        return lambda x: sparse_matvec(self.idx, self.S, self.kappas[s], x)

    def expv(self, s, v, tau):
        """exp(tau A_s) v by Krylov projection (eq. krylov8); (w, m_eff)."""
        return krylov_expv_substeps(self.A(s), v, tau, self.M, self.substeps)

    def F(self, U, t):
        """F(U, t) = P f(u_h) + P s(., t)."""
        out = self.rx.F(U) if self.has_reaction else [np.zeros_like(u) for u in U]
        for s in range(self.nspecies):
            for lam, Sm in self.sources[s]:
                out[s] = out[s] + np.exp(lam * t) * Sm
        return out

    def J(self, U, xs):
        if not self.has_reaction:
            return [np.zeros_like(x) for x in xs]
        return self.rx.J(U, xs)

    def newton(self, W, c=None):
        """Solve U - c F(U, t^{n+1}) = W (c = dt/2 for IIF2)."""
        dt2 = 0.5 * self.dt if c is None else c
        U = [w.copy() for w in W]
        wnorm = float(np.sqrt(sum(float(w @ w) for w in W)))
        stop = None
        n = self.idx.dof
        inner_total = 0
        for it in range(NEWTON_MAX + 1):
            Fu = self.F(U, self.t + self.dt)
            G = np.concatenate([U[s] - dt2 * Fu[s] - W[s] for s in range(self.nspecies)])
            g = float(np.linalg.norm(G))
            if stop is None:  # first evaluation, at U = W
                stop = NEWTON_TOL * max(wnorm, g)
            if g <= stop:
                return U, it, inner_total
            if it == NEWTON_MAX:
                break

            def apply(x):
                xs = [x[s * n:(s + 1) * n] for s in range(self.nspecies)]
                Jx = self.J(U, xs)
                return np.concatenate([xs[s] - dt2 * Jx[s] for s in range(self.nspecies)])

            if self.nspecies == 1 and getattr(self.rx, "symmetric", True):
                delta, inner = cg(apply, -G)
            else:
                delta, inner = gmres(apply, -G)
            inner_total += inner
            for s in range(self.nspecies):
                U[s] = U[s] + delta[s * n:(s + 1) * n]
        raise NewtonError("Newton did not converge in %d iterations" % NEWTON_MAX)

    def step(self, U):
        """One IIF2 step (eq. krylov5); U is a list of per-species vectors."""
        dt2 = 0.5 * self.dt
        Fn = self.F(U, self.t)
        W = []
        for s in range(self.nspecies):
            v = U[s] + dt2 * Fn[s]
            w, m_eff = self.expv(s, v, self.dt)
            self.stats["m_eff"].append(m_eff)
            W.append(w)
        return self.finish(W, dt2)

    def finish(self, W, c):
        """The implicit stage of a step whose exponential term is W; advances t."""
        if not self.has_F:
            Unew, it, inner = W, 0, 0
        else:
            Unew, it, inner = self.newton(W, c)
        self.stats["newton"].append(it)
        self.stats["inner"].append(inner)
        self.t += self.dt
        return Unew

    def run(self, U, nsteps):
        U = [np.asarray(u, dtype=np.float64).copy() for u in U]
        for _ in range(nsteps):
            U = self.step(U)
        return U


class IIF3Solver(IIF2Solver):
    """Sparse-grid Krylov IIF3 DG solver (eq. krylov6), IIF2 for the first step."""

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        self.F_prev = None  # F(U^{n-1}) of the last step

    def step(self, U):
        dt = self.dt
        Fn = self.F(U, self.t)
        if self.F_prev is None:
            Unew = super().step(U)  # computes F(U^n) again: the same values
            self.F_prev = Fn
            return Unew
        W = []
        for s in range(self.nspecies):
            w1, m1 = self.expv(s, U[s] + (2.0 / 3.0) * dt * Fn[s], dt)
            w2, m2 = self.expv(s, self.F_prev[s], 2.0 * dt)
            self.stats["m_eff"] += [m1, m2]
            W.append(w1 - (dt / 12.0) * w2)
        self.F_prev = Fn
        return self.finish(W, 5.0 / 12.0 * dt)


def iif_alpha(r):
    """[alpha_1, alpha_0, alpha_{-1}, ..., alpha_{-(r-2)}] of eq. krylov4.

    alpha_{-i} = (1/dt) int_0^dt prod_{k=-1..r-2, k != i} (tau + k dt) / ((k - i) dt) dtau;
    with s = tau / dt each factor is (s + k) / (k - i), integrated over [0, 1].
    """
    nodes = list(range(-1, r - 1))
    out = []
    for i in nodes:
        poly = np.poly1d([1.0])
        for k in nodes:
            if k != i:
                poly = poly * np.poly1d([1.0 / (k - i), k / (k - i)])
        prim = poly.integ()
        out.append(float(prim(1.0) - prim(0.0)))
    return out


class IIFSolver(IIF2Solver):
    """Sparse-grid Krylov IIFr DG solver (eqs. krylov3, krylov4), r >= 2; the
    first steps after a new state use the orders their history allows."""

    def __init__(self, *args, order=3, **kw):
        super().__init__(*args, **kw)
        assert order >= 2
        self.order = order
        self.F_hist = []  # F(U^{n-1}), F(U^{n-2}), ... of the last steps

    def step(self, U):
        dt = self.dt
        Fn = self.F(U, self.t)
        r = min(self.order, 2 + len(self.F_hist))
        alpha = iif_alpha(r)
        W = []
        for s in range(self.nspecies):
            w, m = self.expv(s, U[s] + alpha[1] * dt * Fn[s], dt)
            self.stats["m_eff"].append(m)
            for i in range(1, r - 1):
                wi, mi = self.expv(s, self.F_hist[i - 1][s], (i + 1) * dt)
                self.stats["m_eff"].append(mi)
                w = w + alpha[i + 1] * dt * wi
            W.append(w)
        self.F_hist = ([Fn] + self.F_hist)[: self.order - 2]
        return self.finish(W, alpha[0] * dt)
