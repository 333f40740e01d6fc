"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module only draws random numbers and names problem sizes; it contains
none of the method's arithmetic, so both the CUDA path and the oracle can take
their inputs from it.  All draws use numpy's PCG64 (``default_rng(seed)``).

Workloads (sizes follow the paper's 2D/3D scalar and two-species runs):
  heat2d      u_t = Lap u on [0,1]^2, periodic, level 4, degree 1,
              u_0 = sin(2 pi x) sin(2 pi y), M = 20, dt = 0.01, 10 steps
  cubic3d     d = 3, level 6, degree 2, diffusion diag(1, 0.5, 0.1),
              f(u) = -100 u^3, u_0 = 8 seeded Fourier products (seed 1),
              IIF2, M = 30, dt = 0.005, 20 steps
  schnak2d    d = 2, level 8, degree 2, two species (kappa 0.01 / 0.5),
              f_u = 0.1 - u + u^2 v, f_v = 0.9 - u^2 v, u_0 = 1.0 and
              v_0 = 0.9 plus 0.01 N(0,1) on every coefficient (seed 2),
              IIF2, M = 40, dt = 0.05, 200 steps
  batch       256 scalar instances (seed 3): d in {2,3,4}, level 5..8,
              degree 1..2, kappa_i ~ U(0.05, 1), f = -c u^3 with
              c ~ U(1, 100), 8-mode Fourier u_0; M = 30, dt = 0.005
  served      Poisson arrivals of solve requests (seed 4): d in {3,4},
              level 6..9, degree 1..3, scalar cubic (f = -100 u^3,
              8-mode Fourier u_0) or two-species Schnakenberg (the
              schnak2d constants and noise), 10..100 steps, M = 30,
              dt = 0.005; draws whose finest grid exceeds the nodal budget
              are rejected and counted
"""
import numpy as np

CUBIC = "cubic"
SCHNAKENBERG = "schnakenberg"
HEAT = "heat"


def fourier_modes(rng, d, nmodes=8):
    """amp ~ U(-1,1); wavenumbers ~ U{1,2,3}; factor kind ~ U{sin, cos}."""
    amp = rng.uniform(-1.0, 1.0, nmodes)
    wavenum = rng.integers(1, 4, size=(nmodes, d)).astype(np.int32)
    kind = rng.integers(0, 2, size=(nmodes, d)).astype(np.int32)
    return amp, wavenum, kind


def reaction_terms(kind, c=100.0):
    """Monomial lists per species: (coefficient, exponents by species)."""
    if kind == HEAT:
        return [[]]
    if kind == CUBIC:
        return [[(-float(c), (3,))]]
    if kind == SCHNAKENBERG:
        return [[(0.1, (0, 0)), (-1.0, (1, 0)), (1.0, (2, 1))],
                [(0.9, (0, 0)), (-1.0, (2, 1))]]
    raise ValueError(kind)


def heat2d():
    return dict(name="heat2d", d=2, n=4, k=1, kappas=[[1.0, 1.0]], reaction=reaction_terms(HEAT),
                M=20, dt=0.01, steps=10,
                init=[dict(amp=np.array([1.0]), wavenum=np.array([[1, 1]], np.int32),
                           kind=np.array([[0, 0]], np.int32), const=0.0)])


def cubic3d(n=6, k=2, steps=20, seed=1):
    rng = np.random.default_rng(seed)
    amp, wavenum, kind = fourier_modes(rng, 3)
    return dict(name="cubic3d", d=3, n=n, k=k, kappas=[[1.0, 0.5, 0.1]], reaction=reaction_terms(CUBIC),
                M=30, dt=0.005, steps=steps,
                init=[dict(amp=amp, wavenum=wavenum, kind=kind, const=0.0)])


def schnak2d(n=8, k=2, steps=200, seed=2):
    return dict(name="schnak2d", d=2, n=n, k=k, kappas=[[0.01, 0.01], [0.5, 0.5]],
                reaction=reaction_terms(SCHNAKENBERG), M=40, dt=0.05, steps=steps,
                init=[dict(noise_seed=seed, base=1.0, species=0), dict(noise_seed=seed, base=0.9, species=1)])


def coefficient_noise(seed, dof, nspecies, base, scale=0.01):
    """Per-coefficient noise initial data: base_s on the constant function plus
    scale * N(0,1) on every coefficient, one stream for all species."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nspecies):
        u = scale * rng.standard_normal(dof)
        u[0] += base[s]
        out.append(u)
    return out


def batch_instances(count=256, seed=3, max_nodal_bytes=2 << 30):
    """Scalar cubic instances of uneven size; draws whose finest-grid nodal
    array ((k+1) 2^n)^d exceeds max_nodal_bytes in FP64 are rejected and
    counted (the reaction term reconstructs on the finest full grid)."""
    rng = np.random.default_rng(seed)
    out, rejected = [], 0
    while len(out) < count:
        d = int(rng.integers(2, 5))
        n = int(rng.integers(5, 9))
        k = int(rng.integers(1, 3))
        kappa = rng.uniform(0.05, 1.0, d)
        c = float(rng.uniform(1.0, 100.0))
        amp, wavenum, kind = fourier_modes(rng, d)
        if (((k + 1) << n) ** d) * 8 > max_nodal_bytes:
            rejected += 1
            continue
        out.append(dict(d=d, n=n, k=k, kappas=[list(kappa)], reaction=reaction_terms(CUBIC, c),
                        M=30, dt=0.005, steps=20,
                        init=[dict(amp=amp, wavenum=wavenum, kind=kind, const=0.0)]))
    return out, rejected


def served_requests(count=16, seed=4, max_nodal_bytes=2 << 30, max_steps=100):
    """Solve requests of the served workload and the number of rejected draws.
    Each request is a workload dict (as cubic3d / schnak2d) with a
    precision-independent seeded initial state."""
    rng = np.random.default_rng(seed)
    out, rejected = [], 0
    while len(out) < count:
        d = int(rng.integers(3, 5))
        n = int(rng.integers(6, 10))
        k = int(rng.integers(1, 4))
        kind = CUBIC if rng.random() < 0.5 else SCHNAKENBERG
        steps = int(rng.integers(10, max_steps + 1))
        noise_seed = int(rng.integers(0, 2 ** 31))
        amp, wavenum, kindv = fourier_modes(rng, d)
        if (((k + 1) << n) ** d) * 8 > max_nodal_bytes:
            rejected += 1
            continue
        if kind == CUBIC:
            req = dict(name="served-cubic", d=d, n=n, k=k, kappas=[[1.0, 0.5, 0.1, 0.7][:d]],
                       reaction=reaction_terms(CUBIC, 100.0),
                       init=[dict(amp=amp, wavenum=wavenum, kind=kindv, const=0.0)])
        else:
            req = dict(name="served-schnakenberg", d=d, n=n, k=k, kappas=[[0.01] * d, [0.5] * d],
                       reaction=reaction_terms(SCHNAKENBERG),
                       init=[dict(noise_seed=noise_seed, base=1.0, species=0),
                             dict(noise_seed=noise_seed, base=0.9, species=1)])
        req.update(M=30, dt=0.005, steps=steps)
        out.append(req)
    return out, rejected


def poisson_arrivals(count, rate_per_s, seed=4):
    """Arrival times (s, from 0) of a Poisson stream."""
    rng = np.random.default_rng(seed + 1000)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count)) - 0.0
