"""Synthetic workload definitions: parameter sets and seeds only.

These describe the runs (Kn, gas, cells, particles per cell, force, steps, seeds)
that the tests and the benchmark feed to both the CUDA library and the oracle.  This
module holds none of the DSMC arithmetic; each side derives its own time step,
cross-sections and collision parameters from these inputs.

Shapes follow the paper's workloads (Sec. 3: Delta y = 0.005 cells, 50 to 500
particles per cell, low-speed force-driven flow, long time averages) scaled to the
sizes of the benchmark configurations below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


def f0_force(Kn: float, sigma_p: float = 1.0) -> float:
    """Body force (v0^2/H) whose slip-Stokes channel-mean speed is 1e-3 v0: the mean
    of the Eq. 8 parabola (S = 0) plus first-order slip (Eq. 10),
    u_mean = sqrt(pi) F / (12 Kn) + sigma_P F, with sigma_P := 1."""
    return 1e-3 / (math.sqrt(math.pi) / (12.0 * Kn) + sigma_p)


@dataclass(frozen=True)
class Workload:
    name: str
    omega: float
    Kn: float
    n_cells: int
    ppc: int
    body_force: float
    steps: int
    sample_start: int
    seeds: tuple = (0,)
    group_size: int = 256
    dt_factor: float = 0.2
    extra: dict = field(default_factory=dict)

    @property
    def n_particles(self) -> int:
        return self.n_cells * self.ppc


# Argon hard spheres at Kn = 1: 100 cells, 200 particles per cell, 2,000 steps with the
# last 1,000 sampled, mean speed ~1e-3 v0.
HS_KN1 = Workload("hs_kn1_100c_200ppc", omega=0.5, Kn=1.0, n_cells=100, ppc=200,
                  body_force=f0_force(1.0), steps=2000, sample_start=1001,
                  seeds=tuple(range(16)))

# Argon VHS (omega = 0.81) at Kn = 0.1: 2,000 cells, 25,000 particles per cell
# (5e7 particles), 20,000 steps sampled after step 5,000.
VHS_KN01_50M = Workload("vhs_kn0.1_2000c_25000ppc", omega=0.81, Kn=0.1, n_cells=2000,
                        ppc=25000, body_force=f0_force(0.1), steps=20000,
                        sample_start=5001, seeds=(0, 1, 2, 3))


def scaled(w: Workload, n_cells: int = None, ppc: int = None, **kw) -> Workload:
    """The same physics with fewer cells or particles (parity-test sizes)."""
    d = dict(w.__dict__)
    d.update(kw)
    if n_cells is not None:
        d["n_cells"] = n_cells
    if ppc is not None:
        d["ppc"] = ppc
    d["name"] = f"{w.name}@{d['n_cells']}c_{d['ppc']}ppc"
    return Workload(**d)


def batch_instances(n: int = 256, seed: int = 12345):
    """Independent runs with Kn log-uniform in [0.05, 10], cells uniform in
    {50..1000}, particles per cell uniform in {50..400}, force uniform in
    [0.5, 2] x f0_force(1)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        Kn = float(math.exp(rng.uniform(math.log(0.05), math.log(10.0))))
        out.append(Workload(f"batch{i}", omega=0.5, Kn=Kn,
                            n_cells=int(rng.integers(50, 1001)),
                            ppc=int(rng.integers(50, 401)),
                            body_force=float(rng.uniform(0.5, 2.0) * f0_force(1.0)),
                            steps=2000, sample_start=1001,
                            seeds=(int(rng.integers(0, 2 ** 63 - 1)),)))
    return out


def serving_requests(n: int = 2000, rate: float = 50.0, target_se: float = 0.01,
                     max_steps: int = 200_000, seed: int = 4242):
    """Micro-solve requests: Poisson arrivals at `rate` per second (exponential gaps),
    each a run drawn as in batch_instances (Kn log-uniform in [0.05, 10], 50-1000
    cells, 50-400 particles per cell, force 0.5-2 x f0_force(1), hard spheres, own
    seed), to a relative standard error `target_se` of the channel-mean velocity."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    t -= t[0]
    out = []
    for i, w in enumerate(batch_instances(n, seed=seed + 1)):
        out.append(dict(Kn=w.Kn, n_cells=w.n_cells, ppc=w.ppc, omega=w.omega,
                        body_force=w.body_force, seed=w.seeds[0], arrival=float(t[i]),
                        target_se=float(target_se), max_steps=int(max_steps)))
    return out


def synthetic_windows(n_windows: int, n_cells: int, per_cell: int, u, cxy, seed: int = 0):
    """Raw moment sums of `n_windows` windows of synthetic samples: in every window and
    cell i, `per_cell` velocity triples with vx ~ N(u[i], 1/2), vy ~ N(0, 1/2) with
    covariance cxy[i] with vx, vz ~ N(0, 1/2), summed into the 13 raw moments
    [count, vx, vy, vz, vx^2, vy^2, vz^2, vx vy, vx vz, vy vz, vx v^2, vy v^2, vz v^2].
    Returns an array [n_windows, n_cells, 13] (binary64)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    u = np.asarray(u, np.float64)
    rho = np.asarray(cxy, np.float64) / 0.5
    s = math.sqrt(0.5)
    out = np.empty((n_windows, n_cells, 13))
    for w in range(n_windows):
        z = rng.standard_normal((3, n_cells, per_cell))
        vx = u[:, None] + s * z[0]
        vy = s * (rho[:, None] * z[0] + np.sqrt(1.0 - rho[:, None] ** 2) * z[1])
        vz = s * z[2]
        v2 = vx * vx + vy * vy + vz * vz
        cols = [np.ones_like(vx), vx, vy, vz, vx * vx, vy * vy, vz * vz, vx * vy, vx * vz,
                vy * vz, vx * v2, vy * v2, vz * v2]
        for k, c in enumerate(cols):
            out[w, :, k] = c.sum(axis=1)
    return out


def latin_hypercube(n: int, dims: int = 2, seed: int = 0):
    """n points of a Latin hypercube in [0, 1]^dims: each axis cut into n equal strata,
    one point per stratum, uniform within it, strata paired by independent
    permutations."""
    import numpy as np
    rng = np.random.default_rng(seed)
    u = np.empty((n, dims))
    for d in range(dims):
        u[:, d] = (rng.permutation(n) + rng.uniform(size=n)) / n
    return u


# Range of the Gaussian-process variant's design (the variant is not the paper's
# method): Kn log-uniform over the paper's verification range 0.1-5 (Sec. 3.1) and a
# force factor in [0.5, 2] times F_ma(Kn), the force whose slip-Stokes channel-mean
# speed is 0.02 v0 (Ma ~ 0.02).
GP_KN = (0.1, 5.0)
GP_FORCE = (0.5, 2.0)


def gp_force(Kn: float, factor: float) -> float:
    return factor * 0.02 / (math.sqrt(math.pi) / (12.0 * Kn) + 1.0)


def gp_design(n: int = 64, seed: int = 3):
    """The design points (Kn, F) of the GP variant and their unit-square coordinates."""
    import numpy as np
    u = latin_hypercube(n, 2, seed)
    Kn = np.exp(np.log(GP_KN[0]) + u[:, 0] * (np.log(GP_KN[1]) - np.log(GP_KN[0])))
    f = GP_FORCE[0] + u[:, 1] * (GP_FORCE[1] - GP_FORCE[0])
    F = np.array([gp_force(k, x) for k, x in zip(Kn, f)])
    return Kn, F, u
