"""Physics pins of the whole oracle DSMC step (CPU only).

The paper (arXiv 2311.14140) fixes the problem and its exact relations, not the DSMC
code; these tests check the oracle against what kinetic theory and the paper fix:

* equilibrium: with no force, the state stays a Maxwellian at the wall temperature
  with uniform density (diffuse isothermal walls, Sec. 2.1);
* collision rate: at equilibrium, accepted NTC collisions per cell and step equal
  N(N-1) sigma_ref <g> dt / (2 V) with <g> = 2 sqrt(2/pi) (also for VHS, whose
  <sigma g> equals sigma_ref <g> at the reference temperature);
* free-molecular transient: without collisions, u(y, t) = F E[min(t, tau(y, vy))] over
  vy ~ N(0, 1/2), tau the time since the particle left a wall (1D quadrature);
* momentum balance: the steady shear stress obeys dP_xy/dy = 2F at every Kn (Eq. 1 in
  the units of Eq. 6, rho / P0 = 2 / v0^2);
* near-continuum limit: at Kn = 0.05 the interior velocity is the parabola of Eq. 8
  with S = 0, curvature -sqrt(pi) F / Kn, up to the exact hard-sphere viscosity being
  1.016 times the first Chapman-Enskog value the Kn definition (Eq. 7) uses; the wall
  intercept (the slip, Eq. 10) lies in a band (the paper prints no sigma_P).

Standard errors of time averages are batch means over independent blocks of steps.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest
from scipy import integrate, stats

import oracle

GBAR = 2.0 * math.sqrt(2.0 / math.pi)


@pytest.mark.parametrize("omega,Kn", [(0.5, 1.0), (0.81, 0.5)])
def test_equilibrium_is_preserved(omega, Kn):
    nc, ppc = 100, 200
    s = oracle.OracleSim(omega=omega, Kn=Kn, F=0.0, n_cells=nc, ppc=ppc, seed=21,
                         sample_start=1001)
    assert s.step(2000) == 0
    y, vx, vy, vz = [a.astype(np.float64) for a in s.state()]
    n = y.size
    cdf = lambda a: stats.norm.cdf(np.asarray(a) / math.sqrt(0.5))
    for v in (vx, vy, vz):
        assert abs(v.mean()) < 4 * math.sqrt(0.5 / n)
        assert abs(v.var() - 0.5) < 4 * 0.5 * math.sqrt(2.0 / n)
        assert abs(stats.kurtosis(v, fisher=False) - 3.0) < 4 * math.sqrt(24.0 / n)
        assert stats.kstest(v, cdf).pvalue > 1e-3
    counts = np.bincount(np.minimum((y * nc).astype(int), nc - 1), minlength=nc)
    assert stats.chisquare(counts).pvalue > 1e-3
    acc, ns = s.moments()
    f = oracle.fields(acc, ns, ppc)
    assert ns == 1000
    assert abs(np.average(f["T"], weights=acc[:, 0]) - 1.0) < 0.01
    assert abs(f["n"].mean() - 1.0) < 1e-12


@pytest.mark.parametrize("omega,Kn", [(0.5, 1.0), (0.81, 1.0)])
def test_collision_rate_at_equilibrium(omega, Kn):
    nc, ppc = 100, 200
    s = oracle.OracleSim(omega=omega, Kn=Kn, F=0.0, n_cells=nc, ppc=ppc, seed=4)
    s.step(50)
    p = s.params()
    rate = p["nsig"] * GBAR * p["dt_d"] / (2.0 * ppc)
    s.reset_samples()
    expected = 0.0
    for _ in range(400):
        off = s.cells()[0]
        N = np.diff(off).astype(np.float64)
        expected += (N * (N - 1)).sum() * rate
        s.step(1)
    observed = float(s.cells()[3].sum())
    assert abs(observed - expected) < 4 * math.sqrt(expected)


def _u_free_molecular(y, t, F):
    """F E[min(t, tau)], vy ~ N(0, 1/2): tau = y/vy from the bottom wall for vy > 0 and
    (1-y)/|vy| from the top wall for vy < 0."""
    f = lambda v: math.exp(-v * v) / math.sqrt(math.pi)
    tot = 0.0
    for d in (y, 1.0 - y):
        k = d / t
        tot += t * integrate.quad(f, 0.0, k)[0]
        if d > 0:
            tot += integrate.quad(lambda v: f(v) * d / v, k, np.inf, limit=400)[0]
    return F * tot


@pytest.mark.parametrize("t", [0.5, 2.0, 8.0])
def test_free_molecular_transient(t):
    """Collisionless gas from rest, time step 0.25 (a particle may bounce several times
    in one step): cell-averaged u_x against the closed form, per cell and overall."""
    F, dt, nc, ppc = 1.0, 0.25, 20, 5000
    m = int(round(t / dt))
    zs = []
    for seed in (1, 2):
        s = oracle.OracleSim(Kn=math.inf, F=F, n_cells=nc, ppc=ppc, seed=seed, dt=dt,
                             sample_start=m + 1)
        assert s.step(m + 1) == 0  # the sample of step m+1 is taken at time m dt
        acc, ns = s.moments()
        N = acc[:, 0]
        u = acc[:, 1] / N
        var = acc[:, 4] / N - u ** 2
        ue = np.array([integrate.quad(lambda y: _u_free_molecular(y, t, F), i / nc,
                                      (i + 1) / nc)[0] * nc for i in range(nc)])
        z = (u - ue) / np.sqrt(var / N)
        assert np.abs(z).max() < 4.0
        zs.append(((u - ue) * N).sum() / math.sqrt((var * N).sum()))
    assert abs(np.mean(zs)) * math.sqrt(len(zs)) < 3.5


def _batched_fields(s, n_batches, steps, ppc):
    out = []
    for _ in range(n_batches):
        s.reset_samples()
        s.step(steps)
        acc, ns = s.moments()
        out.append(oracle.fields(acc, ns, ppc))
    return out


def test_momentum_balance():
    """Steady P_xy(y) = F (2y - 1): per cell within 4 standard errors, and the fitted
    slope equals 2F within 3 standard errors (Eq. 1)."""
    Kn, F, nc, ppc = 1.0, 0.05, 50, 200
    s = oracle.OracleSim(Kn=Kn, F=F, n_cells=nc, ppc=ppc, seed=3, dt_factor=0.1)
    s.step(1000)
    fb = _batched_fields(s, 12, 400, ppc)
    P = np.array([f["Pxy"] for f in fb])
    yc = (np.arange(nc) + 0.5) / nc
    pm, pse = P.mean(0), P.std(0, ddof=1) / math.sqrt(len(P))
    assert np.abs((pm - F * (2 * yc - 1)) / pse).max() < 4.0
    A = np.vstack([yc, np.ones(nc)]).T
    slopes = np.array([np.linalg.lstsq(A, p, rcond=None)[0][0] for p in P])
    se = slopes.std(ddof=1) / math.sqrt(len(slopes))
    assert abs(slopes.mean() - 2 * F) < 3 * se + 0.005 * 2 * F


def _near_continuum_run(seed):
    import oracle as o
    Kn, F, nc, ppc = 0.05, 0.04, 100, 200
    s = o.OracleSim(Kn=Kn, F=F, n_cells=nc, ppc=ppc, seed=seed)
    s.step(2500)
    us = []
    for _ in range(5):
        s.reset_samples()
        s.step(1500)
        acc, ns = s.moments()
        us.append(acc[:, 1] / acc[:, 0])
    return np.array(us)


@pytest.mark.slow
def test_near_continuum_parabola_and_slip():
    Kn, F, nc = 0.05, 0.04, 100
    with mp.get_context("spawn").Pool(8) as pool:
        U = np.concatenate(pool.map(_near_continuum_run, list(range(11, 19))))
    yc = (np.arange(nc) + 0.5) / nc
    inner = (yc > 0.1) & (yc < 0.9)  # two mean free paths from each wall
    A = np.vstack([np.ones(inner.sum()), yc[inner] * (1 - yc[inner])]).T
    c = np.array([np.linalg.lstsq(A, u[inner], rcond=None)[0] for u in U])
    curv = 2 * c[:, 1] / (math.sqrt(math.pi) * F / Kn)  # -u'' in units of sqrt(pi)F/Kn
    se = curv.std(ddof=1) / math.sqrt(len(curv))
    assert se < 0.02
    assert abs(curv.mean() - 1 / 1.016) < 0.03
    slip = c[:, 0].mean() / F  # sigma_P of Eq. 10: u(wall) = sigma_P |P_xy(wall)|
    assert 0.8 < slip < 1.3
