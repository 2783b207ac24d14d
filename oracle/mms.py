"""Oracle of the MMS hybrid (Sec. 2, Sec. 3.2): DSMC only in the Knudsen layer next to
a wall, open to the CFD through a Chapman-Enskog interface, its data training the
surrogates that correct the CFD, iterated.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU baseline of the
benchmark may import it; the library never does.

Readings (listed in the design notes):
* the DSMC sub-domain spans the training region, two mean free paths (Kn in channel
  units, the viscosity-based lambda of Eq. 7) rounded up to whole cells of width dy,
  plus a buffer of `buffer` cells next to the interface (Sec. 3.2: 2 lambda and 5
  cells); its own Kn and force follow from its height L_d: Kn / L_d and F L_d;
* by the symmetry of the flow (u(y) = u(1 - y), P(y) = -P(1 - y)) the layer at the
  bottom wall stands for both;
* the interface is an open Chapman-Enskog reservoir at y = L_d with the CFD's velocity
  there (the mean of the two CFD cells next to that face) and the exact stress
  P(L_d) = F (2 L_d - 1); each particle crossing it is re-emitted from the half-range
  flux-weighted Chapman-Enskog distribution, so the particle count stays fixed;
* iteration k sets the interface from the current CFD profile, runs the sub-domain
  `steps` steps (after `warmup` unsampled steps in the first iteration), adds one
  training sample per `window` sampled steps (samples accumulate over iterations),
  retrains all models and solves the CFD with the selected ones; the first CFD profile
  is the no-slip Navier-Stokes one.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import surrogate as S


def layer_geometry(Kn: float, dy: float, buffer: int):
    """(cells in the training region, cells of the sub-domain, its height L_d)."""
    n_train = int(math.ceil(2.0 * Kn / dy - 1e-9))
    n_sub = n_train + int(buffer)
    return n_train, n_sub, n_sub * dy


def interface_velocity(u_cfd, L_d: float) -> float:
    """CFD velocity at the face y = L_d of an n-cell cell-centred profile."""
    n = len(u_cfd)
    f = int(round(L_d * n))
    return 0.5 * (u_cfd[f - 1] + u_cfd[f])


def mms_hybrid(Kn: float, F: float, *, omega: float = 0.5, dy: float = 0.005, ppc: int = 50,
               buffer: int = 5, iterations: int = 3, steps: int = 400, window: int = 20,
               warmup: int = 200, n_cfd: int = 200, seed: int = 0, G: int = 256,
               interface=None):
    """The MMS hybrid (Sec. 2, Sec. 3.2).  `interface`, if given, is a list of (u, P)
    pairs used at the DSMC's open boundary in each iteration instead of the values from
    the current CFD profile (a test drives the oracle with the library's interface
    history this way, so that both sides' DSMC layers run bit for bit alike even where
    rounding of the fitted profiles makes the binary32 interface values differ); the
    values the oracle's own profiles give are returned as "interface_own"."""
    b = S.exponents(Kn)
    n_train, n_sub, L_d = layer_geometry(Kn, dy, buffer)
    sim = oracle.OracleSim(omega=omega, Kn=Kn / L_d, F=F * L_d, n_cells=n_sub, ppc=ppc,
                           seed=seed, G=G, sample_start=0)
    u_cfd = S.cfd(Kn, F, n_cfd)  # no-slip Navier-Stokes to start
    samples, history, own, fit = [], [], [], None
    for it in range(iterations):
        u_if = interface_velocity(u_cfd, L_d)
        p_if = F * (2.0 * L_d - 1.0)
        own.append((u_if, p_if))
        if interface is not None:
            u_if, p_if = interface[it]
        sim.set_open_top(u_if, p_if)
        history.append((float(np.float32(u_if)), float(np.float32(p_if))))
        if it == 0 and warmup:
            sim.step(warmup)
        sim.reset_samples()
        for w in range(steps // window):
            sim.step(window)
            acc, n = sim.moments()
            samples.append(S.training_sample(acc, n, ppc, Kn, F, b, length=L_d, n_train=n_train))
            sim.reset_samples()
        fit = S.train(samples, Kn)
        u_cfd = S.selected_profile(fit, Kn, F, n_cfd, b)
    err = sim.error
    sim.close()
    return {"fit": fit, "profile": u_cfd, "interface": history, "interface_own": own,
            "n_train": n_train,
            "n_sub": n_sub, "L_d": L_d, "b": b, "samples": len(samples), "error": err}
