"""A Gaussian-process variant of the surrogate stage (not the paper's method, which
trains Bayesian ridge regressions per flow case): DSMC runs at Latin-hypercube
(Kn, force) points, all advanced in one batch; each run's windows train the paper's
Bayesian ridge regression surrogates
(``Surrogate``); a GP over the design (``GaussianProcess``) learns each run's slip
coefficient and its stress correction divided by F at the CFD faces; for a new (Kn, F)
the CFD (``cfd_faces``) uses the GP's predictions.  Orchestration only: the DSMC, the
training windows, the evidence maximisation's device part, the GP and the CFD run in
the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W
from .dsmc import DsmcBatch, GaussianProcess, Surrogate, cfd_faces, surrogate_correction

# Hyperparameter grid of the GP (length scales on the unit square, noise variance of the
# standardised outputs); the same grid as the oracle's.
GRID = [(l1, l2, s2) for l1 in (0.05, 0.1, 0.2, 0.4, 0.8) for l2 in (0.25, 1.0, 4.0)
        for s2 in (1e-4, 1e-3, 1e-2, 3e-2, 1e-1, 3e-1)]


def unit_inputs(Kn, F):
    """(Kn, F) -> unit-square inputs of the GP: log Kn over GP_KN, force factor over
    GP_FORCE."""
    Kn = np.asarray(Kn, np.float64)
    u1 = (np.log(Kn) - math.log(W.GP_KN[0])) / (math.log(W.GP_KN[1]) - math.log(W.GP_KN[0]))
    fac = np.asarray(F, np.float64) / np.array([W.gp_force(k, 1.0) for k in Kn])
    u2 = (fac - W.GP_FORCE[0]) / (W.GP_FORCE[1] - W.GP_FORCE[0])
    return np.stack([u1, u2], axis=1)


def run_cases(Kn, F, *, n_cells=100, ppc=100, warmup=2000, windows=40, window=100, seed=0,
              stream=None):
    """DSMC runs of the channel at (Kn_i, F_i) in one batch; returns the fits of their
    surrogates and their time-averaged velocity profiles."""
    defs = [dict(Kn=float(k), n_cells=n_cells, ppc=ppc, omega=0.5, body_force=float(f),
                 seed=seed + 7919 * i) for i, (k, f) in enumerate(zip(Kn, F))]
    b = DsmcBatch(defs, sample_start=0, graph=stream is not None, stream=stream)
    b.step(warmup)
    b.reset_samples()
    sur = [Surrogate(d["Kn"], d["body_force"], n_cells, ppc, stream=stream) for d in defs]
    sums = np.zeros((len(defs), n_cells, 13))
    for w in range(windows):
        b.step(window)
        for i in range(len(defs)):
            m, n = b.moments(i)
            sums[i] += m
            sur[i].add_run(b, i)
    fits = [s.train() for s in sur]
    prof = np.array([sums[i][:, 1] / sums[i][:, 0] for i in range(len(defs))])
    for s in sur:
        s.close()
    b.close()
    return fits, prof


def targets(fits, F, n_cfd=200):
    """Per run: [sigma_P (slip posterior mean), S(y_f) / F at the n_cfd + 1 faces]."""
    rows = []
    for f, Fi in zip(fits, F):
        S = surrogate_correction(f, n_cfd)
        rows.append(np.concatenate([[f["sigma_p"]], S / Fi]))
    return np.array(rows)


def predict_profiles(gp, Kn, F, n_cfd=200):
    out = gp.predict(unit_inputs(Kn, F))
    return np.array([cfd_faces(k, f, n_cfd, o[0], f * o[1:]) for k, f, o in zip(Kn, F, out)])


def run(n_design=64, n_test=8, *, n_cells=100, ppc=200, warmup=2000, windows=160, window=100,
        test_ppc=200, test_windows=160, n_cfd=200, seed=0, stream=None):
    """The whole variant: returns the GP's hyperparameters and, for the held-out cases, the
    CFD and DSMC profiles (10 bins each) and the largest bin difference relative to the
    DSMC's peak velocity."""
    Kn, F, _ = W.gp_design(n_design, seed=3 + seed)
    fits, _ = run_cases(Kn, F, n_cells=n_cells, ppc=ppc, warmup=warmup, windows=windows,
                        window=window, seed=1000 * seed, stream=stream)
    Y = targets(fits, F, n_cfd)
    gp = GaussianProcess(unit_inputs(Kn, F), Y, GRID, stream=stream)
    Kt, Ft, _ = W.gp_design(n_test, seed=101 + seed)
    _, prof_t = run_cases(Kt, Ft, n_cells=n_cells, ppc=test_ppc, warmup=warmup,
                          windows=test_windows, window=window, seed=1000 * seed + 500,
                          stream=stream)
    pred = predict_profiles(gp, Kt, Ft, n_cfd)
    bins = lambda x, k: x.reshape(10, k).mean(axis=1)
    errs = [float(np.abs(bins(p, n_cfd // 10) - bins(d, n_cells // 10)).max() / np.abs(d).max())
            for p, d in zip(pred, prof_t)]
    sel = [(f["sel_v"], f["sel_c"]) for f in fits]
    out = {"hyper": gp.hyper, "errors": errs, "Kn_test": Kt.tolist(), "F_test": Ft.tolist(),
           "selections": sel, "pred": pred, "dsmc": prof_t}
    gp.close()
    return out
