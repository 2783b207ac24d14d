"""Oracle of the Gaussian-process variant of the surrogate stage (not the paper's method,
which uses Bayesian ridge regression per flow case): a GP over the (Kn, force) design of many DSMC runs predicts the slip
coefficient and the stress correction of a new case, and the 1D CFD uses them.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU baseline of the
benchmark may import it; the library never does.

Written from the textbook GP regression (Rasmussen and Williams 2006, Ch. 2 and Sec. 5.4):
squared-exponential covariance k(x, x') = exp(-1/2 sum_d ((x_d - x'_d) / l_d)^2) on
inputs scaled to the unit square, Gaussian noise sigma_n^2; each output column is
standardised (mean, standard deviation) and shares the covariance; K = k(X, X) +
sigma_n^2 I is factored by Cholesky, alpha = K^-1 y, the predictive mean at x* is
k(x*, X) alpha (un-standardised); the log marginal likelihood of the outputs is
sum_o (-1/2 y_o^T alpha_o) - (m/2) log|K| - (n m / 2) log 2 pi, and the hyperparameters
(l_1, l_2, sigma_n^2) are the best point of a fixed grid (readings: the targets of a run
are its slip coefficient and its stress correction divided by F at the CFD faces, from
the paper's Bayesian ridge regression on its own DSMC windows; the grid below).
"""
from __future__ import annotations

import math

import numpy as np

# Hyperparameter grid (length scales on the unit square, noise variance of
# standardised outputs).
GRID = [(l1, l2, s2) for l1 in (0.05, 0.1, 0.2, 0.4, 0.8) for l2 in (0.25, 1.0, 4.0)
        for s2 in (1e-4, 1e-3, 1e-2, 3e-2, 1e-1, 3e-1)]


def kernel(A, B, l1: float, l2: float):
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    d1 = (A[:, None, 0] - B[None, :, 0]) / l1
    d2 = (A[:, None, 1] - B[None, :, 1]) / l2
    return np.exp(-0.5 * (d1 * d1 + d2 * d2))


def standardise(Y):
    Y = np.asarray(Y, np.float64)
    mu = Y.mean(axis=0)
    sd = Y.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return (Y - mu) / sd, mu, sd


def log_marginal(X, Ys, l1, l2, s2):
    """Summed log marginal likelihood of the standardised outputs Ys."""
    n, m = Ys.shape
    K = kernel(X, X, l1, l2) + s2 * np.eye(n)
    L = np.linalg.cholesky(K)
    z = np.linalg.solve(L, Ys)  # L z = y
    return (-0.5 * float(np.sum(z * z)) - m * float(np.sum(np.log(np.diag(L))))
            - 0.5 * n * m * math.log(2.0 * math.pi))


def fit(X, Y, grid=GRID):
    """Best grid point by the log marginal likelihood, with alpha = K^-1 Ys there."""
    Ys, mu, sd = standardise(Y)
    lml = np.array([log_marginal(X, Ys, *g) for g in grid])
    best = int(np.argmax(lml))
    l1, l2, s2 = grid[best]
    n = len(X)
    K = kernel(X, X, l1, l2) + s2 * np.eye(n)
    L = np.linalg.cholesky(K)
    alpha = np.linalg.solve(L.T, np.linalg.solve(L, Ys))
    return {"X": np.asarray(X, np.float64), "alpha": alpha, "mu": mu, "sd": sd, "hyper": grid[best],
            "best": best, "lml": lml}


def predict(model, Xs):
    l1, l2, _ = model["hyper"]
    Ks = kernel(Xs, model["X"], l1, l2)
    return model["mu"] + model["sd"] * (Ks @ model["alpha"])


def cfd_faces(Kn: float, F: float, n: int, sigma_p, S_faces):
    """The finite-volume solve of Eq. 8 (as oracle.surrogate.cfd) with the stress
    correction given at the n + 1 faces."""
    h = 1.0 / n
    S = np.asarray(S_faces, np.float64)
    uw = 0.0 if sigma_p is None else sigma_p * F
    A = np.zeros((n, n))
    r = np.full(n, -h * math.sqrt(math.pi) * F / Kn)
    for i in range(n):
        if i < n - 1:
            A[i, i + 1] += 1.0 / h
            A[i, i] -= 1.0 / h
        else:
            A[i, i] -= 2.0 / h
            r[i] -= 2.0 * uw / h
        r[i] += S[i + 1]
        if i > 0:
            A[i, i] -= 1.0 / h
            A[i, i - 1] += 1.0 / h
        else:
            A[i, i] -= 2.0 / h
            r[i] -= 2.0 * uw / h
        r[i] -= S[i]
    return np.linalg.solve(A, r)
