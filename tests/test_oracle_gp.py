"""Pins of the GP-variant oracle (oracle/gp.py): the Latin hypercube's strata, the
marginal likelihood against scipy's multivariate normal, the predictive mean against a
direct solve of the full covariance (no Cholesky), interpolation of noise-free data, the
grid choosing the generating length scale, and the face-given CFD against the
basis-given one."""
import numpy as np
import pytest
from scipy import stats

from oracle import gp as GP
from oracle import surrogate as S
from paper_2311_14140_gb300 import workloads as W


def test_latin_hypercube_strata():
    u = W.latin_hypercube(64, 2, seed=1)
    for d in range(2):
        assert sorted(np.floor(u[:, d] * 64).astype(int).tolist()) == list(range(64))
    Kn, F, uu = W.gp_design(64, seed=3)
    assert np.all((Kn >= 0.1) & (Kn <= 5.0)) and np.all(F > 0)


def _data(seed, n=30, m=3, l=(0.3, 1.0)):
    rng = np.random.default_rng(seed)
    X = rng.uniform(size=(n, 2))
    K = GP.kernel(X, X, *l) + 1e-8 * np.eye(n)
    scale = np.linspace(0.2, 3.0, m)
    shift = np.linspace(-1.0, 5.0, m)
    Y = np.linalg.cholesky(K) @ rng.normal(size=(n, m)) * scale + shift
    return X, Y


def test_marginal_likelihood_against_scipy():
    X, Y = _data(2)
    Ys, mu, sd = GP.standardise(Y)
    for l1, l2, s2 in ((0.3, 1.0, 1e-3), (0.1, 4.0, 1e-2)):
        K = GP.kernel(X, X, l1, l2) + s2 * np.eye(len(X))
        ref = sum(stats.multivariate_normal(mean=np.zeros(len(X)), cov=K).logpdf(Ys[:, o])
                  for o in range(Ys.shape[1]))
        assert GP.log_marginal(X, Ys, l1, l2, s2) == pytest.approx(ref, rel=1e-10)


def test_prediction_against_direct_solve_and_interpolation():
    X, Y = _data(4)
    model = GP.fit(X, Y)
    l1, l2, s2 = model["hyper"]
    Xs = np.random.default_rng(9).uniform(size=(7, 2))
    K = GP.kernel(X, X, l1, l2) + s2 * np.eye(len(X))
    Ys, mu, sd = GP.standardise(Y)
    ref = mu + sd * (GP.kernel(Xs, X, l1, l2) @ np.linalg.solve(K, Ys))
    np.testing.assert_allclose(GP.predict(model, Xs), ref, rtol=1e-9, atol=1e-12)
    # with the smallest noise on the grid, training points are reproduced closely
    m2 = GP.fit(X, Y, grid=[(l1, l2, 1e-8)])
    np.testing.assert_allclose(GP.predict(m2, X), Y, rtol=1e-4, atol=1e-4 * np.abs(Y).max())


def test_grid_finds_the_generating_length_scale():
    X, Y = _data(6, n=60, m=20, l=(0.2, 4.0))
    model = GP.fit(X, Y)
    assert model["hyper"][0] == 0.2 and model["hyper"][1] == 4.0


def test_face_cfd_equals_basis_cfd():
    Kn, F, n = 0.3, 2e-3, 200
    b = S.exponents(Kn)
    a = (0.2, -0.1, 0.03)
    yf = np.arange(n + 1) / n
    u1 = GP.cfd_faces(Kn, F, n, 1.1, S.stress_correction(yf, a, b))
    u2 = S.cfd(Kn, F, n, 1.1, a, b)
    np.testing.assert_allclose(u1, u2, rtol=1e-12, atol=1e-15)
