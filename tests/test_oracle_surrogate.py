"""Pins of the surrogate oracle (oracle/surrogate.py) to things other than itself:
the printed Table 1, the Gaussian marginal likelihood and posterior written through the
joint Gaussian of (w, t) (scipy's multivariate normal and the Woodbury form, not the
oracle's route), the closed-form solution of Eq. 8 with Eqs. 9-10 and the second-order
convergence of the finite-volume solve, the exact shear stress P = F (2y - 1) the paper
states the macroscopic model returns, exact training samples of a known flow, and the
Occam behaviour of the evidence."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import surrogate as S

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table1_as_printed():
    rows = np.loadtxt(os.path.join(HERE, "golden", "table1_exponents.txt"))
    for kn, b1, b2, b3 in rows:
        assert S.exponents(kn) == (b1, b2, b3)
    # between tabulated values: the nearest in log Kn
    assert S.exponents(0.3) == S.exponents(0.2)
    assert S.exponents(0.35) == S.exponents(0.5)
    assert S.exponents(10.0) == S.exponents(5.0)
    assert S.exponents(0.001) == S.exponents(0.01)


def _data(seed, N=40, M=2, noise=0.3):
    rng = np.random.default_rng(seed)
    Phi = rng.normal(size=(N, M))
    w = rng.normal(size=M)
    return Phi, Phi @ w + noise * rng.normal(size=N), w


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_evidence_is_the_gaussian_marginal_likelihood_at_its_maximum(seed):
    Phi, t, _ = _data(seed)
    r = S.brr(Phi, t)
    a, b = r["alpha"], r["beta"]

    def logml(alpha, beta):
        C = np.eye(len(t)) / beta + Phi @ Phi.T / alpha
        return stats.multivariate_normal(mean=np.zeros(len(t)), cov=C).logpdf(t)

    assert r["log_evidence"] == pytest.approx(logml(a, b), abs=1e-8)
    for fa, fb in ((1.02, 1), (0.98, 1), (1, 1.02), (1, 0.98)):
        assert logml(a * fa, b * fb) < logml(a, b)
    # posterior by conditioning the joint Gaussian of (w, t)
    C = np.eye(len(t)) / b + Phi @ Phi.T / a
    Ci = np.linalg.inv(C)
    m = Phi.T @ Ci @ t / a
    Sg = np.eye(Phi.shape[1]) / a - Phi.T @ Ci @ Phi / a ** 2
    np.testing.assert_allclose(r["m"], m, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r["S"], Sg, rtol=1e-8, atol=1e-12)


def test_zero_order_evidence():
    rng = np.random.default_rng(5)
    t = 0.7 * rng.normal(size=30)
    le, beta = S.log_evidence_zero(t)
    assert beta == pytest.approx(30 / float(t @ t))
    ref = stats.multivariate_normal(mean=np.zeros(30), cov=np.eye(30) / beta).logpdf(t)
    assert le == pytest.approx(ref, abs=1e-9)
    for f in (0.97, 1.03):
        assert stats.multivariate_normal(mean=np.zeros(30),
                                         cov=np.eye(30) / (beta * f)).logpdf(t) < ref


def test_recovers_weights_and_noise():
    rng = np.random.default_rng(11)
    Phi = rng.normal(size=(20000, 3))
    w = np.array([0.5, -1.25, 2.0])
    t = Phi @ w + 0.2 * rng.normal(size=20000)
    r = S.brr(Phi, t)
    sd = np.sqrt(np.diag(r["S"]))
    assert np.all(np.abs(r["m"] - w) < 5 * sd)
    assert r["beta"] == pytest.approx(1 / 0.04, rel=0.03)


def test_model_selection_prefers_the_simplest_model_the_data_support():
    """Pure noise: no corrected model beats Newton's law (C0) by more than a few nats,
    and none falls below it (each contains C0 as its alpha -> infinity limit, which the
    evidence maximisation can always reach).  A real C1 signal: C0 is ruled out."""
    y = (np.arange(1, 99) + 0.5) / 100
    b = S.exponents(0.1)
    phi = S.basis(y, 0.1, b)
    ph = np.tile(phi, (50, 1))
    rng = np.random.default_rng(3)
    for s in range(10):
        t = 0.05 * rng.normal(size=50 * y.size)
        le0 = S.log_evidence_zero(t)[0]
        lek = [S.brr(ph[:, :k], t)["log_evidence"] for k in (1, 2, 3)]
        assert max(lek) - le0 < 3.0
        assert min(lek) - le0 > -1e-6
    a1 = 20 * 0.05 / math.sqrt(float(ph[:, 0] @ ph[:, 0]))  # a 20-sigma weight
    t = ph[:, 0] * a1 + 0.05 * rng.normal(size=50 * y.size)
    le = [S.log_evidence_zero(t)[0]] + [S.brr(ph[:, :k], t)["log_evidence"] for k in (1, 2, 3)]
    p = S.probabilities(le)
    assert p[0] < 1e-6 and np.argmax(p) >= 1


@pytest.mark.parametrize("sp,a", [(None, ()), (1.1, ()), (0.9, (0.3, -0.2)), (1.3, (0.1, 0.05, -0.02))])
def test_cfd_converges_to_the_closed_form_at_second_order(sp, a):
    Kn, F = 0.5, 1e-3
    b = S.exponents(Kn)[:len(a)]
    errs = []
    for n in (100, 200, 400):
        y = (np.arange(n) + 0.5) / n
        u = S.cfd(Kn, F, n, sp, a, b)
        errs.append(np.abs(u - S.exact_profile(Kn, F, y, sp, a, b)).max())
    scale = np.abs(S.exact_profile(Kn, F, np.linspace(0, 1, 11), sp, a, b)).max()
    assert errs[1] < 1e-3 * scale
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_cfd_returns_the_exact_shear_stress_whatever_the_models():
    Kn, F, n = 0.2, 2e-3, 200
    b = S.exponents(Kn)
    for sp, a in ((None, ()), (1.2, (0.4, -0.3, 0.05))):
        u = S.cfd(Kn, F, n, sp, a, b[:len(a)])
        yf = np.arange(1, n) / n
        dudy = (u[1:] - u[:-1]) * n
        P = -(2 * Kn / math.sqrt(math.pi)) * (dudy - S.stress_correction(yf, a, b[:len(a)]))
        np.testing.assert_allclose(P, F * (2 * yf - 1), rtol=0, atol=1e-13)


def _window(u, P, N, steps, ppc, rng):
    """Raw sums of a window whose cells hold exactly the mean velocities u and shear
    stresses P: N samples per cell, vy symmetric, vx vy covariance P / (2 n)."""
    n = N / (steps * ppc)
    acc = np.zeros((u.size, 13))
    acc[:, 0] = N
    acc[:, 1] = N * u
    acc[:, 2] = 0.0
    acc[:, 7] = N * P / (2 * n)
    acc[:, 4] = N * (0.5 + u ** 2)
    acc[:, 5] = acc[:, 6] = N * 0.5
    return acc


def test_training_sample_of_a_navier_stokes_slip_flow():
    Kn, F, sp, n, steps, ppc = 0.3, 1e-3, 1.1, 200, 100, 50
    y = (np.arange(n) + 0.5) / n
    c = math.sqrt(math.pi) * F / (2 * Kn)
    u = sp * F + c * y * (1 - y)
    P = F * (2 * y - 1)
    acc = _window(u, P, steps * ppc, steps, ppc, None)
    s = S.training_sample(acc, steps, ppc, Kn, F, S.exponents(Kn))
    np.testing.assert_allclose(s["x_v"], [F, F])
    h = 1.0 / n
    np.testing.assert_allclose(s["t_v"], sp * F + 0.75 * c * h * h, rtol=1e-12)
    assert np.abs(s["t_c"]).max() < 1e-12       # Newton's law holds exactly
    assert s["phi_c"].shape == (n - 2, 3)
    np.testing.assert_allclose(s["phi_c"], S.basis(y[1:-1], Kn, S.exponents(Kn)))


def test_training_then_bands():
    """Samples of a slip flow with a Knudsen-layer correction plus noise: the slip model
    and a corrected constitutive model are selected, the posterior mean recovers the
    slip coefficient, and Monte Carlo trials with z = 0 give the mean profile."""
    Kn, F, n, steps, ppc = 0.5, 1e-3, 100, 100, 50
    b = S.exponents(Kn)
    y = (np.arange(n) + 0.5) / n
    sp, a = 1.05, (0.2,)
    u0 = S.exact_profile(Kn, F, y, sp, a, b[:1])
    rng = np.random.default_rng(7)
    samples = []
    for j in range(200):
        u = u0 + 2e-5 * rng.normal(size=n)
        P = F * (2 * y - 1) + 2e-5 * rng.normal(size=n)
        samples.append(S.training_sample(_window(u, P, steps * ppc, steps, ppc, rng), steps, ppc,
                                         Kn, F, b))
    fit = S.train(samples, Kn)
    assert fit["sel_v"] == 1 and fit["sel_c"] >= 1
    fv = fit["v"][1]
    # the slip coefficient the wall extrapolation of the noise-free profile implies
    expect = (1.5 * u0[0] - 0.5 * u0[1]) / F
    assert abs(fv["m"][0] - expect) < 4 * math.sqrt(fv["S"][0, 0])
    assert abs(expect - sp) < 0.15 * sp
    z = np.zeros((3, 4))
    mean, sd, prof = S.mc_profiles(fit, Kn, F, 200, b, z)
    np.testing.assert_allclose(mean, S.selected_profile(fit, Kn, F, 200, b), rtol=1e-12)
    assert np.all(sd <= 1e-12 * np.abs(mean).max())
    z = np.array([[1, 0, 0, 0], [-1, 0, 0, 0]], float)
    mean, sd, prof = S.mc_profiles(fit, Kn, F, 200, b, z)
    np.testing.assert_allclose(mean, S.selected_profile(fit, Kn, F, 200, b), rtol=1e-10)
    # the wall value moves by one posterior standard deviation of sigma_P times F
    assert sd[0] == pytest.approx(math.sqrt(2) * math.sqrt(fv["S"][0, 0]) * F, rel=0.05)


def test_selection_takes_the_simplest_of_tied_models():
    """Eq. 17 picks the most probable model; models whose log evidences agree to rounding
    (1e-9 relative) are tied and the simplest (lowest index) is taken, whichever of them
    rounding made largest."""
    assert S.select([-674.977100523768, -674.977100523768, -674.9771005237678,
                     -674.977100523768]) == 0
    assert S.select([-5.0, -4.0, -4.0 + 1e-12, -7.0]) == 1
    assert S.select([-5.0, -4.0, -3.999, -7.0]) == 2
    assert S.select([10.0, 9.0]) == 0 and S.select([9.0, 10.0]) == 1
