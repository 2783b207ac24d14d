"""The surrogate stage on the GPU (dsmc_surrogate_*) against the oracle
(oracle/surrogate.py) on the same seeded synthetic windows: training statistics,
evidence maximisation, model probabilities and selection, posteriors, and the Monte Carlo
bands of the corrected profile with the same standard normals.  Tolerances: both sides
work in binary64; the library accumulates the sufficient statistics in another order
and forms residuals from them (|t - Phi m|^2 = t^T t - 2 m^T Phi^T t + m^T G m), so
agreement is to a few parts in 1e9 of the quantities' scales, not bit for bit."""
import math

import numpy as np
import pytest

from oracle import surrogate as S
from paper_2311_14140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import _build
    _build.build()


def flow(Kn, F, n, sp, a, b):
    """A slip flow with a Knudsen-layer correction: mean vx and the vx-vy covariance
    P / 2 of a sample at the initial density (P = F (2y - 1))."""
    y = (np.arange(n) + 0.5) / n
    return S.exact_profile(Kn, F, y, sp, a, b[:len(a)]), 0.5 * F * (2 * y - 1)


CASES = [
    dict(Kn=0.1, F=2e-3, n=100, sp=1.1, a=(0.3,), windows=60, per_cell=400),
    dict(Kn=1.0, F=5e-3, n=64, sp=1.3, a=(0.2, -0.1), windows=40, per_cell=300),
    dict(Kn=0.5, F=1e-2, n=3, sp=0.9, a=(), windows=30, per_cell=200),   # one interior cell
    dict(Kn=5.0, F=1e-3, n=200, sp=None, a=(), windows=20, per_cell=100),  # no signal
]


def both(case, seed):
    b = S.exponents(case["Kn"])
    u, cxy = flow(case["Kn"], case["F"], case["n"], case["sp"], case["a"], b)
    wins = W.synthetic_windows(case["windows"], case["n"], case["per_cell"], u, cxy, seed=seed)
    from paper_2311_14140_gb300 import Surrogate
    g = Surrogate(case["Kn"], case["F"], case["n"], case["per_cell"])
    samples = []
    for w in wins:
        g.add_window(w, 1)  # per_cell samples = 1 step x per_cell "particles per cell"
        samples.append(S.training_sample(w, 1, case["per_cell"], case["Kn"], case["F"], b))
    return g, g.train(), S.train(samples, case["Kn"]), b


def close(x, y, scale, tol=1e-8):
    assert abs(x - y) <= tol * max(abs(scale), 1e-300), (x, y)


@pytest.mark.parametrize("k", range(len(CASES)))
def test_training_matches_oracle(k):
    g, fg, fo, b = both(CASES[k], seed=100 + k)
    assert fg["n_samples"] == CASES[k]["windows"]
    assert fg["sel_v"] == fo["sel_v"] and fg["sel_c"] == fo["sel_c"]
    for i in range(2):
        close(fg["log_evidence_v"][i], fo["v"][i]["log_evidence"], fo["v"][i]["log_evidence"])
    for i in range(4):
        close(fg["log_evidence_c"][i], fo["c"][i]["log_evidence"], fo["c"][i]["log_evidence"])
    np.testing.assert_allclose(fg["prob_v"], fo["p_v"], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(fg["prob_c"], fo["p_c"], rtol=1e-6, atol=1e-12)
    fv = fo["v"][1]
    close(fg["sigma_p"], fv["m"][0], math.sqrt(fv["S"][0, 0]), 1e-6)
    close(fg["sigma_p_var"], fv["S"][0, 0], fv["S"][0, 0], 1e-6)
    for kk in (1, 2, 3):
        fc = fo["c"][kk]
        sd = np.sqrt(np.diag(fc["S"]))
        for i in range(kk):
            close(fg["m_c"][kk][i], fc["m"][i], sd[i], 1e-6)
            for j in range(kk):
                close(fg["S_c"][kk][3 * i + j], fc["S"][i, j], sd[i] * sd[j], 1e-6)
        close(fg["beta_c"][kk], fc["beta"], fc["beta"], 1e-8)


@pytest.mark.parametrize("k", [0, 1])
def test_bands_match_oracle(k):
    g, fg, fo, b = both(CASES[k], seed=200 + k)
    rng = np.random.default_rng(300 + k)
    z = rng.standard_normal((257, 4))
    mean, sd = g.profile(200, z)
    mo, so, _ = S.mc_profiles(fo, CASES[k]["Kn"], CASES[k]["F"], 200, b, z)
    scale = np.abs(mo).max()
    np.testing.assert_allclose(mean, mo, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(sd, so, rtol=1e-5, atol=1e-9 * scale)
    # a single z = 0 trial is the profile at the posterior means
    m0, s0 = g.profile(200, np.zeros((1, 4)))
    np.testing.assert_allclose(m0, S.selected_profile(fo, CASES[k]["Kn"], CASES[k]["F"], 200, b),
                               rtol=0, atol=1e-10 * scale)
    assert np.all(s0 == 0)


def test_run_windows_are_read_in_place():
    """add_run on a DSMC run equals add_window of the same sums copied to the host, and
    resets the run's sums so that the next call sees the next window."""
    from paper_2311_14140_gb300 import Dsmc, Surrogate
    Kn, F = 1.0, W.f0_force(1.0) * 5
    g = Dsmc(Kn, 100, 50, body_force=F, seed=4, sample_start=1)
    s1 = Surrogate(Kn, F, 100, 50)
    s2 = Surrogate(Kn, F, 100, 50)
    for w in range(5):
        g.step(20)
        m, n = g.moments()
        assert n == 20
        s2.add_window(m, n)
        s1.add_run(g)
        assert g.moments()[1] == 0
    f1, f2 = s1.train(), s2.train()
    for key in ("log_evidence_v", "log_evidence_c", "m_c", "S_c"):
        np.testing.assert_array_equal(f1[key], f2[key])


def test_dsmc_trained_surrogate_selects_slip_at_kn1():
    """A short DSMC training run at Kn = 1 (the paper selects the slip model from the
    first training steps there): 40 windows of 50 steps after a 400-step transient."""
    from paper_2311_14140_gb300 import Dsmc, Surrogate
    Kn, F = 1.0, 20 * W.f0_force(1.0)
    g = Dsmc(Kn, 100, 200, body_force=F, seed=7, sample_start=401)
    g.step(400)
    s = Surrogate(Kn, F, 100, 200)
    for w in range(40):
        g.step(50)
        s.add_run(g)
    f = s.train()
    assert f["sel_v"] == 1 and f["prob_v"][1] > 0.99
    assert 0.5 < f["sigma_p"] < 2.5
    z = np.random.default_rng(1).standard_normal((1000, 4))
    mean, sd = s.profile(200, z)
    assert np.all(sd > 0) and mean[100] > mean[0] > 0
