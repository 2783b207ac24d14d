"""Pins of the MMS-hybrid oracle pieces (oracle/mms.py and the sub-domain form of
oracle/surrogate.training_sample): the sub-domain geometry of Sec. 3.2 (two mean free
paths plus a 5-cell buffer), exact training samples of a Navier-Stokes slip flow seen
through the sub-domain, the interface value of a cell-centred profile, and a short
hybrid run whose bookkeeping (interface history, samples, final profile) follows its
definition."""
import math

import numpy as np
import pytest

from oracle import mms as M
from oracle import surrogate as S


def test_layer_geometry():
    assert M.layer_geometry(0.1, 0.005, 5) == (40, 45, pytest.approx(0.225))
    assert M.layer_geometry(0.01, 0.005, 5) == (4, 9, pytest.approx(0.045))
    assert M.layer_geometry(0.05, 0.005, 5) == (20, 25, pytest.approx(0.125))


def _window(u, P, N, steps, ppc):
    n = N / (steps * ppc)
    acc = np.zeros((u.size, 13))
    acc[:, 0] = N
    acc[:, 1] = N * u
    acc[:, 7] = N * P / (2 * n)
    acc[:, 4] = N * (0.5 + u ** 2)
    acc[:, 5] = acc[:, 6] = N * 0.5
    return acc


def test_subdomain_sample_of_a_slip_flow():
    Kn, F, sp, dy, steps, ppc = 0.1, 2e-3, 1.2, 0.005, 50, 50
    n_train, n_sub, L_d = M.layer_geometry(Kn, dy, 5)
    y = (np.arange(n_sub) + 0.5) * dy
    c = math.sqrt(math.pi) * F / (2 * Kn)
    u = sp * F + c * y * (1 - y)
    P = F * (2 * y - 1)
    s = S.training_sample(_window(u, P, steps * ppc, steps, ppc), steps, ppc, Kn, F,
                          S.exponents(Kn), length=L_d, n_train=n_train)
    np.testing.assert_allclose(s["x_v"], [F])
    np.testing.assert_allclose(s["t_v"], [sp * F + 0.75 * c * dy * dy], rtol=1e-12)
    assert s["t_c"].size == n_train - 1 and np.abs(s["t_c"]).max() < 1e-12
    np.testing.assert_allclose(s["phi_c"], S.basis(y[1:n_train], Kn, S.exponents(Kn)))


def test_interface_velocity_of_a_parabola():
    n, c = 200, 0.3
    y = (np.arange(n) + 0.5) / n
    u = c * y * (1 - y)
    L = 45 / n
    assert M.interface_velocity(u, L) == pytest.approx(c * L * (1 - L) - c / (4 * n * n), rel=1e-12)


def test_short_hybrid_follows_its_definition():
    Kn, F = 0.1, 0.02
    r = M.mms_hybrid(Kn, F, ppc=40, iterations=3, steps=200, window=20, warmup=100, seed=4)
    assert r["error"] == 0 and r["samples"] == 30
    n_train, n_sub, L_d = M.layer_geometry(Kn, 0.005, 5)
    # iteration 0 starts from the no-slip Navier-Stokes profile
    u0 = S.cfd(Kn, F, 200)
    assert r["interface"][0][0] == pytest.approx(M.interface_velocity(u0, L_d), rel=1e-6)
    assert r["interface"][0][1] == pytest.approx(F * (2 * L_d - 1), rel=1e-6)
    # the final profile is the CFD solve with the final fit's selected models
    np.testing.assert_allclose(r["profile"], S.selected_profile(r["fit"], Kn, F, 200, r["b"]))
    assert len(r["interface"]) == 3
