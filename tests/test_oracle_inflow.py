"""Pins of the open Chapman-Enskog boundary of the oracle (the MMS hybrid's DSMC-CFD
interface, Sec. 2 and Sec. 3.2).  Particles re-emitted below y = 1 must follow the
flux-weighted half-range Chapman-Enskog distribution f ~ |c_y| exp(-c^2)
(1 + 2 P c_x c_y), c_y < 0, in the units of Eq. 6; its moments follow in closed form:
<c_x> = -P sqrt(pi)/2, <c_x c_y> = P, <c_x^2> = <c_z^2> = 1/2, <c_y^2> = 1, and with
P = 0 it is the diffuse wall's emission law."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def emissions(n, P, u_top=0.0, seed=3):
    """Particles just above the boundary flying up: each crosses once and is re-emitted
    with a tiny time left, so the returned velocity is the emitted one."""
    out = np.empty((n, 3))
    errs = 0
    for k in range(n):
        (y, vx, vy, vz), err = oracle.move_particle_open(0.999, 0.0, 1.0, 0.0, 0.0015, 0.0,
                                                          seed, 7, k, u_top, P)
        errs |= err
        out[k] = (vx, vy, vz)
    assert errs == 0
    return out


def test_without_shear_it_is_the_wall_emission_law():
    v = emissions(20000, 0.0)
    assert np.all(v[:, 1] < 0)
    speed = -v[:, 1]
    # P(|vy| > a) = exp(-a^2)
    assert stats.kstest(speed, lambda a: 1 - np.exp(-a * a)).pvalue > 1e-3
    for k in (0, 2):
        assert stats.kstest(v[:, k], stats.norm(scale=math.sqrt(0.5)).cdf).pvalue > 1e-3


@pytest.mark.parametrize("P", [0.05, -0.08])
def test_chapman_enskog_moments(P):
    n = 60000
    v = emissions(n, P, u_top=0.02, seed=11)
    cx = v[:, 0] - np.float32(0.02)
    cy = v[:, 1]
    se = lambda x: x.std() / math.sqrt(n)
    assert abs(cx.mean() - (-P * math.sqrt(math.pi) / 2)) < 4 * se(cx)
    assert abs((cx * cy).mean() - P) < 4 * se(cx * cy)
    assert abs((cx * cx).mean() - 0.5) < 4 * se(cx * cx)
    assert abs((cy * cy).mean() - 1.0) < 4 * se(cy * cy)
    assert abs((v[:, 2] ** 2).mean() - 0.5) < 4 * se(v[:, 2] ** 2)


def test_open_boundary_keeps_an_equilibrium_gas():
    """With u = 0, P = 0 and no force the open boundary is indistinguishable from a
    wall at rest: the gas stays Maxwellian and uniform."""
    s = oracle.OracleSim(omega=0.5, Kn=0.5, F=0.0, n_cells=20, ppc=200, seed=5)
    s.set_open_top(0.0, 0.0)
    s.step(200)
    assert s.error == 0
    y, vx, vy, vz = s.state()
    for comp in (vx, vy, vz):
        assert abs(comp.mean()) < 4 * math.sqrt(0.5 / comp.size)
        assert abs(comp.var() - 0.5) < 0.03
    counts = np.histogram(y, bins=10, range=(0, 1))[0]
    assert stats.chisquare(counts).pvalue > 1e-3
