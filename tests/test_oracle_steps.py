"""Pins of the oracle's individual DSMC steps (CPU only): parameters, cell index and
stable sort, collision groups, free flight with walls, and binary collisions."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


def test_nsigma_matches_hard_sphere_textbook_viscosity():
    """For hard spheres the first Chapman-Enskog viscosity is mu = (5/16) sqrt(pi m k T)
    / sigma; with mu0 v0 / (P0 H) = 2 Kn / sqrt(pi) (Eq. 7) this gives
    n sigma H = 5 sqrt(2) pi / (32 Kn)."""
    for Kn in (0.05, 0.1, 1.0, 10.0):
        assert oracle.nsigma(0.5, Kn) == pytest.approx(5 * math.sqrt(2) * math.pi / (32 * Kn),
                                                       rel=1e-14)
    assert oracle.nsigma(0.5, math.inf) == 0.0


@pytest.mark.parametrize("omega,Kn,dt_expected", [(0.5, 1.0, 0.18054), (0.81, 0.1, 0.013679)])
def test_time_step_is_fifth_of_mean_collision_time(omega, Kn, dt_expected):
    s = oracle.OracleSim(omega=omega, Kn=Kn, n_cells=4, ppc=4)
    assert s.params()["dt_d"] == pytest.approx(dt_expected, rel=5e-5)


@pytest.mark.parametrize("omega", [0.5, 0.74, 0.81, 1.0])
def test_vhs_cross_section_normalisation(omega):
    """Bird's VHS reference: at the reference temperature <sigma g> = sigma_ref <g>, with
    <g> = 2 sqrt(2/pi) for the relative speed of two Maxwellian molecules (chi with 3
    degrees of freedom, unit scale in v0 units)."""
    p = oracle.OracleSim(omega=omega, Kn=1.0, n_cells=2, ppc=2).params()
    f = lambda g: math.sqrt(2 / math.pi) * g * g * math.exp(-g * g / 2)
    mean_sg = integrate.quad(lambda g: float(p["cvhs"]) * g ** float(p["vexp"]) * f(g),
                             0, 40)[0]
    assert mean_sg == pytest.approx(2 * math.sqrt(2 / math.pi), rel=2e-7)


def test_cell_of_edges():
    n = 100
    assert oracle.lib().or_cell_of(0.0, n) == 0
    assert oracle.lib().or_cell_of(1.0, n) == n - 1
    assert oracle.lib().or_cell_of(np.nextafter(np.float32(1.0), np.float32(0)), n) == n - 1
    assert oracle.lib().or_cell_of(0.5, n) == 50
    assert oracle.lib().or_cell_of(0.0099, n) == 0


@pytest.mark.parametrize("n,n_cells", [(1, 1), (17, 3), (1000, 7), (100_000, 2000)])
def test_stable_sort_against_brute_force(n, n_cells):
    rng = np.random.default_rng(n + n_cells)
    cell = rng.integers(0, n_cells, size=n).astype(np.int32)
    if n > 10:
        cell[: n // 10] = n_cells - 1  # a crowded cell
    perm, off = oracle.stable_cell_sort(cell, n_cells)
    ref = sorted(range(n), key=lambda p: (cell[p], p))
    assert perm.tolist() == ref
    assert off.tolist() == [0] + np.cumsum(np.bincount(cell, minlength=n_cells)).tolist()


def test_group_partition_invariants():
    """Groups tile the cell in order; all but the last have G particles; the last has
    at least G/2 unless it is the only one; 25,000 particles with G = 256 give 97 groups
    of 256 and one of 168."""
    for G in (2, 4, 8, 64, 256):
        for nc in range(0, 3 * G + 5):
            ng = oracle.group_count(nc, G)
            if nc == 0:
                assert ng == 0
                continue
            sizes = [G] * (ng - 1) + [nc - (ng - 1) * G]
            assert sum(sizes) == nc and min(sizes) >= 1
            assert sizes[-1] < G + G // 2
            if ng > 1:
                assert sizes[-1] >= G // 2
    assert oracle.group_count(25_000, 256) == 98
    assert 25_000 - 97 * 256 == 168
    assert oracle.group_count(300, 256) == 1
    assert oracle.group_count(384, 256) == 2


def test_free_flight_without_wall():
    (y, vx, vy, vz), ok = oracle.move_particle(0.5, 0.1, 0.2, -0.3, 0.25, 0.01, 1, 1, 0)
    assert ok
    f = np.float32
    assert y == f(f(0.5) + f(f(0.2) * f(0.25)))
    assert vx == f(f(0.1) + f(f(0.01) * f(0.25)))
    assert vy == f(0.2) and vz == f(-0.3)


@pytest.mark.parametrize("y0,vy0", [(0.05, -1.0), (0.95, 1.0), (0.01, -3.0)])
def test_wall_hit_reemits_into_gas(y0, vy0):
    dt = 0.1
    hits = 0
    for slot in range(200):
        (y, vx, vy, vz), ok = oracle.move_particle(y0, 0.0, vy0, 0.0, dt, 0.5, 11, 3, slot)
        assert ok and 0.0 <= y <= 1.0
        t_hit = y0 / -vy0 if vy0 < 0 else (1 - y0) / vy0
        t_left = dt - t_hit
        wall = 0.0 if vy0 < 0 else 1.0
        # one bounce unless the emitted particle crosses the whole gap
        if abs(vy) * t_left < 1.0:
            hits += 1
            assert np.sign(vy) == (1 if wall == 0.0 else -1)
            assert y == pytest.approx(wall + vy * t_left, abs=1e-6)
    assert hits > 150


def test_bounce_limit_reported():
    (y, vx, vy, vz), ok = oracle.move_particle(0.5, 0.0, 1.0, 0.0, 1e4, 0.0, 5, 1, 0)
    assert not ok and y in (0.0, 1.0)


def test_collision_conserves_momentum_and_energy():
    """Each accepted collision conserves momentum and energy to binary32 rounding
    (the 1e-5 relative bar, met with a margin)."""
    rng = np.random.default_rng(1)
    worst_p = worst_e = 0.0
    for k in range(20_000):
        vi = rng.normal(0, math.sqrt(0.5), 3).astype(np.float32) + np.float32(rng.normal(0, 2))
        vj = rng.normal(0, math.sqrt(0.5), 3).astype(np.float32)
        a, b, ok = oracle.scatter_pair(vi, vj, seed=3, k=k, cell=k % 7, step=k % 5, group=0)
        assert ok
        p0 = vi.astype(np.float64) + vj
        p1 = a.astype(np.float64) + b
        e0 = (vi.astype(np.float64) ** 2).sum() + (vj.astype(np.float64) ** 2).sum()
        e1 = (a.astype(np.float64) ** 2).sum() + (b.astype(np.float64) ** 2).sum()
        scale = np.abs(vi).sum() + np.abs(vj).sum()
        worst_p = max(worst_p, np.abs(p1 - p0).max() / scale)
        worst_e = max(worst_e, abs(e1 - e0) / e0)
    assert worst_p < 1e-6
    assert worst_e < 1e-5


def test_pair_choice_is_uniform_over_ordered_pairs():
    """The candidate pair from one word (multiply-shift): always i != j within the group;
    for ng = 2..6 the count of words per ordered pair, over an evenly spaced grid of 2^20
    words covering [0, 2^32), is within 1 of equal (exactly as floor/ceil of the share);
    and random words give a chi-square consistent with uniform pairs at ng = 7."""
    rng = np.random.default_rng(12)
    for ng in (2, 3, 5, 17, 256, 383):
        for w in rng.integers(0, 2 ** 32, 2000, dtype=np.uint64):
            i, j = oracle.pair_choice(int(w), ng)
            assert 0 <= i < ng and 0 <= j < ng and i != j
    step = 2 ** 12
    for ng in range(2, 7):
        counts = {}
        for w in range(0, 2 ** 32, step):
            p = oracle.pair_choice(w, ng)
            counts[p] = counts.get(p, 0) + 1
        assert len(counts) == ng * (ng - 1)
        share = (2 ** 32 // step) / (ng * (ng - 1))
        assert max(abs(v - share) for v in counts.values()) <= 1.0
    ng, n = 7, 84_000
    counts = np.zeros((ng, ng))
    for w in rng.integers(0, 2 ** 32, n, dtype=np.uint64):
        i, j = oracle.pair_choice(int(w), ng)
        counts[i, j] += 1
    obs = counts[~np.eye(ng, dtype=bool)]
    exp = n / (ng * (ng - 1))
    chi2 = ((obs - exp) ** 2 / exp).sum()
    from scipy import stats
    assert stats.chi2.sf(chi2, ng * (ng - 1) - 1) > 1e-3


def test_sincos_turn_exact_quarter_turns():
    """The oracle's binary32 sin/cos of 2 pi v: at whole quarter turns the reduced angle
    is exactly 0 and the values are exact."""
    for v, (s, c) in [(0.0, (0.0, 1.0)), (0.25, (1.0, 0.0)), (0.5, (0.0, -1.0)),
                      (0.75, (-1.0, 0.0)), (1.0, (0.0, 1.0))]:
        sn, cs = oracle.sincos_turn(v)
        assert (float(sn), float(cs)) == (s, c), v


def test_sincos_turn_against_libm():
    """Within 3e-7 (a few binary32 ulps of values of order 1) of sin and cos of 2 pi v in
    binary64, over a fine grid of [0, 1] and the octant boundaries, and sin^2 + cos^2
    within 4e-7 of 1: no dropped or mis-signed series term or quadrant."""
    v = np.concatenate([np.linspace(0.0, 1.0, 20_001), np.arange(9) / 8.0,
                        np.arange(9) / 8.0 + 2.0 ** -24, np.arange(1, 9) / 8.0 - 2.0 ** -24])
    v = v.astype(np.float32)
    out = np.array([oracle.sincos_turn(x) for x in v], np.float64)
    ref = 2.0 * np.pi * v.astype(np.float64)
    assert np.abs(out[:, 0] - np.sin(ref)).max() < 3e-7
    assert np.abs(out[:, 1] - np.cos(ref)).max() < 3e-7
    assert np.abs(out[:, 0] ** 2 + out[:, 1] ** 2 - 1.0).max() < 4e-7


def test_collision_direction_is_isotropic():
    vi = np.array([0.3, -0.2, 0.9], np.float32)
    vj = np.array([-0.5, 0.4, 0.1], np.float32)
    g0 = np.linalg.norm(vi.astype(np.float64) - vj)
    n = []
    for k in range(40_000):
        a, b, ok = oracle.scatter_pair(vi, vj, seed=9, k=k, cell=1, step=1, group=0)
        d = a.astype(np.float64) - b
        assert np.linalg.norm(d) == pytest.approx(g0, rel=1e-6)
        n.append(d / np.linalg.norm(d))
    n = np.array(n)
    N = len(n)
    assert np.abs(n.mean(0)).max() < 4 * math.sqrt(1 / 3 / N)
    second = n.T @ n / N
    assert np.abs(second - np.eye(3) / 3).max() < 4 * math.sqrt(4 / 45 / N) + 1e-9
    # uniform on the sphere: each component is uniform on [-1, 1]
    from scipy import stats
    for c in range(3):
        assert stats.kstest(n[:, c], lambda x: (np.asarray(x) + 1) / 2).pvalue > 1e-3


@pytest.mark.parametrize("omega", [0.5, 0.74, 0.81, 1.0])
def test_acceptance_probability_is_sigma_g_over_max(omega):
    """NTC accepts a candidate of relative speed g with probability
    sigma(g) g / (sigma g)_max (sigma(g) g = cvhs g^(2 - 2 omega) in sigma_ref v0 units):
    the fraction of a fine uniform grid of u accepted through the threshold g > thr(u)
    matches it."""
    s = oracle.OracleSim(omega=omega, Kn=1.0, n_cells=1, ppc=2)
    p = s.params()
    cv, a = float(p["cvhs"]), float(p["vexp"])
    smax = float(p["smax0"])
    words = (np.arange(4096, dtype=np.uint64) * 2 ** 20 + 2 ** 19).astype(np.uint32)
    us = [oracle.u01(int(x)) for x in words]
    thr = np.array([s.accept_threshold(u, smax) for u in us])
    for g in (0.05, 0.4, 1.0, 1.7, 3.0, 4.9):
        frac = float((g > thr).mean())
        assert abs(frac - min(1.0, cv * g ** a / smax)) < 2.0 / len(us), (g, frac)
