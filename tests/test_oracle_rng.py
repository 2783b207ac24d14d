"""Pins of the oracle's random-number and elementary-function layer (CPU only).

Each check compares the oracle with something other than itself: cuRAND's host
Philox4_32_10 generator (a library that runs on the CPU), the published Philox
known-answer vectors, binary64 libm, and the distributions the DSMC method needs
(N(0,1/2) velocity components of a Maxwellian at the wall temperature in v0 units,
Eq. 6 of the paper, and the flux-weighted half-Maxwellian of a diffuse wall).
"""
import ctypes
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert list(oracle.philox4x32_10(ctr, key)) == out


def _curand_host():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 12345, 0xDEADBEEFCAFEF00D])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's Philox4_32_10 host generator emits philox(ctr=(0, 0, b_lo, b_hi),
    key=(seed_lo, seed_hi)) for block b = 0, 1, 2, ...; a generator offset of 4b
    values starts at block b."""
    cr = _curand_host()
    if cr is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        for start_block in (0, 5, 1000):
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * start_block)) == 0
            n = 64
            buf = np.zeros(n, np.uint32)
            assert cr.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_size_t(n)) == 0
            for b in range(n // 4):
                blk = start_block + b
                ctr = [0, 0, blk & 0xffffffff, blk >> 32]
                key = [seed & 0xffffffff, seed >> 32]
                assert list(oracle.philox4x32_10(ctr, key)) == list(buf[4 * b:4 * b + 4])
    finally:
        cr.curandDestroyGenerator(gen)


def test_u01_open_interval_and_exact():
    """u = (floor(x / 2^9) + 1/2) 2^-23 exactly, for the extreme and a few inner words."""
    for x in (0, 511, 512, 0x80000000, 0xfffffdff, 0xffffffff, 0x12345678):
        assert oracle.u01(x) == ((x >> 9) + 0.5) * 2.0 ** -23
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xffffffff) == 1.0 - 2.0 ** -24


@pytest.mark.parametrize("e", [-25, -24, -10, -3, -2, -1, 0, 1, 3])
def test_ln_error_all_mantissas(e):
    """Every binary32 input of the binade [2^e, 2^(e+1)) against binary64 log: at most
    2 units in the last place of the binary32 result."""
    bits = ((e + 127) << 23) | np.arange(1 << 23, dtype=np.uint32)
    x = bits.view(np.float32)
    r = oracle.ln32_array(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    nz = ref != 0.0
    ulp = np.spacing(np.abs(ref[nz]).astype(np.float32)).astype(np.float64)
    err = np.abs(r[nz] - ref[nz]) / ulp
    assert err.max() <= 2.0
    if e == 0:
        assert r[0] == 0.0  # ln 1 exactly


def test_ln_subnormal_and_exp_range():
    for x in (1e-40, 2.0 ** -140, 3e-39):
        assert abs(oracle.ln32(x) - math.log(x)) <= 2e-6 * abs(math.log(x))
    x = np.linspace(-30.0, 3.0, 1_000_001).astype(np.float32)
    r = oracle.exp32_array(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    err = np.abs(r - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert err.max() <= 2.0
    assert oracle.exp32(0.0) == 1.0


def test_init_velocities_are_maxwellian():
    """N(0, 1/2) per component: mean, variance, kurtosis and Kolmogorov-Smirnov."""
    v = oracle.init_velocities(seed=7, n=200_000).astype(np.float64)
    n = v.shape[0]
    for k in range(3):
        x = v[:, k]
        assert abs(x.mean()) < 4 * math.sqrt(0.5 / n)
        assert abs(x.var() - 0.5) < 4 * 0.5 * math.sqrt(2.0 / n)
        assert abs(stats.kurtosis(x, fisher=False) - 3.0) < 4 * math.sqrt(24.0 / n)
        cdf = lambda a: stats.norm.cdf(np.asarray(a) / math.sqrt(0.5))
        assert stats.kstest(x, cdf).pvalue > 1e-3
    # the three components are uncorrelated
    c = np.corrcoef(v.T)
    assert np.abs(c[np.triu_indices(3, 1)]).max() < 4 / math.sqrt(n)


def test_emission_speed_is_flux_weighted_half_maxwellian():
    """A diffuse wall emits |vy| with density 2 v exp(-v^2) (v0 units), so
    P(|vy| > a) = exp(-a^2) and <|vy|> = sqrt(pi)/2."""
    s = oracle.emission_speeds(seed=3, n=200_000).astype(np.float64)
    assert (s > 0).all()
    n = s.size
    assert abs(s.mean() - math.sqrt(math.pi) / 2) < 4 * math.sqrt((1 - math.pi / 4) / n)
    cdf = lambda a: 1.0 - np.exp(-np.asarray(a) ** 2)
    assert stats.kstest(s, cdf).pvalue > 1e-3
