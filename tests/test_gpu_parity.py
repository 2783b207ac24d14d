"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Deterministic mode: both sides draw the same Philox streams keyed on (step, slot,
bounce) and (step, cell, group, candidate) and round every binary32 operation once,
so particle state, cell offsets (the sort order), (sigma g)_max and collision
counters must agree bit for bit.  The moment sums are binary64 in the oracle.  The CUDA
path's default (DSMC_ACCUM_FP32) adds a collision group's products in binary32 (per lane
at most 24 terms: 12 before and 12 after the collisions, the second and third moments
by fused multiply-add, which skips the product's own rounding of at most half a unit;
then 5 butterfly levels across the warp), rounds each group total to the cell's
fixed-point grid (at most 2^-(42 - e) absolute, e the bit length of the cell's count:
below 1e-9 of sum|product| for every cell here) and adds the integers exactly.  Each
product thus passes through at most 23 + 0.5 + 5 = 28.5 roundings of relative size
2^-24 on partial sums bounded by the sum of |products|, so the sums must agree within
28.5 * 2^-24 * sum|product| + grid < 2e-6 * sum|product|, with sum|product| from the
oracle.  DSMC_ACCUM_FP64 forms the same binary32 products and adds them in binary64:
it differs from the oracle only by the summation order and the grid, within 1e-10 of
sum|product| on the runs below.

Statistical mode: independent seeds on each side; time-averaged velocity, shear
stress and heat flux agree within the combined standard errors.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from paper_2311_14140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MOM_TOL = 2e-6
MOM_TOL_F64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import _build
    _build.build()


def make_pair(omega=0.5, Kn=1.0, n_cells=100, ppc=200, F=0.0, seed=0, G=256, dt=0.0,
              dt_factor=0.2, sample_start=0, collisions=True, **gkw):
    from paper_2311_14140_gb300 import Dsmc
    o = oracle.OracleSim(omega=omega, Kn=Kn, F=F, n_cells=n_cells, ppc=ppc, seed=seed, G=G,
                         dt_factor=dt_factor, dt=dt, sample_start=sample_start,
                         collisions=collisions)
    g = Dsmc(Kn, n_cells, ppc, omega=omega, body_force=F, seed=seed, group_size=G, dt=dt,
             dt_factor=dt_factor, sample_start=sample_start, collisions=collisions, **gkw)
    return o, g


def assert_bitexact(o, g, moments=True, mom_tol=MOM_TOL):
    for name, a, b in zip(("y", "vx", "vy", "vz"), o.state(), g.state()):
        bad = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
        assert bad.size == 0, f"{name}: {bad.size} slots differ, first {bad[:5]}"
    oo, so, co, ao = o.cells()
    og, sg, cg, ag = g.cells()
    np.testing.assert_array_equal(oo, og)
    np.testing.assert_array_equal(so.view(np.uint32), sg.view(np.uint32))
    np.testing.assert_array_equal(co, cg)
    np.testing.assert_array_equal(ao, ag)
    if moments:
        mo, no = o.moments()
        mg, ng = g.moments()
        assert no == ng
        bound = mom_tol * o.abs_moments()
        err = np.abs(mg - mo)
        assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("omega,Kn,ppc,dt,dtf", [
    (0.5, 1.0, 200, 0.0, 0.2), (0.81, 0.1, 25000, 0.0, 0.2), (0.74, 5.0, 50, 0.0, 0.1),
    (0.5, math.inf, 10, 0.25, 0.2), (1.0, 0.05, 7, 0.0, 0.3)])
def test_parameters_match_oracle(omega, Kn, ppc, dt, dtf):
    o, g = make_pair(omega=omega, Kn=Kn, n_cells=3, ppc=ppc if ppc < 1000 else 4, dt=dt,
                     dt_factor=dtf)
    po, pg = o.params(), g.info()
    if ppc >= 1000:  # coef depends on ppc: compare a run with the real ppc too
        o, g = make_pair(omega=omega, Kn=Kn, n_cells=1, ppc=ppc, dt=dt, dt_factor=dtf)
        po, pg = o.params(), g.info()
    for ko, kg in (("dt", "dt_f"), ("F", "F_f"), ("coef", "coef"), ("cvhs", "cvhs"),
                   ("vexp", "vexp"), ("smax0", "smax0"), ("vinv", "vinv"), ("lncv", "lncv")):
        assert np.float32(po[ko]).view(np.uint32) == np.float32(pg[kg]).view(np.uint32), ko
    assert po["nsig"] == pg["nsigma"] and po["dt_d"] == pg["dt"]


def test_initial_state_bitexact():
    o, g = make_pair(n_cells=100, ppc=200, seed=5)
    assert_bitexact(o, g)


@pytest.mark.parametrize("steps", [1, 50])
def test_hard_sphere_kn1_deterministic(steps):
    """Argon hard spheres, Kn = 1, 100 cells x 200 particles, mean speed 1e-3 v0: bit-exact
    state after 1 and 50 steps (all particles in one group per cell)."""
    w = W.HS_KN1
    o, g = make_pair(omega=w.omega, Kn=w.Kn, n_cells=w.n_cells, ppc=w.ppc, F=w.body_force,
                     seed=0)
    o.step(steps)
    g.step(steps)
    assert_bitexact(o, g)


@pytest.mark.parametrize("warps,rows", [(8, 1), (4, 1), (8, 2)])
def test_vhs_kn01_multigroup_deterministic(warps, rows):
    """VHS omega = 0.81 at Kn = 0.1 with 700 particles per cell: 2 or 3 collision groups
    per cell (group size 256, remainder merge), 20 steps, in both CTA shapes."""
    w = W.VHS_KN01_50M
    o, g = make_pair(omega=w.omega, Kn=w.Kn, n_cells=40, ppc=700, F=w.body_force, seed=3,
                     cta_warps=warps, span_rows=rows)
    o.step(20)
    g.step(20)
    assert_bitexact(o, g)


@pytest.mark.parametrize("case", [
    # up to 1,365 cells a CTA per span: 1,000 spans of one cell, particles crossing ~13
    # cells a step
    dict(Kn=0.1, omega=0.81, n_cells=1000, ppc=1200, span_particles=1024, spans=1000),
    # the same with two sort rows per span (a CTA per row)
    dict(Kn=0.1, omega=0.81, n_cells=1000, ppc=1200, span_particles=1024, span_rows=2,
         spans=1000),
    # rows of ~8,400 records: two 32-record slices per warp and round
    dict(Kn=0.1, omega=0.81, n_cells=1000, ppc=1200, span_particles=8192, spans=143),
    # more cells, a warp per span: 750 spans, the mask table
    dict(Kn=0.1, omega=0.81, n_cells=1500, ppc=800, span_particles=1024, spans=750),
    # the same run in 137 spans: __match_any_sync
    dict(Kn=0.1, omega=0.81, n_cells=1500, ppc=800, span_particles=8192, spans=137),
    # 750 spans of two sort rows each (a warp per row): the mask table on half-spans
    dict(Kn=0.1, omega=0.81, n_cells=1500, ppc=800, span_particles=1024, span_rows=2,
         spans=750),
    # Kn = 1 on 2,000 cells, particles crossing hundreds of cells a step, 1,000 spans:
    # the mask table with slices whose cells span 256 values or more (its fallback)
    dict(Kn=1.0, omega=0.5, n_cells=2000, ppc=600, span_particles=1024, spans=1000),
])
def test_scatter_variants_bitexact(case):
    """The stable scatter runs a CTA per span while its shared memory (nine words per
    cell) leaves room for 4 CTAs per SM (up to 1,365 cells), its warps taking one or, for
    rows averaging 4,096 records or more, two 32-record slices per round; above, a warp
    per span, which ranks same-cell records with a shared-memory mask table when at least four of
    its warps (spans) share an SM (a 152-SM GPU: 608 spans), else with
    __match_any_sync, and falls back to __match_any_sync for a slice whose cells span
    256 values or more.  Each case bit-exact against the oracle over 6 steps."""
    c = dict(case)
    spans = c.pop("spans")
    o, g = make_pair(F=W.f0_force(c["Kn"]), seed=5, **c)
    assert g.info()["n_spans"] == spans
    o.step(6)
    g.step(6)
    assert_bitexact(o, g)


@pytest.mark.parametrize("n_cells,ppc,rows,kernel", [
    (256, 1100, 1, "fused"), (257, 1100, 1, "spans"), (128, 1100, 2, "fused"),
    (129, 1100, 2, "spans"), (1024, 100, 1, "fused"), (1025, 100, 1, "cols")])
def test_span_prefix_kernels_bitexact(n_cells, ppc, rows, kernel):
    """The prefix of the sort matrix down its rows and the new cell offsets: one launch of
    one CTA while the run has at most 1,024 cells and 256 rows (spans x sort rows); with
    more cells but at most 256 rows a thread per cell walking its column, then the offsets;
    else blocks of 32 cells x 32 row segments, then the offsets.  Cases on either side of
    each threshold (spans of 1,024 particles), bit-exact against the oracle over 5 steps."""
    o, g = make_pair(Kn=1.0, n_cells=n_cells, ppc=ppc, F=W.f0_force(1.0), seed=21,
                     span_particles=1024, span_rows=rows)
    info = g.info()
    n_rows = info["n_spans"] * rows
    expect = ("fused" if n_cells <= 1024 and n_rows <= 256 else
              "cols" if n_rows <= 256 else "spans")
    assert expect == kernel, (info["n_spans"], n_rows)
    o.step(5)
    g.step(5)
    assert_bitexact(o, g)


@pytest.mark.parametrize("case", [
    dict(n_cells=1, ppc=2, Kn=1.0),                       # one cell, smallest pair
    dict(n_cells=37, ppc=13, Kn=0.5, F=0.01),             # N = 481, ragged warp tail
    dict(n_cells=500, ppc=1, Kn=1.0),                     # empty and single-particle cells
    dict(n_cells=50, ppc=60, Kn=10.0, F=0.002),           # dt = 1.8: many wall bounces
    dict(n_cells=20, ppc=300, Kn=math.inf, dt=0.3, F=1.0),  # collisionless
    dict(n_cells=30, ppc=100, Kn=0.2, G=2),               # smallest groups
    dict(n_cells=8, ppc=1500, Kn=0.3, G=512, omega=0.81),  # largest groups
    dict(n_cells=64, ppc=250, Kn=1.0, collisions=False),  # sampling without collisions
    dict(n_cells=33, ppc=97, Kn=0.7, sample_start=7, dt_factor=0.5),
    dict(n_cells=16384, ppc=60, Kn=0.5, F=0.002),         # the largest cell count
    dict(n_cells=1, ppc=70000, Kn=0.5, omega=0.81),       # one cell of 274 groups
    dict(n_cells=3, ppc=40000, Kn=2.0, span_particles=1 << 17, span_rows=2),  # a 120,000-
])                                                        # particle span in two sort rows
def test_edge_cases_deterministic(case):
    c = dict(case)
    o, g = make_pair(seed=11, **c)
    o.step(12)
    g.step(12)
    assert_bitexact(o, g)


def test_checkpoint_resume_bitexact():
    """Copying state, (sigma g)_max and the step counter into a fresh handle and going
    on gives the same run as going on without a break (counter-based random numbers)."""
    from paper_2311_14140_gb300 import Dsmc
    kw = dict(omega=0.81, body_force=1e-3, seed=9, sample_start=0)
    a = Dsmc(0.3, 60, 150, **kw)
    a.step(10)
    b = Dsmc(0.3, 60, 150, **kw)
    b.load_state(*a.state(), smax=a.cells()[1], step=10)
    a.step(7)
    b.step(7)
    for u, v in zip(a.state(), b.state()):
        np.testing.assert_array_equal(u.view(np.uint32), v.view(np.uint32))
    np.testing.assert_array_equal(a.cells()[1], b.cells()[1])


def test_bounce_limit_reported_not_trapped():
    """A collisionless step of 1e4 H/v0 makes every particle exceed the bounded wall loop
    (64 bounces): the kernels finish, the error word is set, and the call reports it."""
    from paper_2311_14140_gb300 import Dsmc, DsmcError
    g = Dsmc(math.inf, 4, 8, dt=1e4)
    g.step(1)
    with pytest.raises(DsmcError) as e:
        g.sync()
    assert e.value.status == 4 and "wall-bounces" in str(e.value)
    with pytest.raises(DsmcError):
        g.step(1)
    o = oracle.OracleSim(Kn=math.inf, n_cells=4, ppc=8, dt=1e4)
    assert o.step(1) & 2


def _oracle_run(args):
    import oracle as orc
    from paper_2311_14140_gb300 import workloads as WL
    seed, = args
    w = WL.HS_KN1
    s = orc.OracleSim(omega=w.omega, Kn=w.Kn, F=w.body_force, n_cells=w.n_cells, ppc=w.ppc,
                      seed=seed, sample_start=w.sample_start)
    s.step(w.steps)
    acc, ns = s.moments()
    return orc.fields(acc, ns, w.ppc)


def test_statistical_16_seeds():
    """Argon hard spheres at Kn = 1 (100 cells x 200 particles, 2,000 steps, last 1,000
    sampled): 16 GPU seeds against 16 different oracle seeds.  The channel means of
    velocity, shear stress and heat flux agree within 3 combined standard errors; the
    same quantities averaged over 10 bins of 10 cells (a family of 30 comparisons) within
    3.5, the per-comparison bar that keeps the family-wise false-alarm rate near 1 %
    (Bonferroni: 30 x P(|t_30| > 3.5) = 0.045; 30 x P(|z| > 3.5) = 0.014), where 3 would
    fail one run in ten by chance alone (30 x P(|t_30| > 3) = 0.16)."""
    from paper_2311_14140_gb300 import Dsmc
    w = W.HS_KN1
    gpu = []
    for seed in range(16):
        g = Dsmc(w.Kn, w.n_cells, w.ppc, omega=w.omega, body_force=w.body_force, seed=seed,
                 sample_start=w.sample_start)
        g.step(w.steps)
        gpu.append(g.fields())  # the library's post-processing (dsmc_cell_fields_of)
        g.close()
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        cpu = pool.map(_oracle_run, [(100 + s,) for s in range(16)])
    for q in ("ux", "Pxy", "qx"):
        a = np.array([f[q] for f in gpu]).reshape(16, 10, 10).mean(2)
        b = np.array([f[q] for f in cpu]).reshape(16, 10, 10).mean(2)
        se = np.sqrt(a.var(0, ddof=1) / 16 + b.var(0, ddof=1) / 16)
        z = (a.mean(0) - b.mean(0)) / se
        assert np.abs(z).max() < 3.5, (q, z)
        am, bm = a.mean(1), b.mean(1)
        zc = (am.mean() - bm.mean()) / math.sqrt(am.var(ddof=1) / 16 + bm.var(ddof=1) / 16)
        assert abs(zc) < 3.0, (q, zc)
    # the physics both share: the momentum balance of Eq. 1
    P = np.array([f["Pxy"] for f in gpu])
    yc = (np.arange(w.n_cells) + 0.5) / w.n_cells
    slopes = [np.polyfit(yc, p, 1)[0] for p in P]
    assert abs(np.mean(slopes) - 2 * w.body_force) < 3 * np.std(slopes, ddof=1) / 4 + \
        0.02 * 2 * w.body_force


def test_full_size_vhs_50m_bitexact():
    """The 5e7-particle VHS workload (2,000 cells x 25,000 particles, Kn = 0.1, the
    benchmark's launch configuration): initial state and two steps, bit-exact against
    the oracle."""
    w = W.VHS_KN01_50M
    o, g = make_pair(omega=w.omega, Kn=w.Kn, n_cells=w.n_cells, ppc=w.ppc, F=w.body_force,
                     seed=0)
    assert_bitexact(o, g, moments=False)
    o.step(2)
    g.step(2)
    assert_bitexact(o, g)


@pytest.mark.parametrize("case", [
    dict(omega=0.5, Kn=1.0, n_cells=100, ppc=200, F=8.713e-4),
    dict(omega=0.81, Kn=0.1, n_cells=40, ppc=700, F=4.038e-4),
])
def test_binary64_moment_sums_against_oracle(case):
    """options.accum = DSMC_ACCUM_FP64: the state is the same as with the default (the
    sums never feed back), and the moment sums agree with the oracle's binary64 sums to
    1e-10 of sum|product| after 30 sampled steps; the default binary32 sums agree with
    both within the binary32 bound."""
    from paper_2311_14140_gb300 import Dsmc
    o, g = make_pair(seed=4, **case)
    g2 = Dsmc(case["Kn"], case["n_cells"], case["ppc"], omega=case["omega"],
              body_force=case["F"], seed=4, accum=1)
    o.step(30)
    g.step(30)
    g2.step(30)
    assert_bitexact(o, g2, mom_tol=MOM_TOL_F64)
    m32, _ = g.moments()
    m64, _ = g2.moments()
    assert np.all(np.abs(m32 - m64) <= MOM_TOL * o.abs_moments())
    for u, v in zip(g.state(), g2.state()):
        np.testing.assert_array_equal(u.view(np.uint32), v.view(np.uint32))


@pytest.mark.parametrize("accum", [0, 1])
def test_moment_sums_reproducible(accum):
    """The moment sums are a pure function of the run: two identical runs, and runs
    with other span partitions and CTA shapes (which change which warp takes which
    collision group, and in what order groups finish), give bit-identical sums."""
    from paper_2311_14140_gb300 import Dsmc
    kw = dict(omega=0.81, body_force=1e-3, seed=21, accum=accum)
    runs = [Dsmc(0.2, 300, 900, **kw), Dsmc(0.2, 300, 900, **kw),
            Dsmc(0.2, 300, 900, span_particles=8192, **kw),
            Dsmc(0.2, 300, 900, cta_warps=4, span_rows=2, **kw)]
    ref = None
    for g in runs:
        g.step(15)
        m, n = g.moments()
        if ref is None:
            ref = (m, n)
        else:
            assert n == ref[1]
            np.testing.assert_array_equal(m.view(np.uint64), ref[0].view(np.uint64))
        g.close()


def test_accumulation_modes_over_1000_sampled_steps():
    """The benchmark's physics (VHS omega = 0.81, Kn = 0.1, its force) on 40 cells x 700
    particles, 1,000 sampled steps: the binary64 mode's sums against the oracle's within
    1e-10 of sum|product| (summation order and the fixed-point grid are its only
    differences), the default binary32 mode's within the binary32 bound 2e-6, and the
    state bit-exact in both."""
    from paper_2311_14140_gb300 import Dsmc
    w = W.VHS_KN01_50M
    o, g32 = make_pair(omega=w.omega, Kn=w.Kn, n_cells=40, ppc=700, F=w.body_force, seed=8)
    g64 = Dsmc(w.Kn, 40, 700, omega=w.omega, body_force=w.body_force, seed=8, accum=1)
    o.step(1000)
    g32.step(1000)
    g64.step(1000)
    assert_bitexact(o, g64, mom_tol=MOM_TOL_F64)
    assert_bitexact(o, g32, mom_tol=MOM_TOL)
