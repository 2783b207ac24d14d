"""Batched runs (dsmc_create_batch) through the C ABI.

An instance of a batch draws its random numbers from its own seed, step, cells and
slots, so it must evolve bit for bit as the same run on its own, and hence as the
oracle.  The span partition of the step passes, the tuner and CUDA-graph replay change
only how work is split and launched, so none of them may change a single bit either.
Moment sums of two CUDA runs are compared bit for bit (group totals combine exactly in
fixed point, whatever the order); against the oracle's binary64 sums, within the
tolerance of the parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_2311_14140_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MOM_TOL = 2e-6

# Uneven instances: hard spheres and VHS, several Kn (one collisionless), forces,
# cell counts and particles per cell, including a one-cell and a ragged instance.
DEFS = [
    dict(Kn=1.0, n_cells=100, ppc=200, omega=0.5, body_force=W.f0_force(1.0), seed=0),
    dict(Kn=0.1, n_cells=40, ppc=700, omega=0.81, body_force=W.f0_force(0.1), seed=3),
    dict(Kn=5.0, n_cells=37, ppc=13, omega=0.74, body_force=0.01, seed=17),
    dict(Kn=0.3, n_cells=1, ppc=900, omega=1.0, body_force=0.0, seed=5),
    dict(Kn=0.05, n_cells=211, ppc=55, omega=0.5, body_force=2e-3, seed=2 ** 40 + 7),
    dict(Kn=2.0, n_cells=64, ppc=250, omega=0.81, body_force=-5e-3, seed=99),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import _build
    _build.build()


class Member:
    """Instance i of a batch with the accessors of a single run."""

    def __init__(self, b, i):
        self.b, self.i = b, i

    def state(self):
        return self.b.state(self.i)

    def cells(self):
        return self.b.cells(self.i)

    def moments(self):
        return self.b.moments(self.i)


def assert_same_run(ref, got, abs_moments=None):
    for name, a, b in zip(("y", "vx", "vy", "vz"), ref.state(), got.state()):
        bad = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
        assert bad.size == 0, f"{name}: {bad.size} slots differ, first {bad[:5]}"
    for a, b in zip(ref.cells(), got.cells()):
        np.testing.assert_array_equal(a.view(np.uint32) if a.dtype == np.float32 else a,
                                      b.view(np.uint32) if b.dtype == np.float32 else b)
    ma, na = ref.moments()
    mb, nb = got.moments()
    assert na == nb
    if abs_moments is not None:  # against the oracle's binary64 sums
        bound = MOM_TOL * abs_moments
        err = np.abs(mb - ma)
        assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    else:  # two CUDA runs: group totals combine exactly, so the sums are bit-identical
        np.testing.assert_array_equal(mb.view(np.uint64), ma.view(np.uint64))


def batch(defs, **kw):
    from paper_2311_14140_gb300 import DsmcBatch
    return DsmcBatch(defs, **kw)


def single(d, **kw):
    from paper_2311_14140_gb300 import Dsmc
    return Dsmc(**d, **kw)


@pytest.mark.parametrize("G", [256, 8])
def test_batch_members_match_single_runs(G):
    b = batch(DEFS, group_size=G, sample_start=5)
    b.step(25)
    for i, d in enumerate(DEFS):
        s = single(d, group_size=G, sample_start=5)
        s.step(25)
        assert_same_run(s, Member(b, i))


def test_batch_members_match_oracle():
    b = batch(DEFS, sample_start=3)
    b.step(12)
    for i in (0, 2, 3):
        d = DEFS[i]
        o = oracle.OracleSim(omega=d["omega"], Kn=d["Kn"], F=d["body_force"],
                             n_cells=d["n_cells"], ppc=d["ppc"], seed=d["seed"], G=256,
                             dt_factor=0.2, dt=0.0, sample_start=3, collisions=True)
        o.step(12)
        assert_same_run(o, Member(b, i), abs_moments=o.abs_moments())


def test_moments_all_is_the_concatenation():
    b = batch(DEFS)
    b.step(6)
    allm, ns = b.moments_all()
    for i in range(len(DEFS)):
        m, n = b.moments(i)
        np.testing.assert_array_equal(allm[b.cell_base[i]:b.cell_base[i + 1]], m)
        assert ns[i] == n == 6


@pytest.mark.parametrize("span,warps,rows", [(1024, 8, 1), (4096, 4, 2), (65536, 8, 2),
                                             (2048, 4, 1)])
def test_partition_does_not_change_results(span, warps, rows):
    ref = batch(DEFS)
    ref.step(10)
    b = batch(DEFS, span_particles=span, cta_warps=warps, span_rows=rows)
    b.step(4)
    b.set_options(span_particles=2048, cta_warps=12 - warps, span_rows=3 - rows)
    b.step(3)
    b.set_options(span_particles=span, cta_warps=warps, span_rows=rows)
    b.step(3)
    for i in range(len(DEFS)):
        assert_same_run(Member(ref, i), Member(b, i))


def test_batch_with_a_member_of_many_spans():
    """A member of 300 one-cell spans makes the batch's sort matrix too tall for the
    column-walk prefix (more than 256 rows): the batch takes the segmented prefix kernel,
    its members alone take either; every member still matches its run alone."""
    defs = [dict(Kn=1.0, n_cells=300, ppc=1100, omega=0.5, body_force=W.f0_force(1.0),
                 seed=8), DEFS[1], DEFS[2]]
    b = batch(defs, span_particles=1024, sample_start=2)
    b.step(6)
    assert b.info(0)["n_spans"] == 300
    for i, d in enumerate(defs):
        s = single(d, span_particles=1024, sample_start=2)
        s.step(6)
        assert_same_run(s, Member(b, i))


def test_autotune_keeps_the_run():
    ref = batch(DEFS)
    b = batch(DEFS)
    best, ms = b.autotune(steps_per_trial=2)
    assert best >= 1024 and ms > 0
    steps = b.info(0)["step"]
    assert steps >= 3
    ref.step(steps)
    for i in range(len(DEFS)):
        assert_same_run(Member(ref, i), Member(b, i))
    assert b.info(0)["span_particles"] == best
    assert b.info(0)["cta_warps"] in (4, 8)


def test_graph_replay_matches_direct_launches():
    import torch
    stream = torch.cuda.Stream()
    ref = batch(DEFS, sample_start=20)
    ref.step(45)
    with torch.cuda.stream(stream):
        b = batch(DEFS, sample_start=20, graph=True, stream=stream.cuda_stream)
        b.step(3)   # direct steps, then replays starting from another buffer parity
        b.step(35)  # two replays of 16 steps and three direct steps
        b.step(7)
        stream.synchronize()
    for i in range(len(DEFS)):
        assert_same_run(Member(ref, i), Member(b, i))
    one = single(DEFS[1], sample_start=20)
    one.step(45)
    with torch.cuda.stream(stream):
        g = single(DEFS[1], sample_start=20, graph=True, stream=stream.cuda_stream)
        g.step(45)
        stream.synchronize()
    assert_same_run(one, g)


def test_load_state_of_one_member_restores_it():
    a = batch(DEFS, sample_start=0)
    a.step(10)
    saved = a.state(4)
    smax = a.cells(4)[1]
    a.step(5)
    b = batch(DEFS, sample_start=0)
    b.step(10)
    # scramble member 4, then restore it from the checkpoint
    b.step(3)
    b.load_state(4, *saved, smax=smax, step=10)
    b.step(5)
    # member 4 continues from step 10 as in `a`; the others ran 18 steps
    sa = a.state(4)
    sb = b.state(4)
    for x, y in zip(sa, sb):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    assert b.info(4)["step"] == 15 and b.info(0)["step"] == 18
    c = single(DEFS[0], sample_start=0)
    c.step(18)
    for x, y in zip(c.state(), b.state(0)):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))


def test_full_size_batch_members_match_single_runs():
    """The 256 uneven instances of the batched workload (Kn log-uniform in [0.05, 10],
    50-1000 cells, 50-400 particles per cell): three steps in one batch, compared with
    five members run alone (smallest, largest, lowest and highest Kn, one more)."""
    insts = W.batch_instances(256)
    defs = [dict(Kn=w.Kn, n_cells=w.n_cells, ppc=w.ppc, omega=w.omega,
                 body_force=w.body_force, seed=w.seeds[0]) for w in insts]
    b = batch(defs)
    b.autotune(steps_per_trial=1)
    n = b.info(0)["step"]
    sizes = [d["n_cells"] * d["ppc"] for d in defs]
    kns = [d["Kn"] for d in defs]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argmin(kns)),
            int(np.argmax(kns)), 77}
    for i in sorted(pick):
        s = single(defs[i])
        s.step(n)
        assert_same_run(s, Member(b, i))


def test_many_tiny_instances_match_single_runs():
    """4,096 instances of one to three cells and a few particles each (HS, Kn 0.3-3, own
    seeds): a batch far wider than the GPU's grid of spans, every instance a CTA of its
    own, the per-instance prefix kernels at full width.  Sampled members bit-exact
    against the same runs alone after 12 steps."""
    rng = np.random.default_rng(77)
    defs = [dict(Kn=float(10 ** rng.uniform(-0.5, 0.5)), n_cells=int(rng.integers(1, 4)),
                 ppc=int(rng.integers(2, 9)), omega=0.5, body_force=2e-3, seed=int(s))
            for s in range(4096)]
    b = batch(defs, sample_start=3)
    b.step(12)
    for i in (0, 1, 777, 2048, 4095):
        g = single(defs[i], sample_start=3)
        g.step(12)
        assert_same_run(g, Member(b, i))
