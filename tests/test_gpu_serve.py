"""Pools (instances added and removed while the handle runs) and the request loop.

An instance added to a pool is set up exactly as a run created on its own and draws its
random numbers from its own seed, step, cells and slots, so whatever else is in the
pool, before or after it, its state must be bit for bit that of the same run alone
after the same number of its own steps.  The request loop must return, for every
request, the channel sums of that run alone after the steps it reports.
"""
import numpy as np
import pytest

from paper_2311_14140_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import _build
    _build.build()


A = dict(Kn=1.0, n_cells=100, ppc=200, omega=0.5, body_force=W.f0_force(1.0), seed=0)
B = dict(Kn=0.1, n_cells=40, ppc=700, omega=0.81, body_force=W.f0_force(0.1), seed=3)
C = dict(Kn=5.0, n_cells=37, ppc=13, omega=0.74, body_force=0.01, seed=17)
D_ = dict(Kn=0.05, n_cells=211, ppc=55, omega=0.5, body_force=2e-3, seed=2 ** 40 + 7)


def vx_tol(m):
    """Tolerance of a sum of sampled vx between two runs whose states agree bit for bit:
    their per-cell sums are then bit-identical (group totals combine exactly, whatever
    warp takes which group), and only the order in which the cells' binary64 sums are
    added into the channel total differs (the device's reduction against numpy's), so the
    totals agree to 1e-12 * sum |vx|, with sum |vx| <= sqrt(count * sum vx^2)
    (Cauchy-Schwarz)."""
    return 1e-12 * np.sqrt(m[:, 0].sum() * m[:, 4].sum())


def alone(d, steps, **kw):
    from paper_2311_14140_gb300 import Dsmc
    g = Dsmc(**d, **kw)
    g.step(steps)
    return g


def same_state(g, pool, i):
    for x, y in zip(g.state(), pool.state(i)):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    for x, y in zip(g.cells(), pool.cells(i)):
        np.testing.assert_array_equal(x, y)


def pool(**kw):
    from paper_2311_14140_gb300 import DsmcPool
    return DsmcPool(max_particles=200_000, max_cells=2000, max_instances=8,
                    max_cells_per_instance=1000, **kw)


def test_members_added_and_removed_mid_run_evolve_as_alone():
    p = pool(sample_start=4)
    ia = p.add(**A)
    ib = p.add(**B)
    p.step(10)
    ic = p.add(**C)          # joins at the pool's step 10
    p.step(7)
    p.remove(ia)             # frees A's ranges and id
    idd = p.add(**D_)        # reuses them
    assert idd == ia
    p.step(9)
    assert p.size() == 3
    same_state(alone(B, 26, sample_start=4), p, ib)
    same_state(alone(C, 16, sample_start=4), p, ic)
    same_state(alone(D_, 9, sample_start=4), p, idd)
    assert p.info(ic)["step"] == 16 and p.info(idd)["step"] == 9


def test_pool_refuses_what_does_not_fit_and_recovers():
    from paper_2311_14140_gb300 import DsmcError
    p = pool()
    big = dict(A, n_cells=500, ppc=300)    # 150,000 particles
    i = p.add(**big)
    with pytest.raises(DsmcError) as e:
        p.add(**big)                        # 300,000 > 200,000 slots
    assert e.value.status == 2 and "no room" in str(e.value)
    p.step(3)
    p.remove(i)
    j = p.add(**big)
    p.step(5)
    same_state(alone(big, 5), p, j)


def test_channel_sums_are_the_cell_sums():
    p = pool(sample_start=2)
    ids = [p.add(**d) for d in (A, B, C)]
    p.step(12)
    cs = p.channel_sums()
    for i in ids:
        m, n = p.moments(i)
        assert cs[i, 0] == m[:, 0].sum()
        np.testing.assert_allclose(cs[i, 1], m[:, 1].sum(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("graph", [False, True])
def test_serve_results_equal_the_same_runs_alone(graph):
    """Six requests arriving at once into a pool that holds three of them at a time,
    each to a 30 % standard error (capped at 640 steps); every result is then replayed
    as a run of its own for the steps the loop reports.  With graph replay the pool's
    membership changes between replays (admissions and removals invalidate the graph)."""
    import torch
    defs = [A, B, C, D_, dict(A, seed=5, Kn=2.0), dict(C, seed=9, n_cells=80)]
    reqs = [dict(d, arrival=0.0, target_se=0.3, max_steps=640) for d in defs]
    from paper_2311_14140_gb300 import DsmcPool
    # graph capture needs a stream other than the legacy default one
    stream = torch.cuda.Stream() if graph else torch.cuda.current_stream()
    kw = dict(graph=True, stream=stream.cuda_stream) if graph else {}
    with torch.cuda.stream(stream):
        p = DsmcPool(max_particles=60_000, max_cells=1000, max_instances=8,
                     max_cells_per_instance=400, sample_start=8, **kw)
        res = p.serve(reqs, epoch_steps=16, batches=4)
        stream.synchronize()
    assert p.size() == 0
    for r, d in zip(res, defs):
        assert r["converged"] in (0, 1) and r["finished"] >= r["admitted"] >= 0.0
        assert r["steps"] % 16 == 0 and 0 < r["steps"] <= 640
        g = alone(d, r["steps"], sample_start=8)
        m, n = g.moments()
        assert r["count"] == m[:, 0].sum()
        assert abs(r["sum_vx"] - m[:, 1].sum()) <= vx_tol(m)
        if r["converged"] == 1:
            assert r["u_se"] <= 0.3 * abs(r["u_mean"])
    # A, B and C fill the pool (48,576 of 60,000 slots): D waits for one of them
    assert res[3]["admitted"] >= min(res[k]["finished"] for k in range(3))


def test_solve_alone_matches_serving_one_request():
    from paper_2311_14140_gb300 import DsmcPool, solve
    req = dict(B, arrival=0.0, target_se=0.5, max_steps=320)
    s = solve(req, epoch_steps=16, batches=4, sample_start=8)
    p = DsmcPool(max_particles=60_000, max_cells=1000, max_instances=4,
                 max_cells_per_instance=400, sample_start=8)
    r = p.serve([req], epoch_steps=16, batches=4)[0]
    assert s["steps"] == r["steps"] and s["count"] == r["count"]
    # the same per-cell sums reduced over the instance's cells by the same kernel
    assert s["sum_vx"] == r["sum_vx"]


def test_served_requests_and_pool_members_match_the_oracle():
    """The oracle, not the library, as the reference of served work.  Three small requests
    (hard spheres, VHS omega = 0.74, Kn 0.3-4) are served together; for each, the oracle
    runs the same instance for the steps the loop reports: the sampled particle count
    must agree exactly and the channel sum of vx within the DSMC parity bound
    (2e-6 of the oracle's sum of |vx|).  A pool member that joins mid-run is also
    compared with the oracle bit for bit (state, cell offsets, (sigma g)_max)."""
    import oracle
    from paper_2311_14140_gb300 import DsmcPool
    defs = [dict(Kn=1.0, n_cells=30, ppc=50, omega=0.5, body_force=2e-3, seed=31),
            dict(Kn=0.3, n_cells=24, ppc=80, omega=0.74, body_force=1e-3, seed=32),
            dict(Kn=4.0, n_cells=40, ppc=30, omega=0.5, body_force=5e-3, seed=33)]
    reqs = [dict(d, arrival=0.0, target_se=0.3, max_steps=320) for d in defs]
    p = DsmcPool(max_particles=20_000, max_cells=400, max_instances=4,
                 max_cells_per_instance=100, sample_start=8)
    res = p.serve(reqs, epoch_steps=16, batches=4)
    for r, d in zip(res, defs):
        assert r["converged"] in (0, 1) and r["steps"] > 0
        o = oracle.OracleSim(omega=d["omega"], Kn=d["Kn"], F=d["body_force"],
                             n_cells=d["n_cells"], ppc=d["ppc"], seed=d["seed"],
                             sample_start=8)
        o.step(r["steps"])
        m, _ = o.moments()
        assert r["count"] == m[:, 0].sum()
        assert abs(r["sum_vx"] - m[:, 1].sum()) <= 2e-6 * o.abs_moments()[:, 1].sum()
        o.close()
    # a member added to a running pool against the oracle
    q = DsmcPool(max_particles=20_000, max_cells=400, max_instances=4,
                 max_cells_per_instance=100, sample_start=3)
    q.add(**defs[0])
    q.step(5)
    i = q.add(**defs[1])
    q.step(11)
    d = defs[1]
    o = oracle.OracleSim(omega=d["omega"], Kn=d["Kn"], F=d["body_force"], n_cells=d["n_cells"],
                         ppc=d["ppc"], seed=d["seed"], sample_start=3)
    o.step(11)
    for x, y in zip(o.state(), q.state(i)):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    oo, so, _, _ = o.cells()
    og, sg, _, _ = q.cells(i)
    np.testing.assert_array_equal(oo, og)
    np.testing.assert_array_equal(so.view(np.uint32), sg.view(np.uint32))
    o.close()
