"""The C-ABI library on the CPU side (no GPU needed): it loads, exports every symbol
that include/dsmc.h declares, and rejects bad arguments before touching the device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2311_14140_gb300 import dsmc as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^DSMC_API\s+[\w\s\*]+?\b(dsmc_\w+)\(", text, re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2311_14140_gb300 import _build
    _build.build()
    return D.load_library()


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ("dsmc_create", "dsmc_step", "dsmc_sample_moments", "dsmc_destroy"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = D.default_options()
    assert (o.dt_factor, o.dt, o.sample_start, o.group_size, o.collisions, o.profile,
            o.span_particles, o.cta_warps, o.span_rows, o.graph, o.accum) == \
        (0.2, 0.0, 0, 256, 1, 0, 0, 0, 0, 0, 0)
    # the ctypes mirror of dsmc_options has the C struct's size (accum sits in what was
    # the padding before the stream pointer)
    assert ctypes.sizeof(D.Options) == 64 and D.Options.accum.offset == 52
    assert lib.dsmc_kernel_count() == 7
    assert lib.dsmc_kernel_name(0) == b"init"
    assert lib.dsmc_status_string(4) == b"device limit reached"


def test_workspace_bytes_grow_with_size(lib):
    a = lib.dsmc_workspace_bytes(100, 200)
    b = lib.dsmc_workspace_bytes(2000, 25000)
    assert 0 < a < b
    assert b >= 8 * 4 * 2000 * 25000  # two SoA copies of y, vx, vy, vz
    assert lib.dsmc_workspace_bytes(0, 10) == 0


def _create(lib, gas=None, Kn=1.0, wall_T=273.0, F=0.0, n_cells=10, ppc=10, opt=None):
    g = D.Gas(6.63e-26, 4.17e-10, 0.5, 273.0) if gas is None else gas
    h = ctypes.c_void_p()
    o = D.default_options() if opt is None else opt
    st = lib.dsmc_create_in(ctypes.byref(g), Kn, wall_T, F, n_cells, ppc, 0, ctypes.byref(o),
                            None, 0, ctypes.byref(h))
    return st, lib.dsmc_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(Kn=0.0), "Kn"), (dict(Kn=-1.0), "Kn"), (dict(Kn=math.nan), "Kn"),
    (dict(wall_T=0.0), "wall_T"), (dict(F=math.inf), "body_force"),
    (dict(n_cells=0), "n_cells"), (dict(ppc=0), "ppc"),
    (dict(n_cells=70000, ppc=1), "16384"), (dict(n_cells=50000, ppc=50000), "2^31 - 2^24"),
    (dict(Kn=math.inf), "time step"),
])
def test_bad_arguments_are_rejected(lib, kw, needle):
    st, msg = _create(lib, **kw)
    assert st == 1 and needle in msg


def test_bad_gas_and_options_rejected(lib):
    st, msg = _create(lib, gas=D.Gas(6.63e-26, 4.17e-10, 0.4, 273.0))
    assert st == 1 and "omega" in msg
    st, msg = _create(lib, gas=D.Gas(-1.0, 4.17e-10, 0.5, 273.0))
    assert st == 1 and "mass" in msg
    for field, val in (("group_size", 3), ("group_size", 1024), ("dt_factor", 0.0),
                       ("dt", -1.0), ("span_particles", 1000), ("span_particles", 1 << 25),
                       ("cta_warps", 6), ("cta_warps", 16), ("span_rows", 3), ("graph", 1),
                       ("accum", 2), ("accum", -1)):
        o = D.default_options()
        setattr(o, field, val)
        st, msg = _create(lib, opt=o)
        assert st == 1 and "options" in msg, (field, msg)


def _batch(lib, defs, opt=None):
    arr = (D.Instance * len(defs))(*[D.make_instance(**d) for d in defs])
    h = ctypes.c_void_p()
    o = D.default_options() if opt is None else opt
    st = lib.dsmc_create_batch(arr, len(defs), ctypes.byref(o), None, 0, ctypes.byref(h))
    return st, lib.dsmc_last_error().decode()


def test_batch_arguments_are_rejected(lib):
    ok = dict(Kn=1.0, n_cells=10, ppc=10)
    st, msg = _batch(lib, [ok, dict(ok, Kn=-1.0)])
    assert st == 1 and "instance 1" in msg and "Kn" in msg
    st, msg = _batch(lib, [ok, ok, dict(ok, n_cells=20000)])
    assert st == 1 and "instance 2" in msg and "16384" in msg
    # each instance alone is within limits, together they are not
    big = dict(Kn=1.0, n_cells=10000, ppc=150000)
    st, msg = _batch(lib, [big, big])
    assert st == 1 and "total" in msg
    h = ctypes.c_void_p()
    assert lib.dsmc_create_batch(None, 1, None, None, 0, ctypes.byref(h)) == 1
    arr = (D.Instance * 1)(D.make_instance(**ok))
    assert lib.dsmc_create_batch(arr, 0, None, None, 0, ctypes.byref(h)) == 1


def test_batch_workspace_is_the_sum_of_its_parts(lib):
    defs = [dict(Kn=1.0, n_cells=50 + 7 * i, ppc=40 + 3 * i) for i in range(5)]
    arr = (D.Instance * 5)(*[D.make_instance(**d) for d in defs])
    total = lib.dsmc_batch_workspace_bytes(arr, 5)
    singles = sum(lib.dsmc_workspace_bytes(d["n_cells"], d["ppc"]) for d in defs)
    assert total > 0 and total <= singles
    assert total >= sum(2 * 16 * d["n_cells"] * d["ppc"] for d in defs)
    assert lib.dsmc_batch_workspace_bytes(arr, 0) == 0
    assert lib.dsmc_batch_size(None) == 0


def test_binding_structs_match_the_header(tmp_path):
    """sizeof and every field offset of the header's structs, as a C compiler lays them
    out, equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    structs = {"dsmc_gas": D.Gas, "dsmc_options": D.Options, "dsmc_info": D.Info,
               "dsmc_instance": D.Instance, "dsmc_pool_limits": D.PoolLimits,
               "dsmc_request": D.Request, "dsmc_serve_options": D.ServeOptions,
               "dsmc_request_result": D.RequestResult, "dsmc_surrogate_fit": D.SurrogateFit,
               "dsmc_mms_params": D.MmsParams, "dsmc_mms_result": D.MmsResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dsmc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(x.split()[:2]): int(x.split()[2]) for x in out if x}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_pool_limits_are_checked(lib):
    bad = [D.PoolLimits(0, 10, 4, 10), D.PoolLimits(1 << 20, 10, 0, 10),
           D.PoolLimits(1 << 20, 10, 4, 20), D.PoolLimits(1 << 20, 100000, 4, 20000)]
    for lim in bad:
        assert lib.dsmc_pool_workspace_bytes(ctypes.byref(lim)) == 0
        h = ctypes.c_void_p()
        assert lib.dsmc_pool_create(ctypes.byref(lim), None, None, 0, ctypes.byref(h)) == 1
    ok = D.PoolLimits(1 << 20, 10000, 64, 1000)
    assert lib.dsmc_pool_workspace_bytes(ctypes.byref(ok)) >= 32 * (1 << 20)
    i = ctypes.c_int()
    inst = D.make_instance(Kn=1.0, n_cells=10, ppc=10)
    assert lib.dsmc_pool_add(None, ctypes.byref(inst), ctypes.byref(i)) == 1
    assert lib.dsmc_pool_remove(None, 0) == 1
    assert lib.dsmc_channel_sums(None, None) == 1


def test_serve_arguments_are_checked(lib):
    so = D.serve_options()
    assert (so.epoch_steps, so.batches, so.max_active, so.time_limit) == (32, 16, 0, 0.0)
    inst = D.make_instance(Kn=1.0, n_cells=10, ppc=10)
    res = (D.RequestResult * 2)()
    reqs = (D.Request * 2)(D.Request(inst, 1.0, 0.01, 100), D.Request(inst, 0.5, 0.01, 100))
    # a NULL pool, then requests out of order, then bad targets: all rejected on the host
    assert lib.dsmc_serve(None, reqs, 2, ctypes.byref(so), res) == 1
    r1 = (D.Request * 1)(D.Request(inst, 0.0, 0.0, 100))
    assert lib.dsmc_solve(r1, None, ctypes.byref(so), res) == 1
    assert "target_se" in lib.dsmc_last_error().decode()
    bad = D.serve_options(batches=1)
    r2 = (D.Request * 1)(D.Request(inst, 0.0, 0.01, 100))
    assert lib.dsmc_solve(r2, None, ctypes.byref(bad), res) == 1


def test_surrogate_table_and_arguments(lib):
    """The library's own copy of Table 1 (typed from the paper) equals the printed one."""
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table1_exponents.txt"))
    for kn, b1, b2, b3 in rows:
        assert D.surrogate_exponents(kn) == (b1, b2, b3)
    h = ctypes.c_void_p()
    for args in ((0.0, 1e-3, 10, 5), (1.0, 0.0, 10, 5), (1.0, 1e-3, 2, 5), (1.0, 1e-3, 10, 0)):
        assert lib.dsmc_surrogate_create(*args, None, None, ctypes.byref(h)) == 1
    assert lib.dsmc_surrogate_train(None, None) == 1
    assert lib.dsmc_surrogate_destroy(None) == 0


def test_mms_arguments_are_checked(lib):
    p = D.MmsParams()
    assert lib.dsmc_default_mms_params(ctypes.byref(p)) == 0
    assert (p.dy, p.ppc, p.buffer, p.n_cfd) == (0.005, 50, 5, 200)
    r = D.MmsResult()
    prof = np.empty(200)
    p.Kn, p.body_force = 0.1, 0.0          # no force
    assert lib.dsmc_mms_run(ctypes.byref(p), None, prof.ctypes.data, None, 0, None,
                            ctypes.byref(r)) == 1
    p.body_force, p.Kn = 1e-3, 0.3          # 2 lambda + buffer above half the channel
    assert lib.dsmc_mms_run(ctypes.byref(p), None, prof.ctypes.data, None, 0, None,
                            ctypes.byref(r)) == 1
    assert "half the channel" in lib.dsmc_last_error().decode()
    assert lib.dsmc_set_open_top(None, 0, 0.0, 0.0) == 1


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.dsmc_step(None, 1) == 1
    assert lib.dsmc_sync(None) == 1
    assert lib.dsmc_destroy(None) == 0
    assert lib.dsmc_autotune(None, 1, None, None) == 1
    assert lib.dsmc_sample_moments_of(None, 0, None, None) == 1


def test_missing_library_fails_loudly(tmp_path):
    saved = D._lib
    try:
        D._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            D.load_library(str(tmp_path / "libdsmc.so"))
    finally:
        D._lib = saved


def _random_sums(rng, n_cells, n_samples, ppc, u=(0.01, -0.002, 0.0), P=0.003):
    """Raw sums of a sheared Maxwellian sample: per cell, count particles with velocity
    components N(u_i, 1/2) and a prescribed vx-vy covariance, summed as the sampler sums
    them (plain numpy; none of the method's arithmetic)."""
    out = np.zeros((n_cells, 13))
    for c in range(n_cells):
        n = n_samples * ppc + int(rng.integers(-ppc, ppc))
        cov = np.array([[0.5, P / 2, 0.0], [P / 2, 0.5, 0.0], [0.0, 0.0, 0.5]])
        v = rng.multivariate_normal(u, cov, size=n)
        v2 = (v ** 2).sum(1)
        x, y, z = v.T
        out[c] = [n, x.sum(), y.sum(), z.sum(), (x * x).sum(), (y * y).sum(), (z * z).sum(),
                  (x * y).sum(), (x * z).sum(), (y * z).sum(), (x * v2).sum(), (y * v2).sum(),
                  (z * v2).sum()]
    return out


def test_cell_fields_match_the_oracle_definitions(lib):
    """dsmc_cell_fields (host code of the library) against the oracle's plain numpy
    post-processing of the same raw sums, and against values known from the sample:
    density, mean velocity, temperature 1 (T0) of N(u, 1/2) components, shear stress
    2 n cov(vx, vy), zero heat flux of a Gaussian."""
    import oracle
    rng = np.random.default_rng(7)
    ppc, ns = 40, 25
    acc = _random_sums(rng, 6, ns, ppc)
    acc[3] = 0.0  # a cell that was never sampled
    got = D.fields(acc, ns, ppc)
    want = oracle.fields(acc, ns, ppc)
    for k in ("n", "ux", "uy", "uz", "T", "Pxy", "qx", "qy"):
        a, b = got[k], want[k]
        live = np.arange(6) != 3
        np.testing.assert_allclose(a[live], b[live], rtol=1e-12, atol=1e-15, err_msg=k)
        if k != "n":
            assert np.isnan(a[3]), k
    assert got["n"][3] == 0.0
    live = np.arange(6) != 3
    n_total = acc[live, 0]
    np.testing.assert_allclose(got["n"][live], n_total / (ns * ppc))
    # statistical agreement with the sampled distribution (1,000 particles per cell)
    assert np.all(np.abs(got["ux"][live] - 0.01) < 5 * np.sqrt(0.5 / n_total))
    assert np.all(np.abs(got["T"][live] - 1.0) < 0.2)
    assert np.all(np.abs(got["Pxy"][live] - 2 * got["n"][live] * 0.0015) < 0.2)
    assert np.all(np.abs(got["qz"][live]) < 0.2)


def test_cell_fields_reject_bad_arguments(lib):
    out = np.zeros((2, D.NFIELD))
    acc = np.ones((2, 13))
    assert lib.dsmc_cell_fields(D._ptr(acc), 0, 10, 2, D._ptr(out)) == 1
    assert lib.dsmc_cell_fields(D._ptr(acc), 5, 0, 2, D._ptr(out)) == 1
    assert lib.dsmc_cell_fields(None, 5, 10, 2, D._ptr(out)) == 1
