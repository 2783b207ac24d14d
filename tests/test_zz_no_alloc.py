"""The allocation-free cell sort, dsmc_sort_cells_static, against the oracle's sort.

Who needs it: callers that cannot allocate device memory when they sort, for example
a plug-in running inside a host runtime that owns all GPU memory and lends it no
allocator, or a tight loop that must not pay the device-wide synchronisation that
cudaMalloc/cudaFree bring.  The entry point keeps its scratch in a fixed array inside
the library, so this test checks, through the C ABI, that it sorts exactly like the
oracle's stable counting sort (cell index of each particle by the oracle's own
binary32 rule, then a stable sort by cell) on several calls in a row, i.e. that
nothing a previous call left in the shared scratch leaks into the next result.
Sorting is index work, so the comparison is bit for bit.  The library's usual sort
(dsmc_load_state) is checked against the same expectation on the first call.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _state(rng, n):
    y = rng.random(n, dtype=np.float32)
    y[:: max(1, n // 7)] = 1.0  # particles on the top wall go to the last cell
    y[1:: max(1, n // 5)] = 0.0
    v = rng.normal(0.0, 0.7, size=(3, n)).astype(np.float32)
    return y, v[0].copy(), v[1].copy(), v[2].copy()


def _oracle_sort(host, n_cells):
    """Sorted arrays and offsets from the oracle alone (cell rule and stable sort)."""
    import oracle
    L = oracle.lib()
    cell = np.array([L.or_cell_of(float(v), n_cells) for v in host[0]], np.int32)
    perm, off = oracle.stable_cell_sort(cell, n_cells)
    return [a[perm] for a in host], off


def _entry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import _build
    from paper_2311_14140_gb300.dsmc import load_library
    _build.build()
    lib = load_library()
    fn = lib.dsmc_sort_cells_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 9 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return torch, lib, fn


def test_static_scratch_sort_matches_oracle_on_consecutive_calls():
    torch, lib, fn = _entry()
    from paper_2311_14140_gb300 import Dsmc
    stream = torch.cuda.current_stream()

    # Three calls in a row: a size, a larger one, then the first size with new data.
    for call, (n_cells, ppc, seed) in enumerate([(300, 97, 1), (2000, 60, 2), (300, 97, 3)]):
        rng = np.random.default_rng(seed)
        n = n_cells * ppc
        host = _state(rng, n)
        want, want_off = _oracle_sort(host, n_cells)
        dev_in = [torch.from_numpy(a).cuda() for a in host]
        dev_out = [torch.full((n,), np.nan, dtype=torch.float32, device="cuda") for _ in range(4)]
        offset = torch.full((n_cells + 1,), -7, dtype=torch.int32, device="cuda")
        st = fn(*[t.data_ptr() for t in dev_in], *[t.data_ptr() for t in dev_out],
                offset.data_ptr(), n, n_cells, stream.cuda_stream)
        assert st == 0, lib.dsmc_last_error().decode()
        torch.cuda.synchronize()
        got_off = offset.cpu().numpy()
        assert got_off[n_cells] == n  # no device-side error (else -1)
        np.testing.assert_array_equal(got_off, want_off)
        for name, got, exp in zip(("y", "vx", "vy", "vz"), dev_out, want):
            g = got.cpu().numpy()
            assert np.array_equal(g.view(np.uint32), exp.view(np.uint32)), (call, name)
        if call == 0:  # the handle's sort agrees with the same expectation
            ref = Dsmc(1.0, n_cells, ppc, seed=seed)
            ref.load_state(*host, step=0)
            for name, a, b in zip(("y", "vx", "vy", "vz"), ref.state(), want):
                assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), name
            np.testing.assert_array_equal(ref.cells()[0], want_off)
            ref.close()


def test_static_scratch_sort_rejects_sizes_and_overlaps():
    torch, lib, fn = _entry()
    n, n_cells = 64, 4
    bufs = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(8)]
    off = torch.zeros(n_cells + 1, dtype=torch.int32, device="cuda")
    p = [b.data_ptr() for b in bufs]
    ok_args = p[:4] + p[4:8] + [off.data_ptr()]
    assert fn(*ok_args, 16, 60000, None) == 1
    assert "51200" in lib.dsmc_last_error().decode()
    assert fn(*ok_args, 0, n_cells, None) == 1
    assert fn(None, *ok_args[1:], n, n_cells, None) == 1
    # an output equal to an input, or starting inside one
    bad = list(ok_args)
    bad[5] = p[1]  # vx_out = vx
    assert fn(*bad, n, n_cells, None) == 1
    assert "overlaps an input" in lib.dsmc_last_error().decode()
    bad = list(ok_args)
    bad[4] = p[0] + 4 * (n // 2)  # y_out inside y
    assert fn(*bad, n, n_cells, None) == 1
    bad = list(ok_args)
    bad[8] = p[3] + 8  # offsets inside vz
    assert fn(*bad, n, n_cells, None) == 1
    # two outputs sharing memory
    bad = list(ok_args)
    bad[7] = p[6] + 4  # vz_out inside vy_out
    assert fn(*bad, n, n_cells, None) == 1
    assert "two output arrays overlap" in lib.dsmc_last_error().decode()
    # the valid call still runs after the rejections
    assert fn(*ok_args, n, n_cells, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert off.cpu().numpy()[n_cells] == n
