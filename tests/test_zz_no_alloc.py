"""The allocation-free cell sort, dsmc_sort_cells_static, against the handle's sort.

Who needs it: callers that cannot allocate device memory when they sort, for example
a plug-in running inside a host runtime that owns all GPU memory and lends it no
allocator, or a tight loop that must not pay the device-wide synchronisation that
cudaMalloc/cudaFree bring.  The entry point keeps its scratch in a fixed array inside
the library, so this test checks, through the C ABI, that it sorts exactly like the
handle-based path (dsmc_load_state, the library's usual sort into cells) on several
calls in a row, i.e. that nothing a previous call left in the shared scratch leaks
into the next result.  Sorting is index work, so the comparison is bit for bit.
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


def test_static_scratch_sort_matches_handle_sort_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_14140_gb300 import Dsmc, _build
    from paper_2311_14140_gb300.dsmc import load_library
    _build.build()
    lib = load_library()
    fn = lib.dsmc_sort_cells_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 9 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    stream = torch.cuda.current_stream()

    # Three calls in a row: a size, a larger one, then the first size with new data.
    for call, (n_cells, ppc, seed) in enumerate([(300, 97, 1), (2000, 600, 2), (300, 97, 3)]):
        rng = np.random.default_rng(seed)
        n = n_cells * ppc
        host = _state(rng, n)
        dev_in = [torch.from_numpy(a).cuda() for a in host]
        dev_out = [torch.full((n,), np.nan, dtype=torch.float32, device="cuda") for _ in range(4)]
        offset = torch.full((n_cells + 1,), -1, dtype=torch.int32, device="cuda")
        st = fn(*[t.data_ptr() for t in dev_in], *[t.data_ptr() for t in dev_out],
                offset.data_ptr(), n, n_cells, stream.cuda_stream)
        assert st == 0, lib.dsmc_last_error().decode()
        torch.cuda.synchronize()

        ref = Dsmc(1.0, n_cells, ppc, seed=seed)  # any run of the right size
        ref.load_state(*host, step=0)
        want = ref.state()
        want_off = ref.cells()[0]
        ref.close()
        for name, got, exp in zip(("y", "vx", "vy", "vz"), dev_out, want):
            g = got.cpu().numpy()
            assert np.array_equal(g.view(np.uint32), exp.view(np.uint32)), (call, name)
        np.testing.assert_array_equal(offset.cpu().numpy(), want_off)


def test_static_scratch_sort_rejects_sizes_beyond_its_limits():
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
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    assert fn(p, p, p, p, p, p, p, p, p, 16, 60000, None) == 1
    assert "51200" in lib.dsmc_last_error().decode()
    assert fn(p, p, p, p, p, p, p, p, p, 0, 4, None) == 1
    assert fn(None, p, p, p, p, p, p, p, p, 16, 4, None) == 1
