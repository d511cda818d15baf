"""trk_jtj_rows_noalloc, the allocation-free [J r]^T [J r] entry point for callers that may not allocate
device memory (a frame loop that must not call the CUDA allocator once running, or a host whose device
memory belongs to another allocator or a fixed budget).

Checked through the C ABI against an FP64 product of the same rows, at the tolerance of the
trk_jtj_rows tests (1e-5 of sqrt(diag_i diag_j)), on two calls in a row, and against trk_jtj_rows: bit
for bit while both use the same CTAs (n_rows <= 152 * 256), within that tolerance beyond.  Collected last
so that a stop at the first failure has run every other test; it also passes alone in a fresh process
(the first call does the per-device set-up)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402

SAME_CTAS_MAX_ROWS = 152 * 256


def _call(name, rows, n, nc, ld, out, stream):
    lib = trk.lib()
    f = getattr(lib, name)
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(ctypes.c_void_p(rows), n, nc, ld, ctypes.c_void_p(out), ctypes.c_void_p(stream))


def _rel_err(got, ref):
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref))) + 1e-30
    return (np.abs(got - ref) / scale).max()


def test_noalloc_matches_fp64_product_on_two_calls():
    stream = torch.cuda.current_stream().cuda_stream
    # 50,010 rows take all 152 CTAs of the fixed scratch (trk_jtj_rows would take 196); the second call
    # is a smaller, ragged case that leaves the first call's partials in the unused part of the scratch
    cases = [(50010, 56, 56, 1), (3001, 33, 40, 2)]
    for n, nc, ld, seed in cases:
        rng = np.random.default_rng(seed)
        J = (rng.normal(size=(n, nc)) * rng.uniform(0.01, 1.0, nc)).astype(np.float32)
        rows = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
        rows[:, :nc] = torch.from_numpy(J)
        alloc = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
        got = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
        assert _call("trk_jtj_rows_noalloc", rows.data_ptr(), n, nc, ld, got.data_ptr(), stream) == trk.TRK_OK
        assert _call("trk_jtj_rows", rows.data_ptr(), n, nc, ld, alloc.data_ptr(), stream) == trk.TRK_OK
        torch.cuda.synchronize()
        g, a = got.cpu().numpy(), alloc.cpu().numpy()
        J64 = J.astype(np.float64)
        ref = J64.T @ J64
        assert np.isfinite(g).all()
        assert _rel_err(g, ref) < 1e-5, (n, _rel_err(g, ref))
        assert np.array_equal(g, g.T)
        if n <= SAME_CTAS_MAX_ROWS:
            assert np.array_equal(g, a)
        else:
            assert _rel_err(g, a) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    rows = torch.zeros((4, 96), dtype=torch.float32, device="cuda")
    out = torch.zeros((96, 96), dtype=torch.float64, device="cuda")
    st = _call("trk_jtj_rows_noalloc", rows.data_ptr(), 4, 81, 96, out.data_ptr(), 0)
    assert st == trk.TRK_ERR_INVALID_ARG
    assert b"n_cols" in trk.lib().trk_last_error()
