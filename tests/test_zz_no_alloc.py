"""trk_jtj_rows_noalloc, the allocation-free [J r]^T [J r] entry point for callers that may not allocate
device memory, checked through the C ABI against trk_jtj_rows (which takes its scratch from the
stream-ordered allocator) on two calls in a row.  Collected last so that a stop at the first failure has
run every other test; it also passes alone in a fresh process (the first call does the per-device
set-up)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _call(name, rows, n, nc, ld, out, stream):
    lib = trk.lib()
    f = getattr(lib, name)
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(ctypes.c_void_p(rows), n, nc, ld, ctypes.c_void_p(out), ctypes.c_void_p(stream))


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(50010, 56, 56, 1), (3001, 33, 40, 2)]  # the second call uses a smaller, ragged case
    for n, nc, ld, seed in cases:
        rng = np.random.default_rng(seed)
        J = (rng.normal(size=(n, nc)) * rng.uniform(0.01, 1.0, nc)).astype(np.float32)
        rows = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
        rows[:, :nc] = torch.from_numpy(J)
        ref = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
        got = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
        assert _call("trk_jtj_rows", rows.data_ptr(), n, nc, ld, ref.data_ptr(), stream) == trk.TRK_OK
        assert _call("trk_jtj_rows_noalloc", rows.data_ptr(), n, nc, ld, got.data_ptr(), stream) == trk.TRK_OK
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        scale = np.sqrt(np.outer(np.diag(r), np.diag(r))) + 1e-30
        assert np.isfinite(g).all()
        assert (np.abs(g - r) / scale).max() < 1e-5  # the tolerance of the trk_jtj_rows tests


def test_noalloc_rejects_sizes_beyond_its_scratch():
    rows = torch.zeros((4, 96), dtype=torch.float32, device="cuda")
    out = torch.zeros((96, 96), dtype=torch.float64, device="cuda")
    st = _call("trk_jtj_rows_noalloc", rows.data_ptr(), 4, 81, 96, out.data_ptr(), 0)
    assert st == trk.TRK_ERR_INVALID_ARG
    assert b"n_cols" in trk.lib().trk_last_error()
