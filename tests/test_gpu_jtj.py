"""The standalone [J r]^T [J r] contraction (trk_jtj_rows) against an FP64 product of the same rows.

Tolerance: each entry is a sum of FP32 products formed and summed per CTA in FP32, so its error is a
few 1e-7 of the sum of the magnitudes of its terms; checked at 1e-5 of sqrt(diag_i diag_j)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _ref(J):
    J64 = J.astype(np.float64)
    return J64.T @ J64


def _run(J, nc, ld):
    n = J.shape[0]
    dev = torch.zeros((max(n, 1), ld), dtype=torch.float32, device="cuda")
    if n:
        dev[:n, :nc] = torch.from_numpy(J)
    out = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    trk.jtj_rows(dev.data_ptr(), n, nc, ld, out.data_ptr(), st.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n,nc,ld", [(50010, 56, 56), (1, 1, 1), (257, 80, 96), (100003, 33, 40), (300, 17, 17)])
def test_matches_fp64_product(n, nc, ld):
    rng = np.random.default_rng(n + nc)
    J = (rng.normal(size=(n, nc)) * rng.uniform(0.01, 1.0, nc)).astype(np.float32)
    got = _run(J, nc, ld)
    ref = _ref(J)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref))) + 1e-30
    assert (np.abs(got - ref) / scale).max() < 1e-5
    assert np.array_equal(got, got.T)


def test_zero_rows_give_zeros():
    got = _run(np.zeros((0, 8), np.float32), 8, 8)
    assert np.all(got == 0)


def test_invalid_arguments_are_rejected():
    with pytest.raises(trk.TrkError) as e:
        trk.jtj_rows(0, 10, 8, 8, 0, 0)
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
    dev = torch.zeros((4, 90), device="cuda")
    out = torch.zeros((90, 90), dtype=torch.float64, device="cuda")
    with pytest.raises(trk.TrkError):
        trk.jtj_rows(dev.data_ptr(), 4, 90, 90, out.data_ptr(), 0)
