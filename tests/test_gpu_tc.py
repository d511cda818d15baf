"""The tensor-core contraction [J r]^T [J r] (trk_jtj_rows_tc, Eqs. JTJ and JTr) against the oracle's FP64
normal equations of the same FP32 rows.

Error bound of an entry (a, b), from the arithmetic: each value x is split as hi + lo with
|x - hi - lo| <= u^2 |x| (u = 2^-8 for BF16, 2^-11 for TF32); the product drops lo_a lo_b, so each product
is off by at most 3 u^2 |x_a x_b|.  The products are summed in FP32 within a chain of at most 512 rows
(3 MMAs per row), then with Kahan compensation across chains and in FP64 across CTAs, which adds at most
(3 * 512 + 2) 2^-24 of sum_k |x_ka x_kb|.  So |err| <= (3 u^2 + 1538 * 2^-24) sum_k |x_ka x_kb|."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402

U = {trk.PRECISION_BF16X3: 2.0 ** -8, trk.PRECISION_TF32X3: 2.0 ** -11}


def _bound(prec):
    return 3 * U[prec] ** 2 + 1538 * 2.0 ** -24


def _rows(n, nc, seed):
    """Rows shaped like [J r]: columns of different scales (rotations about far joints are large,
    translations ~1, the residual ~1e-3), mixed signs."""
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(np.log(1e-3), np.log(2.0), nc))
    R = rng.normal(size=(n, nc)) * scale
    if nc > 1:
        R[:, -1] = rng.normal(scale=1.5e-3, size=n)
    return R.astype(np.float32)


def _ref(R):
    n, nc = R.shape
    JTJ, _ = oracle.normal_eq(R, np.zeros(n), np.ones(n, np.int32))
    return JTJ


def _run(R, nc, ld, prec):
    n = R.shape[0]
    dev = torch.zeros((max(n, 1), ld), dtype=torch.float32, device="cuda")
    if n:
        dev[:n, :nc] = torch.from_numpy(R)
    out = torch.full((nc, nc), np.nan, dtype=torch.float64, device="cuda")
    trk.jtj_rows_tc(dev.data_ptr(), n, nc, ld, prec, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [(50010, 56, 56), (1, 1, 1), (257, 80, 96), (100003, 33, 40), (300, 17, 17), (64, 16, 16), (65, 64, 64),
         (4097, 80, 80), (200000, 56, 60)]


@pytest.mark.parametrize("prec", [trk.PRECISION_BF16X3, trk.PRECISION_TF32X3])
@pytest.mark.parametrize("n,nc,ld", CASES)
def test_within_the_split_precision_bound(prec, n, nc, ld):
    R = _rows(n, nc, n + 7 * nc)
    got = _run(R, nc, ld, prec)
    ref = _ref(R)
    mag = np.abs(R.astype(np.float64)).T @ np.abs(R.astype(np.float64))
    err = np.abs(got - ref) / np.maximum(mag, 1e-300)
    print(f"prec {prec} n {n} nc {nc}: max rel err {err.max():.3e}, rms {np.sqrt((err ** 2).mean()):.3e}")
    assert np.isfinite(got).all()
    assert err.max() <= _bound(prec)


@pytest.mark.parametrize("prec", [trk.PRECISION_BF16X3, trk.PRECISION_TF32X3])
def test_lo_terms_are_used(prec):
    """Without the hi*lo products the error would be ~u = 2^-8 / 2^-11 of the magnitudes; the split keeps
    the typical error near u^2."""
    R = _rows(20000, 56, 3)
    got = _run(R, 56, 56, prec)
    ref = _ref(R)
    mag = np.abs(R.astype(np.float64)).T @ np.abs(R.astype(np.float64))
    rms = np.sqrt((((got - ref) / mag) ** 2).mean())
    assert rms < 4 * U[prec] ** 2


def test_deterministic_and_zero_rows():
    R = _rows(30001, 40, 11)
    a = _run(R, 40, 40, trk.PRECISION_BF16X3)
    b = _run(R, 40, 40, trk.PRECISION_BF16X3)
    assert np.array_equal(a, b)
    z = _run(np.zeros((0, 8), np.float32), 8, 8, trk.PRECISION_TF32X3)
    assert np.all(z == 0)


def test_invalid_arguments_are_rejected():
    dev = torch.zeros((4, 90), device="cuda")
    out = torch.zeros((90, 90), dtype=torch.float64, device="cuda")
    with pytest.raises(trk.TrkError) as e:
        trk.jtj_rows_tc(dev.data_ptr(), 4, 90, 90, trk.PRECISION_BF16X3, out.data_ptr(), 0)
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
    with pytest.raises(trk.TrkError) as e:
        trk.jtj_rows_tc(dev.data_ptr(), 4, 8, 8, trk.PRECISION_FP32, out.data_ptr(), 0)
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
