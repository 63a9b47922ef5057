"""The library's table-driven FP64 exponential against CUDA's exp, through the C ABI."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_exp_within_two_ulp_of_cuda_exp():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39 as C
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-60, 10, 1 << 20), rng.uniform(-1e-3, 1e-3, 1 << 16),
                        rng.uniform(-500, 500, 1 << 16),
                        [0.0, -0.0, 1e-300, -1e-300, 700.0, -700.0, 800.0, -800.0, np.inf,
                         -np.inf, np.nan, 1.0, -1.0, np.log(2.0)]])
    xd = torch.as_tensor(x, device="cuda")
    y = torch.empty_like(xd)
    ref = torch.empty_like(xd)
    s = torch.cuda.current_stream()
    C.check(C.lbm39_selftest_exp(xd.data_ptr(), y.data_ptr(), ref.data_ptr(), len(x),
                                 s.cuda_stream))
    torch.cuda.synchronize()
    y, ref = y.cpu().numpy(), ref.cpu().numpy()
    fin = np.isfinite(ref) & (ref > 1e-300)
    ulp = np.abs(y[fin] - ref[fin]) / np.spacing(ref[fin])
    assert ulp.max() <= 2.0, ulp.max()
    # special values follow CUDA's exp
    same = ~fin
    assert np.array_equal(np.isnan(y[same]), np.isnan(ref[same]))
    assert np.array_equal(y[same & ~np.isnan(ref)], ref[same & ~np.isnan(ref)])
