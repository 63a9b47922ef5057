"""The step's reciprocals against CUDA's division, through the C ABI: the FP64 one (Newton's
method from the hardware estimate; 1/rho and the pivots of the Newton solve) within 2 ulp, and
the FP32 one of the Knudsen-sensor screen within the 1 ulp its error bound assumes."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_reciprocals_against_cuda_division():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39 as C
    rng = np.random.default_rng(11)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 1 << 20)),
                        rng.uniform(0.05, 20.0, 1 << 18),        # densities and pivots
                        -np.exp(rng.uniform(-20, 20, 1 << 16)),  # negative values
                        2.0 ** np.arange(-100, 101), [1.0, 3.0, 0.1, 1.4, 0.6004]])
    xd = torch.as_tensor(x, device="cuda")
    y, ref = torch.empty_like(xd), torch.empty_like(xd)
    y32 = torch.empty(len(x), dtype=torch.float32, device="cuda")
    ref32 = torch.empty_like(y32)
    s = torch.cuda.current_stream()
    C.check(C.lbm39_selftest_rcp(xd.data_ptr(), y.data_ptr(), ref.data_ptr(), y32.data_ptr(),
                                 ref32.data_ptr(), len(x), s.cuda_stream))
    torch.cuda.synchronize()
    y, ref, y32, ref32 = (t.cpu().numpy() for t in (y, ref, y32, ref32))
    ulp = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 2.0, ulp.max()
    assert np.array_equal(y[-206:-5], ref[-206:-5])  # powers of two are exact
    ulp32 = np.abs(y32.astype(np.float64) - ref32) / np.spacing(np.abs(ref32))
    assert ulp32.max() <= 1.0, ulp32.max()
