"""The tensor-core contraction tile (tcgen05.mma, BF16 operands staged in
128-byte-swizzled shared memory, FP32 accumulators in TMEM) against an exact
product of the same BF16 values.  BF16 x BF16 products are exact in FP32, so
the only difference is the FP32 summation order: bounded by 256 u sum|a b|."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2009_01614_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("N", [16, 48, 128, 256])
def test_tile_matches_exact_product(built, N):
    g = torch.Generator().manual_seed(N)
    a = torch.randn(128, 256, generator=g).to(torch.bfloat16)
    b = torch.randn(N, 256, generator=g).to(torch.bfloat16)
    # structured rows: a row of ones and a one-hot column pin the layout
    a[0] = 1
    b[0] = 0
    b[0, 255] = 1
    ad, bd = a.cuda().contiguous(), b.cuda().contiguous()
    d = torch.empty(128, N, dtype=torch.float32, device="cuda")
    pkg.isax_tc_selftest(ad.data_ptr(), bd.data_ptr(), N, d.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    ref = a.double() @ b.double().T
    bound = 256 * 2.0 ** -24 * (a.double().abs() @ b.double().abs().T) + 1e-30
    err = (d.cpu().double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    np.testing.assert_array_equal(d[:, 0].cpu().numpy(), a[:, 255].float().numpy())
