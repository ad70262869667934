"""The FP64 fused multiply-add rate the FP64 particle pass is compared with."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_measured():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic

    build()
    a, b = pic.pic_fp64_fma_rate(2048), pic.pic_fp64_fma_rate(8192)
    # a GPU's FP64 rate: well above a CPU core, below GB300's FP32 rate
    assert 100.0 < a < 60000.0 and 100.0 < b < 60000.0
    # longer runs measure the same rate to within launch overhead
    assert abs(a - b) < 0.25 * max(a, b)
    with pytest.raises(pic.PicError):
        pic.pic_fp64_fma_rate(1)
