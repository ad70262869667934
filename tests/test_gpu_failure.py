"""Failure detection on the GPU without a fault: a bounded wait of the
library's grid barrier runs out (its partner block is never launched),
returns its status, and the context keeps working."""
import time

import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_2969_gb300 import build
    from paper_1001_2969_gb300 import pic as P

    build()
    return P


def test_bounded_wait_gives_up_and_the_context_stays_usable(pic):
    t0 = time.perf_counter()
    assert pic.pic_selftest_wait(1 << 16) is True
    assert time.perf_counter() - t0 < 10.0
    cfg = W.scaled(W.config("c1"), 2000)
    h = pic.pic_init(cfg)
    assert pic.pic_step(h, 2) == 0
    assert list(pic.pic_get_counts(h)["n_alive"]) != [0, 0]
    with pytest.raises(pic.PicError):
        pic.pic_selftest_wait(10)  # below the smallest limit
