"""The square-root bounds behind every distance bound (u, lb; Sec. I).

The library bounds sqrt(v) by the hardware approximation moved two steps of
the bit pattern down / up.  kmeans_selftest_sqrt checks, on the device, that
lo >= 0 and lo^2 <= v <= hi^2 hold exactly for all 2^31 non-negative floats;
a failure there would void the exactness of every filter.
"""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    return kpynq


@pytest.mark.gpu
def test_sqrt_bounds_hold_for_every_float(kp):
    assert kp.kmeans_selftest_sqrt() == 0
