"""The error paths, made to happen without faulting the GPU.

* KM_ETIMEOUT: the bounded-wait self-test waits on an mbarrier that nothing
  arrives at; the wait must give up, the status must come back, and the
  device must stay usable (a fit right after it is exact).
* KM_ENOMEM: the allocation-failure hook makes the n-th device allocation of
  a context fail on the host side; kmeans_init must return KM_ENOMEM with a
  message, hand back no context, and leave the library usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1905_09345_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    oracle.build()
    return kpynq


def _small_fit_is_exact(kp):
    w = synth.small_blobs(N=3000, D=16, K=12, G=3, seed=5)
    km = kp.KMeans(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.C0).cuda(), w.G)
    lab = torch.empty(w.N, dtype=torch.int32, device="cuda")
    C = torch.empty(w.K, w.D, device="cuda")
    km.fit(10, 0.0, lab, C)
    km.close()
    ref, _, _, _ = oracle.lloyd_assign(w.X.astype(np.float64), C.cpu().numpy().astype(np.float64))
    return np.array_equal(lab.cpu().numpy(), ref)


def test_bounded_wait_times_out_and_device_stays_usable(kp):
    for polls in (1, 64, 1024):
        assert kp.kmeans_selftest_timeout(polls) == kp.KM_ETIMEOUT
        assert "gave up" in kp.kmeans_last_error(None)
    assert _small_fit_is_exact(kp)


@pytest.mark.parametrize("after", [0, 1, 5, 12])
def test_allocation_failure_returns_enomem(kp, after):
    w = synth.small_blobs(N=2000, D=16, K=8, G=2, seed=6)
    X, C0 = torch.from_numpy(w.X).cuda(), torch.from_numpy(w.C0).cuda()
    kp.kmeans_debug_fail_alloc(after)
    try:
        with pytest.raises(kp.KMeansError) as e:
            kp.KMeans(X, C0, w.G)
        assert e.value.status == kp.KM_ENOMEM
        assert kp.kmeans_last_error(None)
    finally:
        kp.kmeans_debug_fail_alloc(-1)
    assert _small_fit_is_exact(kp)
