"""bfloat16-stored points (kmeans_options.dtype = KM_DTYPE_BF16).

The library widens the bfloat16 values to an exact FP32 copy at init, so a
fit on the bfloat16 bit patterns must equal, label for label and iteration
for iteration, a fit on the same values handed over as FP32; and the result
is checked against the oracle the way every fit is: labels equal to the
oracle's FP64 argmin over the returned centroids, objective within 1e-5 of
the oracle's J of that pair.  Covers host and device inputs, both dense
engines, and the widening itself (bit patterns read back through torch).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1905_09345_gb300 import synth  # noqa: E402

OBJECTIVE_RTOL = 1e-5


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    return kpynq


def _workload(N, D, K, seed):
    rng = np.random.default_rng(seed)
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="blob_lognormal",
                                  scale_args=(0.0, 0.5))
    X32 = synth.to_bf16(X)
    C0 = synth.sample_init(rng, X32, K)
    return X32, synth.bf16_bits(X), C0


def _fit(kp, X, C0, G, iters, **kw):
    N, K, D = X.shape[0], C0.shape[0], C0.shape[1]
    km = kp.KMeans(X, C0, G, **kw)
    lab = torch.empty(N, dtype=torch.int32, device="cuda")
    C = torch.empty(K, D, device="cuda")
    r = km.fit(iters, 0.0, lab, C)
    km.close()
    return r, lab.cpu().numpy(), C.cpu().numpy()


def _check_against_oracle(X32, lab, C, J):
    ref, _, _, _ = oracle.lloyd_assign(X32.astype(np.float64), C.astype(np.float64))
    assert np.array_equal(lab, ref)
    _, _, Jref = oracle.lloyd_update(X32.astype(np.float64), ref, C.astype(np.float64))
    assert abs(J - Jref) <= OBJECTIVE_RTOL * Jref + 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("N,D,K,G,dense", [
    (20000, 64, 128, 13, 0),     # tensor-core dense passes
    (20000, 64, 128, 13, 1),     # FP32 dense passes
    (9001, 128, 300, 30, 0),     # K > 256: FP32 dense passes, ragged tail
    (5003, 13, 40, 4, 0),        # D not a multiple of 4
], ids=["tc", "fp32", "k300", "d13"])
def test_bf16_fit_equals_fp32_fit_and_oracle(kp, N, D, K, G, dense):
    X32, bits, C0 = _workload(N, D, K, seed=N + D)
    r32, lab32, C32 = _fit(kp, torch.from_numpy(X32).cuda(), torch.from_numpy(C0).cuda(), G, 15, dense=dense)
    # device bfloat16 tensor (dtype inferred) and host uint16 bit patterns
    xb = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    rb, labb, Cb = _fit(kp, xb, torch.from_numpy(C0).cuda(), G, 15, dense=dense)
    rh, labh, Ch = _fit(kp, bits, C0, G, 15, dense=dense, dtype=kp.KM_DTYPE_BF16)
    for r, lab, C in ((rb, labb, Cb), (rh, labh, Ch)):
        assert r.n_iter == r32.n_iter
        assert np.array_equal(lab, lab32)
        np.testing.assert_allclose(C, C32, rtol=1e-6, atol=1e-6)
        _check_against_oracle(X32, lab, C, r.objective)


@pytest.mark.gpu
def test_bf16_widening_is_exact(kp):
    """The FP32 copy the library keeps holds exactly the bfloat16 values:
    with K = N every point is its own centroid after one assignment, so the
    returned centroids are the widened points themselves."""
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((64, 8)) * 3.0).astype(np.float32)
    X[0, :] = [0.0, 1e-30, -1e-30, 1e15, -1e15, 1.0 / 3.0, 65504.0, -7.0e-3]
    bits = synth.bf16_bits(X)
    X32 = synth.to_bf16(X)
    km = kp.KMeans(bits, X32.copy(), 4, dtype=kp.KM_DTYPE_BF16)
    C = torch.empty(64, 8, device="cuda")
    lab = torch.empty(64, dtype=torch.int32, device="cuda")
    km.fit(1, 0.0, lab, C)
    km.close()
    assert np.array_equal(lab.cpu().numpy(), np.arange(64))
    assert np.array_equal(C.cpu().numpy(), X32)
