"""k-means++ seeding on the GPU (kmeans_init_kmeanspp) against O4.

The draw is exact by construction (FP64 squared distances in the oracle's
summation order, integer weights, input uniforms), so the chosen indices must
equal O4's bit for bit, and the centroids must be those rows of X.  Shapes
cover one and many chunks of 1024 points, ragged N, K = N, and duplicated
points (all weights zero, so that the draw falls back to the uniform one).
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


def _seed(kp, X, K, u):
    N, D = X.shape
    C = torch.empty(K, D, dtype=torch.float32, device="cuda")
    idx = torch.empty(K, dtype=torch.int64, device="cuda")
    kp.kmeans_init_kmeanspp(torch.from_numpy(np.ascontiguousarray(X)).cuda(), N, D, K, u, C, idx)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), C.cpu().numpy()


CASES = [(5000, 16, 32, 1), (100003, 64, 256, 2), (1024, 3, 1024, 3), (777, 130, 40, 4), (262144, 64, 128, 5)]


@pytest.mark.parametrize("N,D,K,seed", CASES, ids=[f"N{c[0]}_D{c[1]}_K{c[2]}" for c in CASES])
def test_kmeanspp_matches_oracle(kp, N, D, K, seed):
    rng = np.random.default_rng(seed)
    X, _ = synth.gaussian_mixture(rng, N, D, max(2, min(K, 64)), centre_range=10.0, scale="fixed",
                                  scale_args=(1.0,))
    u = rng.uniform(size=K)
    idx, C = _seed(kp, X, K, u)
    ref, _ = oracle.kmeanspp(X.astype(np.float64), K, u)
    assert np.array_equal(idx, ref), np.flatnonzero(idx != ref)[:5]
    assert np.array_equal(C, X[ref])


def test_kmeanspp_duplicates_fall_back_to_uniform(kp):
    """Five distinct points, each ten times: after five centres every weight
    is zero and the draw is floor(u * N)."""
    rng = np.random.default_rng(8)
    base = rng.normal(size=(5, 4)).astype(np.float32)
    X = np.repeat(base, 10, axis=0)[rng.permutation(50)]
    u = rng.uniform(size=9)
    idx, C = _seed(kp, X, 9, u)
    ref, dmin = oracle.kmeanspp(X.astype(np.float64), 9, u)
    assert np.array_equal(idx, ref)
    assert np.all(dmin == 0.0)
    assert list(idx[5:]) == [int(np.floor(v * 50)) for v in u[5:]]


def test_fit_from_kmeanspp_centres(kp):
    """A filtered fit from the GPU-seeded centres: labels exact against the
    oracle over the returned centroids."""
    w = synth.anisotropic_1m(N=1 << 16)
    u = np.random.default_rng(3).uniform(size=w.K)
    _, C0 = _seed(kp, w.X, w.K, u)
    km = kp.KMeans(torch.from_numpy(w.X).cuda(), torch.from_numpy(C0).cuda(), w.G)
    lab = torch.empty(w.N, dtype=torch.int32, device="cuda")
    C = torch.empty(w.K, w.D, device="cuda")
    r = km.fit(30, 1e-4, lab, C)
    km.close()
    ref, _, _, _ = oracle.lloyd_assign(w.X.astype(np.float64), C.cpu().numpy().astype(np.float64))
    assert np.array_equal(lab.cpu().numpy(), ref)
    assert r.n_iter >= 1
