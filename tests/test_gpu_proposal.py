"""The learned group proposal (kmeans_set_proposal, kmeans_mlp_predict).

* (The network's own checks against O3 -- gradients, Adam, predictions --
  are in test_gpu_mlp.py.)
* A seeded iteration 0 keeps the filtered method exact: with a trained
  proposal, a random one and a deliberately wrong one, every fit equals the
  fit without a proposal (iterations, labels, objective) and its final
  labels are the oracle's FP64 argmin over the returned centroids.
* A trained proposal saves distance evaluations in iteration 0.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_1905_09345_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    return kpynq


def _dev_params(params):
    return {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in params.items()}


def _problem(seed=0, N=20000, D=32, K=256, G=26):
    rng = np.random.default_rng(seed)
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="blob_uniform", scale_args=(0.3, 1.5))
    C0 = synth.sample_init(rng, X, K)
    return X, C0, G


def _fit(kp, X, C0, G, params=None, iters=12):
    km = kp.KMeans(torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), G)
    if params is not None:
        km.set_proposal(_dev_params(params))
    lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    C = torch.empty(C0.shape, dtype=torch.float32, device="cuda")
    r = km.fit(iters, 0.0, lab, C)
    km.close()
    return r, lab.cpu().numpy(), C.cpu().numpy()


def test_seeded_iteration_zero_keeps_labels_exact(kp):
    X, C0, G = _problem()
    N, D = X.shape
    K = C0.shape[0]
    base, lab0, C_0 = _fit(kp, X, C0, G)
    # a trained proposal: O3 fitted to the groups of the oracle's final labels
    o = oracle.lloyd_fit(X.astype(np.float64), C0.astype(np.float64), 12)
    grp = oracle.contiguous_groups(K, G)
    y = grp[o["labels"]]
    trained = mlp.train(X[:8192], y[:8192], hidden=64, classes=G, seed=1, epochs=20, batch=512, lr=3e-3)
    rng = np.random.default_rng(9)
    random_ = mlp.init_params(D, 64, G, seed=2)
    wrong = {k: v.copy() for k, v in trained.items()}
    wrong["b3"] = wrong["b3"] + 1e3 * (np.arange(G) == rng.integers(0, G))  # always one fixed group
    for name, params in (("trained", trained), ("random", random_), ("wrong", wrong)):
        r, lab, C = _fit(kp, X, C0, G, params)
        assert r.n_iter == base.n_iter, name
        assert np.array_equal(lab, lab0), name
        assert abs(r.objective - base.objective) <= 1e-9 * base.objective, name
        ref, _, _, _ = oracle.lloyd_assign(X.astype(np.float64), C.astype(np.float64))
        assert np.array_equal(lab, ref), name
        if name == "trained":
            assert r.stats[0]["n_dist"] < 0.5 * N * K, r.stats[0]["n_dist"]
            assert r.stats[0]["path"] == kp.KM_PATH_FILTERED


def test_proposal_rejects_bad_calls(kp):
    X, C0, G = _problem(N=2000, K=32, G=4)
    params = _dev_params(mlp.init_params(X.shape[1], 16, G, seed=0))
    km = kp.KMeans(torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), G, algo=kp.KM_ALGO_LLOYD)
    with pytest.raises(kp.KMeansError) as e:
        km.set_proposal(params)
    assert e.value.status == kp.KM_EINVAL
    km.close()
    km = kp.KMeans(torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), G)
    with pytest.raises(kp.KMeansError) as e:
        kp.kmeans_set_proposal(km.ctx, params["W1"], None, params["W2"], params["b2"], params["W3"], params["b3"], 16)
    assert e.value.status == kp.KM_EINVAL
    km.set_proposal(params)
    km.set_proposal(None)  # removed again
    r = km.fit(5)
    assert r.stats[0]["path"] != kp.KM_PATH_FILTERED
    km.close()
