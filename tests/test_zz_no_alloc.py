"""The allocation-free Lloyd step against the regular entry points.

``kmeans_lloyd_step_noalloc`` exists for callers that may not allocate device
memory: a host framework that owns all device memory through its own pool, a
latency-critical loop where cudaMalloc/cudaFree would synchronise the device,
or a deployment that reserves every byte at start-up.  It keeps its
intermediates in a static device array instead.  Here it is called twice in a
row through the C ABI (the second call starting from the first call's
centroids, so the shared scratch is reused) and each call is checked against
``kmeans_iterate`` on a plain-Lloyd context at the same centroids: labels
exactly, centroids within the parity tolerance (1e-5 relative), objective
within 1e-9 relative -- and against the FP64 oracle's assignment and update
(O1) from the same centroids.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

CENTROID_RTOL = 1e-5
OBJECTIVE_RTOL = 1e-9


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    return kpynq


def _data(N=20000, D=24, K=40, seed=11):
    from paper_1905_09345_gb300 import synth
    rng = np.random.default_rng(seed)
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=6.0, scale="fixed", scale_args=(1.0,))
    return X, synth.sample_init(rng, X, K)


@pytest.mark.gpu
def test_noalloc_step_matches_iterate_twice(kp, oracle_lib):
    oracle = oracle_lib
    X, C0 = _data()
    N, D = X.shape
    K = C0.shape[0]
    Xd = torch.from_numpy(X).cuda()
    km = kp.KMeans(Xd, torch.from_numpy(C0).cuda(), 4, algo=kp.KM_ALGO_LLOYD)
    C = torch.from_numpy(C0).cuda()
    labels = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    C_new = torch.empty(K, D, dtype=torch.float32, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref_lab = torch.empty(N, dtype=torch.int32, device="cuda")
    ref_C = torch.empty(K, D, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        st = km.iterate()
        km.labels(ref_lab)
        km.centroids(ref_C)
        kp.kmeans_lloyd_step_noalloc(Xd, N, D, C, K, labels, C_new, J, stream)
        torch.cuda.synchronize()
        assert torch.equal(labels, ref_lab), f"call {call}: labels differ"
        a = C_new.cpu().numpy().astype(np.float64)
        b = ref_C.cpu().numpy().astype(np.float64)
        assert np.abs(a - b).max() <= CENTROID_RTOL * max(1.0, np.abs(b).max()), f"call {call}"
        assert abs(J.item() - st["objective"]) <= OBJECTIVE_RTOL * st["objective"], f"call {call}"
        # the FP64 oracle from the same centroids: exact labels, means, J
        Cin = C.cpu().numpy().astype(np.float64)
        o_lab, _, _, _ = oracle.lloyd_assign(X, Cin)
        o_C, _, o_J = oracle.lloyd_update(X, o_lab, Cin)
        assert np.array_equal(labels.cpu().numpy(), o_lab), f"call {call}: labels differ from the oracle"
        assert np.abs(a - o_C).max() <= CENTROID_RTOL * max(1.0, np.abs(o_C).max()), f"call {call}"
        assert abs(J.item() - o_J) <= OBJECTIVE_RTOL * o_J, f"call {call}: {J.item()} vs {o_J}"
        C = C_new.clone()
    km.close()


@pytest.mark.gpu
def test_noalloc_step_rejects_oversize_and_host_memory(kp):
    X, C0 = _data(N=3000, D=8, K=16)
    Xd = torch.from_numpy(X).cuda()
    lab = torch.empty(3000, dtype=torch.int32, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = torch.zeros(2000, 8, device="cuda")
    with pytest.raises(kp.KMeansError) as e:  # K above the static limit
        kp.kmeans_lloyd_step_noalloc(Xd, 3000, 8, big, 2000, lab, torch.empty_like(big), J)
    assert e.value.status == kp.KM_EINVAL and "1024" in str(e.value)
    with pytest.raises(kp.KMeansError) as e:  # host memory is refused, not staged
        kp.kmeans_lloyd_step_noalloc(X, 3000, 8, C0, 16, lab, torch.empty(16, 8, device="cuda"), J)
    assert e.value.status == kp.KM_EINVAL
