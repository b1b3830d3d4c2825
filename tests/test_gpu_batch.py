"""The batched form: many independent problems fitted by one graph launch.

Every problem is checked the way a single fit is: its labels must be the
oracle's FP64 argmin over its returned centroids, bit for bit, its objective
the oracle's J of that pair (1e-5), and the whole batch must equal the same
problems fitted one by one with KMeans (identical labels and iterations).
"""
import os

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


def _problems(n=8, seed0=100, n_hi=6000, k_hi=96):
    specs = synth.batched_problems(n, seed0=seed0, n_lo=500, n_hi=n_hi, k_lo=4, k_hi=k_hi)
    ws = [synth.batched_problem(s) for s in specs]
    return [(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.C0).cuda(), w.G) for w in ws], ws


def _final_check(w, lab, C, J):
    ref, _, _, _ = oracle.lloyd_assign(w.X.astype(np.float64), C.astype(np.float64))
    assert np.array_equal(lab, ref)
    _, _, Jref = oracle.lloyd_update(w.X.astype(np.float64), ref, C.astype(np.float64))
    assert abs(J - Jref) <= OBJECTIVE_RTOL * Jref + 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("algo", [0, 1], ids=["filtered", "lloyd"])
def test_batch_matches_oracle_and_single_fits(kp, algo):
    probs, ws = _problems()
    b = kp.KMeansBatch(probs, algo=algo)
    b.fit(25, 0.0)
    for i, ((X, C0, G), w) in enumerate(zip(probs, ws)):
        N, D, K = w.X.shape[0], w.X.shape[1], w.C0.shape[0]
        lab = torch.empty(N, dtype=torch.int32, device="cuda")
        C = torch.empty(K, D, device="cuda")
        J, n_it = b.get(i, lab, C)
        lab, C = lab.cpu().numpy(), C.cpu().numpy()
        _final_check(w, lab, C, J)
        km = kp.KMeans(X, C0, G, algo=algo)
        lab1 = torch.empty(N, dtype=torch.int32, device="cuda")
        r = km.fit(25, 0.0, lab1)
        km.close()
        assert r.n_iter == n_it, (i, r.n_iter, n_it)
        assert np.array_equal(lab1.cpu().numpy(), lab), i
    b.close()


@pytest.mark.gpu
def test_batch_reset_and_refit_repeat(kp):
    probs, ws = _problems(n=5, seed0=300)
    b = kp.KMeansBatch(probs)
    first = []
    for rep in range(2):
        if rep:
            b.reset()
        b.fit(20, 1e-4)
        out = []
        for i, w in enumerate(ws):
            lab = torch.empty(w.X.shape[0], dtype=torch.int32, device="cuda")
            J, n = b.get(i, lab)
            out.append((lab.cpu().numpy(), J, n))
        if rep == 0:
            first = out
        else:
            for (l0, J0, n0), (l1, J1, n1) in zip(first, out):
                assert n0 == n1 and np.array_equal(l0, l1)
                assert abs(J0 - J1) <= 1e-9 * J0
    b.close()


@pytest.mark.gpu
def test_batch_tuner_writes_and_reuses_cache(kp, tmp_path):
    probs, ws = _problems(n=6, seed0=500)
    cache = str(tmp_path / "tune.txt")
    b = kp.KMeansBatch(probs, tune_cache=cache)
    assert os.path.exists(cache)
    lines = [ln.split() for ln in open(cache) if ln.strip()]
    assert all(len(ln) == 6 for ln in lines), lines
    table = {(int(a), int(c), int(d)): (float(e), int(f), int(g)) for a, c, d, e, f, g in lines}
    for i, w in enumerate(ws):
        N, D = w.X.shape
        K = w.C0.shape[0]
        key = (D, int(np.ceil(np.log2(K))) if K > 1 else 0, int(np.ceil(np.log2(N))))
        assert key in table
        sw, dense, grab = table[key]
        assert b.switch(i) == pytest.approx(sw)
        assert sw in (0.5, 0.7, 0.9, 1.0)
        assert dense in (kp.KM_DENSE_AUTO, kp.KM_DENSE_FP32) and grab in (32, 64, 128)
        assert b.tuning(i) == (pytest.approx(sw), dense, grab)
    b.fit(10)
    b.close()
    # a second batch reads the cache instead of tuning again
    mtime = os.path.getmtime(cache)
    b2 = kp.KMeansBatch(probs, tune_cache=cache)
    assert os.path.getmtime(cache) == mtime
    b2.close()


@pytest.mark.gpu
def test_batch_rejects_bad_calls(kp):
    probs, _ = _problems(n=2, seed0=700)
    b = kp.KMeansBatch(probs)
    with pytest.raises(kp.KMeansError) as e:
        b.fit(0)
    assert e.value.status == kp.KM_EINVAL
    with pytest.raises(kp.KMeansError) as e:
        b.get(5)
    assert e.value.status == kp.KM_EINVAL
    b.close()


@pytest.mark.gpu
def test_batch_reads_older_cache_lines(kp, tmp_path):
    """A cache line of the older "D logK logN switch" form is read with the
    default engine and queue schedule."""
    probs, ws = _problems(n=3, seed0=800)
    cache = tmp_path / "old.txt"
    keys = {(w.X.shape[1], int(np.ceil(np.log2(w.C0.shape[0]))) if w.C0.shape[0] > 1 else 0,
             int(np.ceil(np.log2(w.X.shape[0])))) for w in ws}
    cache.write_text("".join(f"{d} {k} {n} 0.900\n" for d, k, n in sorted(keys)))
    b = kp.KMeansBatch(probs, tune_cache=str(cache))
    for i in range(len(ws)):
        assert b.tuning(i) == (pytest.approx(0.9), kp.KM_DENSE_AUTO, 32)
    b.fit(8)
    for i, w in enumerate(ws):
        lab = torch.empty(w.X.shape[0], dtype=torch.int32, device="cuda")
        C = torch.empty(w.C0.shape, device="cuda")
        J, _ = b.get(i, lab, C)
        _final_check(w, lab.cpu().numpy(), C.cpu().numpy(), J)
    b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("grab", [64, 128])
def test_survivor_queue_schedule_keeps_labels(kp, grab):
    """A larger survivor queue claim per warp changes only the schedule: the
    fit equals the default one label for label."""
    w = synth.anisotropic_1m(N=1 << 15, seed=4)
    X, C0 = torch.from_numpy(w.X).cuda(), torch.from_numpy(w.C0).cuda()
    out = []
    for g in (0, grab):
        opt = kp.kmeans_default_options()
        opt.surv_grab = g
        opt.dense_switch = 1.0
        ctx = kp.kmeans_init(X, w.N, w.D, w.K, w.G, C0, opt)
        lab = torch.empty(w.N, dtype=torch.int32, device="cuda")
        n_iter, J = kp.kmeans_fit(ctx, 12, 0.0, lab)
        st = [kp.kmeans_get_stats(ctx, t) for t in range(n_iter)]
        kp.kmeans_destroy(ctx)
        out.append((lab.cpu().numpy(), n_iter, J, [s["n_dist"] for s in st]))
    # the cluster sums take their FP64 atomic additions in another order, so
    # the objective may differ in the last bits; labels and iterations may not
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    assert abs(out[0][2] - out[1][2]) <= 1e-9 * out[0][2]
