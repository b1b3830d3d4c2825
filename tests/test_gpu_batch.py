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
    table = {(int(a), int(c), int(d)): float(e) for a, c, d, e in lines}
    for i, w in enumerate(ws):
        N, D = w.X.shape
        K = w.C0.shape[0]
        key = (D, int(np.ceil(np.log2(K))) if K > 1 else 0, int(np.ceil(np.log2(N))))
        assert key in table
        assert b.switch(i) == pytest.approx(table[key])
        assert table[key] in (0.5, 0.7, 0.9, 1.0)
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
