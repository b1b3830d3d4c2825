"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Lockstep: before each iteration the GPU's centroids C^t are downloaded; the
oracle assigns every point to them in FP64 and must give exactly the GPU's
labels (the library settles every point the FP32 error bound cannot decide in
FP64, with the oracle's summation order, so no near-tie exception is needed;
near-ties are still counted).  The GPU's update C^{t+1} must match the
oracle's update of those labels within 1e-5 relative, and the GPU objective
J_t the oracle's J(a_t, C^t) within 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09345_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CENTROID_RTOL = 1e-5
OBJECTIVE_RTOL = 1e-9


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    oracle.build()
    return kpynq


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(1.0, np.abs(b).max()))


def get_C(km):
    out = torch.empty(km.K, km.D, dtype=torch.float32, device="cuda")
    return km.centroids(out).cpu().numpy().astype(np.float64)


def get_labels(km):
    out = torch.empty(km.N, dtype=torch.int32, device="cuda")
    return km.labels(out).cpu().numpy()


def tc_expected(D, K, G, smem=232448, algo=0):
    """Mirror of the tensor-core kernels' eligibility (shape and shared memory):
    one accumulator block for K <= 256, streamed centroid blocks above (both
    the filtered method and plain Lloyd)."""
    Dt = {32: 64, 64: 64, 128: 128}.get(D)  # operand copies zero-padded to 64 / 128
    if Dt is None:
        return False
    if K > 256:
        Kp = (K + 127) // 128 * 128
        if Kp > 4096:
            return False
        most = 0
        for j in range(Kp // 64):
            c0, c1 = 64 * j, min(64 * (j + 1), K) - 1
            if c0 >= K:
                break
            most = max(most, c1 * G // K - c0 * G // K + 1)
        srow = (most + 2) | 1
        na = Dt // 64
        a_stage = b_stage = 2 * na * 128 * 128
        stage = 2 * 4 * 32 * srow * 4
        for bst in (2, 1):
            off = 2 * a_stage + bst * b_stage + Kp * 8 + (Kp // 32 * 4 + 15) // 16 * 16 + stage
            off = (off + 7) // 8 * 8 + (4 + 2 * bst + 8 + 1) * 8 + 16
            if 1024 + off <= smem:
                return True
        return False
    Kp = (K + 31) // 32 * 32
    na = Dt // 64
    Gp = (G + 3) // 4 * 4
    fixed = 1024 + 2 * na * Kp * 128 + Kp * 4 + ((G + 1) * 4 + 15) // 16 * 16 + 2 * 128 * (Gp + 1) * 4 + 64 * 8 + 64
    return fixed + 2 * 2 * na * 128 * 128 <= smem


def lockstep(kp, X, C0, G, iters, algo=0, check_bounds=False, report=None, dense=0, dense_switch=0.0, grouping=0):
    """Run `iters` iterations in lockstep with the oracle; returns the list of
    per-iteration GPU stats."""
    N, D = X.shape
    K = C0.shape[0]
    km = kp.KMeans(dev(X), dev(C0), G, algo=algo, dense=dense, dense_switch=dense_switch, grouping=grouping)
    X64 = X.astype(np.float64)
    prev = None
    stats = []
    near = 0
    if grouping == kp.KM_GROUP_CLUSTERED:  # the library's grouping, in the caller's centroid numbering
        grp = np.empty(K, np.int32)
        G = km.groups(grp)
    else:
        grp = oracle.contiguous_groups(K, G)
    for t in range(iters):
        Ct = get_C(km)
        st = km.iterate()
        lab = get_labels(km)
        ref, d1, d2, ch = oracle.lloyd_assign(X64, Ct, prev)
        near += int(oracle.near_ties(d1, d2).sum()) if K > 1 else 0
        bad = np.flatnonzero(lab != ref)
        assert bad.size == 0, f"t={t}: {bad.size} labels differ, first {bad[:5]} gpu {lab[bad[:5]]} ref {ref[bad[:5]]}"
        assert st["n_changed"] == ch, (t, st["n_changed"], ch)
        assert st["iter"] == t
        Cn_ref, counts, J = oracle.lloyd_update(X64, ref, Ct)
        Cn = get_C(km)
        assert rel_err(Cn, Cn_ref) <= CENTROID_RTOL, (t, rel_err(Cn, Cn_ref))
        # FP32 centroids are the FP64 means rounded: within 2 ulp (plus the
        # FP64 summation-order difference for coordinates that cancel to ~0)
        tol = 2 * np.spacing(np.abs(Cn_ref).astype(np.float32)) + 1e-10 * (1 + np.abs(Cn_ref).max())
        assert np.all(np.abs(Cn - Cn_ref) <= tol), t
        assert abs(st["objective"] - J) <= OBJECTIVE_RTOL * J + 1e-12, (t, st["objective"], J)
        assert 0 <= st["n_dist"] <= N * K
        if check_bounds and algo == 0:
            u = np.empty(N, np.float32)
            lbg = np.empty(N, np.float32)
            lb = np.empty((N, G), np.float32)
            km.bounds(u, lbg, lb)
            dd = np.sqrt(np.maximum(((X64[:, None, :] - Cn[None, :, :]) ** 2).sum(-1), 0))
            da = dd[np.arange(N), lab]
            assert np.all(u >= da * (1 - 1e-12)), f"t={t}: upper bound below distance"
            dd[np.arange(N), lab] = np.inf
            assert np.all(lbg <= dd.min(1) * (1 + 1e-12)), f"t={t}: global lower bound above distance"
            for g in range(G):
                m = np.where((grp == g)[None, :], dd, np.inf).min(1)
                assert np.all(lb[:, g] <= m * (1 + 1e-12)), f"t={t}: group {g} lower bound above distance"
        if t > 0 and algo == 0 and dense_switch >= 1.0:
            assert st["path"] == kp.KM_PATH_FILTERED, (t, st["path"])
        if (t == 0 or algo == kp.KM_ALGO_LLOYD) and grouping == kp.KM_GROUP_CONTIGUOUS:
            want = kp.KM_PATH_DENSE_TC if (dense == 0 and tc_expected(D, K, G, algo=algo)) else kp.KM_PATH_DENSE_FP32
            assert st["path"] == want, (t, st["path"], want)
        stats.append(st)
        prev = ref
    if report is not None:
        report["near_ties"] = near
    km.close()
    return stats


def test_small_blobs_lockstep(kp):
    """Plain filtered K-means, FP32: N=16,384, D=16, K=16, G=2, 20 iterations."""
    w = synth.small_blobs()
    for sw in (0.0, 1.0):  # default dense switch; filtered path forced
        rep = {}
        st = lockstep(kp, w.X, w.C0, w.G, w.max_iter, report=rep, dense_switch=sw)
        assert st[0]["n_dist"] == w.N * w.K
        # the filters remove work once the centroids settle
        late = [s for s in st[5:] if s["path"] == kp.KM_PATH_FILTERED]
        assert late and sum(s["n_dist"] for s in late) < 0.5 * w.N * w.K * len(late)


def test_small_blobs_fit_matches_oracle_run(kp):
    w = synth.small_blobs()
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    lab = torch.empty(w.N, dtype=torch.int32, device="cuda")
    C = torch.empty(w.K, w.D, device="cuda")
    r = km.fit(w.max_iter, 0.0, lab, C)
    o = oracle.lloyd_fit(w.X, w.C0, w.max_iter, 0.0)
    assert r.n_iter == o["n_iter"]
    lab = lab.cpu().numpy()
    Cg = C.cpu().numpy().astype(np.float64)
    assert rel_err(Cg, o["centroids"]) <= CENTROID_RTOL
    # against the independent FP64 trajectory only near-ties may differ
    _, d1, d2, _ = oracle.lloyd_assign(w.X, o["centroids"])
    diff = o["labels"] != lab
    assert not np.any(diff & ~oracle.near_ties(d1, d2))
    assert abs(r.objective - o["objective"]) <= 1e-5 * o["objective"]
    # final labels / objective: exact against the returned centroids
    ref, _, _, _ = oracle.lloyd_assign(w.X, Cg)
    assert np.array_equal(lab, ref)
    assert abs(r.objective - oracle.lloyd_objective(w.X, lab, Cg)) <= OBJECTIVE_RTOL * r.objective
    for t, s in enumerate(r.stats):
        assert abs(s["objective"] - o["J_hist"][t]) <= 1e-5 * o["J_hist"][t]
    km.close()


EDGE = [
    # (N, D, K, G, iters) -- ragged sizes, every register width, generic D
    (1000, 3, 7, 2, 8),
    (1001, 17, 33, 5, 8),
    (2048, 64, 64, 64, 6),
    (2048, 64, 64, 1, 6),
    (777, 130, 20, 4, 6),
    (300, 8, 1, 1, 3),
    (2000, 1, 5, 2, 8),
    (3001, 128, 100, 10, 5),
    (4099, 32, 40, 40, 6),
    (513, 4, 9, 3, 10),
]


@pytest.mark.parametrize("dense", [0, 1], ids=["auto", "fp32"])
@pytest.mark.parametrize("N,D,K,G,iters", EDGE, ids=[f"N{e[0]}_D{e[1]}_K{e[2]}_G{e[3]}" for e in EDGE])
def test_edge_shapes_lockstep(kp, N, D, K, G, iters, dense):
    rng = np.random.default_rng(N * 7 + D)
    X, _ = synth.gaussian_mixture(rng, N, D, max(K, 2), centre_range=4.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    lockstep(kp, X, C0, G, iters, check_bounds=(N * K <= 200000), dense=dense,
             dense_switch=1.0 if dense else 0.0)


LLOYD_SHAPES = EDGE[:6] + [(5000, 64, 256, 26, 4), (3001, 32, 33, 4, 5),
                           # K > 256: streamed centroid blocks on the tensor cores
                           (5000, 64, 300, 30, 3), (3001, 128, 600, 60, 3), (4000, 32, 1024, 103, 2)]


@pytest.mark.parametrize("dense", [0, 1], ids=["auto", "fp32"])
@pytest.mark.parametrize("N,D,K,G,iters", LLOYD_SHAPES, ids=[f"N{e[0]}_D{e[1]}_K{e[2]}_G{e[3]}" for e in LLOYD_SHAPES])
def test_plain_lloyd_lockstep(kp, N, D, K, G, iters, dense):
    rng = np.random.default_rng(N * 11 + D)
    X, _ = synth.gaussian_mixture(rng, N, D, max(K, 2), centre_range=4.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    st = lockstep(kp, X, C0, G, iters, algo=kp.KM_ALGO_LLOYD, dense=dense)
    assert all(s["n_dist"] == N * K for s in st)


@pytest.mark.parametrize("D", [32, 64, 128])
def test_tensor_core_near_ties(kp, D):
    """Points placed (almost) half-way between two centroids, far from the
    origin so that the TF32 error window is wide: every one must be settled
    exactly (FP32, then FP64) to the oracle's label."""
    rng = np.random.default_rng(D)
    K, N = 96, 4096
    C0 = (rng.uniform(-3, 3, (K, D)) + 40.0).astype(np.float32)
    a = rng.integers(0, K, N)
    b = (a + 1 + rng.integers(0, K - 1, N)) % K
    w = (0.5 + rng.uniform(-1e-6, 1e-6, N))[:, None]
    X = (w * C0[a] + (1 - w) * C0[b] + rng.normal(0, 1e-4, (N, D))).astype(np.float32)
    X[: N // 8] = (0.5 * C0[a[: N // 8]] + 0.5 * C0[b[: N // 8]]).astype(np.float32)  # exact midpoints
    for algo in (0, 1):
        st = lockstep(kp, X, C0, 8, 2, algo=algo)
        assert st[0]["n_recheck"] > 0


@pytest.mark.parametrize("algo", [0, 1], ids=["filtered", "lloyd"])
@pytest.mark.parametrize("offset", [1e4, 1e5])
def test_objective_far_from_origin(kp, offset, algo):
    """Unit-spread blobs shifted by a large common offset (raw features are
    often far from the origin): the objective comes from per-cluster sums, and
    must still agree with the oracle's direct FP64 sum of squared distances
    within 1e-9 relative in every iteration (the lockstep check).  Summed
    about the origin, ||x||^2 / J per point is ~1e8-1e10 here, which a
    48-bit partial sum would turn into a relative error of up to ~1e-5."""
    rng = np.random.default_rng(int(offset) // 1000 + 7 * algo)
    N, D, K = 8192, 64, 32
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=10.0, scale="fixed", scale_args=(1.0,))
    X = (X.astype(np.float64) + offset).astype(np.float32)
    C0 = synth.sample_init(rng, X, K)
    st = lockstep(kp, X, C0, 4, 6, algo=algo)
    assert all(s["objective"] < 200.0 * N * D for s in st)  # J is O(N D centre_range^2), not O(N D offset^2)


@pytest.mark.parametrize("G", [12, 150])
def test_survivor_thread_per_point_d128(kp, G):
    """The thread-per-point survivor kernel at 128 coordinates (the point in
    registers; K = 600 centroids are too many for shared memory, so their rows
    are read through L1/L2), filtered path in every iteration after the first:
    with the bound rows prefetched into L1 (G = 12) and without (G = 150, rows
    too long for every resident thread's row to fit), labels, centroids and
    objective in lockstep with the oracle."""
    rng = np.random.default_rng(31 + G)
    N, D, K = 8192, 128, 600
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=6.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    st = lockstep(kp, X, C0, G, 6, dense_switch=1.0)
    assert any(s["path"] == kp.KM_PATH_FILTERED for s in st[1:])


def test_skewed_reduced_lockstep(kp):
    """The skewed workload's recipe at N=65,536 (power-law sizes, features on
    very different scales far from the origin, integer features, outliers,
    duplicates), from k-means++ centres: every iteration checked, with bounds
    on the filtered path throughout and with the default switch."""
    w = synth.skewed_mixture(N=1 << 16)
    idx, _ = oracle.kmeanspp(w.X.astype(np.float64), w.K, w.meta["pp_u"])
    C0 = w.X[idx]
    lockstep(kp, w.X, C0, w.G, 8)
    lockstep(kp, w.X, C0, w.G, 8, check_bounds=True, dense_switch=1.0)


CLUSTERED = [(3000, 16, 24, 5, 8, 0), (5000, 64, 256, 26, 6, 0), (4000, 128, 300, 30, 4, 0),
             (3001, 32, 600, 60, 4, 0), (2000, 8, 40, 8, 8, 1)]


@pytest.mark.parametrize("N,D,K,G,iters,dense", CLUSTERED, ids=[f"N{c[0]}_D{c[1]}_K{c[2]}_G{c[3]}_e{c[5]}" for c in CLUSTERED])
def test_clustered_grouping_lockstep(kp, N, D, K, G, iters, dense):
    """Groups of nearby centroids (KM_GROUP_CLUSTERED): the context orders its
    centroids group by group, yet labels (exact, in the caller's numbering),
    centroids and objective equal the oracle's every iteration, and every
    group bound holds for the library's groups -- on the survivor kernels for
    D <= 64 and D > 64, both tensor-core engines and the FP32 engine."""
    rng = np.random.default_rng(N + K)
    X, _ = synth.gaussian_mixture(rng, N, D, max(2, K // 2), centre_range=6.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    lockstep(kp, X, C0, G, iters, grouping=kp.KM_GROUP_CLUSTERED, dense=dense, check_bounds=N * K <= 1_500_000,
             dense_switch=1.0)
    lockstep(kp, X, C0, G, iters, grouping=kp.KM_GROUP_CLUSTERED, dense=dense)


@pytest.mark.parametrize("G,per,D,Gqs", [(10, 12, 8, (1, 4, 10, 30)), (40, 15, 40, (1, 33, 40, 70))])
def test_clustered_grouping_equals_oracle(kp, G, per, D, Gqs):
    """The library's clustered grouping (Lloyd over the centroids with its own
    kernels) is the oracle's, with empty groups dropped and the rest numbered
    in the order of their seeds; well-separated centroid clouds, so no group
    assignment is a near-tie.  The second case spans several member chunks of
    the update (K = 600) and more groups than a warp has lanes."""
    rng = np.random.default_rng(12)
    clouds = rng.uniform(-50, 50, (G, D))
    C0 = (clouds[rng.permutation(np.repeat(np.arange(G), per))] + rng.normal(0, 0.5, (G * per, D))).astype(np.float32)
    X = np.concatenate([C0, C0 + rng.normal(0, 0.1, C0.shape).astype(np.float32)])
    for Gq in Gqs:
        km = kp.KMeans(dev(X), dev(C0), Gq, grouping=kp.KM_GROUP_CLUSTERED)
        grp = np.empty(C0.shape[0], np.int32)
        ng = km.groups(grp)
        km.close()
        ref = oracle.clustered_groups(C0.astype(np.float64), Gq)
        used = np.unique(ref)  # ascending seed index
        ren = np.full(Gq, -1)
        ren[used] = np.arange(len(used))
        assert ng == len(used), (Gq, ng, len(used))
        assert np.array_equal(grp, ren[ref]), Gq


@pytest.mark.parametrize("D", [4, 64])
def test_clustered_grouping_exact_ties(kp, D):
    """Every centre given twice, the copies far apart in index order, with
    groups of nearby centroids: the copies land in the same group but at
    different positions of the context's order, and every point (equidistant
    from both copies in every iteration) must take the copy with the lower
    caller index."""
    rng = np.random.default_rng(15)
    k = 8
    centres = np.zeros((k, 2), np.float32)
    centres[:, 0] = np.arange(k) * 10 - 35
    centres[:, 1] = rng.choice(np.arange(-40, 41, 10), size=k)
    o = np.arange(-2, 3, dtype=np.float32)
    off = np.stack(np.meshgrid(o, o), -1).reshape(-1, 2)
    X = np.zeros((k * off.shape[0], D), np.float32)
    X[:, :2] = (centres[:, None, :] + off[None]).reshape(-1, 2)
    X = X[rng.permutation(X.shape[0])]
    C0 = np.zeros((2 * k, D), np.float32)
    perm = rng.permutation(k)
    C0[:k, :2] = centres[perm]
    C0[k:, :2] = centres[perm[::-1]]
    for sw in (0.0, 1.0):
        st = lockstep(kp, X, C0, 4, 4, dense_switch=sw, grouping=kp.KM_GROUP_CLUSTERED)
        assert all(s["n_recheck"] > 0 for s in st)


def test_bounds_stay_valid(kp):
    w = synth.small_blobs(N=3000, D=16, K=24, G=5, seed=4)
    lockstep(kp, w.X, w.C0, w.G, 12, check_bounds=True, dense_switch=1.0)
    lockstep(kp, w.X, w.C0, w.G, 12, check_bounds=True, dense_switch=0.01)


def test_exact_ties_go_to_lowest_index(kp):
    """Integer points and centroids placed symmetrically: many exact ties,
    including duplicated centroids; the lowest index must win everywhere."""
    g = np.arange(-6, 7, dtype=np.float32)
    X = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    X = np.concatenate([X, np.zeros((X.shape[0], 2), np.float32)], 1)  # D = 4
    C0 = np.array([[-1, 0, 0, 0], [1, 0, 0, 0], [0, -1, 0, 0], [0, 1, 0, 0], [-1, 0, 0, 0], [3, 3, 0, 0]],
                  np.float32)
    st = lockstep(kp, X, C0, 2, 6)
    assert st[0]["n_recheck"] > 0  # the ties went through the FP64 settle


@pytest.mark.parametrize("D", [4, 64])
@pytest.mark.parametrize("dense_switch", [0.0, 1.0])
def test_persistent_exact_ties(kp, D, dense_switch):
    """Blobs of integer offsets (symmetric about integer centres) and every
    centre given twice, the copies in the other group: each point is exactly
    as far from both copies in every iteration (the first copy's mean stays
    its centre, the second copy stays empty), so every iteration settles
    near-ties -- on the survivor path with the filters alone (dense_switch
    1), in the dense passes otherwise, where D = 64 runs on the tensor cores
    -- and the lowest index must win each time.  Many ties per warp exercise
    the warp-wide settles one request after another."""
    rng = np.random.default_rng(5)
    k = 8
    centres = rng.choice(np.arange(-40, 41, 10), size=(k, 2), replace=True).astype(np.float32)
    centres[:, 0] = np.arange(k) * 10 - 35  # distinct centres
    o = np.arange(-2, 3, dtype=np.float32)
    off = np.stack(np.meshgrid(o, o), -1).reshape(-1, 2)
    X = np.zeros((k * off.shape[0], D), np.float32)
    X[:, :2] = (centres[:, None, :] + off[None]).reshape(-1, 2)
    X = X[rng.permutation(X.shape[0])]
    C0 = np.zeros((2 * k, D), np.float32)
    C0[:k, :2] = centres
    C0[k:, :2] = centres
    st = lockstep(kp, X, C0, 2, 4, dense_switch=dense_switch)
    assert all(s["n_recheck"] > 0 for s in st), [s["n_recheck"] for s in st]
    if dense_switch >= 1.0:
        assert all(s["path"] == kp.KM_PATH_FILTERED for s in st[1:]), [s["path"] for s in st]
    if D == 64:
        assert st[0]["path"] == kp.KM_PATH_DENSE_TC


def test_k_equals_n(kp):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((64, 5)).astype(np.float32)
    km = kp.KMeans(dev(X), dev(X), 8)
    lab = torch.empty(64, dtype=torch.int32, device="cuda")
    r = km.fit(5, 0.0, lab)
    assert np.array_equal(lab.cpu().numpy(), np.arange(64))
    assert abs(r.objective) <= 1e-9 and r.n_iter == 2
    km.close()


def test_host_pointers_match_device_pointers(kp):
    w = synth.small_blobs(N=5000, D=16, K=16, G=4, seed=2)
    a = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    la = torch.empty(w.N, dtype=torch.int32, device="cuda")
    Ca = torch.empty(w.K, w.D, device="cuda")
    ra = a.fit(30, 1e-4, la, Ca)
    b = kp.KMeans(w.X, w.C0, w.G)  # NumPy (host) inputs
    lb_ = np.empty(w.N, np.int32)
    Cb = np.empty((w.K, w.D), np.float32)
    rb = b.fit(30, 1e-4, lb_, Cb)
    assert ra.n_iter == rb.n_iter
    assert np.array_equal(la.cpu().numpy(), lb_)
    assert np.allclose(Ca.cpu().numpy(), Cb, rtol=1e-6, atol=1e-6)
    assert abs(ra.objective - rb.objective) <= 1e-9 * ra.objective
    a.close()
    b.close()


def test_tol_stop_and_continue(kp):
    """fit() honours tol like the oracle, and a later fit() continues."""
    w = synth.small_blobs(N=8000, D=16, K=16, G=4, seed=5)
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    o = oracle.lloyd_fit(w.X, w.C0, 50, 1e-3)
    r = km.fit(50, 1e-3)
    assert r.n_iter == o["n_iter"]
    assert abs(r.objective - o["objective"]) <= 1e-5 * o["objective"]
    t0 = km.iteration
    r2 = km.fit(3, 0.0)
    assert km.iteration == t0 + r2.n_iter
    km.close()


def test_iterate_then_fit_and_max_iter_zero(kp):
    w = synth.small_blobs(N=4000, D=16, K=12, G=3, seed=6)
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    lab = torch.empty(w.N, dtype=torch.int32, device="cuda")
    r0 = km.fit(0, 0.0, lab)  # assignment to C0 only
    ref, _, _, _ = oracle.lloyd_assign(w.X, w.C0)
    assert r0.n_iter == 0 and np.array_equal(lab.cpu().numpy(), ref)
    km.close()
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    km.iterate()
    km.iterate()
    r = km.fit(40, 0.0, lab)
    o = oracle.lloyd_fit(w.X, w.C0, 42, 0.0)
    assert 2 + r.n_iter == o["n_iter"]
    assert np.array_equal(lab.cpu().numpy(), o["labels"])
    km.close()


def test_validate_rejects_nan(kp):
    X = np.ones((100, 4), np.float32)
    X[17, 2] = np.nan
    with pytest.raises(kp.KMeansError) as e:
        kp.KMeans(dev(X), dev(X[:4] * 0 + 1), 1, validate=True)
    assert e.value.status == kp.KM_EINVAL


def test_long_runs_rebase_and_grow_tables(kp):
    """More iterations than the drift tables hold at first (64 versions):
    the library rebases the lazy bounds (and grows the tables for a long
    fit) and the labels stay exact and the bounds valid."""
    w = synth.small_blobs(N=3000, D=8, K=40, G=6, seed=8)
    X64 = w.X.astype(np.float64)
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    for _ in range(70):
        Ct = get_C(km)
        km.iterate()
        ref, _, _, _ = oracle.lloyd_assign(X64, Ct)
        assert np.array_equal(get_labels(km), ref)
    assert km.iteration == 70
    r = km.fit(200, 0.0)  # needs more table rows than allocated: grows
    C = get_C(km)
    ref, _, _, _ = oracle.lloyd_assign(X64, C)
    assert np.array_equal(get_labels(km), ref)
    u = np.empty(w.N, np.float32)
    lbg = np.empty(w.N, np.float32)
    km.bounds(u, lbg)
    dd = np.sqrt(((X64[:, None, :] - C[None]) ** 2).sum(-1))
    lab = get_labels(km)
    assert np.all(u >= dd[np.arange(w.N), lab] * (1 - 1e-12))
    dd[np.arange(w.N), lab] = np.inf
    assert np.all(lbg <= dd.min(1) * (1 + 1e-12))
    assert r.n_iter >= 1
    km.close()


# ---------------------------------------------------------------------------
# the large workload: N=1,048,576, D=64, K=256, G=26
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def aniso():
    return synth.anisotropic_1m()


def test_aniso_reduced_lockstep(kp):
    """Same recipe at N=65,536: every iteration checked, with bounds."""
    w = synth.anisotropic_1m(N=1 << 16)
    lockstep(kp, w.X, w.C0, w.G, 8)
    st = lockstep(kp, w.X, w.C0, w.G, 8, dense_switch=1.0)  # filtered path throughout
    assert st[-1]["n_dist"] < 0.2 * w.N * w.K


def test_aniso_full_size(kp, aniso):
    """Full size, in the launch configuration the benchmark times: three
    lockstep iterations over all points, then the fit to convergence with
    sampled label checks and exact objective / centroid checks."""
    w = aniso
    X64 = w.X.astype(np.float64)
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    prev = None
    for t in range(2):
        Ct = get_C(km)
        st = km.iterate()
        lab = get_labels(km)
        ref, d1, d2, ch = oracle.lloyd_assign(X64, Ct, prev)
        assert np.array_equal(lab, ref), t
        assert st["n_changed"] == ch
        Cn_ref, _, J = oracle.lloyd_update(X64, ref, Ct)
        assert rel_err(get_C(km), Cn_ref) <= CENTROID_RTOL
        assert abs(st["objective"] - J) <= OBJECTIVE_RTOL * J
        prev = ref
    labt = torch.empty(w.N, dtype=torch.int32, device="cuda")
    Ct = torch.empty(w.K, w.D, device="cuda")
    r = km.fit(w.max_iter - 2, w.tol, labt, Ct)
    lab = labt.cpu().numpy()
    C = Ct.cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(0).choice(w.N, 1 << 15, replace=False)
    ref, _, _, _ = oracle.lloyd_assign(X64[idx], C)
    assert np.array_equal(lab[idx], ref)
    J = oracle.lloyd_objective(X64, lab, C)
    assert abs(r.objective - J) <= OBJECTIVE_RTOL * J
    assert all(s["path"] in (kp.KM_PATH_FILTERED, kp.KM_PATH_DENSE_TC) for s in r.stats)
    km.close()


def test_tensor_core_settle_many_groups(kp):
    """More than 64 groups: the tensor-core pass cannot name the window's
    groups in its 64-bit mask, so the settle kernel scans every centroid.
    Points near the midpoints of centroid pairs keep it busy."""
    rng = np.random.default_rng(21)
    N, D, K, G = 6000, 64, 256, 80
    C0 = (rng.uniform(-3, 3, (K, D)) + 25.0).astype(np.float32)
    a = rng.integers(0, K, N)
    b = (a + 1 + rng.integers(0, K - 1, N)) % K
    w = (0.5 + rng.uniform(-1e-3, 1e-3, N))[:, None]
    X = (w * C0[a] + (1 - w) * C0[b] + rng.normal(0, 1e-2, (N, D))).astype(np.float32)
    st = lockstep(kp, X, C0, G, 3, dense_switch=1e-6)  # dense in every iteration
    assert all(s["path"] == kp.KM_PATH_DENSE_TC for s in st)


def test_survivor_centroids_not_staged(kp):
    """K x D too large for the survivor kernel to stage the centroids in
    shared memory (1024 x 68 floats): the filtered path reads them from
    global memory."""
    rng = np.random.default_rng(22)
    N, D, K, G = 8000, 64, 1024, 100
    X, _ = synth.gaussian_mixture(rng, N, D, 256, centre_range=8.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    st = lockstep(kp, X, C0, G, 4, dense_switch=1.0)
    assert all(s["path"] == kp.KM_PATH_FILTERED for s in st[1:])


def test_final_assignment_stats(kp):
    """kmeans_get_stats(-1): the record of the last fit's final assignment."""
    w = synth.small_blobs(N=5000, D=16, K=12, G=3, seed=7)
    km = kp.KMeans(dev(w.X), dev(w.C0), w.G)
    with pytest.raises(kp.KMeansError) as e:
        km.final_stats()
    assert e.value.status == kp.KM_ESTATE
    r = km.fit(30, 1e-4)
    f = km.final_stats()
    assert f["iter"] == r.n_iter and f["done"] == 1
    assert f["path"] in (kp.KM_PATH_FILTERED, kp.KM_PATH_DENSE_FP32, kp.KM_PATH_DENSE_TC)
    assert abs(f["objective"] - r.objective) <= 1e-12 * r.objective
    km.reset(dev(w.C0))
    with pytest.raises(kp.KMeansError):
        km.final_stats()
    km.close()


# more centroids than one accumulator block: the tensor-core pass streams the
# centroids in blocks of 128 (ragged tails, several tiles per CTA, G over 64,
# a single group)
KBLOCKED = [
    (40000, 64, 300, 30, 4),
    (100003, 128, 520, 100, 3),
    (20000, 64, 1024, 103, 3),
    (5000, 128, 257, 1, 3),
    (30000, 32, 600, 60, 3),   # 32 coordinates, zero-padded to 64 in the operand copies
]


@pytest.mark.parametrize("N,D,K,G,iters", KBLOCKED, ids=[f"N{e[0]}_D{e[1]}_K{e[2]}_G{e[3]}" for e in KBLOCKED])
def test_kblocked_tensor_core_lockstep(kp, N, D, K, G, iters):
    rng = np.random.default_rng(N + K)
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="blob_lognormal", scale_args=(0.0, 0.5))
    C0 = synth.sample_init(rng, X, K)
    st = lockstep(kp, X, C0, G, iters, check_bounds=(N * K <= 25_000_000))
    assert st[0]["path"] == kp.KM_PATH_DENSE_TC


def test_kblocked_matches_fp32_engine_and_near_ties(kp):
    """Points half-way between two of 300 centroids: the streamed tensor-core
    pass must queue them, and the settle (candidates from the written group
    bounds) must give the oracle's labels; the whole fit equals the FP32
    engine's."""
    rng = np.random.default_rng(77)
    K, N, D = 300, 30000, 64
    C0 = (rng.uniform(-3, 3, (K, D)) + 40.0).astype(np.float32)
    a = rng.integers(0, K, N)
    b = (a + 1 + rng.integers(0, K - 1, N)) % K
    w = (0.5 + rng.uniform(-1e-6, 1e-6, N))[:, None]
    X = (w * C0[a] + (1 - w) * C0[b] + rng.normal(0, 1e-4, (N, D))).astype(np.float32)
    X[: N // 8] = (0.5 * C0[a[: N // 8]] + 0.5 * C0[b[: N // 8]]).astype(np.float32)
    st = lockstep(kp, X, C0, 30, 2)
    assert st[0]["n_recheck"] > 0 and st[0]["n_settle"] > 0
    outs = []
    for dense in (0, 1):
        km = kp.KMeans(dev(X), dev(C0), 30, dense=dense)
        lab = torch.empty(N, dtype=torch.int32, device="cuda")
        r = km.fit(6, 0.0, lab)
        outs.append((r.n_iter, lab.cpu().numpy(), r.objective))
        km.close()
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    assert abs(outs[0][2] - outs[1][2]) <= 1e-9 * outs[1][2]


@pytest.mark.parametrize("D,K", [(64, 48), (32, 300), (17, 20)], ids=["tc", "tc_streamed", "fp32"])
def test_pinned_host_input_matches_device(kp, D, K):
    """Page-locked host X: the tensor-core split reads it directly and makes the
    device copy in the same pass; the fit must equal the one from device X."""
    rng = np.random.default_rng(D + K)
    N = 7001
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=10.0, scale="fixed", scale_args=(1.0,))
    C0 = synth.sample_init(rng, X, K)
    outs = []
    for src in (torch.from_numpy(X).cuda(), torch.from_numpy(X).pin_memory()):
        km = kp.KMeans(src, torch.from_numpy(C0).cuda(), max(1, K // 10))
        lab = torch.empty(N, dtype=torch.int32, device="cuda")
        r = km.fit(10, 0.0, lab)
        outs.append((r.n_iter, lab.cpu().numpy(), r.objective))
        km.close()
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    assert abs(outs[0][2] - outs[1][2]) <= 1e-9 * outs[0][2]
