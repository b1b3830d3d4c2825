"""Pins for the FP64 oracle, independent of the oracle's own code.

Each check below is fixed by something other than the oracle itself: a
hand-derived worked example, a closed form, an independent library routine
(scipy ``cdist``, numpy ``bincount``, scikit-learn's Lloyd), an invariant of
Lloyd's algorithm, or -- for the filtered oracle O2 -- the brute-force oracle O1
it must equal label-for-label (the filters of KPynq, Sec. I, only remove
distance computations).  ``test_planted_mistakes_are_caught`` compiles copies of
the oracle with one plausible mistake each and checks that some pin fails.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lloyd_worked_examples.json")


def _rng_data(seed, N, D, K, spread=3.0):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-spread, spread, (K, D))
    X = centres[rng.integers(0, K, N)] + rng.standard_normal((N, D))
    C0 = X[rng.choice(N, K, replace=False)]
    return X, C0


# ---------------------------------------------------------------------------
# pin checks: each returns a list of failure messages (empty = pass)
# ---------------------------------------------------------------------------
def check_golden(lib=None):
    bad = []
    for case in json.load(open(GOLDEN))["cases"]:
        X = np.array(case["X"], np.float64)
        C0 = np.array(case["C0"], np.float64)
        r = oracle.lloyd_fit(X, C0, case["max_iter"], case["tol"], lib=lib)
        nm = case["name"]
        if r["n_iter"] != case["n_iter"]:
            bad.append(f"{nm}: n_iter {r['n_iter']} != {case['n_iter']}")
            continue
        if not np.allclose(r["J_hist"], case["J_hist"], rtol=1e-13, atol=1e-12):
            bad.append(f"{nm}: J_hist {r['J_hist']} != {case['J_hist']}")
        if list(r["changed_hist"]) != case["changed_hist"]:
            bad.append(f"{nm}: changed {r['changed_hist']} != {case['changed_hist']}")
        if list(r["labels"]) != case["labels"]:
            bad.append(f"{nm}: labels {r['labels']} != {case['labels']}")
        if not np.allclose(r["centroids"], case["centroids"], rtol=1e-14, atol=1e-14):
            bad.append(f"{nm}: centroids {r['centroids'].tolist()}")
        if not np.isclose(r["objective"], case["objective"], rtol=1e-13, atol=1e-12):
            bad.append(f"{nm}: objective {r['objective']} != {case['objective']}")
    return bad


def check_assign_vs_cdist(lib=None):
    bad = []
    for seed, (N, D, K) in enumerate([(500, 7, 13), (300, 1, 4), (200, 33, 9)]):
        X, C0 = _rng_data(100 + seed, N, D, K)
        C = C0 + 0.37  # centroids away from the data points
        labels, d1, d2, ch = oracle.lloyd_assign(X, C, lib=lib)
        ref = cdist(X, C, "sqeuclidean")
        srt = np.sort(ref, axis=1)
        if not np.array_equal(labels, np.argmin(ref, axis=1)):
            bad.append(f"assign labels differ from cdist argmin ({N},{D},{K})")
        if not np.allclose(d1, srt[:, 0], rtol=1e-12) or not np.allclose(d2, srt[:, 1], rtol=1e-12):
            bad.append(f"assign top-2 distances differ from cdist ({N},{D},{K})")
        if ch != N:
            bad.append("changed count without prev != N")
    return bad


def check_update_vs_bincount(lib=None):
    bad = []
    X, C0 = _rng_data(7, 400, 5, 10)
    labels = np.random.default_rng(8).integers(0, 9, 400).astype(np.int32)  # cluster 9 empty
    C_new, counts, J = oracle.lloyd_update(X, labels, C0, lib=lib)
    cnt = np.bincount(labels, minlength=10)
    S = np.zeros((10, 5))
    np.add.at(S, labels, X)
    ref = np.where(cnt[:, None] > 0, S / np.maximum(cnt, 1)[:, None], C0)
    if not np.allclose(C_new, ref, rtol=1e-13, atol=1e-13):
        bad.append("update differs from bincount means")
    if not np.array_equal(counts, cnt):
        bad.append("update counts differ from bincount")
    Jref = float(np.sum((X - C0[labels]) ** 2))
    if not np.isclose(J, Jref, rtol=1e-12):
        bad.append(f"update J {J} != {Jref} (must use the assigning centroids)")
    return bad


def check_closed_forms(lib=None):
    bad = []
    X, _ = _rng_data(11, 257, 6, 3)
    r = oracle.lloyd_fit(X, X[:1], 5, 0.0, lib=lib)
    mu = X.mean(axis=0)
    if not np.allclose(r["centroids"][0], mu, rtol=1e-13, atol=1e-13):
        bad.append("K=1 centroid != mean")
    if not np.isclose(r["objective"], X.shape[0] * X.var(axis=0).sum(), rtol=1e-11):
        bad.append("K=1 objective != N * total variance")
    if r["n_iter"] != 2:
        bad.append(f"K=1 n_iter {r['n_iter']} != 2")
    Y, _ = _rng_data(12, 40, 3, 4)
    r = oracle.lloyd_fit(Y, Y, 5, 0.0, lib=lib)
    if not np.array_equal(r["labels"], np.arange(40)) or r["objective"] != 0.0 or r["n_iter"] != 2:
        bad.append("K=N with C0=X must give identity labels, J=0, n_iter=2")
    return bad


def check_blobs_recovered(lib=None):
    bad = []
    rng = np.random.default_rng(5)
    K, D = 6, 4
    centres = rng.uniform(-1000, 1000, (K, D))
    blob = np.repeat(np.arange(K), 50)
    X = centres[blob] + rng.standard_normal((K * 50, D))
    C0 = X[[50 * k + 3 for k in range(K)]]
    r = oracle.lloyd_fit(X, C0, 20, 0.0, lib=lib)
    if not np.array_equal(r["labels"], blob):
        bad.append("separated blobs not recovered")
    means = np.stack([X[blob == k].mean(0) for k in range(K)])
    if not np.allclose(r["centroids"], means, rtol=1e-12, atol=1e-9):
        bad.append("blob centroids != blob means")
    return bad


def check_lloyd_invariants(lib=None):
    bad = []
    for seed in range(3):
        X, C0 = _rng_data(20 + seed, 600, 4, 12, spread=2.0)
        r = oracle.lloyd_fit(X, C0, 200, 0.0, lib=lib)
        Jh = r["J_hist"]
        if np.any(np.diff(Jh) > 1e-12 * Jh[:-1]):
            bad.append("objective increased")
        if r["n_iter"] >= 200:
            bad.append("did not converge")
            continue
        lab = r["labels"]
        d = cdist(X, r["centroids"], "sqeuclidean")
        if not np.array_equal(lab, np.argmin(d, axis=1)):
            bad.append("converged labels are not nearest centroids")
        for k in range(12):
            if np.any(lab == k) and not np.allclose(r["centroids"][k], X[lab == k].mean(0), rtol=1e-12, atol=1e-12):
                bad.append("converged centroid is not the mean of its points")
                break
        if not np.isclose(r["objective"], d[np.arange(600), lab].sum(), rtol=1e-12):
            bad.append("final objective != sum of nearest squared distances")
    return bad


def check_sklearn(lib=None):
    sk = pytest.importorskip("sklearn.cluster")
    bad = []
    for seed in range(3):
        X, C0 = _rng_data(30 + seed, 2000, 5, 8)
        m = 40
        r = oracle.lloyd_fit(X, C0, m, 0.0, lib=lib)
        km = sk.KMeans(n_clusters=8, init=C0, n_init=1, max_iter=m, tol=0.0, algorithm="lloyd")
        km.fit(X)
        if km.n_iter_ != r["n_iter"]:
            bad.append(f"sklearn n_iter {km.n_iter_} != {r['n_iter']}")
        if not np.array_equal(km.labels_, r["labels"]):
            bad.append("sklearn labels differ")
        if not np.allclose(km.cluster_centers_, r["centroids"], rtol=1e-9, atol=1e-9):
            bad.append("sklearn centroids differ")
        if not np.isclose(km.inertia_, r["objective"], rtol=1e-9):
            bad.append("sklearn inertia differs")
    return bad


def _o1_trajectory(X, C0, max_iter, tol, lib=None):
    """O1 step by step: labels of every iteration."""
    C = np.array(C0, np.float64)
    hist, Js, prev, Jp = [], [], None, 0.0
    for t in range(max_iter):
        lab, _, _, ch = oracle.lloyd_assign(X, C, prev, lib=lib)
        C, _, J = oracle.lloyd_update(X, lab, C, lib=lib)
        hist.append(lab)
        Js.append(J)
        prev = lab
        stop = ch == 0 or (t >= 1 and (Jp - J) < tol * Jp)
        Jp = J
        if stop:
            break
    return np.array(hist), np.array(Js), C


def check_ti_equals_lloyd(lib_ti=None, lib=None):
    bad = []
    cases = [(0, 500, 4, 20), (1, 800, 8, 32), (2, 300, 2, 7), (3, 600, 16, 50)]
    for seed, N, D, K in cases:
        X, C0 = _rng_data(40 + seed, N, D, K, spread=4.0)
        hist, Js, C = _o1_trajectory(X, C0, 60, 0.0, lib=lib)
        for G in sorted({1, 2, max(1, K // 10), K}):
            r = oracle.ti_fit(X, C0, G, 60, 0.0, lib=lib_ti)
            if r["n_iter"] != len(hist):
                bad.append(f"O2 n_iter {r['n_iter']} != O1 {len(hist)} (K={K},G={G})")
                continue
            if not np.array_equal(r["labels_hist"], hist):
                t = int(np.argmax(np.any(r["labels_hist"] != hist, axis=1)))
                bad.append(f"O2 labels differ from O1 at iteration {t} (K={K},G={G})")
            if not np.allclose(r["J_hist"], Js, rtol=1e-12):
                bad.append(f"O2 J differs (K={K},G={G})")
            if not np.allclose(r["centroids"], C, rtol=1e-13, atol=1e-13):
                bad.append(f"O2 centroids differ (K={K},G={G})")
    return bad


def check_ti_bounds(lib_ti=None):
    """u >= d(x, c_a) and lb_g <= min_{c in g, c != a} d(x, c) after every
    assignment (distances from scipy cdist)."""
    bad = []
    for seed, (N, D, K, G) in enumerate([(400, 3, 24, 5), (300, 6, 16, 16), (300, 2, 9, 1)]):
        X, C0 = _rng_data(60 + seed, N, D, K, spread=3.0)
        st = oracle.TIState(X, C0, G, lib=lib_ti)
        for t in range(15):
            st.assign()
            d = cdist(st.X, st.C)
            da = d[np.arange(N), st.a]
            if np.any(st.u < da * (1 - 1e-12)):
                bad.append(f"upper bound below d(x, c_a) at t={t}")
                break
            for g in range(G):
                mask = st.grp == g
                dd = np.where(mask[None, :], d, np.inf)
                dd[np.arange(N), st.a] = np.inf
                if np.any(st.lb[:, g] > dd.min(axis=1) * (1 + 1e-12) + 1e-300):
                    bad.append(f"group lower bound above min distance at t={t}, g={g}")
                    break
            st.update()
    return bad


def check_ti_skips(lib_ti=None):
    """On separated blobs the filters must remove most distance evaluations."""
    bad = []
    rng = np.random.default_rng(9)
    K, D, per = 40, 8, 60
    centres = rng.uniform(-50, 50, (K, D))
    X = centres[np.repeat(np.arange(K), per)] + rng.standard_normal((K * per, D))
    C0 = X[rng.choice(K * per, K, replace=False)]
    r = oracle.ti_fit(X, C0, 4, 100, 0.0, lib=lib_ti)
    c = r["cnt_hist"]
    frac = c[:, oracle.CNT_DIST].sum() / (K * per * K * r["n_iter"])
    if frac > 0.5:
        bad.append(f"filtered oracle evaluated {frac:.2f} of all distances")
    if c[-1, oracle.CNT_GLOBAL] + c[-1, oracle.CNT_TIGHT] < 0.5 * K * per:
        bad.append("global filter kept < 50% of points at the last iteration")
    return bad


def check_ti_golden(lib_ti=None):
    """The filtered oracle on the hand-derived examples, for every G."""
    bad = []
    for case in json.load(open(GOLDEN))["cases"]:
        X = np.array(case["X"], np.float64)
        C0 = np.array(case["C0"], np.float64)
        for G in range(1, C0.shape[0] + 1):
            r = oracle.ti_fit(X, C0, G, case["max_iter"], case["tol"], lib=lib_ti)
            nm = f"{case['name']} G={G}"
            if r["n_iter"] != case["n_iter"]:
                bad.append(f"{nm}: n_iter {r['n_iter']}")
            elif list(r["labels"]) != case["labels"]:
                bad.append(f"{nm}: labels {r['labels']}")
            elif not np.allclose(r["centroids"], case["centroids"], rtol=1e-14, atol=1e-14):
                bad.append(f"{nm}: centroids")
            elif not np.isclose(r["objective"], case["objective"], rtol=1e-13, atol=1e-12):
                bad.append(f"{nm}: objective")
            elif not np.allclose(r["J_hist"], case["J_hist"], rtol=1e-13, atol=1e-12):
                bad.append(f"{nm}: J_hist")
    return bad


COUNTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "o2_filter_counts.json")


def check_ti_counts(lib_ti=None):
    """O2's per-iteration filter counters against hand-derived traces (the
    derivation of every count is written in the fixture)."""
    bad = []
    for case in json.load(open(COUNTS))["cases"]:
        X = np.array(case["X"], np.float64)
        C0 = np.array(case["C0"], np.float64)
        r = oracle.ti_fit(X, C0, case["G"], case["max_iter"], case["tol"], lib=lib_ti)
        nm = case["name"]
        if r["n_iter"] != case["n_iter"]:
            bad.append(f"{nm}: n_iter {r['n_iter']}")
            continue
        got = r["cnt_hist"].tolist()
        if got != case["cnt_hist"]:
            bad.append(f"{nm}: counters {got} != {case['cnt_hist']}")
        if "labels" in case and list(r["labels"]) != case["labels"]:
            bad.append(f"{nm}: labels {r['labels']}")
        if "J_hist" in case and not np.allclose(r["J_hist"], case["J_hist"], rtol=1e-13, atol=1e-12):
            bad.append(f"{nm}: J_hist {r['J_hist']}")
        if "centroids" in case and not np.allclose(r["centroids"], case["centroids"], rtol=1e-14, atol=1e-14):
            bad.append(f"{nm}: centroids")
    return bad


def check_ti_init_bounds_exact(lib_ti=None):
    """After iteration 0 the bounds are exact by definition: u = d(x, c_a) and
    lb_g = min over c in g, c != a of d(x, c) (+inf if g holds only a)."""
    bad = []
    for seed, (N, D, K, G) in enumerate([(300, 3, 24, 5), (200, 5, 7, 7), (100, 2, 6, 1)]):
        X, C0 = _rng_data(80 + seed, N, D, K)
        st = oracle.TIState(X, C0, G, lib=lib_ti)
        st.assign()
        d = cdist(st.X, st.C)
        if not np.array_equal(st.a, np.argmin(d, axis=1)):
            bad.append("iteration-0 labels are not nearest centroids")
        if not np.allclose(st.u, d[np.arange(N), st.a], rtol=1e-13):
            bad.append("iteration-0 upper bound != d(x, c_a)")
        d[np.arange(N), st.a] = np.inf
        for g in range(G):
            ref = np.where((st.grp == g)[None, :], d, np.inf).min(axis=1)
            if not np.allclose(st.lb[:, g], ref, rtol=1e-13):
                bad.append(f"iteration-0 lower bound of group {g} != exact minimum")
                break
    return bad


ALL_O1 = [check_golden, check_assign_vs_cdist, check_update_vs_bincount, check_closed_forms,
          check_blobs_recovered, check_lloyd_invariants, check_sklearn]


# ---------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("check", ALL_O1, ids=lambda f: f.__name__)
def test_o1_pin(oracle_lib, check):
    assert check() == []


def test_o2_equals_o1_every_iteration(oracle_lib):
    assert check_ti_equals_lloyd() == []


def test_o2_bounds_valid(oracle_lib):
    assert check_ti_bounds() == []


def test_o2_filters_skip_work(oracle_lib):
    assert check_ti_skips() == []


def test_o2_golden(oracle_lib):
    assert check_ti_golden() == []


def test_o2_counters_hand_derived(oracle_lib):
    assert check_ti_counts() == []


def test_o2_init_bounds_exact(oracle_lib):
    assert check_ti_init_bounds_exact() == []


def test_near_tie_rule():
    d1 = np.array([1.0, 1.0, 0.0, 4.0])
    d2 = np.array([1.0, (1 + 2e-6) ** 2, 0.0, 4.0 * (1 + 1e-7) ** 2])
    assert list(oracle.near_ties(d1, d2)) == [True, False, True, True]


LLOYD_MUTANTS = [
    ("tie to highest index", [("if (s < b1) {", "if (s <= b1) {")]),
    ("last dimension dropped", [("for (int32_t i = 0; i < D; ++i) {\n        double t", "for (int32_t i = 0; i < D - 1; ++i) {\n        double t")]),
    ("L1 instead of squared", [("s = s + t * t;", "s = s + fabs(t);")]),
    ("mean off by one", [("S[j] / (double)cnt[k]", "S[j] / (double)(cnt[k] + 1)")]),
    ("empty cluster zeroed", [(": C_old[j];", ": 0.0;")]),
    ("objective with new centroids", [("o1_objective(X, N, D, labels, C_old, K);", "o1_objective(X, N, D, labels, C_new, K);")]),
    ("sum row index", [("double *s = S + (int64_t)labels[n] * D;", "double *s = S + (int64_t)labels[n];")]),
    ("tol test inverted", [("(J_prev - J) < tol * J_prev", "(J_prev - J) > tol * J_prev")]),
    ("no final assignment", [("o1_assign(X, N, D, C, K, NULL, labels, NULL, NULL);\n    if (J_final)", "if (J_final)")]),
    ("second distance not tracked", [("} else if (s < b2) {", "} else if (s < b2 && 0) {")]),
]

TI_MUTANTS = [
    ("drift not added to u", [("double ub = u[n] + delta[al];", "double ub = u[n];")]),
    ("group drift not subtracted", [("lbn[g] = row[g] - delta_g[g];", "lbn[g] = row[g];")]),
    ("point filter without drift", [("double bound = lbo[g] - delta[c];", "double bound = lbo[g];")]),
    ("old label not re-added", [("if (g == grp[al] && best != al && da < row[g]) row[g] = da;", "")]),
    ("group drift is a min", [("if (delta[k] > delta_g[grp[k]])", "if (delta[k] < delta_g[grp[k]])")]),
    ("best kept in its group bound", [("if (grp[c] == g && c != best && cand[c] < v)", "if (grp[c] == g && cand[c] < v)")]),
    ("init bound includes label", [("if (k != best && sqrt(s[k]) < row[grp[k]])", "if (sqrt(s[k]) < row[grp[k]])")]),
    ("tie in scan to later index", [("(sc == bs && c < best)", "(sc == bs && c > best)")]),
    ("filter on squared vs root", [("if (beyond(m, ub)) {", "if (beyond(m * m, ub)) {")]),
    # the skip counters (one plausible bookkeeping mistake each)
    ("tight counted as global", [("cnt[CNT_TIGHT] += 1;", "cnt[CNT_GLOBAL] += 1;")]),
    ("global filter not counted", [("cnt[CNT_GLOBAL] += 1;", "")]),
    ("group filter counted when scanning",
     [("cnt[CNT_GROUP] += 1;\n                continue;\n            }\n            scanned[g] = 1;",
       "continue;\n            }\n            scanned[g] = 1;\n            cnt[CNT_GROUP] += 1;")]),
    ("point filter counted after the distance",
     [("cand[c] = bound;\n                    cnt[CNT_POINT] += 1;", "cand[c] = bound;"),
      ("cnt[CNT_DIST] += 1;\n                cand[c] = sqrt(sc);",
       "cnt[CNT_DIST] += 1;\n                cnt[CNT_POINT] += 1;\n                cand[c] = sqrt(sc);")]),
    ("tightening not counted as a distance", [("double da = sqrt(sa);\n        cnt[CNT_DIST] += 1;", "double da = sqrt(sa);")]),
    ("every scanned point counted as changed", [("if (best != al) cnt[CNT_CHANGED] += 1;", "cnt[CNT_CHANGED] += 1;")]),
    ("iteration 0 counts K - 1 distances", [("cnt[CNT_DIST] += K;", "cnt[CNT_DIST] += K - 1;")]),
]


@pytest.mark.parametrize("name,repl", LLOYD_MUTANTS, ids=[m[0] for m in LLOYD_MUTANTS])
def test_planted_mistake_in_o1_is_caught(tmp_path, oracle_lib, name, repl):
    lib = oracle.compile_variant("lloyd", repl, str(tmp_path))
    failures = []
    for check in ALL_O1[:-1]:  # scikit-learn not needed to catch these
        failures += check(lib=lib)
    assert failures, f"no pin caught the planted mistake: {name}"


@pytest.mark.parametrize("name,repl", TI_MUTANTS, ids=[m[0] for m in TI_MUTANTS])
def test_planted_mistake_in_o2_is_caught(tmp_path, oracle_lib, name, repl):
    lib = oracle.compile_variant("ti", repl, str(tmp_path))
    failures = (check_ti_equals_lloyd(lib_ti=lib) + check_ti_bounds(lib_ti=lib) + check_ti_skips(lib_ti=lib)
                + check_ti_golden(lib_ti=lib) + check_ti_init_bounds_exact(lib_ti=lib) + check_ti_counts(lib_ti=lib))
    assert failures, f"no pin caught the planted mistake: {name}"
