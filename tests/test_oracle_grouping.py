"""Pins for the clustered grouping and for O2 under any grouping (CPU).

The filtered method's labels may not depend on how the centroids are
grouped: O2 with the clustered grouping, with a random grouping and with
groups left empty must equal O1 label for label in every iteration.  The
clustered grouping itself is checked against what defines it: a fixed point
of nearest-centre assignment for well-separated centroid clusters, the
degenerate G = 1 and G = K cases, and membership in range.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09345_gb300 import synth


def test_clustered_groups_degenerate_and_range():
    C = np.random.default_rng(0).standard_normal((40, 3))
    assert np.array_equal(oracle.clustered_groups(C, 1), np.zeros(40, np.int32))
    assert np.array_equal(oracle.clustered_groups(C, 40), np.arange(40, dtype=np.int32))
    g = oracle.clustered_groups(C, 7)
    assert g.dtype == np.int32 and g.shape == (40,) and g.min() >= 0 and g.max() < 7
    with pytest.raises(ValueError):
        oracle.clustered_groups(C, 41)


def test_clustered_groups_find_separated_clusters():
    # three tight clouds of centroids far apart, seeded with one row from each
    rng = np.random.default_rng(1)
    far = np.array([[0.0, 0.0], [100.0, 0.0], [0.0, 100.0]])
    C = np.concatenate([far, far[rng.integers(0, 3, 57)] + rng.standard_normal((57, 2))])
    truth = np.argmin(((C[:, None] - far[None]) ** 2).sum(-1), axis=1)
    assert np.array_equal(oracle.clustered_groups(C, 3), truth.astype(np.int32))


def test_clustered_groups_is_nearest_centre_of_its_groups():
    w = synth.anisotropic_1m(N=4096, K=64, G=7, seed=5)
    C = w.C0.astype(np.float64)
    g = oracle.clustered_groups(C, 7, iters=50)  # converged
    centres = np.stack([C[g == j].mean(0) for j in range(7) if (g == j).any()])
    ids = [j for j in range(7) if (g == j).any()]
    d = ((C[:, None] - centres[None]) ** 2).sum(-1)
    assert np.array_equal(np.asarray(ids)[np.argmin(d, axis=1)], g)


@pytest.mark.parametrize("kind", ["clustered", "random", "empty"])
def test_o2_labels_equal_o1_under_any_grouping(kind):
    w = synth.anisotropic_1m(N=3000, K=48, G=6, seed=11)
    X, C0 = w.X.astype(np.float64), w.C0.astype(np.float64)
    K, G = C0.shape[0], 6
    if kind == "clustered":
        grp = oracle.clustered_groups(C0, G)
    elif kind == "random":
        grp = np.random.default_rng(2).integers(0, G, K).astype(np.int32)
    else:  # groups 1 and 4 hold no centroid
        grp = np.random.default_rng(3).choice([0, 2, 3, 5], K).astype(np.int32)
    # O1's trajectory: brute-force assignment and update, iteration by iteration
    hist, C, prev = [], C0.copy(), None
    for _ in range(10):
        lab, _, _, ch = oracle.lloyd_assign(X, C, prev)
        C, _, _ = oracle.lloyd_update(X, lab, C)
        hist.append(lab)
        prev = lab
        if ch == 0:
            break
    o2 = oracle.ti_fit(X, C0, G, 10, grp=grp)
    assert o2["n_iter"] == len(hist)
    for t in range(o2["n_iter"]):
        assert np.array_equal(o2["labels_hist"][t], hist[t]), t
    assert np.allclose(o2["centroids"], C, rtol=1e-13, atol=1e-13)
    # the filters removed work in the filtered iterations
    assert o2["cnt_hist"][1:, oracle.CNT_DIST].sum() < (o2["n_iter"] - 1) * X.shape[0] * K
