"""Pins of O4 (oracle/kmeanspp.c), the k-means++ seeding oracle.

* Hand-derived draws on 1-D points (derivations below).
* The draw's distribution: sweeping u over a fine grid, the fraction of u
  that picks point i equals D(x_i)^2 / sum D^2 (D from scipy's cdist, not from
  the oracle) -- the defining property of D^2 sampling.
* The returned squared distances equal cdist's minimum over the chosen
  centres; distinct points give distinct centres.
* Planted mistakes in the oracle must make a pin fail.
"""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle

# (X, u, expected indices, derivation)
HAND = [
    ([0, 1, 3, 10], [0.0, 0.5], [0, 3],
     "first floor(0*4)=0; D^2=[0,1,9,100], max 100 = 0.78125*2^7 -> scale 2^25; W=110*2^25, "
     "T=55*2^25; running sums 0, 2^25, 10*2^25, 110*2^25: the first above T is x=10 (index 3)"),
    ([0, 1, 3, 10], [0.99, 0.05, 0.9], [3, 0, 2],
     "first floor(0.99*4)=3 (x=10); D^2=[100,81,49,0], scale 2^25, W=230*2^25, T=floor(11.5*2^25): "
     "the first running sum 100*2^25 exceeds it -> index 0; then D^2=[0,1,9,0], max 9 = 0.5625*2^4 -> "
     "scale 2^28, W=10*2^28, T=floor(0.9*10*2^28)=9*2^28 (the FP64 product rounds to it): running sums "
     "0, 2^28, 10*2^28 -> index 2 (x=3)"),
    ([0, 1, 3, 10], [0.0, 0.0], [0, 1],
     "first 0; D^2=[0,1,9,100], T=floor(0*W)=0: the first running sum above 0 is x=1's (index 1); "
     "the chosen centre itself (weight 0) can never be drawn again"),
    ([5, 5, 5], [0.1, 0.7], [0, 2],
     "first floor(0.3)=0; every D^2 is 0, so W=0 and the draw is uniform: floor(0.7*3)=2"),
]


def check_hand(lib=None):
    bad = []
    for X, u, want, _ in HAND:
        idx, _ = oracle.kmeanspp(np.array(X, np.float64)[:, None], len(u), np.array(u), lib=lib)
        if list(idx) != want:
            bad.append(f"{X} {u}: {list(idx)} != {want}")
    return bad


def check_distribution(lib=None):
    """Second centre over a grid of u: frequencies proportional to D^2."""
    bad = []
    rng = np.random.default_rng(1)
    X = rng.normal(0, 3, (7, 2))
    grid = (np.arange(200000) + 0.5) / 200000
    d2 = cdist(X, X[[2]], "sqeuclidean")[:, 0]
    want = d2 / d2.sum()
    picks = [oracle.kmeanspp(X, 2, np.array([2.5 / 7, u]), lib=lib)[0][1] for u in grid[::50]]
    counts = np.bincount(picks, minlength=len(X)) / len(picks)
    if np.abs(counts - want).max() > 2e-3:
        bad.append(f"D^2 sampling frequencies {counts} != {want}")
    return bad


def check_dmin_and_distinct(lib=None):
    bad = []
    rng = np.random.default_rng(2)
    for N, D, K in ((500, 3, 20), (64, 8, 64), (1000, 16, 50)):
        X = rng.normal(0, 1, (N, D))
        idx, dmin = oracle.kmeanspp(X, K, rng.uniform(size=K), lib=lib)
        if len(set(idx.tolist())) != K:
            bad.append("repeated centre among distinct points")
        ref = cdist(X, X[idx], "sqeuclidean").min(axis=1)
        if not np.allclose(dmin, ref, rtol=1e-12, atol=1e-12):
            bad.append("returned squared distances are not the minimum over the chosen centres")
    return bad


ALL = [check_hand, check_distribution, check_dmin_and_distinct]


@pytest.mark.parametrize("check", ALL, ids=lambda f: f.__name__)
def test_o4_pin(oracle_lib, check):
    assert check() == []


MUTANTS = [
    ("distance not minimised", [("if (s < d[n]) d[n] = s;", "d[n] = s;")]),
    ("weights from D instead of D^2", [("W += (uint64_t)floor(ldexp(d[n], 32 - e));",
                                        "W += (uint64_t)floor(ldexp(sqrt(d[n]), 32 - e));"),
                                       ("run += (uint64_t)floor(ldexp(d[n], 32 - e));",
                                        "run += (uint64_t)floor(ldexp(sqrt(d[n]), 32 - e));")]),
    ("running sum reaches instead of exceeds", [("if (run > T) {", "if (run >= T) {")]),
    ("first centre fixed", [("pick = uniform_index(u[0], N);", "pick = 0;")]),
    ("uniform draw uses the first uniform", [("pick = uniform_index(u[j], N);", "pick = uniform_index(u[0], N);")]),
]


@pytest.mark.parametrize("name,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_in_o4_is_caught(tmp_path, oracle_lib, name, repl):
    lib = oracle.compile_variant("pp", repl, str(tmp_path))
    failures = []
    for check in ALL:
        failures += check(lib=lib)
    assert failures, f"no pin caught the planted mistake: {name}"
