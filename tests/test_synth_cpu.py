"""The seeded input generators (CPU): the recipes the parity tests and the
bench draw their inputs from, checked against their stated parameters."""
import numpy as np

from paper_1905_09345_gb300 import synth


def test_same_seed_same_inputs():
    a, b = synth.anisotropic_1m(N=4096, seed=7), synth.anisotropic_1m(N=4096, seed=7)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.C0, b.C0) and np.array_equal(a.blob, b.blob)
    c = synth.anisotropic_1m(N=4096, seed=8)
    assert not np.array_equal(a.X, c.X)


def test_mixture_counts_scales_and_centres():
    rng = np.random.default_rng(0)
    N, D, k = 40000, 8, 5
    X, blob = synth.gaussian_mixture(rng, N, D, k, centre_range=50.0, scale="axis_uniform",
                                     scale_args=(0.5, 2.0))
    assert X.dtype == np.float32 and X.shape == (N, D)
    counts = np.bincount(blob, minlength=k)
    assert counts.max() - counts.min() <= 1 and counts.sum() == N  # equal weights
    sd = np.stack([X[blob == j].std(0) for j in range(k)])
    assert sd.min() > 0.45 and sd.max() < 2.1  # per-axis stds drawn from U[0.5, 2.0]
    mu = np.stack([X[blob == j].mean(0) for j in range(k)])
    assert np.abs(mu).max() < 50.5  # centres in U[-50, 50]^D
    rng = np.random.default_rng(1)
    _, blob = synth.gaussian_mixture(rng, N, D, k, centre_range=5.0, scale="fixed", scale_args=(1.0,),
                                     weights="dirichlet")
    assert np.bincount(blob, minlength=k).sum() == N


def test_sample_init_distinct_rows():
    w = synth.anisotropic_1m(N=5000, K=300, seed=3)
    assert w.C0.shape == (300, 64) and w.C0.flags["C_CONTIGUOUS"]
    rows = {r.tobytes() for r in w.C0}
    assert len(rows) == 300
    xs = {r.tobytes() for r in w.X}
    assert rows <= xs


def test_bf16_round_to_nearest_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even pattern (1.0)
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e38, 1e-40], np.float32)
    r = synth.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    x = np.random.default_rng(2).standard_normal(10000).astype(np.float32) * 100
    y = synth.to_bf16(x)
    # nearest: no other bfloat16 value is closer
    up = (y.view(np.uint32) + 0x10000).view(np.float32)
    dn = (y.view(np.uint32) - 0x10000).view(np.float32)
    e = np.abs(x.astype(np.float64) - y)
    assert np.all(e <= np.abs(x.astype(np.float64) - up)) and np.all(e <= np.abs(x.astype(np.float64) - dn))
    bits = synth.bf16_bits(x)
    assert bits.dtype == np.uint16
    assert np.array_equal((bits.astype(np.uint32) << 16).view(np.float32), y)


def test_highdim_stored_as_bfloat16():
    w = synth.highdim_4m(N=3000, K=100, G=10)
    assert w.meta["storage"] == "bf16"
    assert np.all((w.X.view(np.uint32) & 0xFFFF) == 0)
    assert np.all((w.C0.view(np.uint32) & 0xFFFF) == 0)  # sampled rows of X


def test_proposal_family_fixed_across_sample_seeds():
    a = synth.proposal_family(1, N=8192, K=64, G=7)
    b = synth.proposal_family(9, N=8192, K=64, G=7)
    assert np.array_equal(a.C0, b.C0)                  # the family fixes C0 (and the centres)
    assert not np.array_equal(a.X, b.X)                # the sample seed redraws the points
    assert np.array_equal(np.sort(a.blob), np.sort(b.blob))  # equal weights in both


def test_batched_problem_parameters():
    specs = synth.batched_problems(64, n_lo=1000, n_hi=200000)
    for s in specs:
        assert 1000 <= s["N"] <= 200000 and s["D"] in (8, 32, 64, 128)
        assert 1 <= s["K"] <= min(512, s["N"]) and s["G"] == max(1, s["K"] // 10)
    w = synth.batched_problem(specs[0])
    assert w.X.shape == (specs[0]["N"], specs[0]["D"]) and np.array_equal(w.C0, w.X[: specs[0]["K"]])
    assert w.max_iter == 25
