"""The proposal network on the tensor cores (kmeans_mlp_*) against O3, the
FP64 oracle of the same network.

The network computes its products in bfloat16 with FP32 accumulation, so it
is compared with O3 evaluated at the bfloat16 values of its weights and
inputs; what remains is the rounding of the activations and backpropagated
gradients to bfloat16 (a numpy emulation of exactly those roundings puts
the gradient error at <= 0.35% of each tensor's largest entry on these
shapes), against a tolerance of 1e-2.  A transposed operand, a dropped GELU
derivative or a flipped sign is an O(1) error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_1905_09345_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-2
NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


@pytest.fixture(scope="module")
def kp():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    oracle.build()
    return kpynq


def bf(a):
    """bfloat16 value (round to nearest even) of each entry, as float64."""
    a32 = np.ascontiguousarray(a, np.float32)
    return (synth.bf16_bits(a32).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def at_compute_precision(params):
    return {k: (bf(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
            for k, v in params.items()}


def dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def random_params(D, H, G, seed):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(D, H, G, seed=seed)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.1, params[k].shape)
    return params


@pytest.mark.parametrize("D,H,G,B", [(32, 64, 40, 256), (32, 256, 410, 1024), (20, 48, 7, 128), (128, 96, 300, 384)])
def test_gradient_matches_oracle(kp, D, H, G, B):
    """Forward + backward of one batch: the loss and the gradient of every
    parameter against O3's backpropagation (the proposal family's shape
    D=32, H=256, G=410 included)."""
    rng = np.random.default_rng(D * 1000 + H + G)
    params = random_params(D, H, G, seed=D + H + G)
    X = rng.normal(0, 1.5, (B, D)).astype(np.float32)
    y = rng.integers(0, G, B).astype(np.int32)
    loss_ref, g_ref = mlp.loss_and_grad(at_compute_precision(params), bf(X), y)
    net = kp.MLP(D, H, G)
    net.set_params({k: dev(v) for k, v in params.items()})
    grad = torch.empty(net.n_params(), dtype=torch.float32, device="cuda")
    loss = net.gradient(dev(X), dev(y, np.int32), grad)
    g = net.split(grad.cpu().numpy().astype(np.float64))
    assert abs(loss - loss_ref) <= GRAD_RTOL * loss_ref, (loss, loss_ref)
    for k in NAMES:
        err = float(np.abs(g[k] - g_ref[k]).max())
        scale = float(np.abs(g_ref[k]).max())
        assert err <= GRAD_RTOL * scale, (k, err, scale)
    net.close()


def test_adam_steps_match_oracle(kp):
    """Two full-batch Adam steps (seed ~0: the same rows each step) equal O3's
    Adam applied to the network's own gradients at each step (bias-corrected
    moments at t = 1 and t = 2)."""
    D, H, G, B = 16, 64, 10, 256
    rng = np.random.default_rng(4)
    params = random_params(D, H, G, seed=5)
    X = rng.normal(0, 1.0, (B, D)).astype(np.float32)
    y = rng.integers(0, G, B).astype(np.int32)
    Xd, yd = dev(X), dev(y, np.int32)
    net = kp.MLP(D, H, G)
    net.set_params({k: dev(v) for k, v in params.items()})
    lr = 1e-2
    state = mlp.adam_init(params)
    cur = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}
    grad = torch.empty(net.n_params(), dtype=torch.float32, device="cuda")
    out = {k: torch.empty(s, dtype=torch.float32, device="cuda") for k, s in net.shapes().items()}
    for step in range(2):
        net.gradient(Xd, yd, grad)
        g = net.split(grad.cpu().numpy().astype(np.float64))
        mlp.adam_step(cur, g, state, lr=lr)
        net.train(Xd, yd, 0, steps=1, batch=B, lr=lr, seed=(1 << 64) - 1)
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in net.get_params(out).items()}
        for k in NAMES:
            err = float(np.abs(got[k] - cur[k]).max())
            assert err <= 1e-6 + 1e-3 * lr, (step, k, err)
        cur = got  # the next step starts from the network's FP32 weights
    net.close()


def test_predict_matches_oracle(kp):
    """Inference (kmeans_mlp_predict_net and the standalone kmeans_mlp_predict)
    equals O3's argmax wherever O3's two largest logits are further apart than
    the bfloat16 activations can move them, and is a near-maximal class
    elsewhere."""
    rng = np.random.default_rng(3)
    N, D, H, G = 5003, 32, 64, 40
    params = random_params(D, H, G, seed=7)
    X = rng.normal(0, 2.0, (N, D)).astype(np.float32)
    logits, _ = mlp.forward(at_compute_precision(params), bf(X))
    ref = np.argmax(logits, axis=1)
    srt = np.sort(logits, axis=1)
    scale = np.abs(logits).max(axis=1) + 1.0
    # bfloat16 activations move a logit by at most 0.37% of `scale` on these
    # inputs (numpy emulation of the roundings): a gap of 1e-2 * scale is safe
    clear = (srt[:, -1] - srt[:, -2]) > 1e-2 * scale
    assert clear.mean() > 0.9
    dp = {k: dev(v) for k, v in params.items()}
    net = kp.MLP(D, H, G)
    net.set_params(dp)
    for how in ("net", "standalone"):
        pred = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        if how == "net":
            net.predict(dev(X), pred)
        else:
            kp.kmeans_mlp_predict(dev(X), N, D, *[dp[k] for k in kp.MLP_NAMES], H, G, pred)
        got = pred.cpu().numpy()
        assert np.array_equal(got[clear], ref[clear]), how
        assert np.all(logits[np.arange(N), got] >= srt[:, -1] - 1e-2 * scale), how
    net.close()


def test_training_learns_separable_classes(kp):
    """Adam on batches drawn on the device learns 12 well-separated Gaussian
    classes (held-out accuracy > 0.98) and lowers the loss."""
    rng = np.random.default_rng(11)
    D, H, G, N = 16, 64, 12, 24000
    X, cls = synth.gaussian_mixture(rng, N, D, G, centre_range=6.0, scale="fixed", scale_args=(0.7,))
    net = kp.MLP(D, H, G, seed=3)
    Xd, yd = dev(X[:20000]), dev(cls[:20000], np.int32)
    loss0, _ = net.train(Xd, yd, 0, steps=1, batch=512, lr=3e-3, seed=9)
    loss1, acc1 = net.train(Xd, yd, 0, steps=300, batch=512, lr=3e-3, seed=10)
    assert loss1 < 0.5 * loss0, (loss0, loss1)
    pred = torch.empty(4000, dtype=torch.int32, device="cuda")
    net.predict(dev(X[20000:]), pred)
    acc = float((pred.cpu().numpy() == cls[20000:]).mean())
    assert acc > 0.98, acc
    net.close()


def test_gpu_trained_proposal_cuts_iteration_zero(kp):
    """The network trained on the GPU on the groups of a fit's final labels
    (kmeans_mlp_train with K > 0) seeds iteration 0 of a second fit: labels,
    iterations and objective equal the fit without a proposal, and iteration
    0 evaluates far fewer than N*K distances."""
    rng = np.random.default_rng(0)
    N, D, K, G = 20000, 32, 256, 26
    X, _ = synth.gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="blob_uniform", scale_args=(0.3, 1.5))
    C0 = synth.sample_init(rng, X, K)
    Xd, C0d = dev(X), dev(C0)
    base = kp.KMeans(Xd, C0d, G)
    lab0 = torch.empty(N, dtype=torch.int32, device="cuda")
    r0 = base.fit(12, 0.0, lab0)
    base.close()
    net = kp.MLP(D, 64, G, seed=1)
    loss, acc = net.train(Xd, lab0, K, steps=600, batch=1024, lr=3e-3, seed=2)
    params = net.get_params({k: torch.empty(s, dtype=torch.float32, device="cuda")
                             for k, s in net.shapes().items()})
    km = kp.KMeans(Xd, C0d, G)
    km.set_proposal(params)
    lab = torch.empty(N, dtype=torch.int32, device="cuda")
    C = torch.empty(K, D, dtype=torch.float32, device="cuda")
    r = km.fit(12, 0.0, lab, C)
    km.close()
    net.close()
    assert r.n_iter == r0.n_iter
    assert torch.equal(lab, lab0)
    assert abs(r.objective - r0.objective) <= 1e-9 * r0.objective
    ref, _, _, _ = oracle.lloyd_assign(X.astype(np.float64), C.cpu().numpy().astype(np.float64))
    assert np.array_equal(lab.cpu().numpy(), ref)
    assert r.stats[0]["path"] == kp.KM_PATH_FILTERED
    assert r.stats[0]["n_dist"] < 0.5 * N * K, (r.stats[0]["n_dist"], acc)
