"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol ``include/*.h`` declares, and rejects bad arguments before touching the
device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1905_09345_gb300 import build, kpynq
    build.build()
    return kpynq


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"KM_API\s+[\w\s\*]+?\b(\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["kmeans_init", "kmeans_iterate", "kmeans_fit", "kmeans_get_labels", "kmeans_get_centroids",
              "kmeans_destroy", "kmeans_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert missing == []


def test_binding_uses_c_names(L):
    for n in declared_symbols():
        assert hasattr(L, n), f"binding lacks {n}"


BAD = [
    dict(N=0, D=4, K=1, G=1),
    dict(N=10, D=0, K=1, G=1),
    dict(N=10, D=4097, K=1, G=1),
    dict(N=10, D=4, K=0, G=1),
    dict(N=10, D=4, K=11, G=1),
    dict(N=10, D=4, K=4, G=0),
    dict(N=10, D=4, K=4, G=5),
    dict(N=1 << 31, D=4, K=4, G=1),
    dict(N=100000, D=4, K=65536, G=1),
]


@pytest.mark.parametrize("a", BAD, ids=lambda a: ",".join(f"{k}={v}" for k, v in a.items()))
def test_init_rejects_bad_sizes(L, a):
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(16, a["N"], a["D"], a["K"], a["G"], 16)
    assert e.value.status == L.KM_EINVAL
    assert L.kmeans_last_error(None)


def test_init_rejects_null_and_bad_options(L):
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(0, 10, 4, 2, 1, 16)
    assert e.value.status == L.KM_EINVAL
    opt = L.kmeans_default_options()
    opt.algo = 7
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(16, 10, 4, 2, 1, 16, opt)
    assert e.value.status == L.KM_EINVAL
    opt = L.kmeans_default_options()
    opt.dense = 5
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(16, 10, 4, 2, 1, 16, opt)
    assert e.value.status == L.KM_EINVAL
    opt = L.kmeans_default_options()
    opt.dense_switch = -1.0
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(16, 10, 4, 2, 1, 16, opt)
    assert e.value.status == L.KM_EINVAL
    opt = L.kmeans_default_options()
    opt.reserved[2] = 1
    with pytest.raises(L.KMeansError) as e:
        L.kmeans_init(16, 10, 4, 2, 1, 16, opt)
    assert e.value.status == L.KM_EINVAL
    for field, bad in (("dtype", 7), ("dtype", -1), ("pad0", 1), ("pad1", 1), ("surv_grab", 16),
                       ("surv_grab", 48), ("surv_grab", 2048), ("surv_grab", -32)):
        opt = L.kmeans_default_options()
        setattr(opt, field, bad)
        with pytest.raises(L.KMeansError) as e:
            L.kmeans_init(16, 10, 4, 2, 1, 16, opt)
        assert e.value.status == L.KM_EINVAL, field
    assert L.kmeans_default_options().dtype == L.KM_DTYPE_F32


def test_dtype_inference():
    from paper_1905_09345_gb300 import kpynq
    import numpy as np
    torch = pytest.importorskip("torch")
    assert kpynq._dtype_of(np.zeros((2, 2), np.float32), None) == kpynq.KM_DTYPE_F32
    assert kpynq._dtype_of(np.zeros((2, 2), np.uint16), kpynq.KM_DTYPE_BF16) == kpynq.KM_DTYPE_BF16
    assert kpynq._dtype_of(torch.zeros(2, 2, dtype=torch.bfloat16), None) == kpynq.KM_DTYPE_BF16
    assert kpynq._dtype_of(torch.zeros(2, 2), None) == kpynq.KM_DTYPE_F32


def test_null_context_calls(L):
    lib = L.lib()
    assert lib.kmeans_iterate(None, None) == L.KM_EINVAL
    assert lib.kmeans_fit(None, 1, 0.0, None, None, None, None) == L.KM_EINVAL
    lib.kmeans_destroy(None)
    assert L.kmeans_launch_count() >= 0
    # the proposal entry points reject bad arguments before any device work
    assert lib.kmeans_set_proposal(None, None, None, None, None, None, None, 0) == L.KM_EINVAL
    assert lib.kmeans_mlp_predict(None, 10, 4, None, None, None, None, None, None, 8, 3, None, None) == L.KM_EINVAL
    fake = 16  # any non-NULL address: the size checks come first
    assert lib.kmeans_mlp_predict(fake, 0, 4, fake, fake, fake, fake, fake, fake, 8, 3, fake, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_predict(fake, 10, 4, fake, fake, fake, fake, fake, fake, 300, 3, fake, None) == L.KM_EINVAL
    assert "hidden" in L.kmeans_last_error(None)
    lib.kmeans_selftest_sqrt.restype = __import__("ctypes").c_int
    assert lib.kmeans_selftest_sqrt(None) == L.KM_EINVAL
    assert L.kmeans_selftest_timeout(0) == L.KM_EINVAL
    assert L.kmeans_selftest_timeout(1 << 17) == L.KM_EINVAL


def test_default_options(L):
    o = L.kmeans_default_options()
    assert o.algo == L.KM_ALGO_FILTERED and o.grouping == L.KM_GROUP_CONTIGUOUS and not o.stream


def test_mlp_entry_points_reject_bad_arguments(L):
    """The proposal network's entry points check sizes and pointers before any
    device work."""
    lib = L.lib()
    out = ctypes.c_void_p()
    for D, H, G in ((0, 8, 4), (257, 8, 4), (8, 0, 4), (8, 257, 4), (8, 8, 0), (8, 8, 513)):
        assert lib.kmeans_mlp_create(ctypes.byref(out), D, H, G, 0, None) == L.KM_EINVAL, (D, H, G)
        assert out.value is None
        assert "range" in L.kmeans_mlp_last_error(None)
    assert lib.kmeans_mlp_create(None, 8, 8, 4, 0, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_set_params(None, None, None, None, None, None, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_get_params(None, None, None, None, None, None, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_gradient(None, None, None, 128, None, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_train(None, None, 1, None, 0, 1, 128, 1e-3, 1, None, None) == L.KM_EINVAL
    assert lib.kmeans_mlp_predict_net(None, None, 1, None) == L.KM_EINVAL
    lib.kmeans_mlp_destroy(None)


def test_noalloc_wrapper_checks_types_and_shapes(L):
    """kmeans_lloyd_step_noalloc's Python wrapper refuses arrays whose element
    type, shape or layout the C call would misread."""
    import numpy as np
    N, D, K = 100, 8, 4
    X = np.zeros((N, D), np.float32)
    C = np.zeros((K, D), np.float32)
    lab = np.zeros(N, np.int32)
    J = np.zeros(1, np.float64)
    bad = [
        dict(X=X.astype(np.float64)), dict(C=C.astype(np.float64)), dict(C_new=np.zeros((K, D + 1), np.float32)),
        dict(labels=lab.astype(np.int64)), dict(objective=np.zeros(1, np.float32)),
        dict(X=np.zeros((D, N), np.float32).T),  # not C-contiguous
    ]
    for b in bad:
        args = dict(X=X, C=C, labels=lab, C_new=np.zeros((K, D), np.float32), objective=J)
        args.update(b)
        with pytest.raises(L.KMeansError) as e:
            L.kmeans_lloyd_step_noalloc(args["X"], N, D, args["C"], K, args["labels"], args["C_new"],
                                        args["objective"])
        assert e.value.status == L.KM_EINVAL, b
