"""hm_matvec_noalloc: the H-matvec for callers that cannot allocate device
memory at call time (fixed-budget servers, code where cudaMalloc would
synchronise the device or is not allowed).  Its scratch is a fixed array
inside the library; this checks, through the C ABI, that two calls in a row
give the same result as hm_matvec, that host threads racing on the first
call (the scratch address is looked up and cached then) all get the right
product, and that a problem too large for the fixed scratch is refused with a
clear error.  Collected last on purpose."""
import ctypes
import threading

import numpy as np
import pytest

from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu

CASES = [
    ("levy1d_n4095", W.levy_1d(4095), W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32)),
    ("frac2d_n40", W.frac_lap_2d(40, 0.75), W.default_opts(leaf=64, aca_tol=1e-8, max_rank=32)),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _noalloc(H, x, y, alpha, beta, gamma, w1, w2):
    lib = hmat.load()
    s = lib.hm_matvec_noalloc(H.handle, alpha, beta, ctypes.c_void_p(x.data_ptr()), gamma,
                              ctypes.c_void_p(w1.data_ptr()), ctypes.c_void_p(w2.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    hmat._check(s)


def test_threads_racing_on_the_first_call():
    """Eight host threads make the process's first hm_matvec_noalloc calls at
    the same moment (ctypes releases the GIL, so the address lookup and its
    cache race for real).  They share one stream, as the header asks of calls
    that share the scratch, so the products are serialised on the GPU: each
    must equal hm_matvec's."""
    name, prob, opts = CASES[0]
    H = hmat.HMatrix(prob, opts)
    N = H.n
    rng = np.random.default_rng(11)
    xs = [dev(rng.standard_normal(N)) for _ in range(8)]
    refs = [host(H.matvec(x, alpha=1.0, beta=-1e-3, gamma=0.0, w1=x, w2=x)) for x in xs]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    gate = threading.Barrier(len(xs))
    errors = []

    def work(i):
        try:
            gate.wait()
            with torch.cuda.stream(stream):
                _noalloc(H, xs[i], ys[i], 1.0, -1e-3, 0.0, xs[i], xs[i])
        except Exception as e:  # reported below, on the test's thread
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(xs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not errors, errors
    torch.cuda.synchronize()
    for i, (y, ref) in enumerate(zip(ys, refs)):
        got = host(y)
        assert np.all(np.isfinite(got)), i
        assert np.max(np.abs(got - ref)) <= 1e-13 * (np.max(np.abs(ref)) + 1e-300), i
    H.sync()


@pytest.mark.parametrize("name,prob,opts", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_matvec_twice(name, prob, opts):
    H = hmat.HMatrix(prob, opts)
    N = H.n
    rng = np.random.default_rng(5)
    alpha, beta, gamma = 0.9, -7e-4, 0.3
    for call in range(2):
        x, w1, w2 = (dev(rng.standard_normal(N)) for _ in range(3))
        ref = host(H.matvec(x, alpha=alpha, beta=beta, gamma=gamma, w1=w1, w2=w2))
        y = torch.full_like(x, float("nan"))
        _noalloc(H, x, y, alpha, beta, gamma, w1, w2)
        got = host(y)
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.all(np.isfinite(got)), call
        # the same product up to rounding (hm_matvec multiplies the jump part in
        # double-float arithmetic, 2^-47; the matvec tests allow 50 aca_tol)
        assert np.max(np.abs(got - ref)) <= 1e-13 * scale, call
    H.sync()


def test_noalloc_refuses_too_large():
    prob = W.levy_1d(262143)
    H = hmat.HMatrix(prob, W.default_opts(leaf=256, aca_tol=1e-8, max_rank=16))
    x = torch.zeros(H.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(hmat.HMError) as ei:
        _noalloc(H, x, y, 1.0, 1.0, 0.0, x, x)
    assert "fixed scratch" in str(ei.value)
