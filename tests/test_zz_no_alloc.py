"""The allocation-free norms entry point (mlbm_norms_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory (a memory pool owning the device, loops
that cannot take cudaMalloc's implicit synchronisation): its scratch is a fixed array in the
library's device memory.  This file is collected last so that, run after the other tests, it
also sees a device that other calls have already used; it must pass alone as well.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
LIMIT = 16_777_216


def _call(a, b, c, d, n, out):
    L = mlbm.lib()
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.mlbm_norms_noalloc(p(a), p(b), p(c), p(d), ctypes.c_int64(n), p(out), stream)


def _weights():
    import mlbm_inputs as mi

    xy = mi.jittered_lattice(8, 0.3, seed=1)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=9, degree=2, dx_ml=0.1))
    return mlbm.build_weights(cloud)


def test_noalloc_norms_match_allocating_entry_point_on_consecutive_calls():
    w = _weights()
    dev = torch.device("cuda:0")
    # two calls in a row with different sizes and data: the shared scratch keeps the first
    # call's partial sums, which the second must not pick up
    for n, seed, two in ((LIMIT, 1, True), (1_000_003, 2, True), (12_345, 3, False)):
        g = torch.Generator(device=dev).manual_seed(seed)
        a, b, c, d = (torch.randn(n, dtype=torch.float64, device=dev, generator=g) for _ in range(4))
        if not two:
            c = d = None
        out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        assert _call(a, b, c, d, n, out) == mlbm.OK, mlbm.lib().mlbm_last_error()
        want = mlbm.norms(w, a, b, c, d)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-13)


def test_noalloc_norms_empty_and_limit():
    dev = torch.device("cuda:0")
    a = torch.zeros(4, dtype=torch.float64, device=dev)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    assert _call(a, a, None, None, 0, out) == mlbm.OK
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0]
    # beyond the limit: rejected on the host, nothing launched
    assert _call(a, a, None, None, LIMIT + 1, out) == mlbm.EINVAL
    assert b"limit" in mlbm.lib().mlbm_last_error()


def test_noalloc_norms_leave_device_memory_untouched():
    """The point of the entry point: after a first call (which looks up the scratch address),
    further calls change the device's free memory by nothing.  The Python wrapper goes through
    the same entry point and gives the same sums as the allocating one."""
    w = _weights()
    dev = torch.device("cuda:0")
    n = 3_000_001
    g = torch.Generator(device=dev).manual_seed(7)
    a, b, c, d = (torch.randn(n, dtype=torch.float64, device=dev, generator=g) for _ in range(4))
    out = torch.empty(3, dtype=torch.float64, device=dev)
    assert _call(a, b, c, d, n, out) == mlbm.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        assert _call(a, b, c, d, n, out) == mlbm.OK
        mlbm.norms_noalloc(a, b, c, d, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    np.testing.assert_allclose(out.cpu().numpy(), mlbm.norms(w, a, b, c, d), rtol=1e-13)


def test_noalloc_norms_reject_one_sided_second_component():
    """c and d come together or not at all: one of them alone is rejected before any launch."""
    dev = torch.device("cuda:0")
    a = torch.ones(16, dtype=torch.float64, device=dev)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    assert _call(a, a, a, None, 16, out) == mlbm.EINVAL
    assert _call(a, a, None, a, 16, out) == mlbm.EINVAL
    assert b"both" in mlbm.lib().mlbm_last_error()
    assert np.isnan(out.cpu().numpy()).all()
