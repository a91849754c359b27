"""Device stencil build (mlbm_build_cloud_device): Morton order, N_L-nearest-neighbour stencils
by (d^2, original index), departure nodes, bounce-back masks, force directions and the
transposed stencil, built by kernels, against the host build (every array bit for bit) and the
oracle's brute force (Sec. 2.2, Sec. 2.3, Sec. 3)."""
import time

import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _periodic(k, deg, dx, mode=None):
    d = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=k, degree=deg, dx_ml=dx)
    if mode is not None:
        d["stencil_mode"] = mode
    return d


def _annulus(k, deg, dx, mode=None):
    d = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=k, degree=deg, dx_ml=dx)
    if mode is not None:
        d["stencil_mode"] = mode
    return d


def _same_cloud(xy, segs, offs=None):
    """Host and device builds of the same arguments; every exported array must agree."""
    h = mlbm.build_cloud(xy, segs, offs)
    d = mlbm.build_cloud(xy, segs, offs, device=True)
    np.testing.assert_array_equal(d.perm(), h.perm())
    for s in range(h.nseg):
        np.testing.assert_array_equal(d.stencil(s), h.stencil(s))
        np.testing.assert_array_equal(d.departure_nodes(s), h.departure_nodes(s))
    np.testing.assert_array_equal(d.bounce_mask(), h.bounce_mask())
    return h, d


@pytest.mark.parametrize("n_side,k,deg", [(32, 12, 2), (20, 30, 4), (13, 9, 2), (24, 45, 6), (20, 100, 2)])
def test_periodic_device_build_matches_host_and_oracle(n_side, k, deg):
    xy = mi.jittered_lattice(n_side, 0.3, seed=n_side + k)
    _, d = _same_cloud(xy, _periodic(k, deg, 1.0 / n_side))
    np.testing.assert_array_equal(d.stencil(0), oracle.stencils(xy, k, box=(1.0, 1.0)))


def test_exact_lattice_ties_match_oracle():
    """On an exact lattice most distances tie: ranks fall back to the original index."""
    xy = mi.lattice(16)
    _, d = _same_cloud(xy, _periodic(12, 2, 1.0 / 16))
    np.testing.assert_array_equal(d.stencil(0), oracle.stencils(xy, 12, box=(1.0, 1.0)))


def test_tiny_cloud_scans_every_cell():
    """So few nodes that the search block wraps onto itself at once."""
    xy = mi.jittered_lattice(3, 0.3, seed=2)
    _, d = _same_cloud(xy, _periodic(9, 2, 0.2))
    np.testing.assert_array_equal(d.stencil(0), oracle.stencils(xy, 9, box=(1.0, 1.0)))


def test_collinear_cloud():
    """Degenerate extent: every node on one line (a single row of cells)."""
    x = np.linspace(0.1, 0.9, 40)
    xy = np.stack([x, np.full_like(x, 0.5)])
    _same_cloud(xy, _annulus(5, 1, 0.01))


@pytest.mark.parametrize("mode", [None, "nearest"])
def test_annulus_device_build_matches_host(mode):
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[2000], seed=4)
    dx = 1.0 / 40
    m = mlbm.STENCIL_NEAREST if mode else None
    _, d = _same_cloud(xy, _annulus(20, 3, dx, m))
    np.testing.assert_array_equal(d.bounce_mask(), oracle.bounce_mask(xy, dx, 0.5, 1.0))
    if mode:
        ex, ey = oracle.d2q9()[:2]
        want = np.array([[oracle.knn(xy, (xy[0, i] - ex[k] * dx, xy[1, i] - ey[k] * dx), 1)[0]
                          for i in range(xy.shape[1])] for k in range(1, 9)])
        np.testing.assert_array_equal(d.departure_nodes(0), want)


def test_nearest_periodic_departure_nodes_match_oracle():
    n_side, K, deg, dx = 24, 16, 2, 2.5 / 24
    xy = mi.jittered_lattice(n_side, 0.3, seed=7)
    _, d = _same_cloud(xy, _periodic(K, deg, dx, mlbm.STENCIL_NEAREST))
    sidx, _ = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode="paper")
    np.testing.assert_array_equal(d.departure_nodes(0), sidx[1:, 0, :])


def test_batched_segments_device_build_matches_host():
    parts, segs = [], []
    specs = [(8, 9, 2, "p"), (12, 16, 3, "p"), (5, 6, 1, "p"), (20, 34, 5, "p"), (16, 12, 2, "pn")]
    for s, (n_side, k, deg, kind) in enumerate(specs):
        parts.append(mi.jittered_lattice(n_side, 0.3, seed=50 + s))
        segs.append(_periodic(k, deg, 0.5 / n_side, mlbm.STENCIL_NEAREST if kind == "pn" else None))
    xa, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=6)
    parts.append(xa)
    segs.append(_annulus(15, 2, 1.0 / 40))
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    _same_cloud(np.concatenate(parts, axis=1), segs, offs)


def test_duplicate_nodes_rejected():
    xy = mi.jittered_lattice(10, 0.3, seed=3)
    xy[:, 17] = xy[:, 42]
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_cloud(xy, _periodic(9, 2, 0.1), device=True)
    assert e.value.code == mlbm.EINVAL
    assert "duplicate" in str(e.value)


def _t(a):
    return torch.as_tensor(a, dtype=torch.float64, device=DEV)


def test_forced_annulus_steps_and_adjoint_identical_from_either_build():
    """Force directions and the transposed stencil are not exported: the forced, wall-bounded
    FP64 steps and the deterministic adjoint pull from the two builds must agree bit for bit."""
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[2000], seed=4)
    seg = _annulus(15, 2, 0.05)
    params = [(0.9, 1e-4, 1.0)]
    n = xy.shape[1]
    rng = np.random.default_rng(5)
    rho, u, v = 1 + 1e-3 * rng.standard_normal(n), 1e-3 * rng.standard_normal(n), 1e-3 * rng.standard_normal(n)
    outs = []
    for device in (False, True):
        c = mlbm.build_cloud(xy, seg, device=device)
        w = mlbm.build_weights(c)
        a = torch.empty(9 * n, dtype=torch.float64, device=DEV)
        b = torch.empty_like(a)
        mlbm.init(w, params, mlbm.F64, _t(rho), _t(u), _t(v), a)
        f0 = a.clone()
        for _ in range(10):
            mlbm.step(w, params, mlbm.F64, a, b)
            a, b = b, a
        lam = torch.as_tensor(np.random.default_rng(6).standard_normal(9 * n), device=DEV)
        lam_prev = torch.empty_like(lam)
        grad = torch.zeros(2, dtype=torch.float64, device=DEV)
        mlbm.adjoint_step(w, params, mlbm.F64, f0, lam, lam_prev, grad)
        outs.append((a.cpu().numpy(), lam_prev.cpu().numpy(), grad.cpu().numpy()))
    for x, y in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(x, y)


def test_full_size_device_build_matches_host():
    """2048^2 jittered cloud, N_L = 30: the whole stencil table and the permutation agree with
    the host build; the device build is the faster of the two."""
    xy = mi.jittered_lattice(2048, 0.3, seed=3)
    seg = _periodic(30, 4, 1.0 / 2048)
    torch.cuda.synchronize()
    mlbm.build_cloud(mi.jittered_lattice(64, 0.3, seed=3), _periodic(30, 4, 1.0 / 64), device=True)  # warm-up
    t0 = time.perf_counter()
    d = mlbm.build_cloud(xy, seg, device=True)
    t_dev = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = mlbm.build_cloud(xy, seg)
    t_host = time.perf_counter() - t0
    np.testing.assert_array_equal(d.perm(), h.perm())
    np.testing.assert_array_equal(d.stencil(0), h.stencil(0))
    print(f"device build {t_dev:.3f} s, host build {t_host:.3f} s")
    assert t_dev < t_host
