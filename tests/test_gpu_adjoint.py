"""GPU adjoint: each reverse kernel against central finite differences of the GPU forward, and
whole rollouts (sqrt(T) checkpointing) against the oracle's autograd reference gradient."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")
from oracle import torch_ref  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _annulus(h_key=1000, K=15, deg=2, dx=1.0 / 40, seed=3, upload=True):
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[h_key], seed=seed)
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=deg, dx_ml=dx)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    sidx = W = None
    if upload:
        sidx, W = oracle.weights(xy, K, deg, dx)
        w.upload(W[1:], sidx[1].astype(np.int32))
    return xy, dx, cloud, w, sidx, W


def _t(a):
    return torch.as_tensor(a, dtype=torch.float64, device=DEV).contiguous()


def _rand_state(w, params, xy, seed=0):
    rng = np.random.default_rng(seed)
    n = xy.shape[1]
    f = torch.empty(9 * w.n, dtype=torch.float64, device=DEV)
    mlbm.init(w, params, mlbm.F64, _t(1 + 1e-3 * rng.standard_normal(n)),
              _t(3e-3 * rng.standard_normal(n)), _t(3e-3 * rng.standard_normal(n)), f)
    f += _t(1e-4 * rng.standard_normal(9 * w.n))  # off-equilibrium part
    return f


def _step(w, params, s):
    out = torch.empty_like(s)
    mlbm.step(w, params, mlbm.F64, s, out)
    return out


@pytest.mark.parametrize("from_next", [False, True], ids=["recompute", "from_next"])
def test_adjoint_step_matches_finite_differences(from_next):
    """Both routes of the reverse step (fhat recomputed by interpolation, or taken from the
    forward's output) against central differences of the forward."""
    xy, dx, cloud, w, _, _ = _annulus()
    tau, g = 0.9, 2e-5
    params = [(tau, g, 1.0)]
    s = _rand_state(w, params, xy)
    rng = np.random.default_rng(5)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad,
                      s_next=_step(w, params, s) if from_next else None)
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)
    h = 1e-6
    fdt = (torch.dot(lam, _step(w, [(tau + h, g, 1.0)], s)) - torch.dot(lam, _step(w, [(tau - h, g, 1.0)], s))) / (2 * h)
    assert float(grad[0]) == pytest.approx(float(fdt), rel=1e-6)
    hg = 1e-6
    fdg = (torch.dot(lam, _step(w, [(tau, g + hg, 1.0)], s)) - torch.dot(lam, _step(w, [(tau, g - hg, 1.0)], s))) / (2 * hg)
    assert float(grad[1]) == pytest.approx(float(fdg), rel=1e-6)


def test_adjoint_transpose_dot_product_periodic():
    """<S x, y> = <x, S^T y> for the linear part: with tau = 1 the collision Jacobian at rest is
    a projector, so compare against finite differences on a periodic cloud instead."""
    xy = mi.jittered_lattice(24, 0.3, seed=4)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=16, degree=3, dx_ml=0.5 / 24))
    w = mlbm.build_weights(cloud)
    params = [(0.75, 0.0, 1.0)]
    s = _rand_state(w, params, xy, seed=2)
    rng = np.random.default_rng(6)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad)
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)


def test_moments_and_init_adjoints_match_finite_differences():
    xy, dx, cloud, w, _, _ = _annulus()
    tau, g = 0.9, 2e-5
    params = [(tau, g, 1.0)]
    n = xy.shape[1]
    s = _rand_state(w, params, xy, seed=3)
    rng = np.random.default_rng(7)
    dr, du, dv = (_t(rng.standard_normal(n)) for _ in range(3))
    lam = torch.empty_like(s)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    mlbm.moments_adjoint(w, params, mlbm.F64, s, dr, du, dv, lam, grad)
    v = _t(rng.standard_normal(9 * w.n))

    def J(state, p=params):
        r, u, vv = mlbm.moments(w, p, mlbm.F64, state)
        return torch.dot(dr, r) + torch.dot(du, u) + torch.dot(dv, vv)

    eps = 1e-6
    fd = (J(s + eps * v) - J(s - eps * v)) / (2 * eps)
    assert float(torch.dot(lam, v)) == pytest.approx(float(fd), rel=1e-7)
    fdg = (J(s, [(tau, g + 1e-7, 1.0)]) - J(s, [(tau, g - 1e-7, 1.0)])) / 2e-7
    assert float(grad[1]) == pytest.approx(float(fdg), rel=1e-6)
    # init adjoint
    rho0 = 1 + 1e-3 * rng.standard_normal(n)
    u0, v0 = 2e-3 * rng.standard_normal(n), 2e-3 * rng.standard_normal(n)
    lam0 = _t(rng.standard_normal(9 * w.n))
    d0 = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in range(3)]
    grad.zero_()
    mlbm.init_adjoint(w, params, mlbm.F64, _t(rho0), _t(u0), _t(v0), lam0, d0[0], d0[1], d0[2], grad)

    def I(r, u, vv, p=params):
        f = torch.empty(9 * w.n, dtype=torch.float64, device=DEV)
        mlbm.init(w, p, mlbm.F64, _t(r), _t(u), _t(vv), f)
        return torch.dot(lam0, f)

    d = rng.standard_normal(n)
    for which in range(3):
        args_p = [rho0.copy(), u0.copy(), v0.copy()]
        args_m = [rho0.copy(), u0.copy(), v0.copy()]
        args_p[which] = args_p[which] + 1e-6 * d
        args_m[which] = args_m[which] - 1e-6 * d
        fd = (I(*args_p) - I(*args_m)) / 2e-6
        assert float(d0[which].cpu().numpy() @ d) == pytest.approx(float(fd), rel=1e-7)
    fdg = (I(rho0, u0, v0, [(tau, g + 1e-7, 1.0)]) - I(rho0, u0, v0, [(tau, g - 1e-7, 1.0)])) / 2e-7
    assert float(grad[1]) == pytest.approx(float(fdg), rel=1e-6)


def _profile_loss(xy, r, u, v, g, tau, dx):
    """Velocity-profile mismatch: sum_i (|u_i| - u_target(r_i))^2 with the analytic profile of
    eq. (bch_solution) as the target."""
    rr = np.hypot(xy[0], xy[1])
    target = oracle.annulus_velocity(rr / dx, g, oracle.lattice_viscosity(tau), 0.5 / dx, 1.0 / dx)
    tt = torch.as_tensor(np.abs(target), dtype=torch.float64, device=u.device)
    speed = torch.sqrt(u * u + v * v + 1e-30)
    return ((speed - tt) ** 2).sum()


@pytest.mark.parametrize("checkpoint", [None, 1, 7])
def test_rollout_gradient_matches_oracle_autograd(checkpoint):
    from paper_2306_01525_gb300.autograd import rollout

    xy, dx, cloud, w, sidx, W = _annulus()
    n = xy.shape[1]
    tau, g, steps = 0.9, 5e-5, 40
    rng = np.random.default_rng(11)
    rho0 = 1 + 1e-4 * rng.standard_normal(n)
    u0, v0 = 1e-4 * rng.standard_normal(n), 1e-4 * rng.standard_normal(n)
    # GPU
    tt = torch.tensor(tau, dtype=torch.float64, device=DEV, requires_grad=True)
    gt = torch.tensor(g, dtype=torch.float64, device=DEV, requires_grad=True)
    r0, a0, b0 = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True) for a in (rho0, u0, v0))
    r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=mlbm.F64, checkpoint=checkpoint)
    _profile_loss(xy, r, u, v, g, tau, dx).backward()
    # oracle autograd (same shape vectors)
    T = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tc, gc, rc0, ac0, bc0 = T(tau), T(g), T(rho0), T(u0), T(v0)
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    fdir = oracle.azimuthal_force(xy, 1.0)
    rr, uu, vv = torch_ref.rollout(sidx, W, tc, gc, fdir, mask, rc0, ac0, bc0, steps)
    _profile_loss(xy, rr, uu, vv, g, tau, dx).backward()
    assert tt.grad.item() == pytest.approx(tc.grad.item(), rel=1e-8)
    assert gt.grad.item() == pytest.approx(gc.grad.item(), rel=1e-8)
    for gpu, ref in ((r0, rc0), (a0, ac0), (b0, bc0)):
        np.testing.assert_allclose(gpu.grad.cpu().numpy(), ref.grad.numpy(), rtol=1e-7,
                                   atol=1e-8 * np.abs(ref.grad.numpy()).max())


def test_fp32_rollout_gradient_close_to_fp64_reference():
    from paper_2306_01525_gb300.autograd import rollout

    xy, dx, cloud, w, sidx, W = _annulus()
    n = xy.shape[1]
    tau, g, steps = 0.9, 5e-5, 40
    grads = {}
    for dt in (mlbm.F64, mlbm.F32):
        tt = torch.tensor(tau, dtype=torch.float64, device=DEV, requires_grad=True)
        gt = torch.tensor(g, dtype=torch.float64, device=DEV, requires_grad=True)
        r0 = torch.ones(n, dtype=torch.float64, device=DEV, requires_grad=True)
        a0 = torch.zeros(n, dtype=torch.float64, device=DEV, requires_grad=True)
        b0 = torch.zeros(n, dtype=torch.float64, device=DEV, requires_grad=True)
        r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=dt)
        _profile_loss(xy, r, u, v, g, tau, dx).backward()
        grads[dt] = (tt.grad.item(), gt.grad.item())
    assert grads[mlbm.F32][0] == pytest.approx(grads[mlbm.F64][0], rel=1e-3)
    assert grads[mlbm.F32][1] == pytest.approx(grads[mlbm.F64][1], rel=1e-3)


def test_fp32_rollout_gradient_within_1e4_of_oracle_and_finite_differences():
    """The adjoint workload's recipe at test size: an annulus of about 2k scattered nodes,
    N_L 24, P_3, tau 0.7, 300 FP32 steps with sqrt(T) checkpoints, loss = velocity-profile
    mismatch against eq. (bch_solution).  The FP32 gradients with respect to tau, g and the
    initial density agree with the oracle's autograd (FP64, same shape vectors) and with central
    differences of the FP64 forward to 1e-4 relative."""
    from paper_2306_01525_gb300.autograd import rollout

    xy, dx, cloud, w, sidx, W = _annulus(h_key=2000, K=24, deg=3, dx=1.0 / 40, seed=5)
    n = xy.shape[1]
    tau, g, steps = 0.7, 1e-5, 300
    rng = np.random.default_rng(21)
    rho0 = 1 + 1e-4 * rng.standard_normal(n)
    zeros = np.zeros(n)

    def gpu(dtype, tau_, g_, grad):
        tt = torch.tensor(tau_, dtype=torch.float64, device=DEV, requires_grad=grad)
        gt = torch.tensor(g_, dtype=torch.float64, device=DEV, requires_grad=grad)
        r0, a0, b0 = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=grad)
                      for a in (rho0, zeros, zeros))
        r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=dtype)
        L = _profile_loss(xy, r, u, v, g, tau, dx)
        if not grad:
            return float(L)
        L.backward()
        return tt.grad.item(), gt.grad.item(), r0.grad.cpu().numpy()

    gtau, gg, grho = gpu(mlbm.F32, tau, g, True)
    # oracle autograd reference
    T = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tc, gc, rc0, ac0, bc0 = T(tau), T(g), T(rho0), T(zeros), T(zeros)
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    fdir = oracle.azimuthal_force(xy, 1.0)
    rr, uu, vv = torch_ref.rollout(sidx, W, tc, gc, fdir, mask, rc0, ac0, bc0, steps)
    _profile_loss(xy, rr, uu, vv, g, tau, dx).backward()
    assert gtau == pytest.approx(tc.grad.item(), rel=1e-4)
    assert gg == pytest.approx(gc.grad.item(), rel=1e-4)
    ref = rc0.grad.numpy()
    assert np.linalg.norm(grho - ref) <= 1e-4 * np.linalg.norm(ref)
    # central differences of the FP64 forward
    fdt = (gpu(mlbm.F64, tau + 1e-5, g, False) - gpu(mlbm.F64, tau - 1e-5, g, False)) / 2e-5
    fdg = (gpu(mlbm.F64, tau, g + 1e-8, False) - gpu(mlbm.F64, tau, g - 1e-8, False)) / 2e-8
    assert gtau == pytest.approx(fdt, rel=1e-4)
    assert gg == pytest.approx(fdg, rel=1e-4)


def test_rollout_gradient_matches_central_differences_20k():
    """Annulus with ~20k scattered nodes, N_L = 24, P_3, 200 FP64 steps: dL/dtau and dL/dg from
    the adjoint agree with central finite differences of the GPU forward to 1e-4."""
    from paper_2306_01525_gb300.autograd import rollout

    xy, dx, cloud, w, _, _ = _annulus(h_key=20000, K=24, deg=3, dx=1.0 / 320, seed=5, upload=False)
    n = xy.shape[1]
    tau, g, steps = 0.7, 1e-5, 200
    ones, zeros = np.ones(n), np.zeros(n)

    def loss(tau_, g_, grad=False):
        tt = torch.tensor(tau_, dtype=torch.float64, device=DEV, requires_grad=grad)
        gt = torch.tensor(g_, dtype=torch.float64, device=DEV, requires_grad=grad)
        r0, a0, b0 = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=grad) for a in (ones, zeros, zeros))
        r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=mlbm.F64)
        L = _profile_loss(xy, r, u, v, g, tau, dx)
        if grad:
            L.backward()
            return tt.grad.item(), gt.grad.item()
        return float(L)

    gtau, gg = loss(tau, g, grad=True)
    h = 1e-5
    fdt = (loss(tau + h, g) - loss(tau - h, g)) / (2 * h)
    fdg = (loss(tau, g + 1e-8) - loss(tau, g - 1e-8)) / 2e-8
    assert gtau == pytest.approx(fdt, rel=1e-4)
    assert gg == pytest.approx(fdg, rel=1e-4)


@pytest.mark.parametrize("from_next", [False, True], ids=["recompute", "from_next"])
def test_fp32_adjoint_step_close_to_fp64_and_deterministic(from_next):
    """The FP32 reverse step (transpose of the difference-form FP32 forward) agrees with the FP64
    reverse step to FP32 accuracy, and repeats bit for bit."""
    xy, dx, cloud, w, _, _ = _annulus(upload=False)
    params = [(0.9, 2e-5, 1.0)]
    n = xy.shape[1]
    rng = np.random.default_rng(8)
    fields = [_t(1 + 1e-3 * rng.standard_normal(n)), _t(3e-3 * rng.standard_normal(n)),
              _t(3e-3 * rng.standard_normal(n))]
    pert = _t(1e-4 * rng.standard_normal(9 * w.n))
    lam = _t(rng.standard_normal(9 * w.n))
    out = {}
    for dt, td in ((mlbm.F64, torch.float64), (mlbm.F32, torch.float32)):
        # the same physical state in each storage form (FP32: deviations from omega_k rho0)
        s = torch.empty(9 * w.n, dtype=td, device=DEV)
        mlbm.init(w, params, dt, *fields, s)
        s += pert.to(td)
        sn = None
        if from_next:
            sn = torch.empty_like(s)
            mlbm.step(w, params, dt, s, sn)
        lp = torch.empty(9 * w.n, dtype=td, device=DEV)
        g = torch.zeros(2, dtype=torch.float64, device=DEV)
        mlbm.adjoint_step(w, params, dt, s, lam.to(td), lp, g, s_next=sn)
        out[dt] = (lp.double(), g.clone())
        lp2 = torch.empty_like(lp)
        g2 = torch.zeros(2, dtype=torch.float64, device=DEV)
        mlbm.adjoint_step(w, params, dt, s, lam.to(td), lp2, g2, s_next=sn)
        assert torch.equal(lp, lp2) and torch.equal(g, g2)
    a, b = out[mlbm.F64][0], out[mlbm.F32][0]
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) < 1e-5
    np.testing.assert_allclose(out[mlbm.F32][1].cpu().numpy(), out[mlbm.F64][1].cpu().numpy(), rtol=1e-4)


@pytest.mark.parametrize("n_side", [200, 600])
@pytest.mark.parametrize("from_next", [False, True], ids=["recompute", "from_next"])
def test_adjoint_step_large_tiles_matches_finite_differences(from_next, n_side):
    """Clouds large enough for 128-node tiles (40k nodes) and 512-node tiles (360k nodes): the
    tiled reverse step against central differences of the forward."""
    xy = mi.jittered_lattice(n_side, 0.3, seed=12)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=12, degree=2,
                                      dx_ml=1.0 / n_side))
    w = mlbm.build_weights(cloud)
    params = [(0.8, 1e-5, 1.0)]
    s = _rand_state(w, params, xy, seed=13)
    rng = np.random.default_rng(14)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad,
                      s_next=_step(w, params, s) if from_next else None)
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)
    h = 1e-6
    fdt = (torch.dot(lam, _step(w, [(0.8 + h, 1e-5, 1.0)], s)) - torch.dot(lam, _step(w, [(0.8 - h, 1e-5, 1.0)], s))) / (2 * h)
    assert float(grad[0]) == pytest.approx(float(fdt), rel=1e-6)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_adjoint_from_next_state_agrees_with_recompute(dtype):
    """The reverse step that takes fhat's moments and non-equilibrium part from the forward's
    output equals the one that recomputes fhat by interpolation, to rounding (FP64: 1e-11; FP32:
    the non-equilibrium part is divided by 1 - 1/tau = -0.43, 1e-5); near tau = 1 the library
    recomputes whatever it is given, so both calls give the same bits."""
    xy, dx, cloud, w, _, _ = _annulus(upload=False)
    dt, td = (mlbm.F64, torch.float64) if dtype == "f64" else (mlbm.F32, torch.float32)
    n = xy.shape[1]
    rng = np.random.default_rng(21)
    fields = [_t(1 + 1e-3 * rng.standard_normal(n)), _t(3e-3 * rng.standard_normal(n)),
              _t(3e-3 * rng.standard_normal(n))]
    pert = _t(1e-4 * rng.standard_normal(9 * w.n)).to(td)
    lam = _t(rng.standard_normal(9 * w.n)).to(td)
    for tau, same_bits in ((0.7, False), (1.0, True), (1.05, True), (1.2, False)):
        params = [(tau, 3e-5, 1.0)]
        s = torch.empty(9 * w.n, dtype=td, device=DEV)
        mlbm.init(w, params, dt, *fields, s)
        s += pert
        sn = torch.empty_like(s)
        mlbm.step(w, params, dt, s, sn)
        res = []
        for nxt in (None, sn):
            lp = torch.empty_like(s)
            g = torch.zeros(2, dtype=torch.float64, device=DEV)
            mlbm.adjoint_step(w, params, dt, s, lam, lp, g, s_next=nxt)
            res.append((lp.double(), g.cpu().numpy()))
        (a, ga), (b, gb) = res
        if same_bits:
            assert torch.equal(a, b) and np.array_equal(ga, gb)
            continue
        tol = 1e-11 if dtype == "f64" else 1e-5
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) < tol
        np.testing.assert_allclose(gb, ga, rtol=tol if dtype == "f64" else 1e-4)


@pytest.mark.parametrize("taus", [(0.8, 0.7, 1.3), (0.8, 1.02, 1.3)], ids=["from_next", "recompute"])
def test_adjoint_step_batched_segments_match_finite_differences(taus):
    """Three independent runs of uneven size, stencil and degree in one weights object (one
    reverse step over all their tiles): the transposed step and each segment's dL/dtau and dL/dg
    against central differences.  With tau = 1.02 in one segment (|1 - 1/tau| < 1/16) the whole
    call takes the recompute route."""
    cases = [(16, 12, 2), (20, 16, 3), (12, 9, 2)]
    parts, segs = [], []
    for s, (ns, K, deg) in enumerate(cases):
        parts.append(mi.jittered_lattice(ns, 0.3, seed=90 + s))
        segs.append(dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=0.7 / ns))
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    w = mlbm.build_weights(mlbm.build_cloud(xy, segs, offs))
    gs = (2e-5, -1e-5, 3e-5)
    params = [(t, g, 1.0) for t, g in zip(taus, gs)]
    s = _rand_state(w, params, xy, seed=31)
    rng = np.random.default_rng(32)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(2 * len(cases), dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad, s_next=_step(w, params, s))
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)
    for seg in range(len(cases)):
        for c, h in ((0, 1e-6), (1, 1e-6)):
            lo, hi = [list(p) for p in params], [list(p) for p in params]
            lo[seg][c] -= h
            hi[seg][c] += h
            f = (torch.dot(lam, _step(w, [tuple(p) for p in hi], s)) -
                 torch.dot(lam, _step(w, [tuple(p) for p in lo], s))) / (2 * h)
            assert float(grad[2 * seg + c]) == pytest.approx(float(f), rel=1e-6), (seg, c)


def test_adjoint_step_many_segments_match_finite_differences():
    """Ten segments in one weights object: more than the pull kernel reduces itself, so the
    per-segment gradient sums go through the separate reduction launch; each segment's dL/dtau
    and dL/dg against central differences (from the forward's next state, FP64)."""
    parts, segs = [], []
    for s in range(10):
        ns = 10 + s % 4
        parts.append(mi.jittered_lattice(ns, 0.3, seed=140 + s))
        segs.append(dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=9 + (s % 3), degree=2, dx_ml=0.6 / ns))
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    w = mlbm.build_weights(mlbm.build_cloud(xy, segs, offs))
    params = [(0.75 + 0.05 * s, 1e-5 * (s - 4), 1.0) for s in range(10)]
    st = _rand_state(w, params, xy, seed=41)
    rng = np.random.default_rng(42)
    lam = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(20, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, st, lam, lam_prev, grad, s_next=_step(w, params, st))
    for seg in (0, 3, 9):
        for c in (0, 1):
            lo, hi = [list(p) for p in params], [list(p) for p in params]
            lo[seg][c] -= 1e-6
            hi[seg][c] += 1e-6
            f = (torch.dot(lam, _step(w, [tuple(p) for p in hi], st)) -
                 torch.dot(lam, _step(w, [tuple(p) for p in lo], st))) / 2e-6
            assert float(grad[2 * seg + c]) == pytest.approx(float(f), rel=1e-6), (seg, c)


def test_upload_after_adjoint_rebuilds_its_coefficients():
    """Shape vectors uploaded after a reverse step replace the adjoint's transposed
    coefficients too: the next reverse step equals that of a fresh weights object holding the
    uploaded vectors, bit for bit (and differs from the step before the upload)."""
    xy, dx, cloud, w, _, _ = _annulus(upload=False)
    params = [(0.9, 2e-5, 1.0)]
    s = _rand_state(w, params, xy, seed=21)
    rng = np.random.default_rng(22)
    lam = _t(rng.standard_normal(9 * w.n))

    def reverse(wt):
        lp = torch.empty_like(lam)
        g = torch.zeros(2, dtype=torch.float64, device=DEV)
        mlbm.adjoint_step(wt, params, mlbm.F64, s, lam, lp, g, s_next=_step(wt, params, s))
        return lp, g

    before, _ = reverse(w)
    sidx, W = oracle.weights(xy, 15, 2, dx)
    idx = sidx[1].astype(np.int32)
    w.upload(W[1:], idx)
    after, g_after = reverse(w)
    fresh = mlbm.build_weights(cloud)
    fresh.upload(W[1:], idx)
    ref, g_ref = reverse(fresh)
    assert torch.equal(after, ref) and torch.equal(g_after, g_ref)
    assert not torch.equal(after, before)
