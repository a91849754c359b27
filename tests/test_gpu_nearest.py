"""Nearest-node stencils on the GPU (MLBM_STENCIL_NEAREST): each departure point x_i - e_k dx_ml
is interpolated in the stencil of the Eulerian node nearest to it (Sec. 2.3, appendix
algorithm), against the oracle's "paper" mode; and the paper's convergence study at a fixed
streaming distance (Fig. tgv_conv_P): refining the cloud drives the meshless error onto the
lattice-LBM error at dx = dx_ml."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(a, dtype=torch.float64, device=DEV)


def _periodic_nearest(n_side, K, deg, dx, seed):
    xy = mi.jittered_lattice(n_side, 0.3, seed=seed)
    seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=dx,
               stencil_mode=mlbm.STENCIL_NEAREST)
    cloud = mlbm.build_cloud(xy, seg)
    return xy, cloud, mlbm.build_weights(cloud)


@pytest.mark.parametrize("n_side,K,deg,ratio", [(24, 16, 2, 2.5), (20, 25, 4, 1.5)])
def test_nearest_weights_and_departure_nodes_match_oracle(n_side, K, deg, ratio):
    dx = ratio / n_side
    xy, cloud, w = _periodic_nearest(n_side, K, deg, dx, seed=7)
    assert w.n_bad == 0
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode="paper")
    np.testing.assert_array_equal(cloud.departure_nodes(0), sidx[1:, 0, :])
    err = np.max(np.abs(w.download(0) - W[1:]))
    assert err <= {2: 1e-9, 4: 1e-7}[deg], err


@pytest.mark.parametrize("dtype,tol,n_side,K,deg,steps", [("f64", 1e-12, 24, 16, 3, 60), ("f32", None, 24, 16, 3, 60),
                                                        ("f64", 1e-12, 200, 9, 1, 20)])
def test_nearest_step_matches_oracle(dtype, tol, n_side, K, deg, steps):
    """Oracle shape vectors uploaded; FP64 agrees per step to 1e-12, FP32 within 1e-6 relative
    L2 of the velocity after the run (dx_ml = 2 h: departure points beyond the own stencil).
    24^2 nodes run one-warp tiles, 200^2 the 128-node tiles."""
    dx, tau = 2.0 / n_side, 0.8
    xy, cloud, w = _periodic_nearest(n_side, K, deg, dx, seed=8)
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode="paper")
    w.upload(W[1:], oracle.stencils(xy, K, box=(1.0, 1.0)).astype(np.int32))
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.02)
    st = oracle.Stepper(sidx, W, tau)
    f = oracle.init_equilibrium(rho, u, v)
    dt = mlbm.F64 if dtype == "f64" else mlbm.F32
    a = torch.empty(9 * w.n, dtype=torch.float64 if dtype == "f64" else torch.float32, device=DEV)
    b = torch.empty_like(a)
    mlbm.init(w, params, dt, _t(rho), _t(u), _t(v), a)
    perm = cloud.perm()
    for it in range(steps):
        mlbm.step(w, params, dt, a, b)
        a, b = b, a
        f = st.step(f)
        if dtype == "f64" and it % 10 == 9:
            post = oracle.collide_field(f, tau)
            got = np.empty_like(post)
            got[:, perm] = a.view(9, -1).cpu().numpy()
            assert np.max(np.abs(got - post)) <= tol * np.max(np.abs(post)), it
    _, ug, vg = mlbm.moments(w, params, dt, a)
    _, uo, vo = oracle.moments_field(f)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - uo) ** 2 + (vg - vo) ** 2) / np.sum(uo ** 2 + vo ** 2))
    assert err <= (1e-11 if dtype == "f64" else 1e-6), err


def test_nearest_annulus_step_with_walls_matches_oracle():
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[2000], seed=4)
    dx, K, deg, tau, g = 0.05, 15, 2, 1.0, 1e-5
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=deg, dx_ml=dx,
               stencil_mode=mlbm.STENCIL_NEAREST)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    sidx, W = oracle.weights(xy, K, deg, dx, mode="paper")
    np.testing.assert_array_equal(cloud.departure_nodes(0), sidx[1:, 0, :])
    w.upload(W[1:], oracle.stencils(xy, K).astype(np.int32))
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    force = oracle.azimuthal_force(xy, g)
    st = oracle.Stepper(sidx, W, tau, mask=mask, force=force)
    n = xy.shape[1]
    rng = np.random.default_rng(3)
    rho, u, v = 1 + 1e-3 * rng.standard_normal(n), 1e-3 * rng.standard_normal(n), 1e-3 * rng.standard_normal(n)
    params = [(tau, g, 1.0)]
    a = torch.empty(9 * n, dtype=torch.float64, device=DEV)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F64, _t(rho), _t(u), _t(v), a)
    f = oracle.init_equilibrium(rho, u, v)
    perm = cloud.perm()
    for it in range(20):
        mlbm.step(w, params, mlbm.F64, a, b)
        a, b = b, a
        f = st.step(f)
    post = oracle.collide_field(f, tau, force)
    got = np.empty_like(post)
    got[:, perm] = a.view(9, -1).cpu().numpy()
    assert np.max(np.abs(got - post)) <= 1e-12 * np.max(np.abs(post))


def _tgv_error(n, K, deg, L, u0, tau, steps):
    xy, cloud, w = _periodic_nearest(n, K, deg, 1.0 / L, seed=60 + n)
    rho, u, v = mi.tgv_initial(xy, u0)
    params = [(tau, 0.0, 1.0)]
    a = torch.empty(9 * w.n, dtype=torch.float64, device=DEV)
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F64, _t(rho), _t(u), _t(v), a)
    res = mlbm.run(w, params, mlbm.F64, a, b, steps)
    _, um, _ = mlbm.moments(w, params, mlbm.F64, res)
    ut, _ = oracle.tgv_velocity(xy[0] * L, xy[1] * L, steps, u0=u0, nu=oracle.lattice_viscosity(tau), L=L)
    return oracle.l2_norm(um.cpu().numpy(), ut)


def test_fixed_streaming_distance_converges_to_lattice_lbm_error():
    """dx_ml = 1/32, Taylor-Green to t_end, N_L = 25: refining the cloud from sqrt(N) = 16 to 128
    (h/dx_ml from 2 to 1/4) brings the P_4 error down onto the lattice-LBM error at dx = 1/32,
    and P_4 is more accurate than P_2 on the coarse clouds (oracle on the same inputs:
    P_4 2.2e-2, 7.0e-3, 6.810e-3, 6.808e-3; lattice LBM 6.808e-3)."""
    L, tau, u0 = 32, 0.8, 0.01
    steps = int(round(oracle.tgv_end_time(nu=oracle.lattice_viscosity(tau), L=L)))
    xy = mi.lattice(L)
    rho, u, v = mi.tgv_initial(xy, u0)
    a = torch.empty(9 * L * L, dtype=torch.float64, device=DEV)
    b = torch.empty_like(a)
    mom = torch.empty(3 * L * L, dtype=torch.float64, device=DEV)
    mlbm.lattice_init(L, L, (tau, 0.0, 1.0), mlbm.F64, _t(rho), _t(u), _t(v), a)
    for _ in range(steps):
        mlbm.lattice_step(L, L, (tau, 0.0, 1.0), mlbm.F64, a, b, mom)
        a, b = b, a
    ut, _ = oracle.tgv_velocity(xy[0] * L, xy[1] * L, steps, u0=u0, nu=oracle.lattice_viscosity(tau), L=L)
    e_lbm = oracle.l2_norm(mom.view(3, -1)[1].cpu().numpy(), ut)
    e4 = [_tgv_error(n, 25, 4, L, u0, tau, steps) for n in (16, 32, 64, 128)]
    e2 = [_tgv_error(n, 25, 2, L, u0, tau, steps) for n in (16, 32)]
    assert e4[0] > e4[1] > e4[2], e4
    assert abs(e4[3] - e4[2]) <= 1e-3 * e4[2], e4  # saturated
    assert abs(e4[-1] - e_lbm) <= 0.01 * e_lbm, (e4, e_lbm)
    assert e4[0] < e2[0] and e4[1] < e2[1], (e2, e4)


def _rand_state(w, params, n, seed, dtype=mlbm.F64):
    rng = np.random.default_rng(seed)
    td = torch.float64 if dtype == mlbm.F64 else torch.float32
    f = torch.empty(9 * w.n, dtype=td, device=DEV)
    mlbm.init(w, params, dtype, _t(1 + 1e-3 * rng.standard_normal(n)), _t(3e-3 * rng.standard_normal(n)),
              _t(3e-3 * rng.standard_normal(n)), f)
    f += _t(1e-4 * rng.standard_normal(9 * w.n)).to(td)  # off-equilibrium part
    return f


def _step(w, params, s, dtype=mlbm.F64):
    out = torch.empty_like(s)
    mlbm.step(w, params, dtype, s, out)
    return out


def _nearest_cloud(kind, device=False):
    if kind == "annulus":
        xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
        seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=15, degree=2, dx_ml=1.0 / 20,
                   stencil_mode=mlbm.STENCIL_NEAREST)
    else:
        n_side = int(kind)
        xy = mi.jittered_lattice(n_side, 0.3, seed=n_side)
        seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=16 if n_side < 100 else 12,
                   degree=3 if n_side < 100 else 2, dx_ml=2.0 / n_side, stencil_mode=mlbm.STENCIL_NEAREST)
    return xy, mlbm.build_weights(mlbm.build_cloud(xy, seg, device=device))


@pytest.mark.parametrize("kind", ["24", "annulus", "200", "600"])
def test_adjoint_nearest_matches_finite_differences(kind):
    """The reverse step of a nearest-node cloud (each population interpolated in its departure
    node's stencil, Sec. 2.3) against central differences of the forward: the transposed step
    <lam_prev, v> and dL/dtau, dL/dg.  Periodic clouds with dx_ml = 2 h (departure nodes other
    than the node itself) at 576, 40 k and 360 k nodes (one-warp, 128- and 512-node tiles), and
    an annulus with bounce-back walls."""
    xy, w = _nearest_cloud(kind, device=kind in ("200", "600"))
    tau, g = 0.8, 1e-5
    params = [(tau, g, 1.0)]
    s = _rand_state(w, params, xy.shape[1], seed=41)
    rng = np.random.default_rng(42)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad, s_next=_step(w, params, s))
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)
    for c, h in ((0, 1e-6), (1, 1e-6)):
        hi, lo = list(params[0]), list(params[0])
        hi[c] += h
        lo[c] -= h
        f = (torch.dot(lam, _step(w, [tuple(hi)], s)) - torch.dot(lam, _step(w, [tuple(lo)], s))) / (2 * h)
        assert float(grad[c]) == pytest.approx(float(f), rel=1e-6), c


def test_adjoint_nearest_fp32_close_to_fp64_and_deterministic():
    """FP32 reverse step of a nearest-node annulus (transpose of the forward's difference form to
    the departure node's value) against the FP64 reverse step, and bit-for-bit repeatable."""
    xy, w = _nearest_cloud("annulus")
    params = [(0.9, 2e-5, 1.0)]
    n = xy.shape[1]
    rng = np.random.default_rng(43)
    fields = [_t(1 + 1e-3 * rng.standard_normal(n)), _t(3e-3 * rng.standard_normal(n)),
              _t(3e-3 * rng.standard_normal(n))]
    pert = _t(1e-4 * rng.standard_normal(9 * w.n))
    lam = _t(rng.standard_normal(9 * w.n))
    out = {}
    for dt, td in ((mlbm.F64, torch.float64), (mlbm.F32, torch.float32)):
        s = torch.empty(9 * w.n, dtype=td, device=DEV)
        mlbm.init(w, params, dt, *fields, s)
        s += pert.to(td)
        sn = _step(w, params, s, dt)
        res = []
        for _ in range(2):
            lp = torch.empty(9 * w.n, dtype=td, device=DEV)
            g = torch.zeros(2, dtype=torch.float64, device=DEV)
            mlbm.adjoint_step(w, params, dt, s, lam.to(td), lp, g, s_next=sn)
            res.append((lp, g))
        assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
        out[dt] = (res[0][0].double(), res[0][1])
    a, b = out[mlbm.F64][0], out[mlbm.F32][0]
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) < 1e-5
    np.testing.assert_allclose(out[mlbm.F32][1].cpu().numpy(), out[mlbm.F64][1].cpu().numpy(), rtol=1e-4)


def test_adjoint_nearest_needs_next_state():
    """Nearest-node clouds take the reverse step from the forward's output only: without s_next,
    or with |1 - 1/tau| < 1/16 (where that route is ill-conditioned), the call is refused."""
    xy, cloud, w = _periodic_nearest(12, 9, 2, 2.0 / 12, seed=9)
    f = _rand_state(w, [(0.8, 0.0, 1.0)], xy.shape[1], seed=44)
    grad = torch.zeros(2, dtype=torch.float64, device=DEV)
    for tau, sn in ((0.8, None), (1.02, f.clone())):
        with pytest.raises(mlbm.MLBMError) as e:
            mlbm.adjoint_step(w, [(tau, 0.0, 1.0)], mlbm.F64, f, f.clone(), f.clone(), grad, s_next=sn)
        assert e.value.code == mlbm.EINVAL


def test_rollout_gradient_nearest_matches_central_differences():
    """A whole rollout on a nearest-node annulus with walls (sqrt(T) checkpoints, 60 FP64
    steps): dL/dtau, dL/dg and the initial-density gradient (along a random direction) from
    the adjoint against central differences of the GPU forward."""
    from paper_2306_01525_gb300.autograd import rollout

    xy, w = _nearest_cloud("annulus")
    n = xy.shape[1]
    tau, g, steps = 0.8, 1e-5, 60
    rng = np.random.default_rng(45)
    ones, zeros = np.ones(n), np.zeros(n)
    d_rho = rng.standard_normal(n)
    target = 1e-3 * rng.standard_normal(n)

    def loss(tau_, g_, rho0, grad=False):
        tt = torch.tensor(tau_, dtype=torch.float64, device=DEV, requires_grad=grad)
        gt = torch.tensor(g_, dtype=torch.float64, device=DEV, requires_grad=grad)
        r0 = torch.tensor(rho0, dtype=torch.float64, device=DEV, requires_grad=grad)
        a0, b0 = (torch.tensor(a, dtype=torch.float64, device=DEV) for a in (zeros, zeros))
        r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=mlbm.F64)
        L = torch.sum((u - _t(target)) ** 2 + v ** 2) + torch.sum((r - 1.0) ** 2)
        if grad:
            L.backward()
            return tt.grad.item(), gt.grad.item(), float(torch.dot(r0.grad, _t(d_rho)))
        return float(L)

    rho0 = ones + 1e-3 * rng.standard_normal(n)
    gtau, gg, gr = loss(tau, g, rho0, grad=True)
    h = 1e-5
    fdt = (loss(tau + h, g, rho0) - loss(tau - h, g, rho0)) / (2 * h)
    fdg = (loss(tau, g + 1e-8, rho0) - loss(tau, g - 1e-8, rho0)) / 2e-8
    e = 1e-6
    fdr = (loss(tau, g, rho0 + e * d_rho) - loss(tau, g, rho0 - e * d_rho)) / (2 * e)
    assert gtau == pytest.approx(fdt, rel=1e-5)
    assert gg == pytest.approx(fdg, rel=1e-5)
    assert gr == pytest.approx(fdr, rel=1e-6)


def test_rollout_gradient_nearest_matches_oracle_autograd():
    """Nearest-node annulus with walls, the oracle's paper-mode shape vectors uploaded: the
    gradients of a 40-step FP64 rollout (tau, g and the initial fields) equal those of the
    oracle's autograd reference, whose streaming gathers each direction through its own
    (departure-node) stencil."""
    from oracle import torch_ref
    from paper_2306_01525_gb300.autograd import rollout

    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    K, deg, dx = 15, 2, 1.0 / 20
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=deg, dx_ml=dx,
               stencil_mode=mlbm.STENCIL_NEAREST)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    sidx, W = oracle.weights(xy, K, deg, dx, mode="paper")
    w.upload(W[1:], oracle.stencils(xy, K).astype(np.int32))
    n = xy.shape[1]
    tau, g, steps = 0.9, 5e-5, 40
    rng = np.random.default_rng(46)
    rho0 = 1 + 1e-4 * rng.standard_normal(n)
    u0, v0 = 1e-4 * rng.standard_normal(n), 1e-4 * rng.standard_normal(n)
    tgt = 1e-3 * rng.standard_normal(n)

    def loss(r, u, v, T):
        return torch.sum((u - T(tgt)) ** 2 + v ** 2) + torch.sum((r - 1.0) ** 2)

    G = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True)
    tt, gt, r0, a0, b0 = G(tau), G(g), G(rho0), G(u0), G(v0)
    r, u, v = rollout(w, tt, gt, r0, a0, b0, steps, dtype=mlbm.F64)
    loss(r, u, v, lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)).backward()
    C = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tc, gc, rc0, ac0, bc0 = C(tau), C(g), C(rho0), C(u0), C(v0)
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    fdir = oracle.azimuthal_force(xy, 1.0)
    rr, uu, vv = torch_ref.rollout(sidx, W, tc, gc, fdir, mask, rc0, ac0, bc0, steps)
    loss(rr, uu, vv, lambda a: torch.as_tensor(a, dtype=torch.float64)).backward()
    assert tt.grad.item() == pytest.approx(tc.grad.item(), rel=1e-8)
    assert gt.grad.item() == pytest.approx(gc.grad.item(), rel=1e-8)
    for gpu, ref in ((r0, rc0), (a0, ac0), (b0, bc0)):
        np.testing.assert_allclose(gpu.grad.cpu().numpy(), ref.grad.numpy(), rtol=1e-7,
                                   atol=1e-8 * np.abs(ref.grad.numpy()).max())


def test_adjoint_mixed_stencil_rules_matches_finite_differences():
    """An own-rule and a nearest-rule segment in one weights object (one reverse step over both
    kinds of transposed rows): <lam_prev, v> and each segment's dL/dtau, dL/dg against central
    differences of the forward."""
    parts = [mi.jittered_lattice(18, 0.3, seed=71), mi.jittered_lattice(16, 0.3, seed=72)]
    segs = [dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=12, degree=2, dx_ml=0.7 / 18),
            dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=16, degree=3, dx_ml=2.0 / 16,
                 stencil_mode=mlbm.STENCIL_NEAREST)]
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    w = mlbm.build_weights(mlbm.build_cloud(xy, segs, offs))
    params = [(0.8, 2e-5, 1.0), (0.7, -1e-5, 1.0)]
    s = _rand_state(w, params, xy.shape[1], seed=73)
    rng = np.random.default_rng(74)
    lam = _t(rng.standard_normal(9 * w.n))
    v = _t(rng.standard_normal(9 * w.n))
    lam_prev = torch.empty_like(lam)
    grad = torch.zeros(4, dtype=torch.float64, device=DEV)
    mlbm.adjoint_step(w, params, mlbm.F64, s, lam, lam_prev, grad, s_next=_step(w, params, s))
    eps = 1e-5
    fd = (torch.dot(lam, _step(w, params, s + eps * v)) - torch.dot(lam, _step(w, params, s - eps * v))) / (2 * eps)
    assert float(torch.dot(lam_prev, v)) == pytest.approx(float(fd), rel=1e-7)
    for seg in range(2):
        for c, h in ((0, 1e-6), (1, 1e-6)):
            lo, hi = [list(p) for p in params], [list(p) for p in params]
            lo[seg][c] -= h
            hi[seg][c] += h
            f = (torch.dot(lam, _step(w, [tuple(p) for p in hi], s)) -
                 torch.dot(lam, _step(w, [tuple(p) for p in lo], s))) / (2 * h)
            assert float(grad[2 * seg + c]) == pytest.approx(float(f), rel=1e-6), (seg, c)
