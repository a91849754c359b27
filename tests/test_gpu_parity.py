"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated here, derived in the design notes):
  * FP64 step with shared shape vectors: <= 1e-12 relative per step (max |diff| / max |f|).
  * shape vectors, GPU vs oracle (both LU with partial pivoting in FP64 on the same matrix):
    <= WEIGHT_TOL absolute (|w| is O(1); the systems are ill-conditioned, so the two
    factorisations agree to about cond(Phi) * eps rather than eps).
  * FP32 deviation-storage path: <= 1e-6 relative L2 of the velocity after the run.
"""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu

WEIGHT_TOL = {2: 1e-9, 3: 1e-8, 4: 1e-7}
STEP_TOL = 1e-12
FP32_TOL = 1e-6


def _dev():
    return torch.device("cuda:0")


def _periodic(k, deg, dx):
    return dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=k, degree=deg, dx_ml=dx)


def _setup_tgv(n_side, K, deg, ratio=1.0, seed=1, jitter=0.3):
    xy = mi.jittered_lattice(n_side, jitter, seed=seed) if jitter > 0 else mi.lattice(n_side)
    dx = ratio / n_side
    seg = _periodic(K, deg, dx)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    return xy, dx, cloud, w


def _to_orig(w_stored, perm):
    """[c][N] stored order -> original order."""
    out = np.empty_like(w_stored)
    out[:, perm] = w_stored
    return out


def _gpu_init(w, params, dtype, rho, u, v):
    td = torch.float32 if dtype == mlbm.F32 else torch.float64
    f = torch.empty(9 * w.n, dtype=td, device=_dev())
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=_dev()).contiguous()
    mlbm.init(w, params, dtype, t(rho), t(u), t(v), f)
    return f


def _upload_oracle_weights(w, xy, K, deg, dx, box=(1.0, 1.0)):
    sidx, W = oracle.weights(xy, K, deg, dx, box=box)
    w.upload(W[1:], sidx[1].astype(np.int32))
    return sidx, W


# ----------------------------------------------------------------------------- shape vectors

@pytest.mark.parametrize("n_side,K,deg", [(32, 12, 2), (24, 16, 3), (20, 30, 4)])
def test_weights_match_oracle(n_side, K, deg):
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg)
    assert w.n_bad == 0
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0))
    np.testing.assert_array_equal(cloud.stencil(0), sidx[1])
    Wg = w.download(0)
    err = np.max(np.abs(Wg - W[1:]))
    assert err <= WEIGHT_TOL[deg], err


def _collocation_matrix(pts, deg):
    """Phi_L of eq. (rbf_interp_set_augmented) for stencil points pts (2, K): r^3 block, the
    monomials of total degree <= deg, zero block; written here from the definition."""
    K = pts.shape[1]
    d = pts[:, :, None] - pts[:, None, :]
    R = np.hypot(d[0], d[1]) ** 3
    P = np.array([pts[0] ** (t - b) * pts[1] ** b for t in range(deg + 1) for b in range(t + 1)]).T
    m = P.shape[1]
    A = np.zeros((K + m, K + m))
    A[:K, :K], A[:K, K:], A[K:, :K] = R, P, P.T
    return A


@pytest.mark.parametrize("n_side,K,deg", [(24, 34, 5), (24, 45, 6)])
def test_high_degree_weights_match_oracle_within_conditioning(n_side, K, deg):
    """Degrees 5 and 6 with the stencil sizes of the batched sweep (N_L 34 and 45, Sec. 2.3
    eq. poly_sets).  Both sides factorise the same matrix Phi_L (centred, scaled by the stencil
    radius) by LU with partial pivoting in FP64, in different operation orders, so per node they
    may differ by about cond(Phi_L) times the backward error of the factorisation, n eps:
    |w_gpu - w_oracle| <= 8 n cond(Phi_L) eps max|w|, with cond computed here per sampled node.
    The interpolation of f = 0.01 sin(2 pi x) cos(2 pi y) (Fig. interp_test's function) at the
    departure points then has the same error with either set of weights."""
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg)
    assert w.n_bad == 0
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0))
    np.testing.assert_array_equal(cloud.stencil(0), sidx[1])
    Wg = w.download(0)
    n = K + (deg + 1) * (deg + 2) // 2
    eps = np.finfo(np.float64).eps
    worst = 0.0
    for i in range(0, xy.shape[1], 5):
        d = xy[:, sidx[1][:, i]] - xy[:, i:i + 1]
        d -= np.round(d)
        s = np.max(np.hypot(d[0], d[1]))
        cond = np.linalg.cond(_collocation_matrix(d / s, deg))
        tol = 8 * n * cond * eps * max(1.0, np.max(np.abs(W[1:, :, i])))
        err = np.max(np.abs(Wg[:, :, i] - W[1:, :, i]))
        worst = max(worst, err / tol)
        assert err <= tol, (i, err, tol, cond)
    # interpolation error of a smooth field at the departure points, GPU vs oracle weights
    f = lambda x, y: 0.01 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    fx = f(xy[0], xy[1])
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    errs = []
    for Wk in (Wg, W[1:]):
        e2 = t2 = 0.0
        for k in range(1, 9):
            got = np.sum(Wk[k - 1] * fx[sidx[1]], axis=0)
            want = f(xy[0] - ex[k] * dx, xy[1] - ey[k] * dx)
            e2 += np.sum((got - want) ** 2)
            t2 += np.sum(want ** 2)
        errs.append(np.sqrt(e2 / t2))
    assert errs[1] < 1e-3  # a real interpolation, not a degenerate one
    assert abs(errs[0] - errs[1]) <= 1e-6 * errs[1], errs


@pytest.mark.parametrize("n_side,K,deg", [(20, 30, 4), (32, 12, 2), (24, 45, 6)])
def test_fp32_shape_vectors_keep_polynomial_reproduction(n_side, K, deg):
    """The FP32 copy of the shape vectors (Sec. 2.2: the shape vector reproduces every monomial
    of degree <= d) keeps that reproduction far better than rounding each entry to the nearest
    float: the moment errors sum_{j>=1} (w32_j - w64_j) p((x_j - x_c) / r) over the monomials of
    degree 1..d (radius-scaled, about the centre) have an RMS below 0.15 of nearest rounding's
    (about 0.03-0.05 in an emulation of the same rounding), each entry stays within 2^-12 of the
    system's largest |w| of its FP64 value, and the centre entry is the FP64 value rounded."""
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg)
    W64 = w.download(0)
    W32 = w.download_f32(0).astype(np.float64)
    st = cloud.stencil(0)
    d = xy[:, st] - xy[:, st[0:1]]  # [2][K][n] member offsets from the centre (min image)
    d -= np.round(d)
    rad = np.max(np.hypot(d[0], d[1]), axis=0)
    u, v = d[0] / rad, d[1] / rad
    mono = np.array([u ** (t - b) * v ** b for t in range(1, deg + 1) for b in range(t + 1)])  # [m][K][n]
    r_lib, r_rn = [], []
    for k in range(8):
        dl = W32[k, 1:] - W64[k, 1:]
        dr = W64[k, 1:].astype(np.float32).astype(np.float64) - W64[k, 1:]
        r_lib.append(np.einsum("mjn,jn->mn", mono[:, 1:], dl))
        r_rn.append(np.einsum("mjn,jn->mn", mono[:, 1:], dr))
        bound = 2.0 ** -12 * np.max(np.abs(W64[k]), axis=0)
        assert np.all(np.abs(dl) <= bound + np.abs(W64[k, 1:]) * 2.0 ** -23)
        np.testing.assert_array_equal(W32[k, 0], W64[k, 0].astype(np.float32).astype(np.float64))
    rms_lib = np.sqrt(np.mean(np.square(r_lib)))
    rms_rn = np.sqrt(np.mean(np.square(r_rn)))
    assert rms_lib <= 0.15 * rms_rn, (rms_lib, rms_rn)


@pytest.mark.parametrize("K,deg", [(12, 2), (30, 4), (45, 6)])
def test_gpu_weights_reproduce_polynomials(K, deg):
    """Property check independent of the oracle: sum_j w_j p(x_j) = p(departure point)."""
    n_side = 24
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg)
    Wg = w.download(0)
    st = cloud.stencil(0)
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    for i in range(0, xy.shape[1], 37):
        d = xy[:, st[:, i]] - xy[:, i:i + 1]
        d -= np.round(d)
        s = np.max(np.hypot(d[0], d[1]))
        t = d / s
        for k in range(1, 9):
            q = np.array([-ex[k] * dx, -ey[k] * dx]) / s
            for a in range(deg + 1):
                for b in range(deg + 1 - a):
                    got = np.sum(Wg[k - 1, :, i] * t[0] ** a * t[1] ** b)
                    assert abs(got - q[0] ** a * q[1] ** b) < 1e-9


# ----------------------------------------------------------------------------- FP64 step

@pytest.mark.parametrize("n_side,K,deg,ratio", [(32, 12, 2, 1.0), (20, 30, 4, 1.0), (17, 16, 3, 0.5),
                                                 (200, 12, 2, 1.0)])
def test_fp64_step_matches_oracle_per_step(n_side, K, deg, ratio):
    """Shared (oracle) shape vectors uploaded to the GPU: every step agrees to 1e-12.  The
    small clouds run the one-warp tiles (several threads per node), 200^2 nodes the 128-node
    tiles."""
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg, ratio=ratio)
    sidx, W = _upload_oracle_weights(w, xy, K, deg, dx)
    tau = 0.8
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01 * ratio)
    perm = cloud.perm()
    f_or = oracle.init_equilibrium(rho, u, v)
    st = oracle.Stepper(sidx, W, tau)
    fa = _gpu_init(w, params, mlbm.F64, rho, u, v)
    fb = torch.empty_like(fa)
    mom = torch.empty(3 * w.n, dtype=torch.float64, device=_dev())
    n = w.n
    post = oracle.collide_field(f_or, tau)
    got = _to_orig(fa.view(9, n).cpu().numpy(), perm)
    assert np.max(np.abs(got - post)) <= STEP_TOL * np.max(np.abs(post))
    for it in range(12):
        mlbm.step(w, params, mlbm.F64, fa, fb, mom)
        fa, fb = fb, fa
        f_or = st.step(f_or)
        post = oracle.collide_field(f_or, tau)
        got = _to_orig(fa.view(9, n).cpu().numpy(), perm)
        rel = np.max(np.abs(got - post)) / np.max(np.abs(post))
        assert rel <= STEP_TOL, (it, rel)
        r_o, u_o, v_o = oracle.moments_field(f_or)
        m = _to_orig(mom.view(3, n).cpu().numpy(), perm)
        np.testing.assert_allclose(m[0], r_o, rtol=1e-13, atol=0)
        np.testing.assert_allclose(m[1], u_o, rtol=0, atol=1e-14)
        np.testing.assert_allclose(m[2], v_o, rtol=0, atol=1e-14)


def test_moments_entry_point_matches_oracle():
    xy, dx, cloud, w = _setup_tgv(16, 12, 2)
    _upload_oracle_weights(w, xy, 12, 2, dx)
    params = [(0.8, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.02)
    for dtype in (mlbm.F64, mlbm.F32):
        f = _gpu_init(w, params, dtype, rho, u, v)
        r, uu, vv = mlbm.moments(w, params, dtype, f)
        tol = 1e-15 if dtype == mlbm.F64 else 1e-8
        np.testing.assert_allclose(r.cpu().numpy(), rho, atol=tol * 10)
        np.testing.assert_allclose(uu.cpu().numpy(), u, atol=tol)
        np.testing.assert_allclose(vv.cpu().numpy(), v, atol=tol)


def test_fp64_run_own_weights_matches_oracle_run():
    """Configuration of the small Taylor-Green workload: 32^2 jittered, N_L = 12, P_2,
    tau = 0.8, u0 = 0.01, 500 steps; each side with its own shape vectors."""
    xy, dx, cloud, w = _setup_tgv(32, 12, 2)
    tau, steps = 0.8, 500
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01)
    sidx, W = oracle.weights(xy, 12, 2, dx, box=(1.0, 1.0))
    f_or = oracle.Stepper(sidx, W, tau).run(oracle.init_equilibrium(rho, u, v), steps)
    _, u_o, v_o = oracle.moments_field(f_or)
    fa = _gpu_init(w, params, mlbm.F64, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F64, fa, fb, steps)
    _, ug, vg = mlbm.moments(w, params, mlbm.F64, res)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / np.sum(u_o ** 2 + v_o ** 2))
    assert err <= 1e-9, err
    # and the physics: close to the analytic Taylor-Green decay
    nu = oracle.lattice_viscosity(tau)
    ut, _ = oracle.tgv_velocity(xy[0] / dx, xy[1] / dx, steps, u0=0.01, nu=nu, L=1.0 / dx)
    assert oracle.l2_norm(ug, ut) < 0.05


# ----------------------------------------------------------------------------- FP32 path

@pytest.mark.parametrize("n_side,K,deg,steps,seed", [
    (32, 12, 2, 500, 1),    # the small Taylor-Green workload, whole run
    (256, 30, 4, 400, 3),   # 256^2 sub-sample of the large workload's recipe
    # few nodes, large stencil: rounding of the shape vectors would not average out; run to the
    # error-evaluation time of Sec. 3, t_end = ln 10 / (2 nu k^2) = 116.7 -> 117 steps
    (20, 30, 4, 117, 1),
    (24, 45, 6, 300, 1),    # the sweep's largest stencil and degree
])
def test_fp32_run_within_1e6_of_fp64_oracle(n_side, K, deg, steps, seed):
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg, seed=seed)
    tau = 0.8
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01)
    sidx, W = _upload_oracle_weights(w, xy, K, deg, dx)
    f_or = oracle.Stepper(sidx, W, tau).run(oracle.init_equilibrium(rho, u, v), steps)
    _, u_o, v_o = oracle.moments_field(f_or)
    fa = _gpu_init(w, params, mlbm.F32, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F32, fa, fb, steps)
    _, ug, vg = mlbm.moments(w, params, mlbm.F32, res)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / np.sum(u_o ** 2 + v_o ** 2))
    assert err <= FP32_TOL, err


def test_fp32_error_far_beyond_t_end_is_the_fp32_storage_floor():
    """The 400-node cloud run 300 steps, 2.6 t_end: the vortex has decayed to 0.3 % of its
    amplitude, and the error relative to that small field is dominated by the uniform-flow
    mode (undamped by viscosity) of the FP32 state's rounding, accumulated while the field was
    large.  Its expected size is that of the FP64 oracle with FP32-sized rounding noise (each
    stored deviation f - omega rho0 perturbed by up to 2^-24 of itself, uniformly, every step):
    the FP32 path stays within 3x the RMS over four noise realisations, and within 1e-6 of the
    initial amplitude by a wide margin."""
    n_side, K, deg, steps = 20, 30, 4, 300
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg, seed=1)
    tau, u0 = 0.8, 0.01
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, u0)
    sidx, W = _upload_oracle_weights(w, xy, K, deg, dx)
    st = oracle.Stepper(sidx, W, tau)
    f0 = oracle.init_equilibrium(rho, u, v)
    f_or = st.run(f0, steps)
    _, u_o, v_o = oracle.moments_field(f_or)
    nrm = np.sum(u_o ** 2 + v_o ** 2)
    _, _, om = oracle.d2q9()
    model = []
    for r in range(4):
        rng = np.random.default_rng(1000 + r)
        f = f0.copy()
        for _ in range(steps):
            f = st.step(f)
            f = f + 2.0 ** -24 * np.abs(f - om[:, None]) * rng.uniform(-1.0, 1.0, f.shape)
        _, un, vn = oracle.moments_field(f)
        model.append(np.sum((un - u_o) ** 2 + (vn - v_o) ** 2) / nrm)
    floor = np.sqrt(np.mean(model))
    fa = _gpu_init(w, params, mlbm.F32, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F32, fa, fb, steps)
    _, ug, vg = mlbm.moments(w, params, mlbm.F32, res)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / nrm)
    assert err <= 3.0 * floor, (err, floor)
    err_initial = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / np.sum(u ** 2 + v ** 2))
    assert err_initial <= 1e-7, err_initial


def test_fp32_large_recipe_subsample_1e4_steps_within_1e6_of_fp64_oracle():
    """The precision study of the large Taylor-Green workload, checked where the oracle can
    follow it: a 256^2 cloud of the same recipe (seed 3, N_L 30, P_4, tau 0.8, u0 0.01,
    dx_ml = h), 10^4 FP32 steps against 10^4 FP64 oracle steps with the same shape vectors;
    relative L2 of the velocity <= 1e-6.  Both also follow the Taylor-Green decay of
    eq. (tgv_eqs) to the same discretisation error."""
    n_side, K, deg, steps = 256, 30, 4, 10_000
    xy, dx, cloud, w = _setup_tgv(n_side, K, deg, seed=3)
    tau, u0 = 0.8, 0.01
    params = [(tau, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, u0)
    sidx, W = _upload_oracle_weights(w, xy, K, deg, dx)
    f_or = oracle.Stepper(sidx, W, tau).run(oracle.init_equilibrium(rho, u, v), steps)
    _, u_o, v_o = oracle.moments_field(f_or)
    fa = _gpu_init(w, params, mlbm.F32, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F32, fa, fb, steps)
    _, ug, vg = mlbm.moments(w, params, mlbm.F32, res)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / np.sum(u_o ** 2 + v_o ** 2))
    assert err <= FP32_TOL, err
    nu = oracle.lattice_viscosity(tau)
    ut, vt = oracle.tgv_velocity(xy[0] / dx, xy[1] / dx, steps, u0=u0, nu=nu, L=1.0 / dx)
    e_or, e_gpu = oracle.l2_norm(u_o, ut), oracle.l2_norm(ug, ut)
    assert e_or < 0.01
    assert abs(e_gpu - e_or) <= 1e-3 * e_or, (e_gpu, e_or)


# ----------------------------------------------------------------------------- annulus

def _setup_annulus(h, K, deg, dx, seed=3):
    xy, wall = mi.annulus_cloud(h=h, seed=seed)
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=deg, dx_ml=dx)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    return xy, cloud, w


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_annulus_step_with_force_and_bounce_back_matches_oracle(dtype):
    dx = 1.0 / 40
    K, deg, tau, g = 15, 2, 1.0, 1e-5
    xy, cloud, w = _setup_annulus(mi.ANNULUS_H_FOR[1000], K, deg, dx)
    sidx, W = oracle.weights(xy, K, deg, dx)
    w.upload(W[1:], sidx[1].astype(np.int32))
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    assert np.array_equal(cloud.bounce_mask(), mask) and mask.any()
    force = oracle.azimuthal_force(xy, g)
    st = oracle.Stepper(sidx, W, tau, mask=mask, force=force)
    n = xy.shape[1]
    rng = np.random.default_rng(0)
    rho = 1.0 + 1e-3 * rng.standard_normal(n)
    u = 1e-3 * rng.standard_normal(n)
    v = 1e-3 * rng.standard_normal(n)
    params = [(tau, g, 1.0)]
    dt = mlbm.F64 if dtype == "f64" else mlbm.F32
    fa = _gpu_init(w, params, dt, rho, u, v)
    fb = torch.empty_like(fa)
    f_or = oracle.init_equilibrium(rho, u, v)
    perm = cloud.perm()
    steps = 30
    for it in range(steps):
        mlbm.step(w, params, dt, fa, fb)
        fa, fb = fb, fa
        f_or = st.step(f_or)
        if dtype == "f64":
            post = oracle.collide_field(f_or, tau, force)
            got = _to_orig(fa.view(9, n).cpu().numpy(), perm)
            assert np.max(np.abs(got - post)) <= STEP_TOL * np.max(np.abs(post)), it
    r_g, u_g, v_g = mlbm.moments(w, params, dt, fa)
    r_o, u_o, v_o = oracle.moments_field(f_or)
    tol = 1e-13 if dtype == "f64" else 2e-7
    np.testing.assert_allclose(r_g.cpu().numpy(), r_o, atol=tol)
    np.testing.assert_allclose(u_g.cpu().numpy(), u_o, atol=tol * 1e-1)
    np.testing.assert_allclose(v_g.cpu().numpy(), v_o, atol=tol * 1e-1)


def test_annulus_20k_workload_per_step_parity():
    """The annular-channel workload at its own size and in the launch configuration the
    benchmark times (about 20k scattered nodes refined toward the walls, seed 2, N_L = 20, P_3,
    dx_ml = 1/320, tau = 0.7, g = 1e-6, FP64, one-warp tiles): ten steps from a perturbed rest
    state, each stored state equal to the oracle's post-collision populations to 1e-12 (oracle
    shape vectors uploaded, Q20), with the azimuthal force and wall bounce-back."""
    dx, K, deg, tau, g = 1.0 / 320, 20, 3, 0.7, 1e-6
    xy, wall = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[20000], seed=2)
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=deg, dx_ml=dx)
    cloud = mlbm.build_cloud(xy, seg)
    w = mlbm.build_weights(cloud)
    sidx, W = oracle.weights(xy, K, deg, dx)
    w.upload(W[1:], sidx[1].astype(np.int32))
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    assert np.array_equal(cloud.bounce_mask(), mask) and mask.any()
    force = oracle.azimuthal_force(xy, g)
    st = oracle.Stepper(sidx, W, tau, mask=mask, force=force)
    n = xy.shape[1]
    rng = np.random.default_rng(4)
    rho = 1.0 + 1e-4 * rng.standard_normal(n)
    u = 1e-4 * rng.standard_normal(n)
    v = 1e-4 * rng.standard_normal(n)
    params = [(tau, g, 1.0)]
    fa = _gpu_init(w, params, mlbm.F64, rho, u, v)
    fb = torch.empty_like(fa)
    f_or = oracle.init_equilibrium(rho, u, v)
    perm = cloud.perm()
    for it in range(10):
        mlbm.step(w, params, mlbm.F64, fa, fb)
        fa, fb = fb, fa
        f_or = st.step(f_or)
        post = oracle.collide_field(f_or, tau, force)
        got = _to_orig(fa.view(9, n).cpu().numpy(), perm)
        assert np.max(np.abs(got - post)) <= STEP_TOL * np.max(np.abs(post)), it


# ----------------------------------------------------------------------------- batching

def test_batched_segments_match_single_runs_and_oracle():
    cases = [(16, 12, 2, 1.0, 0.8), (20, 16, 3, 0.5, 0.7), (12, 24, 4, 0.25, 1.1), (9, 8, 1, 1.0, 0.9)]
    parts, segs, params = [], [], []
    for s, (ns, K, deg, ratio, tau) in enumerate(cases):
        parts.append(mi.jittered_lattice(ns, 0.3, seed=70 + s))
        segs.append(_periodic(K, deg, ratio / ns))
        params.append((tau, 0.0, 1.0))
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    cloud = mlbm.build_cloud(xy, segs, offs)
    w = mlbm.build_weights(cloud)
    rho = np.ones(xy.shape[1])
    u = np.concatenate([mi.tgv_initial(p, 0.01)[1] for p in parts])
    v = np.concatenate([mi.tgv_initial(p, 0.01)[2] for p in parts])
    fa = _gpu_init(w, params, mlbm.F64, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F64, fa, fb, 40)
    _, ub, vb = mlbm.moments(w, params, mlbm.F64, res)
    ub = ub.cpu().numpy()
    for s, p in enumerate(parts):
        c1 = mlbm.build_cloud(p, segs[s])
        w1 = mlbm.build_weights(c1)
        np.testing.assert_array_equal(w1.download(0), w.download(s))
        _, u1, v1 = mi.tgv_initial(p, 0.01)
        f1 = _gpu_init(w1, [params[s]], mlbm.F64, np.ones(p.shape[1]), u1, v1)
        g1 = torch.empty_like(f1)
        r1 = mlbm.run(w1, [params[s]], mlbm.F64, f1, g1, 40)
        _, us, _ = mlbm.moments(w1, [params[s]], mlbm.F64, r1)
        np.testing.assert_array_equal(us.cpu().numpy(), ub[offs[s]:offs[s + 1]])
        sidx, W = oracle.weights(p, segs[s]["k"], segs[s]["degree"], segs[s]["dx_ml"], box=(1.0, 1.0))
        err = np.max(np.abs(w.download(s) - W[1:]))
        assert err <= 1e-7, (s, err)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_run_until_gives_each_segment_its_own_run(dtype):
    """Segments of uneven size, stencil, degree and tau, each run for its own number of steps in
    one call (even, odd, zero, past a 64-step graph): every segment's result equals a run of
    that segment alone, bit for bit."""
    dt = mlbm.F32 if dtype == "f32" else mlbm.F64
    cases = [(16, 12, 2, 1.0, 0.8, 37), (20, 16, 3, 0.5, 0.7, 0), (12, 24, 4, 0.25, 1.1, 150),
             (9, 8, 1, 1.0, 0.9, 64)]
    parts, segs, params, steps = [], [], [], []
    for s_, (ns, K, deg, ratio, tau, n) in enumerate(cases):
        parts.append(mi.jittered_lattice(ns, 0.3, seed=80 + s_))
        segs.append(_periodic(K, deg, ratio / ns))
        params.append((tau, 0.0, 1.0))
        steps.append(n)
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    w = mlbm.build_weights(mlbm.build_cloud(xy, segs, offs))
    u = np.concatenate([mi.tgv_initial(p, 0.01)[1] for p in parts])
    v = np.concatenate([mi.tgv_initial(p, 0.01)[2] for p in parts])
    fa = _gpu_init(w, params, dt, np.ones(xy.shape[1]), u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run_until(w, params, dt, fa, fb, steps)
    assert res is (fb if max(steps) % 2 else fa)
    rb, ub, vb = (t.cpu().numpy() for t in mlbm.moments(w, params, dt, res))
    for s_, p in enumerate(parts):
        w1 = mlbm.build_weights(mlbm.build_cloud(p, segs[s_]))
        _, u1, v1 = mi.tgv_initial(p, 0.01)
        f1 = _gpu_init(w1, [params[s_]], dt, np.ones(p.shape[1]), u1, v1)
        r1 = mlbm.run(w1, [params[s_]], dt, f1, torch.empty_like(f1), steps[s_])
        ro, uo, vo = (t.cpu().numpy() for t in mlbm.moments(w1, [params[s_]], dt, r1))
        sl = slice(offs[s_], offs[s_ + 1])
        np.testing.assert_array_equal(rb[sl], ro)
        np.testing.assert_array_equal(ub[sl], uo)
        np.testing.assert_array_equal(vb[sl], vo)
    # equal counts: the same as one mlbm_run of the whole cloud
    ga = _gpu_init(w, params, dt, np.ones(xy.shape[1]), u, v)
    gb = torch.empty_like(ga)
    ha = ga.clone()
    r_all = mlbm.run(w, params, dt, ga, gb, 71)
    r_until = mlbm.run_until(w, params, dt, ha, torch.empty_like(ha), [71] * len(cases))
    assert torch.equal(r_all, r_until)
    # no steps at all: the state stays where it is, the other buffer is not written
    za = _gpu_init(w, params, dt, np.ones(xy.shape[1]), u, v)
    keep = za.clone()
    zb = torch.full_like(za, 3.0)
    assert mlbm.run_until(w, params, dt, za, zb, [0] * len(cases)) is za
    assert torch.equal(za, keep) and bool((zb == 3.0).all())
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.run_until(w, params, dt, za, zb, [5, -1, 5, 5])
    assert e.value.code == mlbm.EINVAL
    with pytest.raises(ValueError):
        mlbm.run_until(w, params, dt, za, zb, [5, 5])


def test_weights_objects_with_smaller_halos_leave_earlier_ones_usable():
    """Building weights whose tiles need less shared memory must not shrink what the kernels of
    an existing weights object (and the graphs captured for it) may use."""
    xy, dx, cloud, w = _setup_tgv(24, 30, 4)
    params = [(0.8, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01)
    for dtype in (mlbm.F32, mlbm.F64):
        fa = _gpu_init(w, params, dtype, rho, u, v)
        ref = mlbm.run(w, params, dtype, fa.clone(), torch.empty_like(fa), 70).clone()
        small = mlbm.build_weights(mlbm.build_cloud(mi.jittered_lattice(8, 0.3, seed=2), _periodic(6, 1, 1.0 / 8)))
        assert small.n == 64
        got = mlbm.run(w, params, dtype, fa.clone(), torch.empty_like(fa), 70)
        assert torch.equal(got, ref)
        del small


def test_run_graph_equals_repeated_steps():
    xy, dx, cloud, w = _setup_tgv(24, 12, 2)
    params = [(0.8, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01)
    for dtype in (mlbm.F32, mlbm.F64):
        fa = _gpu_init(w, params, dtype, rho, u, v)
        fb = torch.empty_like(fa)
        ga, gb = fa.clone(), torch.empty_like(fa)
        steps = 131  # two 64-step graph replays plus a tail
        res = mlbm.run(w, params, dtype, fa, fb, steps)
        for _ in range(steps):
            mlbm.step(w, params, dtype, ga, gb)
            ga, gb = gb, ga
        assert torch.equal(res, ga)


def test_run_of_zero_steps_returns_the_input_untouched():
    xy, dx, cloud, w = _setup_tgv(16, 12, 2)
    params = [(0.8, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.01)
    for dtype in (mlbm.F32, mlbm.F64):
        fa = _gpu_init(w, params, dtype, rho, u, v)
        keep = fa.clone()
        fb = torch.full_like(fa, 7.0)
        res = mlbm.run(w, params, dtype, fa, fb, 0)
        assert res is fa and torch.equal(fa, keep) and bool((fb == 7.0).all())


def test_ragged_tail_and_minimal_segment():
    """N not a multiple of the 256-node tile and a segment with exactly N_L nodes."""
    parts = [mi.jittered_lattice(31, 0.3, seed=5), mi.jittered_lattice(3, 0.2, seed=6)]
    segs = [_periodic(12, 2, 1.0 / 31), _periodic(9, 2, 0.1 / 3)]
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    cloud = mlbm.build_cloud(xy, segs, offs)
    w = mlbm.build_weights(cloud)
    assert w.n % 256 != 0
    params = [(0.8, 0.0, 1.0), (0.9, 0.0, 1.0)]
    rho = np.ones(xy.shape[1])
    u = np.concatenate([mi.tgv_initial(p, 0.01)[1] for p in parts])
    v = np.concatenate([mi.tgv_initial(p, 0.01)[2] for p in parts])
    for s, p in enumerate(parts):
        sidx, W = oracle.weights(p, segs[s]["k"], 2, segs[s]["dx_ml"], box=(1.0, 1.0))
        w.upload(W[1:], sidx[1].astype(np.int32), seg=s)
    fa = _gpu_init(w, params, mlbm.F64, rho, u, v)
    fb = torch.empty_like(fa)
    res = mlbm.run(w, params, mlbm.F64, fa, fb, 7)
    _, ug, _ = mlbm.moments(w, params, mlbm.F64, res)
    ug = ug.cpu().numpy()
    for s, p in enumerate(parts):
        sidx, W = oracle.weights(p, segs[s]["k"], 2, segs[s]["dx_ml"], box=(1.0, 1.0))
        _, u1, v1 = mi.tgv_initial(p, 0.01)
        f = oracle.Stepper(sidx, W, params[s][0]).run(
            oracle.init_equilibrium(np.ones(p.shape[1]), u1, v1), 7)
        _, uo, _ = oracle.moments_field(f)
        np.testing.assert_allclose(ug[offs[s]:offs[s + 1]], uo, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- norms, errors

def test_norms_match_numpy():
    xy, dx, cloud, w = _setup_tgv(8, 9, 2)
    rng = np.random.default_rng(3)
    n = 123457
    a, b, c, d = (rng.standard_normal(n) for _ in range(4))
    t = lambda z: torch.as_tensor(z, device=_dev())
    out = mlbm.norms(w, t(a), t(b), t(c), t(d))
    want = [np.sum((a - b) ** 2 + (c - d) ** 2), np.sum(b ** 2 + d ** 2), np.sum(a ** 2 + c ** 2)]
    np.testing.assert_allclose(out, want, rtol=1e-13)
    out1 = mlbm.norms(w, t(a), t(b))
    np.testing.assert_allclose(out1, [np.sum((a - b) ** 2), np.sum(b ** 2), np.sum(a ** 2)], rtol=1e-13)
    # deterministic
    assert np.array_equal(out, mlbm.norms(w, t(a), t(b), t(c), t(d)))


def test_step_argument_errors():
    xy, dx, cloud, w = _setup_tgv(8, 9, 2)
    f = torch.zeros(9 * w.n, dtype=torch.float64, device=_dev())
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.step(w, [(0.4, 0.0, 1.0)], mlbm.F64, f, f.clone())  # tau <= 1/2
    assert e.value.code == mlbm.EINVAL
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.step(w, [(0.8, 0.0, 1.0)], mlbm.F64, f, f)  # in place is not allowed
    assert e.value.code == mlbm.EINVAL
    w32 = mlbm.build_weights(cloud, keep=mlbm.KEEP_W32)
    with pytest.raises(mlbm.MLBMError):
        mlbm.step(w32, [(0.8, 0.0, 1.0)], mlbm.F64, f, f.clone())


def test_singular_stencil_reported():
    """Collinear stencils cannot carry the quadratic monomials: the solver flags them."""
    x = np.linspace(0.05, 0.95, 12)
    xy = np.stack([x, np.full(12, 0.5)])
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.ANNULUS, r_in=0.0, r_out=10.0, k=9,
                                      degree=2, dx_ml=0.01))
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_weights(cloud)
    assert e.value.code == mlbm.ESINGULAR
    w = mlbm.build_weights(cloud, check=False)
    assert w.n_bad == 12
