"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: values printed in the
paper (tests/golden/, each citing its section), textbook identities of the D2Q9 model,
closed-form solutions, special cases that reduce to a library routine (natural cubic spline,
Vandermonde solve, barycentric coordinates), exact invariants and the convergence trends the
paper reports.  No expected value comes from the GPU library.
"""
import os

import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------------------- D2Q9, Sec. 2.1

def test_velocity_set_and_weights_match_paper():
    ex, ey, om = oracle.d2q9()
    for row in _golden_table("d2q9_velocity_set.txt"):
        k, gx, gy, num, den = (int(v) for v in row)
        assert (ex[k], ey[k]) == (gx, gy)
        assert om[k] == pytest.approx(num / den, abs=0, rel=1e-15)
    assert om.sum() == pytest.approx(1.0, abs=1e-15)


def test_opposite_directions():
    ex, ey, _ = oracle.d2q9()
    for k in range(9):
        kk = oracle.opposite(k)
        assert (ex[kk], ey[kk]) == (-ex[k], -ey[k])
        assert oracle.opposite(kk) == k


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moment_identities(seed):
    """Textbook D2Q9 identities: sum feq = rho, sum feq e = rho u,
    sum feq e_a e_b = rho (c_s^2 delta_ab + u_a u_b)."""
    rng = np.random.default_rng(seed)
    ex, ey, _ = oracle.d2q9()
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.2, 0.2, 2)
        f = np.array([oracle.feq(k, rho, u[0], u[1]) for k in range(9)])
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert (f * ex).sum() == pytest.approx(rho * u[0], abs=1e-15)
        assert (f * ey).sum() == pytest.approx(rho * u[1], abs=1e-15)
        assert (f * ex * ex).sum() == pytest.approx(rho * (1 / 3 + u[0] ** 2), rel=1e-14)
        assert (f * ey * ey).sum() == pytest.approx(rho * (1 / 3 + u[1] ** 2), rel=1e-14)
        assert (f * ex * ey).sum() == pytest.approx(rho * u[0] * u[1], abs=1e-15)


def test_equilibrium_at_rest_is_weights():
    _, _, om = oracle.d2q9()
    for k in range(9):
        assert oracle.feq(k, 1.3, 0.0, 0.0) == pytest.approx(1.3 * om[k], rel=1e-15)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0, 1.7])
def test_collision_conserves_mass_and_momentum(tau):
    rng = np.random.default_rng(7)
    ex, ey, _ = oracle.d2q9()
    for _ in range(20):
        f = rng.uniform(0.01, 0.3, 9)
        fp = oracle.collide(f, tau)
        assert fp.sum() == pytest.approx(f.sum(), rel=1e-14)
        assert (fp * ex).sum() == pytest.approx((f * ex).sum(), abs=1e-15)
        assert (fp * ey).sum() == pytest.approx((f * ey).sum(), abs=1e-15)


def test_collision_force_adds_g_to_momentum():
    """The forcing term of Sec. 3 changes momentum by exactly g and leaves mass unchanged."""
    rng = np.random.default_rng(8)
    ex, ey, _ = oracle.d2q9()
    for _ in range(10):
        f = rng.uniform(0.01, 0.3, 9)
        g = rng.uniform(-1e-3, 1e-3, 2)
        fp0 = oracle.collide(f, 0.8)
        fp = oracle.collide(f, 0.8, g[0], g[1])
        assert (fp - fp0).sum() == pytest.approx(0.0, abs=1e-16)
        assert ((fp - fp0) * ex).sum() == pytest.approx(g[0], rel=1e-12)
        assert ((fp - fp0) * ey).sum() == pytest.approx(g[1], rel=1e-12)


def test_collision_tau_one_gives_equilibrium():
    rng = np.random.default_rng(9)
    f = rng.uniform(0.01, 0.3, 9)
    rho, ux, uy = oracle.moments(f)
    fp = oracle.collide(f, 1.0)
    for k in range(9):
        assert fp[k] == pytest.approx(oracle.feq(k, rho, ux, uy), rel=1e-14)


# ----------------------------------------------------------------------------- viscosity reading

def test_viscosity_reading_reproduces_paper_parameters():
    """Sec. 3 prints tau = 0.8, dx = 1/10, dt = 1e-3 and nu = 1; only the reading
    nu = c_s^2 (tau - 1/2) dx^2 / dt reproduces nu = 1 from them."""
    p = {r[0]: float(r[1]) for r in _golden_table("tgv_parameters.txt")}
    nu = oracle.lattice_viscosity(p["tau"]) * p["dx"] ** 2 / p["dt"]
    assert nu == pytest.approx(p["nu"], rel=1e-12)


# ----------------------------------------------------------------------------- closed forms

def test_tgv_solution_solves_navier_stokes():
    """eq. (tgv_eqs) is divergence-free and decays as du/dt = nu lap(u) (the nonlinear term of
    the Taylor-Green vortex is a pure gradient), checked by finite differences."""
    nu, h, t = 0.7, 1e-4, 0.01
    rng = np.random.default_rng(3)
    for x, y in rng.uniform(0, 1, (10, 2)):
        u, v = oracle.tgv_velocity(x, y, t, nu=nu)
        ux_p, _ = oracle.tgv_velocity(x + h, y, t, nu=nu)
        ux_m, _ = oracle.tgv_velocity(x - h, y, t, nu=nu)
        _, vy_p = oracle.tgv_velocity(x, y + h, t, nu=nu)
        _, vy_m = oracle.tgv_velocity(x, y - h, t, nu=nu)
        div = (ux_p - ux_m) / (2 * h) + (vy_p - vy_m) / (2 * h)
        assert abs(div) < 1e-6
        uy_p, _ = oracle.tgv_velocity(x, y + h, t, nu=nu)
        uy_m, _ = oracle.tgv_velocity(x, y - h, t, nu=nu)
        lap = (ux_p + ux_m + uy_p + uy_m - 4 * u) / h ** 2
        ut_p, _ = oracle.tgv_velocity(x, y, t + 1e-6, nu=nu)
        ut_m, _ = oracle.tgv_velocity(x, y, t - 1e-6, nu=nu)
        dudt = (ut_p - ut_m) / 2e-6
        assert dudt == pytest.approx(nu * lap, rel=1e-4, abs=1e-6)


def test_tgv_end_time_is_ten_percent_decay():
    t_end = oracle.tgv_end_time()
    u0, _ = oracle.tgv_velocity(0.0, 0.25, 0.0)
    u1, _ = oracle.tgv_velocity(0.0, 0.25, t_end)
    assert u1 / u0 == pytest.approx(0.1, rel=1e-12)


def test_annulus_profile_solves_azimuthal_balance():
    """eq. (bch_solution) satisfies nu (u'' + u'/r - u/r^2) + g = 0 and no slip at both walls
    (paper geometry R1 = 1, R2 = 2, g = 1e-6)."""
    p = {r[0]: float(r[1]) for r in _golden_table("annulus_parameters.txt")}
    r1, r2, g = p["R1"], p["R2"], p["g"]
    nu = oracle.lattice_viscosity(p["tau"])
    assert oracle.annulus_velocity(r1, g, nu, r1, r2) == pytest.approx(0.0, abs=1e-18)
    assert oracle.annulus_velocity(r2, g, nu, r1, r2) == pytest.approx(0.0, abs=1e-18)
    h = 1e-4
    for r in np.linspace(1.1, 1.9, 9):
        f = lambda s: oracle.annulus_velocity(s, g, nu, r1, r2)
        upp = (f(r + h) - 2 * f(r) + f(r - h)) / h ** 2
        up = (f(r + h) - f(r - h)) / (2 * h)
        res = nu * (upp + up / r - f(r) / r ** 2) + g
        assert abs(res) < 1e-8 * g / 1e-6 * 1e-3
    # flow goes in the direction of the force
    assert oracle.annulus_velocity(1.5, g, nu, r1, r2) > 0


def test_residual_hand_computed():
    """Sec. 3 stop rule, read as ||u^n - u^(n-1)||_2 / ||u^n||_2 over both velocity
    components of all nodes: a 3-node field worked by hand.  Differences (0,-1,0) in u and
    (0,0,1) in v give a numerator of 2; the new field's squares sum to 1 + 4 + 1 = 6, so the
    residual is sqrt(2/6).  A missing square root (1/3), the old field in the denominator
    (sqrt(2/8)) or a single component (sqrt(1/5)) all miss it."""
    u_new, v_new = np.array([1.0, 0.0, 2.0]), np.array([0.0, 1.0, 0.0])
    u_old, v_old = np.array([1.0, 1.0, 2.0]), np.array([0.0, 1.0, -1.0])
    assert oracle.residual(u_new, v_new, u_old, v_old) == pytest.approx(np.sqrt(1.0 / 3.0), rel=1e-15)
    # identical fields: zero; the residual is symmetric in neither argument order
    assert oracle.residual(u_new, v_new, u_new, v_new) == 0.0
    assert oracle.residual(u_old, v_old, u_new, v_new) == pytest.approx(np.sqrt(2.0 / 8.0), rel=1e-15)


def test_l2_norm_hand_computed():
    """eq. (L2norm): sqrt(sum (u - u_true)^2) / sqrt(sum u_true^2).  u = (3, 0, 4) against
    (1, 2, 2): differences (2, -2, 2) give sqrt(12) over sqrt(9), i.e. 2/sqrt(3); without the
    square roots it would be 4/3, normalised by the computed field sqrt(12/25)."""
    u = np.array([3.0, 0.0, 4.0])
    ut = np.array([1.0, 2.0, 2.0])
    assert oracle.l2_norm(u, ut) == pytest.approx(2.0 / np.sqrt(3.0), rel=1e-15)
    assert oracle.l2_norm(ut, ut) == 0.0


def test_speed_rel_error_hand_computed():
    """eq. (vmag_error): e_i = | |U_i| - |U_i,true| | / |U_i,true| with |U| = sqrt(u^2 + v^2).
    Node 0: |U| = 5 against a true speed of 4 gives 1/4 (dividing by the computed speed would
    give 1/5).  Node 1: |U| = 1 against 5 gives 4/5 (positive: the absolute value).  Node 2:
    a rotated velocity of the right magnitude has no speed error.  Node 3: at rest against a
    true speed of 2 gives exactly 1."""
    u = np.array([3.0, 0.6, 0.0, 0.0])
    v = np.array([4.0, 0.8, -2.0, 0.0])
    ut = np.array([0.0, 3.0, 2.0, 2.0])
    vt = np.array([4.0, 4.0, 0.0, 0.0])
    e = oracle.speed_rel_error(u, v, ut, vt)
    np.testing.assert_allclose(e, [0.25, 0.8, 0.0, 1.0], rtol=1e-15, atol=0)


def test_azimuthal_force_points_counter_clockwise():
    """Sec. 3 annulus forcing g = (0, g) in polar coordinates (r, phi): the force is g times the
    unit vector of increasing phi, (-sin phi, cos phi).  At (r, 0) it points along +y, at
    (0, r) along -x, at (-r, 0) along -y; its magnitude is g everywhere."""
    g = 2.5e-6
    xy = np.array([[0.7, 0.0, -0.8, 0.0, 0.6],
                   [0.0, 0.9, 0.0, -0.5, 0.8]])
    gx, gy = oracle.azimuthal_force(xy, g)
    np.testing.assert_allclose(gx, [0.0, -g, 0.0, g, -0.8 * g], rtol=1e-15, atol=1e-22)
    np.testing.assert_allclose(gy, [g, 0.0, -g, 0.0, 0.6 * g], rtol=1e-15, atol=1e-22)
    np.testing.assert_allclose(np.hypot(gx, gy), g, rtol=1e-15)


# ----------------------------------------------------------------------------- shape vectors

def _random_stencil(rng, K, jitter=1.0):
    p = rng.uniform(-jitter, jitter, (2, K))
    p[:, 0] = 0.0
    return p


def _monomial_values(x, y, deg):
    """x^a y^b for a + b <= deg, written from the definition (order irrelevant here)."""
    return np.array([x ** (t - b) * y ** b for t in range(deg + 1) for b in range(t + 1)])


@pytest.mark.parametrize("deg,K", [(1, 6), (2, 12), (3, 16), (4, 25), (5, 30), (6, 45)])
def test_shape_vector_reproduces_polynomials(deg, K):
    """The P_L^T block of eq. (rbf_interp_set_augmented) forces exact reproduction of every
    monomial up to the augmentation degree; with them, sum w = 1."""
    rng = np.random.default_rng(deg * 100 + K)
    for _ in range(5):
        p = _random_stencil(rng, K)
        q = rng.uniform(-0.3, 0.3, 2)
        w = oracle.shape_vector(p[0], p[1], q, deg)
        vals = np.array([_monomial_values(p[0, j], p[1, j], deg) for j in range(K)])
        got = w @ vals
        want = _monomial_values(q[0], q[1], deg)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
        assert w.sum() == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("deg,K", [(2, 12), (4, 25)])
def test_shape_vector_interpolates_at_nodes(deg, K):
    """Evaluated at stencil member j the shape vector is the unit vector e_j (the interpolant
    passes through the data)."""
    rng = np.random.default_rng(11)
    p = _random_stencil(rng, K)
    for j in range(K):
        w = oracle.shape_vector(p[0], p[1], p[:, j], deg)
        e = np.zeros(K)
        e[j] = 1.0
        np.testing.assert_allclose(w, e, atol=1e-10)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_shape_vector_unisolvent_case_is_lagrange_interpolation(deg):
    """With N_L equal to the number of monomials, P_L^T w = p(q) fixes w alone: polynomial
    (Lagrange) interpolation, independent of the radial part; compared with numpy.linalg."""
    rng = np.random.default_rng(deg)
    m = (deg + 1) * (deg + 2) // 2
    p = _random_stencil(rng, m)
    q = rng.uniform(-0.5, 0.5, 2)
    V = np.array([_monomial_values(p[0, j], p[1, j], deg) for j in range(m)])
    w_ref = np.linalg.solve(V.T, _monomial_values(q[0], q[1], deg))
    w = oracle.shape_vector(p[0], p[1], q, deg)
    np.testing.assert_allclose(w, w_ref, atol=1e-10)


def test_shape_vector_triangle_is_barycentric():
    """Three nodes with linear augmentation give the barycentric coordinates of q."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        p = _random_stencil(rng, 3)
        q = rng.uniform(-0.5, 0.5, 2)
        (x1, x2, x3), (y1, y2, y3) = p
        det = (y2 - y3) * (x1 - x3) + (x3 - x2) * (y1 - y3)
        l1 = ((y2 - y3) * (q[0] - x3) + (x3 - x2) * (q[1] - y3)) / det
        l2 = ((y3 - y1) * (q[0] - x3) + (x1 - x3) * (q[1] - y3)) / det
        w = oracle.shape_vector(p[0], p[1], q, 1)
        np.testing.assert_allclose(w, [l1, l2, 1 - l1 - l2], atol=1e-12)


@pytest.mark.parametrize("K", [4, 7, 12])
def test_shape_vector_1d_cubic_is_natural_spline(K):
    """In one dimension, r^3 radial functions with linear augmentation interpolate with the
    natural cubic spline; this pins the radial block R_L and the r^3 basis of Sec. 2.3."""
    from scipy.interpolate import CubicSpline

    rng = np.random.default_rng(K)
    xs = np.sort(rng.uniform(-1, 1, K))
    order = rng.permutation(K)
    px = xs[order] - xs[order][0]
    for q in rng.uniform(px.min(), px.max(), 5):
        w = oracle.shape_vector(px, None, [q], 1, dim=1)
        srt = np.argsort(px)
        for j in range(K):
            data = np.zeros(K)
            data[j] = 1.0
            cs = CubicSpline(px[srt], data[srt], bc_type="natural")
            assert w[j] == pytest.approx(float(cs(q)), abs=1e-10)


def test_shape_vector_scale_and_translation_invariant():
    rng = np.random.default_rng(21)
    p = _random_stencil(rng, 20)
    q = rng.uniform(-0.2, 0.2, 2)
    w = oracle.shape_vector(p[0], p[1], q, 3)
    for s in [1e-3, 0.37, 250.0]:
        w2 = oracle.shape_vector(p[0] * s, p[1] * s, q * s, 3)
        np.testing.assert_allclose(w2, w, atol=1e-9)


def test_shape_vector_cross_check_numpy_solve():
    """Cross-check (not a pin): the same collocation system solved by numpy.linalg."""
    rng = np.random.default_rng(4)
    K, deg = 15, 2
    p = _random_stencil(rng, K)
    q = rng.uniform(-0.3, 0.3, 2)
    s = np.max(np.hypot(p[0], p[1]))
    t, qq = p / s, q / s
    R = np.hypot(t[0][:, None] - t[0][None], t[1][:, None] - t[1][None]) ** 3
    P = np.array([_monomial_values(t[0, j], t[1, j], deg) for j in range(K)])
    m = P.shape[1]
    A = np.block([[R, P], [P.T, np.zeros((m, m))]])
    b = np.concatenate([np.hypot(qq[0] - t[0], qq[1] - t[1]) ** 3,
                        _monomial_values(qq[0], qq[1], deg)])
    np.testing.assert_allclose(oracle.shape_vector(p[0], p[1], q, deg),
                               np.linalg.solve(A, b)[:K], atol=1e-10)


def test_shape_vector_singular_detected():
    p = np.zeros((2, 6))
    p[0] = np.arange(6) * 0.1  # collinear points cannot carry x*y, y^2
    with pytest.raises(np.linalg.LinAlgError):
        oracle.shape_vector(p[0], p[1], [0.05, 0.0], 2)


def test_interpolation_convergence_above_second_order():
    """Fig. (interp_test): f = 0.01 sin(2 pi x) cos(2 pi y) interpolated to the Lagrangian
    points of dx_ml = 1/10 on refining clouds, N_L = 25, each Lagrangian point interpolated in
    the stencil of its nearest Eulerian node (Sec. 2.3); the error converges faster than
    second order for P_2 and P_4, and P_4 is more accurate than P_2."""
    fun = lambda x, y: 0.01 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    errs = {2: [], 4: []}
    sides = [10, 20, 40]
    ex, ey, _ = oracle.d2q9()
    for deg in (2, 4):
        for s in sides:
            xy = mi.jittered_lattice(s, 0.3, seed=s)
            sidx, W = oracle.weights(xy, 25, deg, 0.1, box=(1.0, 1.0), mode="paper")
            fv = fun(xy[0], xy[1])
            num = den = 0.0
            for k in range(1, 9):
                interp = np.sum(W[k] * fv[sidx[k]], axis=0)
                exact = fun(xy[0] - ex[k] * 0.1, xy[1] - ey[k] * 0.1)
                num += np.sum((interp - exact) ** 2)
                den += np.sum(exact ** 2)
            errs[deg].append(np.sqrt(num / den))
    for deg in (2, 4):
        e = np.array(errs[deg])
        slopes = np.log(e[:-1] / e[1:]) / np.log(2.0)
        assert slopes.min() > 2.0, (deg, e, slopes)
    assert all(a < b for a, b in zip(errs[4], errs[2]))


# ----------------------------------------------------------------------------- stencils

def test_knn_brute_force_properties():
    xy = mi.jittered_lattice(12, 0.3, seed=4)
    st = oracle.stencils(xy, 13, box=(1.0, 1.0))
    n = xy.shape[1]
    assert np.all(st[0] == np.arange(n))  # centre first (Sec. 2.2)
    for i in [0, 5, 77, n - 1]:
        d = xy - xy[:, i:i + 1]
        d -= np.round(d)
        d2 = np.sum(d * d, axis=0)
        order = np.lexsort((np.arange(n), d2))
        np.testing.assert_array_equal(st[:, i], order[:13])


def test_knn_ties_broken_by_index():
    """Q5 reading: on an exact lattice 12-NN cuts through four nodes at distance 2h; the lower
    indices are taken."""
    xy = mi.lattice(8)
    st = oracle.stencils(xy, 12, box=(1.0, 1.0))
    i = 27
    d = xy - xy[:, i:i + 1]
    d -= np.round(d)
    d2 = np.round(np.sum(d * d, axis=0) * 64).astype(int)
    want = np.lexsort((np.arange(64), d2))[:12]
    np.testing.assert_array_equal(st[:, i], want)


# ----------------------------------------------------------------------------- streaming

def _numpy_lattice_step(f, n, tau):
    """Textbook LBM on an n x n periodic lattice: the oracle's collision, then the index shift
    of eq. (LBM_streaming) done with numpy.roll."""
    ex, ey, _ = oracle.d2q9()
    post = oracle.collide_field(f, tau)
    out = np.empty_like(post)
    for k in range(9):
        g = post[k].reshape(n, n)  # [iy, ix]
        out[k] = np.roll(np.roll(g, ey[k], axis=0), ex[k], axis=1).ravel()
    return out


def test_lattice_step_is_index_shift():
    n, tau = 12, 0.8
    xy = mi.lattice(n)
    rho, u, v = mi.tgv_initial(xy, 0.05)
    f = oracle.init_equilibrium(rho, u, v)
    a = oracle.lattice_step(f, n, n, tau)
    b = _numpy_lattice_step(f, n, tau)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-16)


@pytest.mark.parametrize("mode", ["own", "paper"])
def test_mlbm_on_lattice_reduces_to_lattice_lbm(mode):
    """Sec. 2.1/2.3: nodes on a periodic lattice with spacing dx_ml make every departure point
    a node, the shape vector a unit vector, and MLBM streaming the LBM index shift."""
    n, tau = 16, 0.8
    xy = mi.lattice(n)
    h = 1.0 / n
    sidx, W = oracle.weights(xy, 9, 2, h, box=(1.0, 1.0), mode=mode)
    st = oracle.Stepper(sidx, W, tau)
    rho, u, v = mi.tgv_initial(xy, 0.05)
    f = oracle.init_equilibrium(rho, u, v)
    g = f.copy()
    for _ in range(20):
        f = st.step(f)
        g = _numpy_lattice_step(g, n, tau)
    np.testing.assert_allclose(f, g, rtol=0, atol=1e-13)


def test_uniform_state_is_preserved():
    xy = mi.jittered_lattice(16, 0.3, seed=2)
    sidx, W = oracle.weights(xy, 12, 2, 1.0 / 16, box=(1.0, 1.0))
    st = oracle.Stepper(sidx, W, 0.8)
    n = xy.shape[1]
    f0 = oracle.init_equilibrium(np.full(n, 1.0), np.full(n, 0.02), np.full(n, -0.01))
    f = st.run(f0, 10)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-13)


def test_direction_zero_weight_is_unit_vector():
    """The rest population's departure point is the node itself, so its shape vector is e_0
    and the rest population needs no interpolation."""
    xy = mi.jittered_lattice(10, 0.3, seed=3)
    sidx, W = oracle.weights(xy, 12, 2, 0.1, box=(1.0, 1.0))
    assert np.all(sidx[0, 0] == np.arange(xy.shape[1]))
    np.testing.assert_allclose(W[0, 0], 1.0, atol=1e-12)
    np.testing.assert_allclose(W[0, 1:], 0.0, atol=1e-12)


def test_paper_and_own_stencils_agree_for_short_streaming():
    """Q3 reading: when every departure point's nearest node is the node itself the paper's
    stencil choice and the own-stencil choice are the same."""
    xy = mi.jittered_lattice(10, 0.3, seed=5)
    h = 0.1
    a = oracle.weights(xy, 12, 2, 0.1 * h, box=(1.0, 1.0), mode="own")
    b = oracle.weights(xy, 12, 2, 0.1 * h, box=(1.0, 1.0), mode="paper")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c = oracle.weights(xy, 12, 2, h, box=(1.0, 1.0), mode="paper")
    assert np.any(c[0] != a[0])


# ----------------------------------------------------------------------------- Taylor-Green runs

def _tgv_run(n_side, K, deg, steps, u0=0.01, tau=0.8, jitter=0.3, seed=1, ratio=1.0):
    xy = mi.jittered_lattice(n_side, jitter, seed=seed) if jitter > 0 else mi.lattice(n_side)
    h = 1.0 / n_side
    dx_ml = ratio * h
    sidx, W = oracle.weights(xy, K, deg, dx_ml, box=(1.0, 1.0))
    st = oracle.Stepper(sidx, W, tau)
    rho, u, v = mi.tgv_initial(xy, u0)
    f = st.run(oracle.init_equilibrium(rho, u, v), steps)
    _, uu, vv = oracle.moments_field(f)
    nu = oracle.lattice_viscosity(tau)
    L = 1.0 / dx_ml
    ut, vt = oracle.tgv_velocity(xy[0] / dx_ml, xy[1] / dx_ml, steps, u0=u0, nu=nu, L=L)
    return oracle.l2_norm(uu, ut), uu, ut


def test_tgv_small_cloud_follows_analytic_decay():
    """Taylor-Green vortex on 32^2 jittered nodes, N_L = 12, P_2, tau = 0.8, dt = dx_ml = h,
    500 steps: the velocity follows eq. (tgv_eqs) within a few percent."""
    err, uu, ut = _tgv_run(32, 12, 2, 500)
    assert err < 0.05, err
    amp = np.sum(uu * ut) / np.sum(ut * ut)
    assert amp == pytest.approx(1.0, abs=0.05)


def test_lattice_lbm_tgv_second_order():
    """Standard LBM is second-order convergent on the Taylor-Green vortex under diffusive
    scaling (Sec. 3): u0 ~ dx, steps to t_end ~ dx^-2."""
    tau = 0.8
    nu = oracle.lattice_viscosity(tau)
    errs = []
    for n in (16, 32, 64):
        xy = mi.lattice(n)
        u0 = 0.04 * 16 / n
        rho, u, v = mi.tgv_initial(xy, u0)
        f = oracle.init_equilibrium(rho, u, v)
        steps = int(round(oracle.tgv_end_time(nu=nu, L=n)))
        for _ in range(steps):
            f = oracle.lattice_step(f, n, n, tau)
        _, uu, _ = oracle.moments_field(f)
        ut, _ = oracle.tgv_velocity(xy[0] * n, xy[1] * n, steps, u0=u0, nu=nu, L=n)
        errs.append(oracle.l2_norm(uu, ut))
    slopes = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2.0)
    assert np.all((slopes > 1.7) & (slopes < 2.3)), (errs, slopes)


def test_mlbm_tgv_higher_degree_is_more_accurate():
    """Sec. 3: raising the polynomial augmentation from P_2 to P_4 lowers the error
    (N_L = 25, dx_ml = h/4, coarse cloud)."""
    e2, _, _ = _tgv_run(16, 25, 2, 200, ratio=0.25, u0=0.0025)
    e4, _, _ = _tgv_run(16, 25, 4, 200, ratio=0.25, u0=0.0025)
    assert e4 < e2, (e2, e4)


# ----------------------------------------------------------------------------- annulus

def test_resting_fluid_with_walls_stays_at_rest():
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    dx_ml = 1.0 / 40
    sidx, W = oracle.weights(xy, 15, 2, dx_ml)
    mask = oracle.bounce_mask(xy, dx_ml, 0.5, 1.0)
    assert mask.any()
    n = xy.shape[1]
    st = oracle.Stepper(sidx, W, 1.0, mask=mask)
    f0 = oracle.init_equilibrium(np.ones(n), np.zeros(n), np.zeros(n))
    f = st.run(f0, 20)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-14)


def test_bounce_mask_flags_only_outgoing_departures():
    xy, wall = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    dx_ml = 1.0 / 200
    mask = oracle.bounce_mask(xy, dx_ml, 0.5, 1.0)
    r = np.hypot(xy[0], xy[1])
    ex, ey, _ = oracle.d2q9()
    # every wall node has unknown populations, interior nodes far from walls have none
    assert np.all(mask[wall] != 0)
    far = (r > 0.5 + 2 * dx_ml) & (r < 1.0 - 2 * dx_ml)
    assert np.all(mask[far] == 0)
    # on the outer wall, population k is unknown when e_k points inward (departure outside)
    outer = np.where(wall & (r > 0.75))[0]
    for i in outer[:20]:
        for k in range(1, 9):
            radial = ex[k] * xy[0, i] + ey[k] * xy[1, i]
            if radial < -0.2:
                assert mask[i] >> k & 1


def test_annulus_steady_profile_matches_analytic():
    """Force-driven flow in the ring r in [0.5, 1] (the paper's R2/R1 = 2 geometry, scaled),
    N_L = 15, P_2, tau = 1, wall bounce-back: the steady azimuthal velocity follows
    eq. (bch_solution)."""
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    dx_ml = 1.0 / 40
    tau, g = 1.0, 1e-6
    sidx, W = oracle.weights(xy, 15, 2, dx_ml)
    mask = oracle.bounce_mask(xy, dx_ml, 0.5, 1.0)
    gx, gy = oracle.azimuthal_force(xy, g)
    n = xy.shape[1]
    st = oracle.Stepper(sidx, W, tau, mask=mask, force=(gx, gy))
    f = oracle.init_equilibrium(np.ones(n), np.zeros(n), np.zeros(n))
    prev = None
    for it in range(200):
        f = st.run(f, 50)
        _, u, v = oracle.moments_field(f)
        if prev is not None and oracle.residual(u, v, *prev) < 1e-7:
            break
        prev = (u, v)
    r = np.hypot(xy[0], xy[1])
    ut = -xy[1] / r * u + xy[0] / r * v
    nu = oracle.lattice_viscosity(tau)
    want = oracle.annulus_velocity(r / dx_ml, g, nu, 0.5 / dx_ml, 1.0 / dx_ml)
    interior = (r > 0.5 + 1e-9) & (r < 1.0 - 1e-9)
    assert oracle.l2_norm(np.hypot(u, v)[interior], np.abs(want[interior])) < 0.06
    # signed: the flow turns the way the force pushes (counter-clockwise for g > 0), as
    # eq. (bch_solution) gives it; a flipped force direction reverses u_theta and fails here
    assert np.all(want[interior] > 0)
    assert oracle.l2_norm(ut[interior], want[interior]) < 0.06
    ur = xy[0] / r * u + xy[1] / r * v
    assert np.max(np.abs(ur)) < 0.05 * np.max(np.abs(want))
