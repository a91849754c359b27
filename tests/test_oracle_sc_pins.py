"""Pins of the oracle's Shan-Chen extension (pseudopotential, interaction force, step) to facts
that do not come from the oracle itself: special values of the pseudopotential, reduction to
the plain step without interaction, the exact discrete gradient of quadratic fields by the
D2Q9 weights (sum_k omega_k e_k = 0, sum_k omega_k e_k e_k = I/3, odd third moments vanish),
the lattice limit of the meshless interpolation, Newton's third law on a lattice, mass
conservation, the linear stability of a uniform state, which changes sign at the critical
coupling G_c = -4 of psi = 1 - exp(-rho) (dp/drho = (1 + G psi psi') / 3 vanishes at
rho = ln 2, where psi = psi' = 1/2), and the coexistence densities of a flat interface, which
the equation of state p = rho / 3 + G psi^2 / 6 fixes through equal pressures and the
mechanical-stability condition int (p_0 - p) psi' / psi^2 drho = 0 (Shan 2008), up to the
discretisation's small deviation."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle


def test_psi_special_values():
    for rho0 in (1.0, 2.5):
        assert oracle.sc_psi(rho0 * np.log(2.0), rho0) == pytest.approx(rho0 / 2, rel=1e-15)
        assert oracle.sc_psi(0.0, rho0) == 0.0
        assert oracle.sc_psi(60.0 * rho0, rho0) == pytest.approx(rho0, rel=1e-15)
        h = 1e-6
        d0 = (oracle.sc_psi(h, rho0) - oracle.sc_psi(-h, rho0)) / (2 * h)
        assert d0 == pytest.approx(1.0, rel=1e-9)  # psi ~ rho for small densities


def _periodic_cloud(n_side=16, K=12, deg=3, dx=None, seed=3, mode="own"):
    xy = mi.jittered_lattice(n_side, 0.3, seed=seed)
    dx = dx if dx is not None else 0.5 / n_side
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode=mode)
    return xy, dx, sidx, W


@pytest.mark.parametrize("mode", ["own", "paper"])
def test_no_interaction_is_the_plain_step(mode):
    xy, dx, sidx, W = _periodic_cloud(dx=(2.0 if mode == "paper" else 0.5) / 16, mode=mode)
    rho, u, v = mi.tgv_initial(xy, 0.02)
    f = oracle.init_equilibrium(rho, u, v)
    a = oracle.Stepper(sidx, W, 0.8)
    b = oracle.ScStepper(sidx, W, 0.8, G=0.0)
    fa, fb = f, f
    for _ in range(5):
        fa, fb = a.step(fa), b.step(fb)
    np.testing.assert_array_equal(fa, fb)


@pytest.mark.parametrize("mode,dx", [("own", 0.03), ("paper", 0.1)])
def test_force_of_a_quadratic_field_is_the_exact_gradient(mode, dx):
    """psi quadratic in x: interpolation with degree >= 2 is exact at every departure point and
    sum_k omega_k psi(x + e_k d) e_k = d grad psi / 3 exactly, so F = -G psi d grad(psi) / 3.
    Under either stencil rule (the nearest-node rule with dx_ml above the spacing, so that the
    departure points are interpolated in other nodes' stencils)."""
    xy = mi.jittered_lattice(14, 0.3, seed=5)  # no periodic box: stencils extrapolate at edges
    G = -4.7
    sidx, W = oracle.weights(xy, 12, 2, dx, mode=mode)
    if mode == "paper":
        assert np.any(sidx[1:, 0, :] != np.arange(xy.shape[1])[None, :])
    x, y = xy
    q = 0.3 + 0.1 * x - 0.05 * y + 0.08 * x * x + 0.04 * x * y - 0.06 * y * y
    gx, gy = 0.1 + 0.16 * x + 0.04 * y, -0.05 + 0.04 * x - 0.12 * y
    fx, fy = oracle.sc_force(sidx, W, q, G)
    np.testing.assert_allclose(fx, -G * q * dx * gx / 3, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fy, -G * q * dx * gy / 3, rtol=0, atol=1e-12)
    # a cubic term is not reproduced by the D2Q9 moments: the pin above is not vacuous
    fx3, _ = oracle.sc_force(sidx, W, q + 0.5 * x ** 3, G)
    assert np.max(np.abs(fx3 + G * (q + 0.5 * x ** 3) * dx * (gx + 1.5 * x * x) / 3)) > 1e-9


def _lattice_state(n, amp, seed):
    xy = mi.lattice(n)
    rng = np.random.default_rng(seed)
    rho = np.log(2.0) * (1 + amp * rng.standard_normal(n * n))
    return xy, oracle.init_equilibrium(rho, np.zeros(n * n), np.zeros(n * n))


def test_meshless_step_on_a_lattice_is_the_lattice_shan_chen_step():
    """Nodes on a periodic lattice with dx_ml = h: every departure point is a node, the shape
    vectors are unit vectors, and the meshless step is the index-shift step."""
    n, tau, G = 12, 0.9, -5.0
    xy, f = _lattice_state(n, 0.02, 1)
    sidx, W = oracle.weights(xy, 9, 2, 1.0 / n, box=(1.0, 1.0))
    st = oracle.ScStepper(sidx, W, tau, G=G)
    a, b = f, f
    for _ in range(10):
        a = st.step(a)
        b = oracle.sc_lattice_step(b, n, n, tau, G)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_lattice_force_obeys_newtons_third_law_and_mass_is_conserved():
    n, tau, G = 16, 1.0, -5.5
    xy, f = _lattice_state(n, 0.05, 2)
    sidx, W = oracle.weights(xy, 9, 2, 1.0 / n, box=(1.0, 1.0))
    rho, _, _ = oracle.moments_field(f)
    fx, fy = oracle.sc_force(sidx, W, oracle.sc_psi(rho), G)
    assert abs(fx.sum()) <= 1e-14 * np.abs(fx).sum()
    assert abs(fy.sum()) <= 1e-14 * np.abs(fy).sum()
    m0 = rho.sum()
    for _ in range(50):
        f = oracle.sc_lattice_step(f, n, n, tau, G)
    assert oracle.moments_field(f)[0].sum() == pytest.approx(m0, rel=1e-13)


@pytest.mark.parametrize("G,grows", [(-3.0, False), (-5.0, True)])
def test_uniform_state_is_unstable_only_beyond_the_critical_coupling(G, grows):
    """A long-wave density perturbation of the uniform state at rho = ln 2 decays for G > -4 and
    grows for G < -4 (sign of the effective squared sound speed (1 + G/4) / 3)."""
    n, tau, amp = 32, 1.0, 1e-3
    xy = mi.lattice(n)
    mode = np.cos(2 * np.pi * xy[0])
    rho = np.log(2.0) * (1 + amp * mode)
    f = oracle.init_equilibrium(rho, np.zeros(n * n), np.zeros(n * n))
    a0 = np.abs(np.dot(oracle.moments_field(f)[0] - np.log(2.0), mode))
    for _ in range(100):
        f = oracle.sc_lattice_step(f, n, n, tau, G)
    a1 = np.abs(np.dot(oracle.moments_field(f)[0] - np.log(2.0), mode))
    assert (a1 > 2 * a0) if grows else (a1 < 0.5 * a0), (a0, a1)


def _mechanical_stability_coexistence(G):
    scipy = pytest.importorskip("scipy")
    from scipy.integrate import quad
    from scipy.optimize import fsolve

    psi = lambda r: 1.0 - np.exp(-r)
    p = lambda r: r / 3.0 + G * psi(r) ** 2 / 6.0

    def eqs(v):
        rg, rl = v
        return [p(rl) - p(rg), quad(lambda r: (p(rg) - p(r)) * np.exp(-r) / psi(r) ** 2, rg, rl, limit=200)[0]]

    return fsolve(eqs, [0.15, 1.9])


@pytest.mark.parametrize("G", [-5.0, -5.5])
def test_flat_interface_coexistence_densities(G):
    """A slab of liquid in its vapour on a 64 x 4 periodic lattice relaxes to the coexistence
    densities of the model's equation of state (within 1.5 %)."""
    nx, ny, tau = 64, 4, 1.0
    ix = np.tile(np.arange(nx), ny)
    rho = np.where((ix >= nx // 4) & (ix < 3 * nx // 4), 2.0, 0.15)
    f = oracle.init_equilibrium(rho, np.zeros(nx * ny), np.zeros(nx * ny))
    for _ in range(4000):
        f = oracle.sc_lattice_step(f, nx, ny, tau, G)
    r = oracle.moments_field(f)[0]
    rho_l, rho_g = r[ix == nx // 2].mean(), r[ix == 0].mean()
    rg, rl = _mechanical_stability_coexistence(G)
    assert rho_l == pytest.approx(rl, rel=0.015) and rho_g == pytest.approx(rg, rel=0.015), (rho_l, rho_g, rl, rg)


def test_field_collision_adds_the_force_to_the_momentum_and_keeps_the_mass():
    """Velocity-shift BGK: the momentum of each node changes by exactly (rho u_eq - rho u) / tau
    = F, its mass not at all; with G = 0 it is the plain collision."""
    xy, dx, sidx, W = _periodic_cloud(n_side=12, K=9, deg=2)
    n = xy.shape[1]
    rng = np.random.default_rng(4)
    f = oracle.init_equilibrium(np.log(2.0) * (1 + 0.05 * rng.standard_normal(n)),
                                0.01 * rng.standard_normal(n), 0.01 * rng.standard_normal(n))
    f = f + 1e-3 * rng.standard_normal(f.shape)
    tau, G = 0.9, -5.0
    post = oracle.sc_collide_field(f, sidx, W, tau, G)
    rho, _, _ = oracle.moments_field(f)
    fx, fy = oracle.sc_force(sidx, W, oracle.sc_psi(rho), G)
    ex, ey, _ = oracle.d2q9()
    d = post - f
    np.testing.assert_allclose(d.sum(axis=0), 0.0, atol=1e-15)
    np.testing.assert_allclose(ex @ d, fx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ey @ d, fy, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(oracle.sc_collide_field(f, sidx, W, tau, 0.0), oracle.collide_field(f, tau))
