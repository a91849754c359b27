"""Standard lattice LBM on the GPU (mlbm_lattice_step) against the oracle's lattice step, and
the paper's finding that the lattice-LBM error at a streaming distance dx is the lower bound the
meshless error approaches at dx_ml = dx as the cloud is refined (Sec. 3, Sec. 4)."""
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


@pytest.mark.parametrize("nx,ny", [(16, 16), (37, 23)])
def test_lattice_step_matches_oracle(nx, ny):
    xy = np.stack(np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny, indexing="xy")).reshape(2, -1)
    rho, u, v = mi.tgv_initial(xy, 0.03)
    tau = 0.7
    f = oracle.init_equilibrium(rho, u, v)
    a = torch.empty(9 * nx * ny, dtype=torch.float64, device=DEV)
    b = torch.empty_like(a)
    mom = torch.empty(3 * nx * ny, dtype=torch.float64, device=DEV)
    mlbm.lattice_init(nx, ny, (tau, 0.0, 1.0), mlbm.F64, _t(rho), _t(u), _t(v), a)
    for it in range(25):
        mlbm.lattice_step(nx, ny, (tau, 0.0, 1.0), mlbm.F64, a, b, mom)
        a, b = b, a
        f = oracle.lattice_step(f, nx, ny, tau)
        post = oracle.collide_field(f, tau)
        got = a.view(9, -1).cpu().numpy()
        assert np.max(np.abs(got - post)) <= 1e-12 * np.max(np.abs(post)), it
    r_o, u_o, v_o = oracle.moments_field(f)
    m = mom.view(3, -1).cpu().numpy()
    np.testing.assert_allclose(m[1], u_o, atol=1e-15)
    np.testing.assert_allclose(m[2], v_o, atol=1e-15)


def _lbm_error(L, u0, tau, steps, dtype):
    xy = mi.lattice(L)
    rho, u, v = mi.tgv_initial(xy, u0)
    td = torch.float64 if dtype == mlbm.F64 else torch.float32
    a = torch.empty(9 * L * L, dtype=td, device=DEV)
    b = torch.empty_like(a)
    mom = torch.empty(3 * L * L, dtype=td, device=DEV)
    mlbm.lattice_init(L, L, (tau, 0.0, 1.0), dtype, _t(rho), _t(u), _t(v), a)
    for _ in range(steps):
        mlbm.lattice_step(L, L, (tau, 0.0, 1.0), dtype, a, b, mom)
        a, b = b, a
    nu = oracle.lattice_viscosity(tau)
    ut, _ = oracle.tgv_velocity(xy[0] * L, xy[1] * L, steps, u0=u0, nu=nu, L=L)
    return oracle.l2_norm(mom.view(3, -1)[1].double().cpu().numpy(), ut)


def _mlbm_error(n, L, K, deg, u0, tau, steps, dtype):
    xy = mi.jittered_lattice(n, 0.3, seed=90 + n)
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=1.0 / L))
    w = mlbm.build_weights(cloud)
    rho, u, v = mi.tgv_initial(xy, u0)
    td = torch.float64 if dtype == mlbm.F64 else torch.float32
    a = torch.empty(9 * w.n, dtype=td, device=DEV)
    b = torch.empty_like(a)
    mlbm.init(w, [(tau, 0.0, 1.0)], dtype, _t(rho), _t(u), _t(v), a)
    res = mlbm.run(w, [(tau, 0.0, 1.0)], dtype, a, b, steps)
    _, um, _ = mlbm.moments(w, [(tau, 0.0, 1.0)], dtype, res)
    nu = oracle.lattice_viscosity(tau)
    ut, _ = oracle.tgv_velocity(xy[0] * L, xy[1] * L, steps, u0=u0, nu=nu, L=L)
    return oracle.l2_norm(um.cpu().numpy(), ut)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lattice_lbm_is_lower_bound_of_meshless_error(dtype):
    """dx_ml = dx = 1/64, Taylor-Green to t_end, P_4, N_L = 24: refining the cloud from 24^2 to
    64^2 nodes brings the meshless error down onto the lattice-LBM error at dx = 1/64 and not
    below it (oracle on the same inputs: 6.5e-3, 2.6e-3, 1.75e-3, 1.71e-3 vs 1.70e-3)."""
    dt = mlbm.F64 if dtype == "f64" else mlbm.F32
    L, tau, u0 = 64, 0.8, 0.01
    steps = int(round(oracle.tgv_end_time(nu=oracle.lattice_viscosity(tau), L=L)))
    e_lbm = _lbm_error(L, u0, tau, steps, dt)
    errs = [_mlbm_error(n, L, 24, 4, u0, tau, steps, dt) for n in (24, 32, 48, 64)]
    assert all(a > b for a, b in zip(errs[:-1], errs[1:])), errs
    assert min(errs) >= 0.97 * e_lbm, (errs, e_lbm)
    assert errs[-1] <= 1.05 * e_lbm, (errs, e_lbm)


@pytest.mark.parametrize("nx,ny", [(4, 4), (8, 5), (132, 7), (256, 3), (1028, 2)])
def test_fp32_four_node_path_equals_the_one_node_path(nx, ny):
    """FP32 with nx a multiple of 4 and 16-byte aligned arrays runs four nodes per thread (16-byte
    loads, neighbours across lanes by shuffles, periodic wrap at the row ends); misaligned
    arrays take the one-node path.  Both compute the same arithmetic per node: bit-identical
    states and moments, steps after step."""
    xy = np.stack(np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny, indexing="xy")).reshape(2, -1)
    rng = np.random.default_rng(nx + ny)
    rho = 1 + 0.02 * rng.standard_normal(nx * ny)
    u, v = 0.03 * rng.standard_normal(nx * ny), 0.03 * rng.standard_normal(nx * ny)
    n = nx * ny
    prm = (0.7, 1e-4, 1.0)
    buf = [torch.empty(9 * n + 1, dtype=torch.float32, device=DEV) for _ in range(4)]
    a4, b4 = buf[0][:9 * n], buf[1][:9 * n]          # aligned
    a1, b1 = buf[2][1:], buf[3][1:]                  # offset by one element: misaligned
    mlbm.lattice_init(nx, ny, prm, mlbm.F32, _t(rho), _t(u), _t(v), a4)
    a1.copy_(a4)
    m4 = torch.empty(3 * n + 1, dtype=torch.float32, device=DEV)
    m1 = torch.empty(3 * n + 1, dtype=torch.float32, device=DEV)
    for _ in range(6):
        mlbm.lattice_step(nx, ny, prm, mlbm.F32, a4, b4, m4[:3 * n])
        mlbm.lattice_step(nx, ny, prm, mlbm.F32, a1, b1, m1[1:])
        a4, b4 = b4, a4
        a1, b1 = b1, a1
        assert torch.equal(a4, a1)
        assert torch.equal(m4[:3 * n], m1[1:])
    assert xy.shape[1] == n
