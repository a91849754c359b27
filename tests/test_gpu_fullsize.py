"""Parity at the full size of the large Taylor-Green workload (2048^2 jittered nodes, N_L = 30,
P_4, dx_ml = h), in the launch configuration the benchmark times: one FP64 and one FP32 step,
checked on sampled nodes that the oracle computes one by one (brute-force stencil over all
4,194,304 nodes, its own shape vectors, its own collide-then-stream)."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu

N_SIDE, K, DEG, TAU, U0, SEED = 2048, 30, 4, 0.8, 0.01, 3
SAMPLES = 40


@pytest.fixture(scope="module")
def big():
    xy = mi.jittered_lattice(N_SIDE, 0.3, seed=SEED)
    dx = 1.0 / N_SIDE
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=DEG, dx_ml=dx))
    w = mlbm.build_weights(cloud)
    return xy, dx, cloud, w


def _oracle_node_step(xy, dx, i, rho, u, v):
    """Moments after one oracle step at node i, from the equilibrium initial state."""
    sidx, W = oracle.node_weights(xy, i, K, DEG, dx, box=(1.0, 1.0))
    members = np.unique(sidx)
    pos = {m: t for t, m in enumerate(members)}
    f0 = oracle.init_equilibrium(rho[members], u[members], v[members])
    post = oracle.collide_field(f0, TAU)
    f1 = np.zeros(9)
    for k in range(9):
        f1[k] = sum(W[k, j] * post[k, pos[sidx[k, j]]] for j in range(K))
    return sidx[1], oracle.moments(f1)


def test_full_size_one_step_sampled_parity(big):
    xy, dx, cloud, w = big
    assert w.n_bad == 0
    n = w.n
    rho, u, v = mi.tgv_initial(xy, U0)
    perm = cloud.perm()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:0")
    params = [(TAU, 0.0, 1.0)]
    got = {}
    for dtype, td in ((mlbm.F64, torch.float64), (mlbm.F32, torch.float32)):
        f0 = torch.empty(9 * n, dtype=td, device="cuda:0")
        f1 = torch.empty_like(f0)
        mom = torch.empty(3 * n, dtype=td, device="cuda:0")
        mlbm.init(w, params, dtype, t(rho), t(u), t(v), f0)
        mlbm.step(w, params, dtype, f0, f1, mom)
        got[dtype] = mom.view(3, n).cpu().numpy().astype(np.float64)
        del f0, f1, mom
    rng = np.random.default_rng(17)
    sample = rng.choice(n, SAMPLES, replace=False)
    st_gpu = cloud.stencil(0)
    for i in sample:
        st_o, (r_o, u_o, v_o) = _oracle_node_step(xy, dx, int(i), rho, u, v)
        np.testing.assert_array_equal(st_gpu[:, i], st_o)
        p = inv[i]
        for dtype, atol in ((mlbm.F64, 1e-9), (mlbm.F32, 1e-8)):
            m = got[dtype][:, p]
            assert abs(m[0] - r_o) < 10 * atol, (i, dtype, m[0], r_o)
            assert abs(m[1] - u_o) < atol, (i, dtype, m[1], u_o)
            assert abs(m[2] - v_o) < atol, (i, dtype, m[2], v_o)


def test_full_size_three_single_steps_sampled_parity(big):
    """Per-step parity at full size over three consecutive steps, in both precisions: each GPU
    step, from the GPU's own state of the previous level, matches at sampled nodes the oracle's
    streaming of that state (its own stencils and shape vectors, checked equal to the GPU's
    stencils) followed by its moments."""
    xy, dx, cloud, w = big
    n = w.n
    rho, u, v = mi.tgv_initial(xy, U0)
    perm = cloud.perm()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:0")
    params = [(TAU, 0.0, 1.0)]
    rng = np.random.default_rng(29)
    sample = rng.choice(n, 16, replace=False)
    st_gpu = cloud.stencil(0)
    node_w = {}
    for i in sample:
        node_w[i] = oracle.node_weights(xy, int(i), K, DEG, dx, box=(1.0, 1.0))
        np.testing.assert_array_equal(st_gpu[:, i], node_w[i][0][1])
    omega = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    for dtype, td, atol in ((mlbm.F64, torch.float64, 1e-9), (mlbm.F32, torch.float32, 1e-8)):
        a = torch.empty(9 * n, dtype=td, device="cuda:0")
        b = torch.empty_like(a)
        mom = torch.empty(3 * n, dtype=td, device="cuda:0")
        mlbm.init(w, params, dtype, t(rho), t(u), t(v), a)
        for step in range(3):
            mlbm.step(w, params, dtype, a, b, mom)
            # the previous level's post-collision populations, original node order (the FP32
            # state holds deviations from omega_k rho0)
            prev = a.view(9, n).cpu().numpy().astype(np.float64)
            if dtype == mlbm.F32:
                prev += omega[:, None]
            post = np.empty_like(prev)
            post[:, perm] = prev
            got = mom.view(3, n).cpu().numpy().astype(np.float64)
            for i in sample:
                sidx, W = node_w[i]
                f = np.array([W[k] @ post[k, sidx[k]] for k in range(9)])
                r_o, u_o, v_o = oracle.moments(f)
                m = got[:, inv[i]]
                assert abs(m[0] - r_o) < 10 * atol, (step, i, dtype, m[0], r_o)
                assert abs(m[1] - u_o) < atol, (step, i, dtype, m[1], u_o)
                assert abs(m[2] - v_o) < atol, (step, i, dtype, m[2], v_o)
            a, b = b, a
        del a, b, mom


def test_full_size_fp32_tracks_fp64(big):
    """Whole-field check at full size: after 200 steps the FP32 deviation-storage path stays
    within 1e-6 relative L2 of the FP64 path (same shape vectors)."""
    xy, dx, cloud, w = big
    n = w.n
    rho, u, v = mi.tgv_initial(xy, U0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:0")
    params = [(TAU, 0.0, 1.0)]
    out = {}
    for dtype, td in ((mlbm.F64, torch.float64), (mlbm.F32, torch.float32)):
        a = torch.empty(9 * n, dtype=td, device="cuda:0")
        b = torch.empty_like(a)
        mlbm.init(w, params, dtype, t(rho), t(u), t(v), a)
        res = mlbm.run(w, params, dtype, a, b, 200)
        out[dtype] = mlbm.moments(w, params, dtype, res)
        del a, b, res
    s = mlbm.norms(w, out[mlbm.F32][1], out[mlbm.F64][1], out[mlbm.F32][2], out[mlbm.F64][2])
    assert np.sqrt(s[0] / s[1]) < 1e-6


def test_largest_cloud_one_step_sampled_parity():
    """Four times the benchmark's node count: 4096^2 jittered nodes (16.8 M), N_L = 12, P_2,
    FP32 tile layout only, stencils built on the device.  Sampled stencils equal the oracle's
    brute force over all nodes, and one FP32 step matches the oracle's step at those nodes."""
    n_side, k, deg = 4096, 12, 2
    xy = mi.jittered_lattice(n_side, 0.3, seed=5)
    dx = 1.0 / n_side
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=k, degree=deg, dx_ml=dx),
                             device=True)
    w = mlbm.build_weights(cloud, keep=mlbm.KEEP_W32)
    assert w.n_bad == 0 and w.n == n_side * n_side
    n = w.n
    rho, u, v = mi.tgv_initial(xy, U0)
    perm = cloud.perm()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:0")
    params = [(TAU, 0.0, 1.0)]
    f0 = torch.empty(9 * n, dtype=torch.float32, device="cuda:0")
    f1 = torch.empty_like(f0)
    mom = torch.empty(3 * n, dtype=torch.float32, device="cuda:0")
    mlbm.init(w, params, mlbm.F32, t(rho), t(u), t(v), f0)
    mlbm.step(w, params, mlbm.F32, f0, f1, mom)
    got = mom.view(3, n).cpu().numpy().astype(np.float64)
    del f0, f1, mom
    st_gpu = cloud.stencil(0)
    rng = np.random.default_rng(23)
    for i in rng.choice(n, 8, replace=False):
        sidx, W = oracle.node_weights(xy, int(i), k, deg, dx, box=(1.0, 1.0))
        np.testing.assert_array_equal(st_gpu[:, i], sidx[1])
        members = np.unique(sidx)
        pos = {m: q for q, m in enumerate(members)}
        post = oracle.collide_field(oracle.init_equilibrium(rho[members], u[members], v[members]), TAU)
        f1n = np.array([sum(W[kk, j] * post[kk, pos[sidx[kk, j]]] for j in range(k)) for kk in range(9)])
        r_o, u_o, v_o = oracle.moments(f1n)
        m = got[:, inv[i]]
        assert abs(m[0] - r_o) < 1e-7 and abs(m[1] - u_o) < 1e-8 and abs(m[2] - v_o) < 1e-8, (i, m, r_o, u_o, v_o)


def test_512_node_tiles_fp32_run_and_fp64_steps_against_oracle():
    """The 512-node tile kernels (the benchmark's launch configuration) against the oracle over
    whole runs, at the smallest cloud of the large recipe that selects them (at least four
    512-node tiles per SM): 560^2 jittered nodes, seed 3, N_L 30, P_4, the oracle's shape vectors
    uploaded.  FP64: three steps, each within 1e-12 of the oracle's step.  FP32: 200 steps
    within 1e-6 relative L2 of the velocity of the FP64 oracle."""
    n_side = 560
    n = n_side * n_side
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert -(-n // 512) >= 4 * sms  # the tile-size rule picks 512-node tiles for this cloud
    xy = mi.jittered_lattice(n_side, 0.3, seed=SEED)
    dx = 1.0 / n_side
    cloud = mlbm.build_cloud(xy, dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=DEG, dx_ml=dx),
                             device=True)
    w = mlbm.build_weights(cloud)
    sidx, W = oracle.weights(xy, K, DEG, dx, box=(1.0, 1.0))
    w.upload(W[1:], sidx[1].astype(np.int32))
    perm = cloud.perm()
    rho, u, v = mi.tgv_initial(xy, U0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda:0")
    params = [(TAU, 0.0, 1.0)]
    st = oracle.Stepper(sidx, W, TAU)
    f_or = oracle.init_equilibrium(rho, u, v)
    # FP64, step by step (the library holds f^post = C(f))
    a = torch.empty(9 * n, dtype=torch.float64, device="cuda:0")
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F64, t(rho), t(u), t(v), a)
    for it in range(3):
        mlbm.step(w, params, mlbm.F64, a, b)
        a, b = b, a
        f_or = st.step(f_or)
        post = oracle.collide_field(f_or, TAU)
        got = np.empty_like(post)
        got[:, perm] = a.view(9, n).cpu().numpy()
        assert np.max(np.abs(got - post)) <= 1e-12 * np.max(np.abs(post)), it
    del a, b
    # FP32, 200 steps
    f_or = st.run(f_or, 197)
    _, u_o, v_o = oracle.moments_field(f_or)
    a = torch.empty(9 * n, dtype=torch.float32, device="cuda:0")
    b = torch.empty_like(a)
    mlbm.init(w, params, mlbm.F32, t(rho), t(u), t(v), a)
    res = mlbm.run(w, params, mlbm.F32, a, b, 200)
    _, ug, vg = mlbm.moments(w, params, mlbm.F32, res)
    ug, vg = ug.cpu().numpy(), vg.cpu().numpy()
    err = np.sqrt(np.sum((ug - u_o) ** 2 + (vg - v_o) ** 2) / np.sum(u_o ** 2 + v_o ** 2))
    assert err <= 1e-6, err
