"""Shan-Chen multiphase steps on the GPU (mlbm_sc_step) against the oracle's Shan-Chen steps:
reduction to the plain step without interaction, per-step parity in FP64, FP32 accuracy, the
lattice limit, and flat interfaces relaxing to the coexistence densities (the extension the
paper's discussion names; model of Shan & Chen 1993)."""
import functools

import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LN2 = float(np.log(2.0))


def _t(a):
    return torch.as_tensor(a, dtype=torch.float64, device=DEV)


def _periodic(xy, K, deg, dx, mode="own"):
    seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=dx,
               stencil_mode=mlbm.STENCIL_NEAREST if mode == "paper" else mlbm.STENCIL_OWN)
    cloud = mlbm.build_cloud(xy, seg)
    return cloud, mlbm.build_weights(cloud)


def _to_stored(post, perm, dtype, rho0=1.0):
    """Oracle populations (original order) -> the library's state (stored order; FP32 holds
    deviations f - omega_k rho0)."""
    s = post[:, perm].copy()
    if dtype == mlbm.F32:
        _, _, om = oracle.d2q9()
        s -= om[:, None] * rho0
    return torch.as_tensor(s.ravel(), dtype=torch.float32 if dtype == mlbm.F32 else torch.float64, device=DEV)


def _from_stored(a, perm, dtype, rho0=1.0):
    s = a.view(9, -1).double().cpu().numpy()
    if dtype == mlbm.F32:
        _, _, om = oracle.d2q9()
        s = s + om[:, None] * rho0
    out = np.empty_like(s)
    out[:, perm] = s
    return out


@pytest.mark.parametrize("mode", ["own", "paper"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_no_interaction_is_the_plain_step(dtype, mode):
    """G = 0: the Shan-Chen step is the plain step bit for bit, under both stencil rules (the
    nearest-node rule with dx_ml = 2 h, departure points beyond the own stencil)."""
    dt = mlbm.F32 if dtype == "f32" else mlbm.F64
    xy = mi.jittered_lattice(32, 0.3, seed=31)
    _, w = _periodic(xy, 16, 3, (2.0 if mode == "paper" else 0.5) / 32, mode)
    params = [(0.8, 0.0, 1.0)]
    rho, u, v = mi.tgv_initial(xy, 0.02)
    td = torch.float32 if dt == mlbm.F32 else torch.float64
    a = torch.empty(9 * w.n, dtype=td, device=DEV)
    mlbm.init(w, params, dt, _t(rho), _t(u), _t(v), a)
    b, c = torch.empty_like(a), torch.empty_like(a)
    mb, mc = torch.empty(3 * w.n, dtype=td, device=DEV), torch.empty(3 * w.n, dtype=td, device=DEV)
    mlbm.step(w, params, dt, a, b, mb)
    mlbm.sc_step(w, params, (0.0, 1.0), dt, a, c, mc)
    assert torch.equal(b, c) and torch.equal(mb, mc)


@pytest.mark.parametrize("mode", ["own", "paper"])
@pytest.mark.parametrize("n_side,K,deg,steps", [(24, 16, 3, 20), (200, 12, 2, 4)])
def test_fp64_steps_match_the_oracle_step_by_step(n_side, K, deg, steps, mode):
    """Oracle shape vectors uploaded; the state after every step is the oracle's Shan-Chen
    post-collision state to 1e-12 relative, and the moments are those of the streamed state.
    24^2 nodes run one-warp tiles, 200^2 the 128-node tiles.  Under the nearest-node rule
    (dx_ml = 2 h) psi at each departure point is interpolated in its nearest node's stencil, as
    the oracle's paper mode does."""
    tau, G = 1.0, -5.0
    dx = (2.0 if mode == "paper" else 0.5) / n_side
    xy = mi.jittered_lattice(n_side, 0.3, seed=32)
    cloud, w = _periodic(xy, K, deg, dx, mode)
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode=mode)
    w.upload(W[1:], oracle.stencils(xy, K, box=(1.0, 1.0)).astype(np.int32))
    n = xy.shape[1]
    rng = np.random.default_rng(5)
    f = oracle.init_equilibrium(LN2 * (1 + 0.05 * rng.standard_normal(n)), np.zeros(n), np.zeros(n))
    perm = cloud.perm()
    a = _to_stored(oracle.sc_collide_field(f, sidx, W, tau, G), perm, mlbm.F64)
    b = torch.empty_like(a)
    mom = torch.empty(3 * n, dtype=torch.float64, device=DEV)
    st = oracle.ScStepper(sidx, W, tau, G)
    params = [(tau, 0.0, 1.0)]
    for it in range(steps):
        mlbm.sc_step(w, params, (G, 1.0), mlbm.F64, a, b, mom)
        a, b = b, a
        f = st.step(f)
        post = oracle.sc_collide_field(f, sidx, W, tau, G)
        got = _from_stored(a, perm, mlbm.F64)
        assert np.max(np.abs(got - post)) <= 1e-12 * np.max(np.abs(post)), it
        r = oracle.moments_field(f)[0]
        m = mom.view(3, -1).cpu().numpy()
        np.testing.assert_allclose(m[0][np.argsort(perm)], r, rtol=1e-12)


@pytest.mark.parametrize("mode", ["own", "paper"])
def test_fp32_follows_the_fp64_oracle(mode):
    n_side, K, deg, tau, G = 24, 16, 3, 1.0, -5.0
    dx = (2.0 if mode == "paper" else 0.5) / n_side
    xy = mi.jittered_lattice(n_side, 0.3, seed=33)
    cloud, w = _periodic(xy, K, deg, dx, mode)
    sidx, W = oracle.weights(xy, K, deg, dx, box=(1.0, 1.0), mode=mode)
    w.upload(W[1:], oracle.stencils(xy, K, box=(1.0, 1.0)).astype(np.int32))
    n = xy.shape[1]
    rng = np.random.default_rng(6)
    f = oracle.init_equilibrium(LN2 * (1 + 0.05 * rng.standard_normal(n)), np.zeros(n), np.zeros(n))
    perm = cloud.perm()
    a = _to_stored(oracle.sc_collide_field(f, sidx, W, tau, G), perm, mlbm.F32)
    b = torch.empty_like(a)
    st = oracle.ScStepper(sidx, W, tau, G)
    # G = -5 lies inside the spinodal region (G_c = -4): the density modes grow exponentially and
    # carry any rounding with them.  The expected size of FP32 rounding after 40 steps is that of
    # the FP64 oracle with FP32-sized noise, each stored deviation f - omega rho0 perturbed by up
    # to 2^-24 of itself every step; the FP32 step rounds several times per population per step
    # (interpolation, psi, force, collision, storage), so it may exceed that model by a small
    # factor: bound 10x the model's RMS over three noise realisations (measured about 6x).
    _, _, om = oracle.d2q9()
    rngs = [np.random.default_rng(99 + r) for r in range(3)]
    fns = [f.copy() for _ in rngs]
    for _ in range(40):
        mlbm.sc_step(w, [(tau, 0.0, 1.0)], (G, 1.0), mlbm.F32, a, b)
        a, b = b, a
        f = st.step(f)
        for r, rng_n in enumerate(rngs):
            fn = st.step(fns[r])
            fns[r] = fn + 2.0 ** -24 * np.abs(fn - om[:, None]) * rng_n.uniform(-1.0, 1.0, fn.shape)
    r_o = oracle.moments_field(f)[0]
    r_g = oracle.moments_field(_from_stored(a, perm, mlbm.F32))[0]
    dev = np.linalg.norm(r_o - r_o.mean())
    err = np.linalg.norm(r_g - r_o) / dev
    model = np.sqrt(np.mean([np.sum((oracle.moments_field(fn)[0] - r_o) ** 2) for fn in fns])) / dev
    assert err <= 10.0 * model, (err, model)
    assert err <= 1e-5, err


def test_lattice_cloud_is_the_lattice_shan_chen_step():
    """Nodes on a periodic lattice with dx_ml = h (GPU-built shape vectors): the meshless step is
    the index-shift Shan-Chen step."""
    n, tau, G = 32, 1.0, -5.5
    xy = mi.lattice(n)
    cloud, w = _periodic(xy, 9, 2, 1.0 / n)
    rng = np.random.default_rng(7)
    f = oracle.init_equilibrium(LN2 * (1 + 0.02 * rng.standard_normal(n * n)), np.zeros(n * n), np.zeros(n * n))
    sidx, W = oracle.weights(xy, 9, 2, 1.0 / n, box=(1.0, 1.0))
    perm = cloud.perm()
    a = _to_stored(oracle.sc_collide_field(f, sidx, W, tau, G), perm, mlbm.F64)
    b = torch.empty_like(a)
    for _ in range(30):
        mlbm.sc_step(w, [(tau, 0.0, 1.0)], (G, 1.0), mlbm.F64, a, b)
        a, b = b, a
        f = oracle.sc_lattice_step(f, n, n, tau, G)
    post = oracle.sc_collide_field(f, sidx, W, tau, G)
    assert np.max(np.abs(_from_stored(a, perm, mlbm.F64) - post)) <= 1e-10 * np.max(np.abs(post))


def _lattice_coexistence(G, tau):
    """Bulk densities of a flat liquid slab in its vapour on a 64 x 4 periodic lattice (oracle)."""
    nx, ny = 64, 4
    ix = np.tile(np.arange(nx), ny)
    f = oracle.init_equilibrium(np.where((ix >= 16) & (ix < 48), 2.0, 0.15), np.zeros(nx * ny), np.zeros(nx * ny))
    for _ in range(4000):
        f = oracle.sc_lattice_step(f, nx, ny, tau, G)
    rr = oracle.moments_field(f)[0]
    return rr[ix == 32].mean(), rr[ix == 0].mean()


_SLAB = dict(n=64, K=16, deg=3, tau=1.0, G=-5.5, steps=2000, seed=34)


@functools.lru_cache(maxsize=1)
def _slab_case():
    """A liquid slab (1/4 <= x < 3/4, tanh edges three spacings wide) in its vapour on a 64^2
    jittered cloud, and the oracle's meshless Shan-Chen run from it (shared by both precisions)."""
    c = _SLAB
    xy = mi.jittered_lattice(c["n"], 0.3, seed=c["seed"])
    sidx, W = oracle.weights(xy, c["K"], c["deg"], 1.0 / c["n"], box=(1.0, 1.0))
    x = xy[0]
    wd = 3.0 / c["n"]
    rho = 0.15 + (2.0 - 0.15) / 2 * (np.tanh((x - 0.25) / wd) - np.tanh((x - 0.75) / wd))
    zero = np.zeros_like(x)
    f0 = oracle.init_equilibrium(rho, zero, zero)
    st = oracle.ScStepper(sidx, W, c["tau"], c["G"])
    f = f0
    for _ in range(c["steps"]):
        f = st.step(f)
    return xy, sidx, W, rho, f0, oracle.moments_field(f)[0]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_flat_interfaces_reach_the_coexistence_densities(dtype):
    """Implementation: from the same state, the GPU's bulk densities after 2000 steps equal those
    of the oracle's meshless run on the same cloud (1e-8 FP64, 1e-4 FP32 relative).  Method: they
    are those of the model's flat interface on a lattice (about 2.30 and 0.104), the liquid
    within 2 %, the vapour, about 20 times less dense and so more sensitive to the interpolation
    of psi across the interface, within 4 % (2.5 % here); the meshless streaming does not
    conserve mass exactly, and across the steep interfaces about 1 % is lost (bound 2 %)."""
    c = _SLAB
    dt = mlbm.F32 if dtype == "f32" else mlbm.F64
    xy, sidx, W, rho, f0, r_o = _slab_case()
    cloud, w = _periodic(xy, c["K"], c["deg"], 1.0 / c["n"])
    w.upload(W[1:], oracle.stencils(xy, c["K"], box=(1.0, 1.0)).astype(np.int32))
    perm = cloud.perm()
    a = _to_stored(oracle.sc_collide_field(f0, sidx, W, c["tau"], c["G"]), perm, dt)
    b = torch.empty_like(a)
    params = [(c["tau"], 0.0, 1.0)]
    for _ in range(c["steps"]):
        mlbm.sc_step(w, params, (c["G"], 1.0), dt, a, b)
        a, b = b, a
    r = oracle.moments_field(_from_stored(a, perm, dt))[0]  # density of the level's streamed state
    x = xy[0]
    liquid = np.abs(x - 0.5) < 0.1
    vapour = np.minimum(x, 1 - x) < 0.1
    # the GPU state is post-collision; its density equals that of the oracle's pre-collision state
    tol = 1e-4 if dt == mlbm.F32 else 1e-8
    assert r[liquid].mean() == pytest.approx(r_o[liquid].mean(), rel=tol)
    assert r[vapour].mean() == pytest.approx(r_o[vapour].mean(), rel=tol)
    rl, rg = _lattice_coexistence(c["G"], c["tau"])
    assert r[liquid].mean() == pytest.approx(rl, rel=0.02), (r[liquid].mean(), rl)
    assert r[vapour].mean() == pytest.approx(rg, rel=0.04), (r[vapour].mean(), rg)
    assert abs(r.sum() - rho.sum()) <= 2e-2 * rho.sum()


def test_walls_are_refused():
    """Walls would need a value of psi beyond the wall (a wetting choice the method leaves
    open): a cloud with bounce-back nodes is refused."""
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    c = mlbm.build_cloud(xy, dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=12, degree=2, dx_ml=0.05))
    w = mlbm.build_weights(c)
    a = torch.zeros(9 * w.n, dtype=torch.float64, device=DEV)
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.sc_step(w, [(0.8, 0.0, 1.0)], (-5.0, 1.0), mlbm.F64, a, a.clone())
    assert e.value.code == mlbm.EINVAL


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mixed_stencil_rules_batched_equal_single_runs(dtype):
    """An own-rule and a nearest-rule segment in one weights object (one launch per pass over
    both): each segment's Shan-Chen steps equal its own single-segment run.  The nearest
    segment bit for bit; the own segment to rounding, because a build holding any nearest
    segment solves every segment through the departure-point table, whose offsets
    (x_i - e_k dx_ml) - x_i round differently from -e_k dx_ml (FP64 shape vectors equal to
    about 1e-16)."""
    dt = mlbm.F32 if dtype == "f32" else mlbm.F64
    td = torch.float32 if dt == mlbm.F32 else torch.float64
    parts = [mi.jittered_lattice(20, 0.3, seed=61), mi.jittered_lattice(16, 0.3, seed=62)]
    segs = [dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=12, degree=2, dx_ml=0.5 / 20),
            dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=16, degree=3, dx_ml=2.0 / 16,
                 stencil_mode=mlbm.STENCIL_NEAREST)]
    params = [(1.0, 0.0, 1.0), (0.9, 0.0, 1.0)]
    scp = [(-5.0, 1.0), (-4.5, 1.0)]
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    xy = np.concatenate(parts, axis=1)
    wb = mlbm.build_weights(mlbm.build_cloud(xy, segs, offs))
    rng = np.random.default_rng(63)
    rho = LN2 * (1 + 0.05 * rng.standard_normal(xy.shape[1]))
    zero = np.zeros(xy.shape[1])

    def run(w, prm, sc, r, n):
        a = torch.empty(9 * w.n, dtype=td, device=DEV)
        mlbm.init(w, prm, dt, _t(r), _t(zero[:n]), _t(zero[:n]), a)
        b = torch.empty_like(a)
        for _ in range(5):
            mlbm.sc_step(w, prm, sc, dt, a, b)
            a, b = b, a
        return a.view(9, -1)

    got = run(wb, params, scp, rho, xy.shape[1])
    for s in range(2):
        ws = mlbm.build_weights(mlbm.build_cloud(parts[s], segs[s]))
        ref = run(ws, [params[s]], [scp[s]], rho[offs[s]:offs[s + 1]], parts[s].shape[1])
        g = got[:, offs[s]:offs[s + 1]]
        if s == 1:
            assert torch.equal(g, ref)
        else:
            tol = 1e-13 if dt == mlbm.F64 else 1e-6
            assert float((g - ref).abs().max()) <= tol * float(ref.abs().max())
