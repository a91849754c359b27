"""Parity on the batched convergence sweep itself: the 64 Taylor-Green runs of uneven size,
stencil, degree and streaming distance as segments of one cloud, one step for all of them in
one launch.  Small runs are compared whole with the oracle (oracle shape vectors uploaded, so
the FP64 step must agree to 1e-12); the 512^2 runs on sampled nodes that the oracle computes
one by one with its own shape vectors."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_sweep_one_step_parity():
    runs = mi.sweep_runs()
    parts, segs, params, us, vs = [], [], [], [], []
    for r in runs:
        xy = mi.jittered_lattice(r["n_side"], 0.3, seed=r["seed"])
        parts.append(xy)
        segs.append(dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=r["K"], degree=r["degree"],
                         dx_ml=r["ratio"] / r["n_side"]))
        params.append((r["tau"], 0.0, 1.0))
        _, u, v = mi.tgv_initial(xy, r["u0"])
        us.append(u)
        vs.append(v)
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    cloud = mlbm.build_cloud(np.concatenate(parts, axis=1), segs, offs)
    w = mlbm.build_weights(cloud)
    assert w.n_bad == 0
    small = [i for i, r in enumerate(runs) if r["n_side"] <= 32]
    oracle_w = {}
    for i in small:
        r = runs[i]
        sidx, W = oracle.weights(parts[i], r["K"], r["degree"], segs[i]["dx_ml"], box=(1.0, 1.0))
        w.upload(W[1:], sidx[1].astype(np.int32), seg=i)
        oracle_w[i] = (sidx, W)
    N = w.n
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)
    a = torch.empty(9 * N, dtype=torch.float64, device=DEV)
    b = torch.empty_like(a)
    mom = torch.empty(3 * N, dtype=torch.float64, device=DEV)
    mlbm.init(w, params, mlbm.F64, t(np.ones(N)), t(np.concatenate(us)), t(np.concatenate(vs)), a)
    mlbm.step(w, params, mlbm.F64, a, b, mom)
    perm = cloud.perm()
    m = np.empty((3, N))
    m[:, perm] = mom.view(3, N).cpu().numpy()
    for i in small:
        sidx, W = oracle_w[i]
        f = oracle.Stepper(sidx, W, params[i][0]).step(
            oracle.init_equilibrium(np.ones(parts[i].shape[1]), us[i], vs[i]))
        r_o, u_o, v_o = oracle.moments_field(f)
        sl = slice(offs[i], offs[i + 1])
        np.testing.assert_allclose(m[1, sl], u_o, rtol=0, atol=1e-14)
        np.testing.assert_allclose(m[2, sl], v_o, rtol=0, atol=1e-14)
        np.testing.assert_allclose(m[0, sl], r_o, rtol=1e-13)
    rng = np.random.default_rng(23)
    for i in [i for i, r in enumerate(runs) if r["n_side"] == 512]:
        r = runs[i]
        for node in rng.choice(parts[i].shape[1], 6, replace=False):
            sidx, W = oracle.node_weights(parts[i], int(node), r["K"], r["degree"], segs[i]["dx_ml"], box=(1.0, 1.0))
            mem = np.unique(sidx)
            pos = {q: t_ for t_, q in enumerate(mem)}
            post = oracle.collide_field(oracle.init_equilibrium(np.ones(mem.size), us[i][mem], vs[i][mem]), r["tau"])
            f1 = [sum(W[k, j] * post[k, pos[sidx[k, j]]] for j in range(r["K"])) for k in range(9)]
            ro, uo, vo = oracle.moments(np.array(f1))
            g = offs[i] + node
            assert abs(m[1, g] - uo) < 1e-9 and abs(m[2, g] - vo) < 1e-9, (i, node)
