"""The adjoint workload at full size, in the launch configuration the benchmark times: an annulus
of about 250k scattered nodes (r in [0.5, 1], refined toward the walls, seed 5), N_L = 24, P_3,
dx_ml = 1/320, tau = 0.7, g = 1e-5, one reverse step from the forward's next state, under the
own-node and the nearest-node rule (Sec. 2.3).  The reference is the oracle's torch restatement
of the same step (streaming with the per-direction stencils and shape vectors, wall
bounce-back, then the BGK collision with the forcing term, FP64 on the CPU) differentiated by
autograd, with the library's FP64 shape vectors and stencils, so that it checks the reverse
kernels on every node; the FP32 reverse step is checked against the FP64 one at FP32 accuracy."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")
from oracle import torch_ref  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
K, DEG, DX, TAU, G = 24, 3, 1.0 / 320, 0.7, 1e-5


@pytest.fixture(scope="module")
def annulus_250k():
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[250000], seed=5)
    mask = oracle.bounce_mask(xy, DX, 0.5, 1.0)
    fdir = oracle.azimuthal_force(xy, 1.0)
    return xy, mask, fdir


def _weights(xy, rule):
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=K, degree=DEG, dx_ml=DX,
               stencil_mode=rule)
    cloud = mlbm.build_cloud(xy, seg, device=True)
    w = mlbm.build_weights(cloud)
    assert w.n_bad == 0
    return cloud, w


def _oracle_layout(cloud, w, rule):
    """sidx, W as the oracle's streaming takes them: [9][K][n], original node order; direction 0
    is the node's own value (centre member, weight 1)."""
    n = w.n
    st = cloud.stencil(0).astype(np.int64)  # [K][n], original numbering, centre first
    W64 = w.download()                       # [8][K][n]
    sidx = np.empty((9, K, n), np.int64)
    sidx[0] = st
    if rule == mlbm.STENCIL_NEAREST:
        dep = cloud.departure_nodes(0)       # [8][n]: node whose stencil interpolates (i, k)
        for k in range(8):
            sidx[k + 1] = st[:, dep[k]]
    else:
        sidx[1:] = st[None]
    W = np.zeros((9, K, n))
    W[0, 0] = 1.0
    W[1:] = W64
    return torch.as_tensor(sidx), torch.as_tensor(W)


def _to_orig(a_stored, perm):
    """[9][n] in the library's stored order -> original node order."""
    a = a_stored.reshape(9, -1)
    out = np.empty_like(a)
    out[:, perm] = a
    return out


def _reference(s_orig, lam_orig, sidx, W, mask, fdir):
    """J^T lam, d<lam, F(s)>/dtau and d<lam, F(s)>/dg for F = collide(stream(s)) (autograd)."""
    bits = torch.stack([(torch.as_tensor(mask.astype(np.int64)) >> k) & 1 for k in range(9)]).bool()
    s = torch.tensor(s_orig, dtype=torch.float64, requires_grad=True)
    tt = torch.tensor(TAU, dtype=torch.float64, requires_grad=True)
    gg = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    fx = torch.as_tensor(fdir[0], dtype=torch.float64)
    fy = torch.as_tensor(fdir[1], dtype=torch.float64)
    out = torch_ref.collide(torch_ref.stream(s, sidx, W, bits), tt, gg * fx, gg * fy)
    (out * torch.as_tensor(lam_orig)).sum().backward()
    return s.grad.numpy(), tt.grad.item(), gg.grad.item()


@pytest.mark.parametrize("rule", ["own", "nearest"])
def test_full_size_reverse_step_matches_oracle_autograd(annulus_250k, rule):
    xy, mask, fdir = annulus_250k
    code = mlbm.STENCIL_OWN if rule == "own" else mlbm.STENCIL_NEAREST
    cloud, w = _weights(xy, code)
    n = w.n
    perm = cloud.perm()
    params = [(TAU, G, 1.0)]
    rng = np.random.default_rng(51)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)
    fields = [t(1 + 1e-3 * rng.standard_normal(n)), t(3e-3 * rng.standard_normal(n)),
              t(3e-3 * rng.standard_normal(n))]
    pert = t(1e-4 * rng.standard_normal(9 * n))
    lam = t(rng.standard_normal(9 * n))
    out = {}
    for dt, td in ((mlbm.F64, torch.float64), (mlbm.F32, torch.float32)):
        # the same physical state in each storage form (FP32: deviations from omega_k rho0)
        s = torch.empty(9 * n, dtype=td, device=DEV)
        mlbm.init(w, params, dt, *fields, s)
        s += pert.to(td)
        sn = torch.empty_like(s)
        mlbm.step(w, params, dt, s, sn)
        lp = torch.empty_like(s)
        g = torch.zeros(2, dtype=torch.float64, device=DEV)
        mlbm.adjoint_step(w, params, dt, s, lam.to(td), lp, g, s_next=sn)
        torch.cuda.synchronize()
        out[dt] = (lp.double().cpu().numpy(), g.cpu().numpy())
        if dt == mlbm.F64:
            s64 = s.cpu().numpy()
    # FP64 reverse step against the oracle's autograd of the same step
    sidx, W = _oracle_layout(cloud, w, code)
    ref, dtau, dg = _reference(_to_orig(s64, perm), _to_orig(lam.cpu().numpy(), perm), sidx, W, mask, fdir)
    got = _to_orig(out[mlbm.F64][0], perm)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    assert out[mlbm.F64][1][0] == pytest.approx(dtau, rel=1e-9)
    assert out[mlbm.F64][1][1] == pytest.approx(dg, rel=1e-9)
    # FP32 reverse step (the kernel the benchmark times under the own-node rule) against it
    a, b = out[mlbm.F64][0], out[mlbm.F32][0]
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    np.testing.assert_allclose(out[mlbm.F32][1], out[mlbm.F64][1], rtol=1e-4)
