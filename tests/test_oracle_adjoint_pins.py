"""Pins of the oracle's autograd reference (oracle.torch_ref): its forward equals the C oracle,
and its gradients equal central finite differences of the C oracle, under both stencil rules
(the nearest-node rule with its per-direction stencils, Sec. 2.3)."""
import numpy as np
import pytest

import mlbm_inputs as mi
import oracle

torch = pytest.importorskip("torch")
from oracle import torch_ref  # noqa: E402


def _annulus_case(steps=30, mode="own"):
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[1000], seed=3)
    dx = 1.0 / 40 if mode == "own" else 1.0 / 20
    sidx, W = oracle.weights(xy, 15, 2, dx, mode=mode)
    if mode == "paper":  # departure points interpolated outside the node's own stencil
        assert np.any(sidx[1:, 0, :] != np.arange(xy.shape[1])[None, :])
    mask = oracle.bounce_mask(xy, dx, 0.5, 1.0)
    fdir = oracle.azimuthal_force(xy, 1.0)
    n = xy.shape[1]
    rng = np.random.default_rng(1)
    rho0 = 1.0 + 1e-3 * rng.standard_normal(n)
    u0 = 2e-3 * rng.standard_normal(n)
    v0 = 2e-3 * rng.standard_normal(n)
    return xy, sidx, W, mask, fdir, rho0, u0, v0, steps


def _c_rollout(sidx, W, tau, g, fdir, mask, rho0, u0, v0, steps):
    force = (g * fdir[0], g * fdir[1])
    st = oracle.Stepper(sidx, W, tau, mask=mask, force=force)
    f = st.run(oracle.init_equilibrium(rho0, u0, v0), steps)
    return oracle.moments_field(f)


def _loss(r, u, v, target):
    return ((u - target[0]) ** 2 + (v - target[1]) ** 2).sum() + ((r - 1.0) ** 2).sum()


@pytest.mark.parametrize("mode", ["own", "paper"])
def test_torch_forward_equals_c_oracle(mode):
    xy, sidx, W, mask, fdir, rho0, u0, v0, steps = _annulus_case(mode=mode)
    tau, g = 0.9, 3e-5
    want = _c_rollout(sidx, W, tau, g, fdir, mask, rho0, u0, v0, steps)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64)
    got = torch_ref.rollout(sidx, W, t(tau), t(g), fdir, mask, t(rho0), t(u0), t(v0), steps)
    for a, b in zip(got, want):
        np.testing.assert_allclose(a.numpy(), b, rtol=0, atol=1e-13)


@pytest.mark.parametrize("mode", ["own", "paper"])
def test_torch_gradients_equal_c_oracle_finite_differences(mode):
    xy, sidx, W, mask, fdir, rho0, u0, v0, steps = _annulus_case(20, mode)
    tau, g = 0.9, 3e-5
    rng = np.random.default_rng(2)
    target = (1e-3 * rng.standard_normal(u0.size), 1e-3 * rng.standard_normal(u0.size))
    T = lambda a, rg=False: torch.tensor(a, dtype=torch.float64, requires_grad=rg)
    tt, gt, r0, a0, b0 = T(tau, True), T(g, True), T(rho0, True), T(u0, True), T(v0, True)
    L = _loss(*torch_ref.rollout(sidx, W, tt, gt, fdir, mask, r0, a0, b0, steps),
              (torch.as_tensor(target[0]), torch.as_tensor(target[1])))
    L.backward()

    def c_loss(tau_, g_, rho_, u_, v_):
        r, u, v = _c_rollout(sidx, W, tau_, g_, fdir, mask, rho_, u_, v_, steps)
        return float(np.sum((u - target[0]) ** 2 + (v - target[1]) ** 2) + np.sum((r - 1.0) ** 2))

    h = 1e-6
    fd_tau = (c_loss(tau + h, g, rho0, u0, v0) - c_loss(tau - h, g, rho0, u0, v0)) / (2 * h)
    assert tt.grad.item() == pytest.approx(fd_tau, rel=1e-5)
    hg = 1e-6
    fd_g = (c_loss(tau, g + hg, rho0, u0, v0) - c_loss(tau, g - hg, rho0, u0, v0)) / (2 * hg)
    assert gt.grad.item() == pytest.approx(fd_g, rel=1e-5)
    d = rng.standard_normal(u0.size)
    hu = 1e-6
    fd_u = (c_loss(tau, g, rho0, u0 + hu * d, v0) - c_loss(tau, g, rho0, u0 - hu * d, v0)) / (2 * hu)
    assert float(a0.grad.numpy() @ d) == pytest.approx(fd_u, rel=1e-5)
