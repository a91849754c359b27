"""Host-buffer steps (mlbm_step_host): a batch of independent states in host memory is copied
in, stepped and copied back with the copies of neighbouring states overlapping the steps; every
result must equal the device step of the same state bit for bit (Sec. 2.3, Sec. 3)."""
import numpy as np
import pytest

import mlbm_inputs as mi

torch = pytest.importorskip("torch")
mlbm = pytest.importorskip("paper_2306_01525_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _setup(n_side=40, K=16, deg=3):
    xy = mi.jittered_lattice(n_side, 0.3, seed=21)
    seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=K, degree=deg, dx_ml=1.0 / n_side)
    w = mlbm.build_weights(mlbm.build_cloud(xy, seg))
    return xy, w


def _states(xy, w, dtype, nb):
    td = torch.float32 if dtype == mlbm.F32 else torch.float64
    out = []
    for b in range(nb):
        rho, u, v = mi.tgv_initial(xy, 0.01 * (b + 1))
        f = torch.empty(9 * w.n, dtype=td, device=DEV)
        t = lambda x: torch.as_tensor(x, dtype=torch.float64, device=DEV)
        mlbm.init(w, [(0.8, 0.0, 1.0)], dtype, t(rho), t(u), t(v), f)
        out.append(f)
    return out


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_batch_of_host_states_equals_device_steps(dtype, pinned):
    dt = mlbm.F32 if dtype == "f32" else mlbm.F64
    xy, w = _setup()
    params = [(0.8, 0.0, 1.0)]
    dev_states = _states(xy, w, dt, 5)
    ins = [s.cpu().pin_memory() if pinned else s.cpu() for s in dev_states]
    outs = [torch.empty_like(t) for t in ins]
    mlbm.step_host(w, params, dt, ins, outs)
    for s, o in zip(dev_states, outs):
        ref = torch.empty_like(s)
        mlbm.step(w, params, dt, s, ref)
        assert torch.equal(ref.cpu(), o)


def test_in_place_and_repeated_calls():
    xy, w = _setup()
    params = [(0.7, 0.0, 1.0)]
    s = _states(xy, w, mlbm.F32, 3)
    host = [t.cpu().pin_memory() for t in s]
    for _ in range(3):  # three steps of each state, results written over the inputs
        mlbm.step_host(w, params, mlbm.F32, host, host)
    for d, h in zip(s, host):
        a, b = d.clone(), torch.empty_like(d)
        r = mlbm.run(w, params, mlbm.F32, a, b, 3)
        assert torch.equal(r.cpu(), h)


def test_argument_errors():
    xy, w = _setup(16, 9, 2)
    good = torch.zeros(9 * w.n, dtype=torch.float32)
    with pytest.raises(ValueError):
        mlbm.step_host(w, [(0.8, 0.0, 1.0)], mlbm.F32, [good.double()], [good])
    with pytest.raises(ValueError):
        mlbm.step_host(w, [(0.8, 0.0, 1.0)], mlbm.F32, [good.cuda()], [good])
    with pytest.raises(ValueError):
        mlbm.step_host(w, [(0.8, 0.0, 1.0)], mlbm.F32, [], [])
    with pytest.raises(mlbm.MLBMError):
        mlbm.step_host(w, [(0.4, 0.0, 1.0)], mlbm.F32, [good], [good])  # tau <= 1/2
