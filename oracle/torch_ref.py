"""FP64 torch-CPU restatement of the oracle's time loop, for autograd reference gradients.

TEST INFRASTRUCTURE ONLY (part of the oracle): the same collide-then-stream step as
``mlbm_oracle.c`` (Sec. 2.1 eq. feq and eq. LBM_collision with the Sec. 3 forcing term,
Sec. 2.3 semi-Lagrangian streaming with per-direction stencils and shape vectors, Sec. 3 wall
bounce-back), written with differentiable torch operations on the CPU in float64, so that
``torch.autograd`` gives the exact gradient of a loss with respect to tau, the force magnitude
g and the initial macroscopic fields.  Its forward pass is pinned to the C oracle and its
gradients to central finite differences of the C oracle (tests/test_oracle_adjoint_pins.py).
"""
from __future__ import annotations

import torch

_EX = torch.tensor([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=torch.float64)
_EY = torch.tensor([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=torch.float64)
_OM = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=torch.float64)
_OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def feq(rho, ux, uy):
    """eq. (feq) for all nine directions: [9][n]."""
    cu = _EX[:, None] * ux + _EY[:, None] * uy
    uu = ux * ux + uy * uy
    return _OM[:, None] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


def moments(f):
    """eq. (macro_var) summed over all nine populations."""
    rho = f.sum(0)
    return rho, (f * _EX[:, None]).sum(0) / rho, (f * _EY[:, None]).sum(0) / rho


def collide(f, tau, gx, gy):
    """eq. (LBM_collision) plus omega_k e_k.g / c_s^2 (Sec. 3)."""
    rho, ux, uy = moments(f)
    force = 3.0 * _OM[:, None] * (_EX[:, None] * gx + _EY[:, None] * gy)
    return f - (f - feq(rho, ux, uy)) / tau + force


def stream(fp, sidx, W, mask_bits):
    """Semi-Lagrangian streaming (Sec. 2.3), then bounce-back of unknown populations (Sec. 3).

    sidx, W: [9][K][n]; mask_bits: [9][n] bool (True where population k is unknown)."""
    fs = torch.stack([(W[k] * fp[k][sidx[k]]).sum(0) for k in range(9)])
    if mask_bits is None:
        return fs
    opp = fs[_OPP]
    return torch.where(mask_bits, opp, fs)


def rollout(sidx, W, tau, g, force_dir, mask, rho0, ux0, uy0, nsteps):
    """Macroscopic fields after nsteps steps from f = f^eq(rho0, u0).

    force_dir: (dx, dy) node arrays of the unit force direction (or None); mask: uint16 bit masks
    per node (or None)."""
    sidx = torch.as_tensor(sidx, dtype=torch.int64)
    W = torch.as_tensor(W, dtype=torch.float64)
    if mask is not None:
        m = torch.as_tensor(mask.astype("int64"))
        bits = torch.stack([(m >> k) & 1 for k in range(9)]).bool()
    else:
        bits = None
    if force_dir is None:
        gx = gy = torch.zeros((), dtype=torch.float64)
    else:
        gx = g * torch.as_tensor(force_dir[0], dtype=torch.float64)
        gy = g * torch.as_tensor(force_dir[1], dtype=torch.float64)
    f = feq(rho0, ux0, uy0)
    for _ in range(nsteps):
        f = stream(collide(f, tau, gx, gy), sidx, W, bits)
    return moments(f)
