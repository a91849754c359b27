"""FP64 CPU oracle of the meshless lattice Boltzmann method (arXiv 2306.01525).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2306_01525_gb300``) and never imports it; the GPU library never imports this.

The arithmetic lives in plain C (``mlbm_oracle.c``, double precision, scalar loops in the
paper's order).  This module builds and loads it and adds the closed-form solutions and error
norms the paper states:

* ``tgv_velocity``       Taylor-Green vortex, eq. (tgv_eqs) of Sec. 3
* ``tgv_end_time``       t_end = ln 10 / (2 nu k^2), Sec. 3
* ``annulus_velocity``   azimuthal profile of the forced annular channel, eq. (bch_solution)
* ``l2_norm``            normalised discrete error norm, eq. (L2norm)
* ``speed_rel_error``    pointwise relative speed error, eq. (vmag_error)
* ``residual``           relative velocity residual used as the steady-state stop, Sec. 3

and the Shan-Chen multiphase extension the paper's discussion names (``sc_psi``, ``sc_force``,
``ScStepper``, ``sc_lattice_step``; model of Shan & Chen 1993, readings as in the library).

Each function is checked against the paper and the mathematics in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

Q = 9


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fused multiply-add contraction, OpenMP over nodes)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            L.orc_feq.restype = d
            L.orc_feq.argtypes = [i32, d, d, d]
            L.orc_opposite.restype = i32
            L.orc_opposite.argtypes = [i32]
            L.orc_d2q9.argtypes = [vp, vp, vp]
            L.orc_moments.argtypes = [vp, vp, vp, vp]
            L.orc_collide.argtypes = [vp, d, d, d, vp]
            L.orc_knn.restype = i32
            L.orc_knn.argtypes = [vp, vp, i64, d, d, i32, d, d, vp]
            L.orc_build_stencils.restype = i32
            L.orc_build_stencils.argtypes = [vp, vp, i64, i32, d, d, vp]
            L.orc_num_monomials.restype = i32
            L.orc_num_monomials.argtypes = [i32, i32]
            L.orc_monomials.argtypes = [i32, i32, d, d, vp]
            L.orc_shape_vector.restype = i32
            L.orc_shape_vector.argtypes = [i32, i32, i32, vp, vp, d, d, vp]
            L.orc_build_weights.restype = i64
            L.orc_build_weights.argtypes = [vp, vp, i64, i32, i32, d, d, d, i32, vp, vp, vp]
            L.orc_node_weights.restype = i32
            L.orc_node_weights.argtypes = [vp, vp, i64, i64, i32, i32, d, d, d, i32, vp, vp]
            L.orc_azimuthal_force.argtypes = [vp, vp, i64, d, vp, vp]
            L.orc_bounce_mask.argtypes = [vp, vp, i64, d, d, d, vp]
            L.orc_init_equilibrium.argtypes = [i64, vp, vp, vp, vp]
            L.orc_step.argtypes = [i64, i32, vp, vp, vp, vp, vp, d, vp, vp, vp]
            L.orc_collide_field.argtypes = [i64, vp, vp, d, vp, vp]
            L.orc_moments_field.argtypes = [i64, vp, vp, vp, vp]
            L.orc_lattice_step.argtypes = [i32, i32, d, vp, vp, vp]
            L.orc_sc_psi.restype = d
            L.orc_sc_psi.argtypes = [d, d]
            L.orc_sc_force.argtypes = [i64, i32, vp, vp, vp, d, vp, vp]
            L.orc_sc_step.argtypes = [i64, i32, vp, vp, vp, vp, d, d, d, vp, vp, vp]
            L.orc_sc_lattice_step.argtypes = [i32, i32, d, d, d, vp, vp, vp]
            L.orc_sc_collide_field.argtypes = [i64, i32, vp, vp, d, d, d, vp, vp, vp]
            L.orc_num_threads.restype = i32
            L.orc_set_threads.argtypes = [i32]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- D2Q9 (Sec. 2.1)

def d2q9():
    """(ex, ey, omega) as stored in the oracle."""
    ex = np.zeros(Q, np.int32)
    ey = np.zeros(Q, np.int32)
    om = np.zeros(Q, np.float64)
    lib().orc_d2q9(_p(ex), _p(ey), _p(om))
    return ex, ey, om


def opposite(k: int) -> int:
    return int(lib().orc_opposite(k))


def feq(k: int, rho: float, ux: float, uy: float) -> float:
    """Equilibrium population k, eq. (feq)."""
    return float(lib().orc_feq(k, rho, ux, uy))


def moments(f):
    """(rho, ux, uy) of nine populations, eq. (macro_var)."""
    f = _f64(f)
    out = np.zeros(3)
    lib().orc_moments(_p(f), _p(out[0:1]), _p(out[1:2]), _p(out[2:3]))
    return float(out[0]), float(out[1]), float(out[2])


def collide(f, tau: float, gx: float = 0.0, gy: float = 0.0):
    """BGK collision with the body-force term of Sec. 3, one node."""
    f = _f64(f)
    out = np.zeros(Q)
    lib().orc_collide(_p(f), tau, gx, gy, _p(out))
    return out


# ----------------------------------------------------------------------------- stencils, weights

def knn(xy, q, K: int, box=(0.0, 0.0)):
    """K nodes nearest to point q by (squared distance, index); min-image if box > 0."""
    x, y = _f64(xy[0]), _f64(xy[1])
    out = np.zeros(K, np.int64)
    rc = lib().orc_knn(_p(x), _p(y), x.size, float(q[0]), float(q[1]), K, box[0], box[1], _p(out))
    if rc != 0:
        raise ValueError("K larger than the number of nodes")
    return out


def stencils(xy, K: int, box=(0.0, 0.0)):
    """Own K-NN stencil of every node, [K][n] int64 (centre first)."""
    x, y = _f64(xy[0]), _f64(xy[1])
    n = x.size
    st = np.zeros((K, n), np.int64)
    rc = lib().orc_build_stencils(_p(x), _p(y), n, K, box[0], box[1], _p(st))
    if rc != 0:
        raise ValueError("K larger than the number of nodes")
    return st


def num_monomials(dim: int, deg: int) -> int:
    return int(lib().orc_num_monomials(dim, deg))


def monomials(dim: int, deg: int, x: float, y: float = 0.0):
    out = np.zeros(num_monomials(dim, deg))
    lib().orc_monomials(dim, deg, x, y, _p(out))
    return out


def shape_vector(px, py, q, deg: int, dim: int = 2):
    """Shape vector w_L(q) of eq. (shape_vector); coordinates relative to the stencil centre."""
    px = _f64(px)
    py = _f64(py) if py is not None else np.zeros_like(px)
    K = px.size
    w = np.zeros(K)
    rc = lib().orc_shape_vector(dim, K, deg, _p(px), _p(py), float(q[0]),
                                float(q[1]) if len(q) > 1 else 0.0, _p(w))
    if rc == -1:
        raise np.linalg.LinAlgError("singular collocation matrix")
    if rc != 0:
        raise ValueError("bad stencil / degree")
    return w


def weights(xy, K: int, deg: int, dx_ml: float, box=(0.0, 0.0), mode: str = "own",
            stencil=None):
    """Per-direction stencil indices and shape vectors, both [9][K][n] (Sec. 2.3).

    mode "own": every direction uses the node's own K-NN stencil; mode "paper": the stencil of
    the Eulerian node nearest to the departure point (appendix algorithm)."""
    x, y = _f64(xy[0]), _f64(xy[1])
    n = x.size
    st = stencils(xy, K, box) if stencil is None else np.ascontiguousarray(stencil, np.int64)
    sidx = np.zeros((Q, K, n), np.int64)
    W = np.zeros((Q, K, n), np.float64)
    nbad = -lib().orc_build_weights(_p(x), _p(y), n, K, deg, dx_ml, box[0], box[1],
                                    1 if mode == "paper" else 0, _p(st), _p(sidx), _p(W))
    if nbad:
        raise np.linalg.LinAlgError(f"{nbad} singular collocation systems")
    return sidx, W


def node_weights(xy, i: int, K: int, deg: int, dx_ml: float, box=(0.0, 0.0), mode="own"):
    """Stencil indices and shape vectors of node i alone, both [9][K], by brute force."""
    x, y = _f64(xy[0]), _f64(xy[1])
    sidx = np.zeros((Q, K), np.int64)
    W = np.zeros((Q, K), np.float64)
    nbad = lib().orc_node_weights(_p(x), _p(y), x.size, int(i), K, deg, dx_ml, box[0], box[1],
                                  1 if mode == "paper" else 0, _p(sidx), _p(W))
    if nbad:
        raise np.linalg.LinAlgError(f"{nbad} singular collocation systems at node {i}")
    return sidx, W


def azimuthal_force(xy, g: float):
    x, y = _f64(xy[0]), _f64(xy[1])
    gx, gy = np.zeros_like(x), np.zeros_like(x)
    lib().orc_azimuthal_force(_p(x), _p(y), x.size, g, _p(gx), _p(gy))
    return gx, gy


def bounce_mask(xy, dx_ml: float, r_in: float, r_out: float):
    x, y = _f64(xy[0]), _f64(xy[1])
    m = np.zeros(x.size, np.uint16)
    lib().orc_bounce_mask(_p(x), _p(y), x.size, dx_ml, r_in, r_out, _p(m))
    return m


# ----------------------------------------------------------------------------- time loop

def init_equilibrium(rho, ux, uy):
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    n = rho.size
    f = np.zeros((Q, n))
    lib().orc_init_equilibrium(n, _p(rho), _p(ux), _p(uy), _p(f))
    return f


class Stepper:
    """Repeated oracle steps on one cloud (COLLIDE then STREAM, then bounce-back)."""

    def __init__(self, sidx, W, tau: float, mask=None, force=None):
        self.sidx = np.ascontiguousarray(sidx, np.int64)
        self.W = _f64(W)
        self.K = self.W.shape[1]
        self.n = self.W.shape[2]
        self.tau = float(tau)
        self.mask = None if mask is None else np.ascontiguousarray(mask, np.uint16)
        self.gx = None if force is None else _f64(force[0])
        self.gy = None if force is None else _f64(force[1])
        self._scratch = np.zeros((Q, self.n))

    def step(self, f):
        f = _f64(f)
        out = np.zeros_like(f)
        lib().orc_step(self.n, self.K, _p(self.sidx), _p(self.W), _p(self.mask), _p(self.gx),
                       _p(self.gy), self.tau, _p(f), _p(out), _p(self._scratch))
        return out

    def run(self, f, nsteps: int):
        for _ in range(nsteps):
            f = self.step(f)
        return f


def collide_field(f, tau: float, force=None):
    f = _f64(f)
    n = f.shape[1]
    out = np.zeros_like(f)
    gx = None if force is None else _f64(force[0])
    gy = None if force is None else _f64(force[1])
    lib().orc_collide_field(n, _p(gx), _p(gy), tau, _p(f), _p(out))
    return out


def moments_field(f):
    f = _f64(f)
    n = f.shape[1]
    rho, ux, uy = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_moments_field(n, _p(f), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


def lattice_step(f, nx: int, ny: int, tau: float):
    """Standard LBM step with index-shift streaming, eq. (LBM_streaming)."""
    f = _f64(f)
    out = np.zeros_like(f)
    scratch = np.zeros_like(f)
    lib().orc_lattice_step(nx, ny, tau, _p(f), _p(out), _p(scratch))
    return out


# ----------------------------------------------------------------------------- Shan-Chen

def sc_psi(rho, rho0: float = 1.0):
    """Shan-Chen pseudopotential psi(rho) = rho0 (1 - exp(-rho / rho0)) (Shan & Chen 1993)."""
    r = np.atleast_1d(_f64(rho))
    out = np.array([lib().orc_sc_psi(float(v), float(rho0)) for v in r])
    return out if np.ndim(rho) else float(out[0])


def sc_force(sidx, W, psi, G: float):
    """Interaction force F_i = -G psi_i sum_k omega_k psi(x_i + e_k dx_ml) e_k, psi at
    x_i + e_k dx_ml interpolated with the shape vector of the opposite direction."""
    sidx = np.ascontiguousarray(sidx, np.int64)
    W = _f64(W)
    K, n = W.shape[1], W.shape[2]
    fx, fy = np.zeros(n), np.zeros(n)
    lib().orc_sc_force(n, K, _p(sidx), _p(W), _p(_f64(psi)), float(G), _p(fx), _p(fy))
    return fx, fy


class ScStepper(Stepper):
    """Shan-Chen steps on a cloud without walls: psi of the current density, interaction force,
    then the collide-and-stream step with that force (plus an optional body force)."""

    def __init__(self, sidx, W, tau: float, G: float, rho0: float = 1.0, force=None):
        super().__init__(sidx, W, tau, mask=None, force=force)
        self.G = float(G)
        self.rho0 = float(rho0)
        self._sc_scratch = np.zeros((Q + 3) * self.n)

    def step(self, f):
        f = _f64(f)
        out = np.zeros_like(f)
        lib().orc_sc_step(self.n, self.K, _p(self.sidx), _p(self.W), _p(self.gx), _p(self.gy),
                          self.tau, self.G, self.rho0, _p(f), _p(out), _p(self._sc_scratch))
        return out


def sc_collide_field(f, sidx, W, tau: float, G: float, rho0: float = 1.0):
    """Shan-Chen collision of a whole field (no streaming): the post-collision state of the
    same level, the form in which the GPU library holds its state."""
    f = _f64(f)
    sidx = np.ascontiguousarray(sidx, np.int64)
    W = _f64(W)
    n = f.shape[1]
    out = np.zeros_like(f)
    scratch = np.zeros(3 * n)
    lib().orc_sc_collide_field(n, W.shape[1], _p(sidx), _p(W), float(tau), float(G), float(rho0),
                               _p(f), _p(out), _p(scratch))
    return out


def sc_lattice_step(f, nx: int, ny: int, tau: float, G: float, rho0: float = 1.0):
    """Shan-Chen step on a periodic nx x ny lattice: psi(x + e_k) at the neighbouring node,
    index-shift streaming."""
    f = _f64(f)
    out = np.zeros_like(f)
    scratch = np.zeros((Q + 3) * f.shape[1])
    lib().orc_sc_lattice_step(nx, ny, float(tau), float(G), float(rho0), _p(f), _p(out), _p(scratch))
    return out


def set_threads(t: int):
    lib().orc_set_threads(int(t))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------------- closed forms

def tgv_velocity(x, y, t, u0=1.0, nu=1.0, L=1.0):
    """Taylor-Green vortex, eq. (tgv_eqs): k = 2 pi / L (L = 1 in the paper)."""
    k = 2.0 * np.pi / L
    decay = np.exp(-2.0 * nu * k * k * t)
    u = u0 * np.cos(k * x) * np.sin(k * y) * decay
    v = -u0 * np.sin(k * x) * np.cos(k * y) * decay
    return u, v


def tgv_end_time(nu=1.0, L=1.0):
    """Time at which the vortex has decayed to 10 % of its amplitude, Sec. 3."""
    k = 2.0 * np.pi / L
    return np.log(10.0) / (2.0 * nu * k * k)


def lattice_viscosity(tau):
    """nu = c_s^2 (tau - 1/2) in lattice units (the reading of the Sec. 2.1 relation that
    reproduces nu = 1 for tau = 0.8, dx = 1/10, dt = 1e-3 of Sec. 3)."""
    return (tau - 0.5) / 3.0


def annulus_velocity(r, g, nu, r1, r2):
    """Azimuthal velocity of force-driven flow between two circles, eq. (bch_solution)."""
    G = g / (3.0 * nu)
    alpha = (r1 * r1 + r1 * r2 + r2 * r2) / (r1 + r2)
    beta = r1 * r1 * r2 * r2 / (r1 + r2)
    return -G * (r * r - alpha * r + beta / r)


def l2_norm(u, u_true):
    """Normalised discrete L2 error, eq. (L2norm)."""
    u = np.asarray(u, np.float64)
    u_true = np.asarray(u_true, np.float64)
    return float(np.sqrt(np.sum((u - u_true) ** 2)) / np.sqrt(np.sum(u_true ** 2)))


def speed_rel_error(u, v, u_true, v_true):
    """Pointwise relative error of the velocity magnitude, eq. (vmag_error)."""
    s = np.sqrt(np.asarray(u) ** 2 + np.asarray(v) ** 2)
    st = np.sqrt(np.asarray(u_true) ** 2 + np.asarray(v_true) ** 2)
    return np.abs(s - st) / st


def residual(u_new, v_new, u_old, v_old):
    """Relative velocity residual between consecutive steps (steady-state stop, Sec. 3)."""
    num = np.sum((u_new - u_old) ** 2 + (v_new - v_old) ** 2)
    den = np.sum(u_new ** 2 + v_new ** 2)
    return float(np.sqrt(num / den))
