"""GB300 meshless lattice Boltzmann method (arXiv 2306.01525): Python binding.

Thin ctypes layer over the C ABI declared in ``include/mlbm.h``.  Every function here only
marshals arguments (torch tensors -> device pointers, the current CUDA stream -> ``void*``);
every step of the method runs in the native library's CUDA kernels.  There is no CPU
fallback: without the compiled library or a CUDA device the calls raise.

Names follow the C ABI without the ``mlbm_`` prefix:

    build_cloud -> Cloud          stencil build, host or device=True GPU (Sec. 2.2, 2.3, Sec. 3)
    build_weights -> Weights      batched FP64 shape-vector solve on the GPU (Sec. 2.2-2.3)
    init, step, run               initial state and the fused pull-stream-collide step
    moments, norms                macroscopic fields (eq. macro_var), eq. (L2norm) sums
    adjoint_step, moments_adjoint, init_adjoint   reverse mode of the above
    sc_step                       Shan-Chen multiphase step (extension named in the discussion)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "MLBMError", "F32", "F64", "PERIODIC", "ANNULUS", "STENCIL_OWN", "STENCIL_NEAREST",
    "KEEP_W32", "KEEP_W64",
    "lib", "Cloud", "Weights", "build_cloud", "build_weights", "init", "step", "run",
    "run_until", "moments", "norms", "norms_noalloc", "fp64_fma_rate", "adjoint_step", "moments_adjoint", "init_adjoint",
    "lattice_init", "lattice_step", "step_host", "sc_step",
]

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ETIMEOUT = 0, -1, -2, -3, -4, -5
PERIODIC, ANNULUS = 0, 1
STENCIL_OWN, STENCIL_NEAREST = 0, 1
F32, F64 = 32, 64
KEEP_W32, KEEP_W64 = 1, 2

_c_int, _c_i64, _c_d, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class SegmentDesc(ctypes.Structure):
    _fields_ = [("geometry", _c_int), ("lx", _c_d), ("ly", _c_d), ("r_in", _c_d),
                ("r_out", _c_d), ("k", _c_int), ("degree", _c_int), ("dx_ml", _c_d),
                ("stencil_mode", _c_int)]


class Params(ctypes.Structure):
    _fields_ = [("tau", _c_d), ("g", _c_d), ("rho0", _c_d)]


class ScParams(ctypes.Structure):
    _fields_ = [("G", _c_d), ("rho_psi", _c_d)]


class MLBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mlbm error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded native library (compiled in-tree on first use if stale)."""
    global _lib
    with _lock:
        if _lib is None:
            import torch  # noqa: F401  (loads the CUDA runtime the library links against)

            path = _build.build()
            L = ctypes.CDLL(path)
            L.mlbm_last_error.restype = ctypes.c_char_p
            L.mlbm_abi_version.restype = _c_int
            L.mlbm_build_cloud.argtypes = [_vp, _c_i64, _vp, _vp, _c_int, ctypes.POINTER(_vp)]
            L.mlbm_build_cloud_device.argtypes = [_vp, _c_i64, _vp, _vp, _c_int, _vp, ctypes.POINTER(_vp)]
            L.mlbm_cloud_free.argtypes = [_vp]
            L.mlbm_cloud_free.restype = None
            L.mlbm_cloud_size.argtypes = [_vp]
            L.mlbm_cloud_size.restype = _c_i64
            L.mlbm_cloud_perm.argtypes = [_vp, _vp]
            L.mlbm_cloud_stencil.argtypes = [_vp, _c_int, _vp]
            L.mlbm_cloud_bounce_mask.argtypes = [_vp, _vp]
            L.mlbm_cloud_departure_nodes.argtypes = [_vp, _c_int, _vp]
            L.mlbm_build_weights.argtypes = [_vp, _c_int, _vp, ctypes.POINTER(_vp), _vp]
            L.mlbm_weights_free.argtypes = [_vp]
            L.mlbm_weights_free.restype = None
            L.mlbm_weights_info.argtypes = [_vp, _vp, _vp]
            L.mlbm_weights_download.argtypes = [_vp, _c_int, _vp]
            L.mlbm_weights_download_f32.argtypes = [_vp, _c_int, _vp]
            L.mlbm_weights_upload.argtypes = [_vp, _c_int, _vp, _vp]
            L.mlbm_init.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp]
            L.mlbm_step.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp]
            L.mlbm_run.argtypes = [_vp, _vp, _c_int, _vp, _vp, _c_i64, _vp]
            L.mlbm_run_until.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp]
            L.mlbm_step_host.argtypes = [_vp, _vp, _c_int, _c_i64, _vp, _vp, _vp]
            L.mlbm_sc_step.argtypes = [_vp, _vp, _vp, _c_int, _vp, _vp, _vp, _vp]
            L.mlbm_moments.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp]
            L.mlbm_norms.argtypes = [_vp, _vp, _vp, _vp, _vp, _c_i64, _vp, _vp]
            L.mlbm_norms_noalloc.argtypes = [_vp, _vp, _vp, _vp, _c_i64, _vp, _vp]
            L.mlbm_lattice_init.argtypes = [_c_i64, _c_i64, _vp, _c_int, _vp, _vp, _vp, _vp, _vp]
            L.mlbm_lattice_step.argtypes = [_c_i64, _c_i64, _vp, _c_int, _vp, _vp, _vp, _vp]
            L.mlbm_adjoint_step.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp]
            L.mlbm_moments_adjoint.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.mlbm_init_adjoint.argtypes = [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                            _vp, _vp]
            L.mlbm_fp64_fma_rate.argtypes = [_c_i64, _c_int, _vp, _c_i64, _vp, _vp]
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise MLBMError(rc, lib().mlbm_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


def _dev_ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return _vp(t.data_ptr())


def _torch_dtype(dtype):
    import torch

    if dtype == F32:
        return torch.float32
    if dtype == F64:
        return torch.float64
    raise ValueError("dtype must be F32 or F64")


def _params(params, nseg):
    if isinstance(params, (tuple, list)) and params and isinstance(params[0], (int, float)):
        params = [params]
    if isinstance(params, dict):
        params = [params]
    if len(params) != nseg:
        raise ValueError(f"need {nseg} parameter sets, got {len(params)}")
    arr = (Params * nseg)()
    for s, p in enumerate(params):
        if isinstance(p, dict):
            arr[s] = Params(float(p["tau"]), float(p.get("g", 0.0)), float(p.get("rho0", 1.0)))
        else:
            vals = list(p) + [None, 0.0, 1.0][len(p):]
            arr[s] = Params(float(vals[0]), float(vals[1]), float(vals[2]))
    return arr


# ----------------------------------------------------------------------------- cloud

class Cloud:
    """Library-owned node cloud (mlbm_build_cloud, or mlbm_build_cloud_device when device=True:
    the same cloud, built by kernels on the current CUDA device)."""

    def __init__(self, xy, segments, offsets=None, device=False, stream=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        if xy.ndim != 2 or xy.shape[0] != 2:
            raise ValueError("xy must have shape (2, n)")
        n = xy.shape[1]
        if isinstance(segments, dict):
            segments = [segments]
        nseg = len(segments)
        if offsets is None:
            if nseg != 1:
                raise ValueError("offsets needed for several segments")
            offsets = [0, n]
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        descs = (SegmentDesc * nseg)()
        for s, d in enumerate(segments):
            descs[s] = SegmentDesc(int(d.get("geometry", PERIODIC)), float(d.get("lx", 0.0)),
                                   float(d.get("ly", 0.0)), float(d.get("r_in", 0.0)),
                                   float(d.get("r_out", 0.0)), int(d["k"]), int(d["degree"]),
                                   float(d["dx_ml"]), int(d.get("stencil_mode", STENCIL_OWN)))
        h = _vp()
        if device:
            _check(lib().mlbm_build_cloud_device(xy.ctypes.data, n, descs, offs.ctypes.data, nseg,
                                                 _stream(stream), ctypes.byref(h)))
        else:
            _check(lib().mlbm_build_cloud(xy.ctypes.data, n, descs, offs.ctypes.data, nseg,
                                          ctypes.byref(h)))
        self._h = h
        self.n = n
        self.nseg = nseg
        self.segments = [dict(d) for d in segments]
        self.offsets = offs.copy()

    @property
    def handle(self):
        return self._h

    def perm(self):
        out = np.zeros(self.n, np.int64)
        _check(lib().mlbm_cloud_perm(self._h, out.ctypes.data))
        return out

    def stencil(self, seg=0):
        ns = int(self.offsets[seg + 1] - self.offsets[seg])
        out = np.zeros((int(self.segments[seg]["k"]), ns), np.int32)
        _check(lib().mlbm_cloud_stencil(self._h, seg, out.ctypes.data))
        return out

    def departure_nodes(self, seg=0):
        """[8][n_seg] int32: the node whose stencil interpolates population k = 1..8 of node i
        (original numbering relative to the segment)."""
        ns = int(self.offsets[seg + 1] - self.offsets[seg])
        out = np.zeros((8, ns), np.int32)
        _check(lib().mlbm_cloud_departure_nodes(self._h, seg, out.ctypes.data))
        return out

    def bounce_mask(self):
        out = np.zeros(self.n, np.uint16)
        _check(lib().mlbm_cloud_bounce_mask(self._h, out.ctypes.data))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.mlbm_cloud_free(h)
            self._h = None


def build_cloud(xy, segments, offsets=None, device=False, stream=None) -> Cloud:
    """Stencil build of a node cloud: on the host, or with device=True on the GPU (identical
    result)."""
    return Cloud(xy, segments, offsets, device=device, stream=stream)


# ----------------------------------------------------------------------------- weights

class Weights:
    """Library-owned device weights object (mlbm_build_weights)."""

    def __init__(self, cloud: Cloud, keep=KEEP_W32 | KEEP_W64, stream=None, check=True):
        h = _vp()
        nbad = ctypes.c_int64(0)
        rc = lib().mlbm_build_weights(cloud.handle, int(keep), _stream(stream), ctypes.byref(h),
                                      ctypes.byref(nbad))
        self._h = h if h.value else None
        self.n_bad = int(nbad.value)
        if rc != OK and not (rc == ESINGULAR and not check and self._h is not None):
            _check(rc)
        self.n = cloud.n
        self.nseg = cloud.nseg
        self.segments = cloud.segments
        self.offsets = cloud.offsets
        self.keep = keep

    @property
    def handle(self):
        return self._h

    def download(self, seg=0):
        """FP64 shape vectors of segment seg, [8][K][n_seg], original order."""
        ns = int(self.offsets[seg + 1] - self.offsets[seg])
        K = int(self.segments[seg]["k"])
        out = np.zeros((8, K, ns), np.float64)
        _check(lib().mlbm_weights_download(self._h, seg, out.ctypes.data))
        return out

    def download_f32(self, seg=0):
        """FP32 shape vectors the FP32 step uses (rounded to keep the polynomial reproduction),
        [8][K][n_seg] float32, original order."""
        ns = int(self.offsets[seg + 1] - self.offsets[seg])
        K = int(self.segments[seg]["k"])
        out = np.zeros((8, K, ns), np.float32)
        _check(lib().mlbm_weights_download_f32(self._h, seg, out.ctypes.data))
        return out

    def upload(self, W, idx, seg=0):
        """Replace segment seg's shape vectors ([8][K][n_seg] FP64, original order); idx must
        equal the library's stencil ([K][n_seg] int32, original numbering)."""
        W = np.ascontiguousarray(W, np.float64)
        idx = np.ascontiguousarray(idx, np.int32)
        _check(lib().mlbm_weights_upload(self._h, seg, W.ctypes.data, idx.ctypes.data))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.mlbm_weights_free(h)
            self._h = None


def build_weights(cloud: Cloud, keep=KEEP_W32 | KEEP_W64, stream=None, check=True) -> Weights:
    return Weights(cloud, keep, stream, check)


# ----------------------------------------------------------------------------- time stepping

def _state(w, dtype, t, name):
    return _dev_ptr(t, _torch_dtype(dtype), 9 * w.n, name)


def init(w: Weights, params, dtype, rho, ux, uy, f_out, stream=None):
    import torch

    _check(lib().mlbm_init(w.handle, _params(params, w.nseg), dtype,
                           _dev_ptr(rho, torch.float64, w.n, "rho"),
                           _dev_ptr(ux, torch.float64, w.n, "ux"),
                           _dev_ptr(uy, torch.float64, w.n, "uy"),
                           _state(w, dtype, f_out, "f_out"), _stream(stream)))


def step(w: Weights, params, dtype, f_in, f_out, moments_out=None, stream=None):
    mom = None if moments_out is None else _dev_ptr(moments_out, _torch_dtype(dtype), 3 * w.n,
                                                    "moments")
    _check(lib().mlbm_step(w.handle, _params(params, w.nseg), dtype,
                           _state(w, dtype, f_in, "f_in"), _state(w, dtype, f_out, "f_out"),
                           mom, _stream(stream)))


def _sc_params(sc, nseg):
    if isinstance(sc, (tuple, list)) and sc and isinstance(sc[0], (int, float)):
        sc = [sc]
    if len(sc) != nseg:
        raise ValueError(f"need {nseg} Shan-Chen parameter pairs, got {len(sc)}")
    arr = (ScParams * nseg)()
    for s, p in enumerate(sc):
        g, rp = (p["G"], p.get("rho_psi", 1.0)) if isinstance(p, dict) else (p[0], p[1] if len(p) > 1 else 1.0)
        arr[s] = ScParams(float(g), float(rp))
    return arr


def sc_step(w: Weights, params, sc, dtype, f_in, f_out, moments_out=None, stream=None):
    """One Shan-Chen multiphase step (mlbm_sc_step): streaming, psi of the streamed density,
    interaction force from psi interpolated at x + e_k dx_ml, collision towards the shifted
    equilibrium.  sc: per segment (G, rho_psi)."""
    mom = None if moments_out is None else _dev_ptr(moments_out, _torch_dtype(dtype), 3 * w.n, "moments")
    _check(lib().mlbm_sc_step(w.handle, _params(params, w.nseg), _sc_params(sc, w.nseg), dtype,
                              _state(w, dtype, f_in, "f_in"), _state(w, dtype, f_out, "f_out"), mom,
                              _stream(stream)))


def _host_state(w, dtype, t, name):
    import torch

    want = _torch_dtype(dtype)
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != want or t.numel() != 9 * w.n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {want} tensor of 9 * N elements")
    return t.data_ptr()


def step_host(w: Weights, params, dtype, f_in, f_out, stream=None):
    """One step for each of a batch of independent states in HOST memory (lists of CPU tensors,
    ideally pinned): copies in, fused step, copies out, pipelined across the batch
    (mlbm_step_host).  Returns when the results are in f_out."""
    if len(f_in) != len(f_out) or not f_in:
        raise ValueError("f_in and f_out must be non-empty lists of the same length")
    nb = len(f_in)
    ins = (_vp * nb)(*[_host_state(w, dtype, t, "f_in") for t in f_in])
    outs = (_vp * nb)(*[_host_state(w, dtype, t, "f_out") for t in f_out])
    _check(lib().mlbm_step_host(w.handle, _params(params, w.nseg), dtype, nb, ins, outs, _stream(stream)))


def run(w: Weights, params, dtype, f_a, f_b, nsteps: int, stream=None):
    """nsteps steps ping-ponging f_a -> f_b -> f_a ...; returns the tensor holding the result."""
    _check(lib().mlbm_run(w.handle, _params(params, w.nseg), dtype,
                          _state(w, dtype, f_a, "f_a"), _state(w, dtype, f_b, "f_b"),
                          int(nsteps), _stream(stream)))
    return f_a if nsteps % 2 == 0 else f_b


def run_until(w: Weights, params, dtype, f_a, f_b, seg_steps, stream=None):
    """Every segment after its own number of steps seg_steps[s]; returns the tensor holding
    the result (f_a when max(seg_steps) is even, else f_b; the other one is scratch)."""
    steps = np.ascontiguousarray(np.asarray(seg_steps, dtype=np.int64).reshape(-1))
    if steps.size != w.nseg:
        raise ValueError(f"seg_steps needs {w.nseg} entries")
    _check(lib().mlbm_run_until(w.handle, _params(params, w.nseg), dtype,
                                _state(w, dtype, f_a, "f_a"), _state(w, dtype, f_b, "f_b"),
                                steps.ctypes.data, _stream(stream)))
    return f_a if int(steps.max(initial=0)) % 2 == 0 else f_b


def moments(w: Weights, params, dtype, f, rho=None, ux=None, uy=None, stream=None):
    """(rho, ux, uy) FP64 in original order of the level whose post-collision state is f."""
    import torch

    dev = f.device
    rho = torch.empty(w.n, dtype=torch.float64, device=dev) if rho is None else rho
    ux = torch.empty(w.n, dtype=torch.float64, device=dev) if ux is None else ux
    uy = torch.empty(w.n, dtype=torch.float64, device=dev) if uy is None else uy
    _check(lib().mlbm_moments(w.handle, _params(params, w.nseg), dtype,
                              _state(w, dtype, f, "f"),
                              _dev_ptr(rho, torch.float64, w.n, "rho"),
                              _dev_ptr(ux, torch.float64, w.n, "ux"),
                              _dev_ptr(uy, torch.float64, w.n, "uy"), _stream(stream)))
    return rho, ux, uy


def norms(w: Weights, a, b, c=None, d=None, stream=None):
    """[sum (a-b)^2 + (c-d)^2, sum b^2 + d^2, sum a^2 + c^2] reduced on the device."""
    import torch

    n = a.numel()
    out = np.zeros(3, np.float64)
    _check(lib().mlbm_norms(w.handle, _dev_ptr(a, torch.float64, n, "a"),
                            _dev_ptr(b, torch.float64, n, "b"),
                            _dev_ptr(c, torch.float64, n, "c") if c is not None else None,
                            _dev_ptr(d, torch.float64, n, "d") if d is not None else None,
                            n, out.ctypes.data, _stream(stream)))
    return out


def norms_noalloc(a, b, c=None, d=None, out=None, stream=None):
    """The sums of ``norms`` into the device tensor ``out`` (3 float64) without any memory
    allocation in the library (for callers that cannot allocate device memory; n is limited to
    16,777,216 and overlapping calls race, see mlbm_norms_noalloc in include/mlbm.h)."""
    import torch

    n = a.numel()
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=a.device)
    _check(lib().mlbm_norms_noalloc(_dev_ptr(a, torch.float64, n, "a"),
                                    _dev_ptr(b, torch.float64, n, "b"),
                                    _dev_ptr(c, torch.float64, n, "c") if c is not None else None,
                                    _dev_ptr(d, torch.float64, n, "d") if d is not None else None,
                                    n, _dev_ptr(out, torch.float64, 3, "out"), _stream(stream)))
    return out


def fp64_fma_rate(iters: int, blocks_per_sm: int, sink, stream=None) -> float:
    """Enqueue the FP64 FMA rate probe (mlbm_fp64_fma_rate); returns the flops it performs.
    ``sink`` is a float64 device tensor of at least blocks_per_sm * SMs elements."""
    import torch

    flops = ctypes.c_double(0.0)
    _check(lib().mlbm_fp64_fma_rate(int(iters), int(blocks_per_sm),
                                    _dev_ptr(sink, torch.float64, sink.numel(), "sink"),
                                    sink.numel(), _stream(stream), ctypes.byref(flops)))
    return flops.value


# ----------------------------------------------------------------------------- lattice LBM

def lattice_init(nx: int, ny: int, params, dtype, rho, ux, uy, f_out, stream=None):
    """Equilibrium initial state of the standard lattice LBM (node index iy * nx + ix)."""
    import torch

    n = nx * ny
    _check(lib().mlbm_lattice_init(nx, ny, _params(params, 1), dtype,
                                   _dev_ptr(rho, torch.float64, n, "rho"),
                                   _dev_ptr(ux, torch.float64, n, "ux"),
                                   _dev_ptr(uy, torch.float64, n, "uy"),
                                   _dev_ptr(f_out, _torch_dtype(dtype), 9 * n, "f_out"),
                                   _stream(stream)))


def lattice_step(nx: int, ny: int, params, dtype, f_in, f_out, moments_out=None, stream=None):
    """One standard lattice LBM step (index-shift streaming, eq. LBM_streaming)."""
    n = nx * ny
    td = _torch_dtype(dtype)
    _check(lib().mlbm_lattice_step(nx, ny, _params(params, 1), dtype,
                                   _dev_ptr(f_in, td, 9 * n, "f_in"), _dev_ptr(f_out, td, 9 * n, "f_out"),
                                   _dev_ptr(moments_out, td, 3 * n, "moments") if moments_out is not None else None,
                                   _stream(stream)))


# ----------------------------------------------------------------------------- adjoint

def adjoint_step(w: Weights, params, dtype, s_prev, lam_next, lam_prev, grad, stream=None,
                 s_next=None):
    """lam_prev = dL/ds^n from lam_next = dL/ds^{n+1}; adds dL/dtau, dL/dg to grad.  s_next,
    the forward's output Step(s_prev), is optional: with it the library takes the interpolated
    populations' moments from it instead of recomputing the interpolation."""
    import torch

    _check(lib().mlbm_adjoint_step(w.handle, _params(params, w.nseg), dtype,
                                   _state(w, dtype, s_prev, "s_prev"),
                                   _state(w, dtype, s_next, "s_next") if s_next is not None else None,
                                   _state(w, dtype, lam_next, "lam_next"),
                                   _state(w, dtype, lam_prev, "lam_prev"),
                                   _dev_ptr(grad, torch.float64, 2 * w.nseg, "grad"),
                                   _stream(stream)))


def moments_adjoint(w: Weights, params, dtype, f, drho, dux, duy, lam, grad, stream=None):
    import torch

    _check(lib().mlbm_moments_adjoint(w.handle, _params(params, w.nseg), dtype,
                                      _state(w, dtype, f, "f"),
                                      _dev_ptr(drho, torch.float64, w.n, "drho"),
                                      _dev_ptr(dux, torch.float64, w.n, "dux"),
                                      _dev_ptr(duy, torch.float64, w.n, "duy"),
                                      _state(w, dtype, lam, "lam"),
                                      _dev_ptr(grad, torch.float64, 2 * w.nseg, "grad"),
                                      _stream(stream)))


def init_adjoint(w: Weights, params, dtype, rho, ux, uy, lam0, drho, dux, duy, grad,
                 stream=None):
    import torch

    _check(lib().mlbm_init_adjoint(w.handle, _params(params, w.nseg), dtype,
                                   _dev_ptr(rho, torch.float64, w.n, "rho"),
                                   _dev_ptr(ux, torch.float64, w.n, "ux"),
                                   _dev_ptr(uy, torch.float64, w.n, "uy"),
                                   _state(w, dtype, lam0, "lam0"),
                                   _dev_ptr(drho, torch.float64, w.n, "drho"),
                                   _dev_ptr(dux, torch.float64, w.n, "dux"),
                                   _dev_ptr(duy, torch.float64, w.n, "duy"),
                                   _dev_ptr(grad, torch.float64, 2 * w.nseg, "grad"),
                                   _stream(stream)))
