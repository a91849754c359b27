"""C-ABI checks that need no GPU: the library loads and exports every function the header
declares, and the host-side stencil build (mlbm_build_cloud) agrees with the oracle's brute
force; argument errors come back as status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import mlbm_inputs as mi
import oracle
import paper_2306_01525_gb300 as mlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mlbm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = _declared_functions()
    assert len(names) >= 15
    L = mlbm.lib()
    for nm in names:
        assert hasattr(L, nm), nm
        assert ctypes.cast(getattr(L, nm), ctypes.c_void_p).value


def test_abi_version():
    assert mlbm.lib().mlbm_abi_version() == 6


def _periodic(k, deg, dx):
    return dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=k, degree=deg, dx_ml=dx)


@pytest.mark.parametrize("n_side,k", [(32, 12), (20, 30), (13, 9)])
def test_periodic_stencils_match_oracle(n_side, k):
    xy = mi.jittered_lattice(n_side, 0.3, seed=n_side)
    c = mlbm.build_cloud(xy, _periodic(k, 2, 1.0 / n_side))
    np.testing.assert_array_equal(c.stencil(0), oracle.stencils(xy, k, box=(1.0, 1.0)))


def test_lattice_ties_match_oracle():
    xy = mi.lattice(16)
    c = mlbm.build_cloud(xy, _periodic(12, 2, 1.0 / 16))
    np.testing.assert_array_equal(c.stencil(0), oracle.stencils(xy, 12, box=(1.0, 1.0)))


def test_annulus_stencils_and_mask_match_oracle():
    xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[2000], seed=4)
    dx = 1.0 / 160
    seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=20, degree=3, dx_ml=dx)
    c = mlbm.build_cloud(xy, seg)
    np.testing.assert_array_equal(c.stencil(0), oracle.stencils(xy, 20))
    np.testing.assert_array_equal(c.bounce_mask(), oracle.bounce_mask(xy, dx, 0.5, 1.0))


def test_permutation_is_morton_and_bijective():
    xy = mi.jittered_lattice(64, 0.3, seed=9)
    c = mlbm.build_cloud(xy, _periodic(12, 2, 1.0 / 64))
    p = c.perm()
    assert np.array_equal(np.sort(p), np.arange(xy.shape[1]))
    # consecutive stored nodes are spatially close (locality of the Z-curve)
    d = np.hypot(*(xy[:, p[1:]] - xy[:, p[:-1]]))
    assert np.median(d) < 2.0 / 64


def test_batched_segments_each_match_oracle():
    parts, segs = [], []
    for s, (n_side, k, deg) in enumerate([(8, 9, 2), (12, 16, 3), (5, 6, 1)]):
        parts.append(mi.jittered_lattice(n_side, 0.3, seed=50 + s))
        segs.append(_periodic(k, deg, 0.5 / n_side))
    offs = np.cumsum([0] + [p.shape[1] for p in parts])
    c = mlbm.build_cloud(np.concatenate(parts, axis=1), segs, offs)
    for s, p in enumerate(parts):
        np.testing.assert_array_equal(c.stencil(s), oracle.stencils(p, segs[s]["k"], box=(1.0, 1.0)))
    perm = c.perm()
    for s in range(3):
        blk = perm[offs[s]:offs[s + 1]]
        assert blk.min() == offs[s] and blk.max() == offs[s + 1] - 1


@pytest.mark.parametrize("bad", [
    dict(k=200),                       # stencil larger than the limit / segment
    dict(k=5, degree=2),               # fewer nodes than monomials
    dict(degree=9),                    # degree above the supported maximum
    dict(dx_ml=0.0),
    dict(lx=0.0),
    dict(geometry=7),
])
def test_bad_descriptors_rejected(bad):
    xy = mi.jittered_lattice(8, 0.3, seed=1)
    seg = _periodic(9, 2, 0.1)
    seg.update(bad)
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_cloud(xy, seg)
    assert e.value.code == mlbm.EINVAL


def test_bad_offsets_rejected():
    xy = mi.jittered_lattice(8, 0.3, seed=1)
    with pytest.raises(mlbm.MLBMError):
        mlbm.build_cloud(xy, [_periodic(9, 2, 0.1)] * 2, [0, 10, 60])
    with pytest.raises(mlbm.MLBMError):
        mlbm.build_cloud(xy, [_periodic(9, 2, 0.1)] * 2, [0, 0, 64])


def test_non_finite_coordinates_rejected():
    xy = mi.jittered_lattice(8, 0.3, seed=1)
    xy[0, 3] = np.nan
    with pytest.raises(mlbm.MLBMError):
        mlbm.build_cloud(xy, _periodic(9, 2, 0.1))


def test_weights_without_gpu_fail_loudly():
    """No CPU fallback: without a CUDA device the GPU entry points return MLBM_ECUDA."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    xy = mi.jittered_lattice(8, 0.3, seed=1)
    c = mlbm.build_cloud(xy, _periodic(9, 2, 0.1))
    h = ctypes.c_void_p()
    rc = mlbm.lib().mlbm_build_weights(c.handle, 0, None, ctypes.byref(h), None)
    assert rc == mlbm.ECUDA
    assert not h.value


def test_device_cloud_build_without_gpu_fails_loudly():
    """The device stencil build checks its arguments like the host build, and without a CUDA
    device returns MLBM_ECUDA (no host fallback)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    xy = mi.jittered_lattice(8, 0.3, seed=1)
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_cloud(xy, _periodic(0, 2, 0.1), device=True, stream=_NullStream())
    assert e.value.code == mlbm.EINVAL
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_cloud(xy, _periodic(9, 2, 0.1), device=True, stream=_NullStream())
    assert e.value.code == mlbm.ECUDA


class _NullStream:
    cuda_stream = 0


@pytest.mark.parametrize("geometry", ["periodic", "annulus"])
def test_departure_nodes_match_oracle_nearest_rule(geometry):
    """Nearest-node stencil mode: the node whose stencil interpolates population k of node i is
    the node nearest to x_i - e_k dx_ml (Sec. 2.3), as the oracle's paper mode finds it."""
    if geometry == "periodic":
        xy = mi.jittered_lattice(20, 0.3, seed=2)
        seg = dict(geometry=mlbm.PERIODIC, lx=1.0, ly=1.0, k=16, degree=3, dx_ml=0.1,
                   stencil_mode=mlbm.STENCIL_NEAREST)
        box = (1.0, 1.0)
    else:
        xy, _ = mi.annulus_cloud(h=mi.ANNULUS_H_FOR[2000], seed=4)
        seg = dict(geometry=mlbm.ANNULUS, r_in=0.5, r_out=1.0, k=15, degree=2, dx_ml=0.05,
                   stencil_mode=mlbm.STENCIL_NEAREST)
        box = (0.0, 0.0)
    c = mlbm.build_cloud(xy, seg)
    sidx, _ = oracle.weights(xy, seg["k"], seg["degree"], seg["dx_ml"], box=box, mode="paper")
    np.testing.assert_array_equal(c.departure_nodes(0), sidx[1:, 0, :])
    own = mlbm.build_cloud(xy, dict(seg, stencil_mode=mlbm.STENCIL_OWN))
    assert np.all(own.departure_nodes(0) == np.arange(xy.shape[1])[None, :])


def test_empty_cloud_rejected():
    """A cloud without nodes has no stencils: the build refuses it instead of returning an
    empty object."""
    with pytest.raises(mlbm.MLBMError) as e:
        mlbm.build_cloud(np.zeros((2, 0)), _periodic(9, 2, 0.1))
    assert e.value.code == mlbm.EINVAL
