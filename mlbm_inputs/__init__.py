"""Seeded synthetic inputs for the meshless LBM workloads (arXiv 2306.01525).

This module holds no arithmetic of the method itself: it only generates node clouds and the
initial macroscopic fields of the two benchmark problems, so that the GPU library and the CPU
oracle can be fed the same inputs.  Both may import it; it imports neither.

The paper's clouds come from the Medusa Poisson-disk generator plus relaxation (Sec. 3), which
is not available here.  They are stood in for by:

* ``jittered_lattice``  -- the periodic unit square, an n x n lattice of cell centres jittered
  uniformly by +-jitter*h per coordinate (Taylor-Green workloads);
* ``lattice``           -- the same without jitter (lattice-reduction checks);
* ``annulus_cloud``     -- a ring r_in <= r <= r_out: wall nodes placed exactly on both circles
  and interior nodes from variable-radius Poisson-disk dart throwing (random sequential
  addition in a seeded priority order), spacing refined toward the walls.
"""
from __future__ import annotations

import numpy as np

__all__ = ["lattice", "jittered_lattice", "annulus_cloud", "tgv_initial", "sweep_runs",
           "ANNULUS_H_FOR"]


def lattice(n_side: int, L: float = 1.0):
    """Cell-centred n_side x n_side lattice on [0, L)^2; node index = iy * n_side + ix.

    Returns xy with shape (2, n_side**2), float64."""
    h = L / n_side
    iy, ix = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    x = (ix.ravel() + 0.5) * h
    y = (iy.ravel() + 0.5) * h
    return np.stack([x, y]).astype(np.float64)


def jittered_lattice(n_side: int, jitter: float = 0.3, seed: int = 1, L: float = 1.0):
    """Lattice of ``lattice`` with each coordinate moved by U(-jitter, jitter) * h, wrapped
    back into [0, L)."""
    xy = lattice(n_side, L)
    h = L / n_side
    rng = np.random.default_rng(seed)
    xy = xy + rng.uniform(-jitter, jitter, size=xy.shape) * h
    return np.mod(xy, L)


def _luby_select(pts, radius_a, radius_b_fn, prio):
    """Greedy maximal independent set in decreasing priority order (dart throwing with
    fixed dart order).  Two points conflict when closer than the mean of their radii."""
    from scipy.spatial import cKDTree

    rad = radius_a
    tree = cKDTree(pts.T)
    pairs = tree.query_pairs(r=float(rad.max()), output_type="ndarray")
    a, b = pairs[:, 0], pairs[:, 1]
    d2 = np.sum((pts[:, a] - pts[:, b]) ** 2, axis=0)
    lim = radius_b_fn(rad[a], rad[b])
    keep = d2 < lim * lim
    a, b = a[keep], b[keep]
    n = pts.shape[1]
    state = np.zeros(n, np.int8)  # 0 undecided, 1 selected, -1 rejected
    while True:
        und = state == 0
        if not und.any():
            break
        e = und[a] & und[b]
        ea, eb = a[e], b[e]
        local_max = und.copy()
        lower = np.where(prio[ea] < prio[eb], ea, eb)
        local_max[lower] = False
        state[local_max] = 1
        sel = local_max
        nb = np.concatenate([eb[sel[ea]], ea[sel[eb]]])
        nb = nb[state[nb] == 0]
        state[nb] = -1
    return state == 1


# Poisson-disk spacing h giving roughly the node counts of the annulus workloads
ANNULUS_H_FOR = {1000: 0.0512, 2000: 0.0356, 20000: 0.0108, 250000: 0.003007}


def annulus_cloud(r_in: float = 0.5, r_out: float = 1.0, h: float = 0.0108, seed: int = 2,
                  wall_ratio: float = 0.6, refine_width: float = 0.2, oversample: float = 6.0,
                  conflict: float = 0.85):
    """Scattered cloud in the ring r_in <= r <= r_out.

    Local spacing s(r) = h * (wall_ratio + (1 - wall_ratio) * clip(d_wall / (refine_width *
    (r_out - r_in)), 0, 1)).  Wall nodes sit exactly on both circles with spacing
    wall_ratio * h and a seeded phase; interior darts are drawn uniformly (rejection from the
    bounding square, thinned to density ~ 1 / s^2) and accepted in a seeded priority order
    unless closer than conflict * mean(s) to an accepted node.  Interior nodes keep at least
    0.5 * s_wall from both circles.

    Returns (xy (2, n) float64, is_wall (n,) bool)."""
    rng = np.random.default_rng(seed)
    width = r_out - r_in
    s_wall = h * wall_ratio

    def spacing(r):
        dw = np.minimum(r - r_in, r_out - r)
        t = np.clip(dw / (refine_width * width), 0.0, 1.0)
        return h * (wall_ratio + (1.0 - wall_ratio) * t)

    walls = []
    for R in (r_in, r_out):
        m = int(np.ceil(2.0 * np.pi * R / s_wall))
        th = 2.0 * np.pi * (np.arange(m) + rng.uniform()) / m
        walls.append(np.stack([R * np.cos(th), R * np.sin(th)]))
    wall = np.concatenate(walls, axis=1)

    area_sq = (2.0 * r_out) ** 2
    n_cand = int(oversample * area_sq / (s_wall * s_wall))
    c = rng.uniform(-r_out, r_out, size=(2, n_cand))
    r = np.sqrt(c[0] * c[0] + c[1] * c[1])
    inside = (r >= r_in + 0.5 * s_wall) & (r <= r_out - 0.5 * s_wall)
    c, r = c[:, inside], r[inside]
    thin = rng.uniform(size=r.size) < (s_wall / spacing(r)) ** 2
    c, r = c[:, thin], r[thin]

    pts = np.concatenate([wall, c], axis=1)
    rad = np.concatenate([np.full(wall.shape[1], s_wall), spacing(r)])
    prio = np.concatenate([np.full(wall.shape[1], 2.0) + np.arange(wall.shape[1]) * 1e-9,
                           rng.uniform(size=r.size)])
    sel = _luby_select(pts, conflict * rad, lambda ra, rb: 0.5 * (ra + rb), prio)
    is_wall = np.zeros(pts.shape[1], bool)
    is_wall[: wall.shape[1]] = True
    return pts[:, sel].astype(np.float64), is_wall[sel]


def tgv_initial(xy, u0: float = 0.01, rho0: float = 1.0, L: float = 1.0):
    """Initial macroscopic fields of the Taylor-Green vortex (Sec. 3, t = 0):
    rho = rho0, u = u0 cos(2 pi x / L) sin(2 pi y / L), v = -u0 sin(2 pi x / L) cos(2 pi y / L).

    u0 is the lattice-unit amplitude (u0 = U0 dt / dx_ml)."""
    x, y = np.asarray(xy[0], np.float64), np.asarray(xy[1], np.float64)
    k = 2.0 * np.pi / L
    u = u0 * np.cos(k * x) * np.sin(k * y)
    v = -u0 * np.sin(k * x) * np.cos(k * y)
    return np.full_like(x, rho0), u, v


# degree -> stencil size used by the batched convergence sweep
SWEEP_K_FOR_DEGREE = {2: 12, 3: 16, 4: 24, 5: 34, 6: 45}


def sweep_runs(small_sides=(16, 32, 64, 128), degrees=(2, 3, 4, 5, 6),
               ratios=(1.0, 0.5, 0.25), big=((512, 2, 1.0), (512, 2, 0.5), (512, 4, 1.0),
                                             (512, 4, 0.5))):
    """The 64 runs of the batched Taylor-Green convergence sweep: sqrt(N) in small_sides x
    interpolation degree x dx_ml refinement ratio (60 runs) plus four 512^2 runs.  Each run is
    a dict with n_side, degree, K, ratio (dx_ml = ratio * h), seed and tau = 0.8."""
    runs = []
    for s in small_sides:
        for d in degrees:
            for r in ratios:
                runs.append(dict(n_side=s, degree=d, K=SWEEP_K_FOR_DEGREE[d], ratio=r))
    for s, d, r in big:
        runs.append(dict(n_side=s, degree=d, K=SWEEP_K_FOR_DEGREE[d], ratio=r))
    for i, run in enumerate(runs):
        run["seed"] = 100 + i
        run["tau"] = 0.8
        # diffusive scaling (Sec. 3): the lattice velocity amplitude scales with dx_ml
        run["u0"] = 0.01 * run["ratio"]
    return runs
