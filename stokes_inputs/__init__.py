"""Seeded synthetic inputs for the 2D porous-pipe Stokes problem.

This module builds the discrete geometry (boundary nodes, unit normals,
quadrature weights, signed curvature, component offsets), boundary data and
interior evaluation targets that both the CPU oracle and the CUDA library
consume. It holds none of the solver's arithmetic: no layer potential, no
completion, no preconditioner, no Krylov step. Everything is a deterministic
function of its arguments and a numpy ``default_rng`` seed.

Geometry conventions (the paper's problem statement, Sec. 2):

* The fluid domain is Omega = Omega_0 minus the union of the pores Omega_k.
  The outer wall Gamma_0 is a smoothed rectangle; we use the superellipse
  |x/a|^p + |y/b|^p = 1 (p = 8), a "rounded off" rectangle like the one of
  Sec. 4. Each pore Gamma_k is a circle.
* Components are stored pores first, outer wall last; unknowns are
  interleaved (sigma_x, sigma_y) per node.
* "n is the unit outward normal" (Sec. 2.1) is read as: n points OUT OF THE
  FLUID. Gamma_0 is traversed counter-clockwise and every pore clockwise, and
  n is the tangent rotated clockwise, (t_y, -t_x). The signed curvature
  kappa = (x'y'' - y'x'')/|x'|^3 is taken along that traversal, so kappa > 0
  on the convex outer wall and kappa = -1/R on a pore of radius R.
* Quadrature weights are the trapezoid rule in the curve's parameter times
  the arclength factor (Sec. 2.2: "the product of the arclength term with
  appropriate quadrature weights"). The outer wall is sampled at equispaced
  arclength, so its weights are all L/n.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "cached_geometry",
    "Geometry", "superellipse_curve", "circle_curve", "assemble_geometry",
    "place_pores", "pipe10_geometry", "pipe1000_geometry", "batch_geometry",
    "coarse_train_geometry", "coarse_eval_geometry", "mlp_initial_params", "batch_config4_geometry",
    "pipe_bc", "reversed_pipe_bc", "outer_shear_bc", "shear_bc",
    "translation_bc", "rotation_bc", "stokeslet_rotlet_bc",
    "stokeslet_rotlet_velocity", "interior_targets", "random_density",
    "superellipse_inside",
]


# ---------------------------------------------------------------------------
# Curves
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Curve:
    """One closed boundary component sampled at n nodes."""
    nodes: np.ndarray      # (n, 2)
    normals: np.ndarray    # (n, 2) unit, out of the fluid
    weights: np.ndarray    # (n,)   arclength quadrature weights
    curvature: np.ndarray  # (n,)   signed, along the traversal
    centre: np.ndarray     # (2,)   circle centre, or area centroid for the wall
    radius: float          # circle radius, or 0 for the wall


def _superellipse_polar(theta, a, b, p):
    """Position and first/second theta-derivatives of the polar superellipse
    r(theta) = (|cos(theta)/a|^p + |sin(theta)/b|^p)^(-1/p), p even."""
    c, s = np.cos(theta), np.sin(theta)
    u, v = c / a, s / b
    du, dv = -s / a, c / b
    g = u**p + v**p
    g1 = p * (u**(p - 1) * du + v**(p - 1) * dv)
    g2 = p * ((p - 1) * u**(p - 2) * du**2 - u**p + (p - 1) * v**(p - 2) * dv**2 - v**p)
    q = 1.0 / p
    r = g**(-q)
    r1 = -q * g**(-q - 1) * g1
    r2 = q * (q + 1) * g**(-q - 2) * g1**2 - q * g**(-q - 1) * g2
    x, y = r * c, r * s
    x1, y1 = r1 * c - r * s, r1 * s + r * c
    x2 = r2 * c - 2 * r1 * s - r * c
    y2 = r2 * s + 2 * r1 * c - r * s
    return x, y, x1, y1, x2, y2


def superellipse_inside(pts, a, b, p=8):
    """Implicit function |x/a|^p + |y/b|^p (< 1 strictly inside)."""
    pts = np.asarray(pts, dtype=np.float64)
    u, v = pts[..., 0] / a, pts[..., 1] / b
    if p == 8:
        u, v = u * u, v * v
        u, v = u * u, v * v
        return u * u + v * v
    return u**p + v**p


def superellipse_curve(a: float, b: float, n: int, p: int = 8,
                       spacing: str = "arclength") -> Curve:
    """Outer wall |x/a|^p + |y/b|^p = 1, counter-clockwise, n nodes.

    spacing="arclength": nodes equispaced in arclength, found by inverting
    the spectrally integrated speed |x'(theta)| of the polar parametrisation
    with Newton's method; weights are L/n.
    spacing="polar": nodes equispaced in the polar angle; weights are
    |x'(theta_j)| 2 pi / n.
    """
    if n < 8 or p % 2:
        raise ValueError("need n >= 8 and even p")
    if spacing == "polar":
        theta = 2.0 * np.pi * np.arange(n) / n
        x, y, x1, y1, x2, y2 = _superellipse_polar(theta, a, b, p)
        speed = np.hypot(x1, y1)
        weights = speed * (2.0 * np.pi / n)
    elif spacing == "arclength":
        # Fourier series of the speed on a fine grid; the speed is analytic
        # and periodic, so its coefficients decay geometrically.
        K = 1 << 15
        tg = 2.0 * np.pi * np.arange(K) / K
        _, _, gx1, gy1, _, _ = _superellipse_polar(tg, a, b, p)
        sp = np.hypot(gx1, gy1)
        coef = np.fft.rfft(sp) / K
        c0 = coef[0].real
        L = 2.0 * np.pi * c0
        ks = np.arange(1, coef.size)
        A = 2.0 * coef[1:].real   # cos coefficients
        B = -2.0 * coef[1:].imag  # sin coefficients
        # drop the FFT round-off floor (~1e-16 c0) so the series stays short
        keep = np.nonzero(np.abs(A) + np.abs(B) > 1e-15 * c0)[0]
        kmax = int(keep.max()) + 1 if keep.size else 1
        ks, A, B = ks[:kmax], A[:kmax], B[:kmax]

        def arclen(th):
            kt = np.outer(th, ks)
            return c0 * th + (np.sin(kt) * (A / ks)).sum(1) + ((1.0 - np.cos(kt)) * (B / ks)).sum(1)

        # initial guess from the cumulative arclength on the fine grid
        s_grid = np.concatenate([[0.0], np.cumsum(0.5 * (sp + np.roll(sp, -1)) * (2 * np.pi / K))])
        t_grid = np.concatenate([tg, [2 * np.pi]])
        s_target = L * np.arange(n) / n
        theta = np.interp(s_target, s_grid * (L / s_grid[-1]), t_grid)
        for _ in range(8):
            _, _, tx1, ty1, _, _ = _superellipse_polar(theta, a, b, p)
            step = (arclen(theta) - s_target) / np.hypot(tx1, ty1)
            theta = theta - step
            if np.max(np.abs(step)) < 1e-15:
                break
        x, y, x1, y1, x2, y2 = _superellipse_polar(theta, a, b, p)
        weights = np.full(n, L / n)
    else:
        raise ValueError(spacing)
    speed = np.hypot(x1, y1)
    nodes = np.stack([x, y], axis=1)
    normals = np.stack([y1, -x1], axis=1) / speed[:, None]
    curvature = (x1 * y2 - y1 * x2) / speed**3
    return Curve(nodes, normals, weights, curvature, np.zeros(2), 0.0)


def circle_curve(centre, radius: float, n: int) -> Curve:
    """Pore of the given radius, traversed clockwise from angle 0, n nodes;
    normals point into the pore (out of the fluid), curvature is -1/R."""
    if n < 8 or radius <= 0:
        raise ValueError("need n >= 8 and radius > 0")
    centre = np.asarray(centre, dtype=np.float64)
    th = 2.0 * np.pi * np.arange(n) / n
    c, s = np.cos(th), np.sin(th)
    nodes = centre[None, :] + radius * np.stack([c, -s], axis=1)
    normals = -np.stack([c, -s], axis=1)
    weights = np.full(n, 2.0 * np.pi * radius / n)
    curvature = np.full(n, -1.0 / radius)
    return Curve(nodes, normals, weights, curvature, centre.copy(), float(radius))


# ---------------------------------------------------------------------------
# Geometry container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Geometry:
    """Discrete boundary: all arrays float64 C-contiguous, pores first."""
    nodes: np.ndarray       # (N, 2)
    normals: np.ndarray     # (N, 2)
    weights: np.ndarray     # (N,)
    curvature: np.ndarray   # (N,)
    offsets: np.ndarray     # (n_comp + 1,) int64
    outer_comp: int         # index of Gamma_0
    centres: np.ndarray     # (n_comp, 2) completion centres (pore centres)
    radii: np.ndarray       # (n_comp,) pore radii, 0 for the wall
    outer_shape: tuple = ()  # (a, b, p) of the outer superellipse, if any
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.offsets[-1])

    @property
    def n_comp(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def n_pores(self) -> int:
        return self.n_comp - 1

    def comp_of_node(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_comp), np.diff(self.offsets))

    def comp_slice(self, k: int) -> slice:
        return slice(int(self.offsets[k]), int(self.offsets[k + 1]))


def assemble_geometry(pores: list, outer: Curve, outer_shape=(), info=None) -> Geometry:
    curves = list(pores) + [outer]
    sizes = [c.nodes.shape[0] for c in curves]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cat = lambda f: np.ascontiguousarray(np.concatenate([getattr(c, f) for c in curves]))
    # The wall's entry in `centres` is its quadrature centroid; it is not
    # used by the completion (only pores carry a Stokeslet/rotlet).
    wall_c = (outer.nodes * outer.weights[:, None]).sum(0) / outer.weights.sum()
    centres = np.array([c.centre for c in pores] + [wall_c], dtype=np.float64).reshape(-1, 2)
    radii = np.array([c.radius for c in pores] + [0.0], dtype=np.float64)
    return Geometry(cat("nodes"), cat("normals"), cat("weights"), cat("curvature"),
                    offsets, len(curves) - 1, centres, radii, tuple(outer_shape), dict(info or {}))


# ---------------------------------------------------------------------------
# Pore placement
# ---------------------------------------------------------------------------

def _disc_inside_superellipse(centres, radii, a, b, p, margin):
    """True where the disc of radius radii+margin lies inside the (convex)
    superellipse, tested on 128 points of the inflated circle."""
    ang = 2 * np.pi * np.arange(128) / 128
    ring = np.stack([np.cos(ang), np.sin(ang)], 1)
    pts = centres[:, None, :] + (radii + margin)[:, None, None] * ring[None]
    return (superellipse_inside(pts, a, b, p) < 1.0).all(1)


_CLEARANCE_CACHE = {}


def _wall_clearance_grid(a, b, p, h, cap):
    """Cell centres of a grid of spacing h over the wall's bounding box and
    each centre's distance to the wall, capped at `cap` or more (negative
    outside). The cap only bounds the search: the placement compares these
    distances with thresholds below `cap`, so a grid computed once with a
    larger cap serves later calls with the same wall and spacing (read-only)."""
    key = (float(a), float(b), int(p), float(h))
    hit = _CLEARANCE_CACHE.get(key)
    if hit is not None and hit[0] >= cap:
        return hit[1]
    cap = max(cap, 0.6)
    out = _wall_clearance_grid_uncached(a, b, p, h, cap)
    for arr in out:
        arr.setflags(write=False)
    _CLEARANCE_CACHE[key] = (cap, out)
    return out


def _wall_clearance_grid_uncached(a, b, p, h, cap):
    from scipy.spatial import cKDTree
    xs = np.arange(-a + h / 2, a, h)
    ys = np.arange(-b + h / 2, b, h)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    fine = superellipse_curve(a, b, 1 << 16, p, spacing="polar").nodes
    d, _ = cKDTree(fine).query(pts, distance_upper_bound=cap)
    d = np.minimum(d, cap)
    inside = superellipse_inside(pts, a, b, p) < 1.0
    return xs, ys, np.where(inside, d, -d).reshape(X.shape)


def place_pores(rng, radii, outer_shape, gap, box=None, largest_first=False,
                shrink=0.95, max_restarts=40, h=None):
    """Sample pore centres uniformly at random subject to: every pair of pores
    and every pore and the wall at least `gap` apart, centres inside `box`
    ((xmin, xmax, ymin, ymax); default: the wall's bounding box).

    Pores are placed one at a time (in the given order, or largest first).
    Each centre is drawn uniformly from the feasible set by rejection from a
    superset of it: a grid keeps each cell centre's clearance (distance to
    the nearest placed disc or to the wall); candidate cells are those whose
    clearance could admit the disc, a point is drawn uniformly inside a
    uniformly chosen candidate cell, and it is accepted only if it passes
    the exact pairwise-gap and wall tests. If some pore has no candidate
    cell, all radii are scaled by `shrink` and placement restarts; the final
    scale is returned. Returns (centres (M,2), radii (M,), scale).
    """
    a, b, p = outer_shape
    radii = np.asarray(radii, dtype=np.float64)
    M = radii.size
    order = np.argsort(-radii, kind="stable") if largest_first else np.arange(M)
    if box is None:
        box = (-a, a, -b, b)
    if h is None:
        h = max(min(a, b) / 200.0, 0.008)
    cap = 2.0 * (radii.max() + gap + h)
    xs, ys, wall_clear = _wall_clearance_grid(a, b, p, h, cap)
    in_box = ((xs[:, None] >= box[0]) & (xs[:, None] <= box[1])
              & (ys[None, :] >= box[2]) & (ys[None, :] <= box[3]))
    slack = h * 0.7072  # half the cell diagonal
    scale = 1.0
    for _ in range(max_restarts):
        rr = radii * scale
        clear = wall_clear.copy()
        pc = np.zeros((M, 2))
        pr = np.zeros(M)
        ok = True
        for cnt, idx in enumerate(order):
            r = rr[idx]
            cand_cells = np.nonzero(in_box & (clear >= r + gap - slack))
            if cand_cells[0].size == 0:
                ok = False
                break
            found = None
            for _attempt in range(10000):
                pick = rng.integers(0, cand_cells[0].size, 64)
                cx = xs[cand_cells[0][pick]] + rng.uniform(-h / 2, h / 2, 64)
                cy = ys[cand_cells[1][pick]] + rng.uniform(-h / 2, h / 2, 64)
                cand = np.stack([cx, cy], 1)
                good = ((cx >= box[0]) & (cx <= box[1]) & (cy >= box[2]) & (cy <= box[3]))
                near_wall = wall_clear[cand_cells[0][pick], cand_cells[1][pick]] < r + gap + slack
                if near_wall.any():
                    nw = np.nonzero(near_wall)[0]
                    good[nw] &= _disc_inside_superellipse(cand[nw], np.full(nw.size, r), a, b, p, gap)
                if cnt:
                    dx = cand[:, 0, None] - pc[None, :cnt, 0]
                    dy = cand[:, 1, None] - pc[None, :cnt, 1]
                    lim = pr[None, :cnt] + r + gap
                    good &= (dx * dx + dy * dy >= lim * lim).all(1)
                if good.any():
                    found = cand[np.argmax(good)]
                    break
            if found is None:
                ok = False
                break
            pc[cnt], pr[cnt] = found, r
            # update the clearance field near the new disc
            reach = r + 2 * rr.max() + 2 * gap + 2 * h
            i0, i1 = np.searchsorted(xs, found[0] - reach), np.searchsorted(xs, found[0] + reach)
            j0, j1 = np.searchsorted(ys, found[1] - reach), np.searchsorted(ys, found[1] + reach)
            dx = xs[i0:i1, None] - found[0]
            dy = ys[None, j0:j1] - found[1]
            clear[i0:i1, j0:j1] = np.minimum(clear[i0:i1, j0:j1], np.sqrt(dx * dx + dy * dy) - r)
        if ok:
            inv = np.empty_like(order)
            inv[order] = np.arange(M)
            return pc[inv], pr[inv], scale
        scale *= shrink
    raise RuntimeError("pore placement failed")


# ---------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------

def _build(rng_seed, outer_shape, n_outer, radius_sampler, n_pores, n_per_pore,
           gap, box, largest_first, info):
    rng = np.random.default_rng(rng_seed)
    radii = radius_sampler(rng, n_pores)
    a, b, p = outer_shape
    centres, radii, scale = place_pores(rng, radii, outer_shape, gap, box=box,
                                        largest_first=largest_first)
    if np.isscalar(n_per_pore):
        n_per_pore = np.full(n_pores, int(n_per_pore))
    pores = [circle_curve(c, r, int(m)) for c, r, m in zip(centres, radii, n_per_pore)]
    outer = superellipse_curve(a, b, n_outer, p)
    info = dict(info, radius_scale=scale, seed=rng_seed)
    return assemble_geometry(pores, outer, outer_shape, info)


def pipe10_geometry(seed: int = 0, n_outer: int = 512, n_pores: int = 10, n_per_pore: int = 64):
    """Outer |x/4|^8 + |y|^8 = 1 (512 nodes); 10 pores, radii U[0.1, 0.2],
    centres uniform in |x| < 3.2, |y| < 0.6, gap >= 0.05; 64 nodes per
    pore (N = 1152 nodes, 2304 unknowns)."""
    return _build(seed, (4.0, 1.0, 8), n_outer,
                  lambda rng, m: rng.uniform(0.1, 0.2, m), n_pores, n_per_pore,
                  0.05, (-3.2, 3.2, -0.6, 0.6), False, {"name": "pipe10"})


def _lognormal_radii(rng, m, median=0.15, sigma=0.3, lo=0.05, hi=0.3):
    return np.clip(rng.lognormal(math.log(median), sigma, m), lo, hi)


def pipe1000_geometry(seed: int = 0, n_outer: int = 8192, n_pores: int = 1000, n_per_pore: int = 128):
    """Outer |x/20|^8 + |y/2|^8 = 1 (8192 nodes); 1000 pores with radii
    lognormal (median 0.15, sigma 0.3) clipped to [0.05, 0.3], gap >= 0.05,
    128 nodes per pore (N = 136,192 nodes, 272,384 unknowns).

    The stated radii cover ~71 % of the area once the gap is added, above the
    random-sequential-adsorption limit, so pores are placed largest first and
    all radii shrink by 0.95 until placement succeeds (scale in info)."""
    return _build(seed, (20.0, 2.0, 8), n_outer, _lognormal_radii, n_pores, n_per_pore,
                  0.05, None, True, {"name": "pipe1000"})


def batch_geometry(index: int, n_pores=None, n_per_pore=None, n_outer=None):
    """One geometry of the uneven multi-geometry batch: pore count uniform in
    [50, 800], nodes per pore in {64, 128, 256}, wall nodes in
    {2048, 4096, 8192}; wall |x/a|^8 + |y/2|^8 = 1 with a set so the pores
    fill ~30 % of the area; radii as in pipe1000_geometry. Seed = index."""
    rng = np.random.default_rng(10_000 + index)
    M = int(rng.integers(50, 801)) if n_pores is None else int(n_pores)
    npp = int(rng.choice([64, 128, 256])) if n_per_pore is None else int(n_per_pore)
    no = int(rng.choice([2048, 4096, 8192])) if n_outer is None else int(n_outer)
    mean_area = math.pi * 0.15**2 * math.exp(2 * 0.3**2)
    area = M * mean_area / 0.30
    # area of |x/a|^8 + |y/b|^8 <= 1 is 4ab Gamma(1+1/8)^2 / Gamma(1+2/8)
    k = 4 * math.gamma(1.125) ** 2 / math.gamma(1.25)
    a = area / (k * 2.0)
    return _build(index, (a, 2.0, 8), no, _lognormal_radii, M, npp, 0.05, None, True,
                  {"name": f"batch{index}"})


def batch_small_geometry(index: int):
    """A geometry of the scaled-down uneven batch: pore count uniform in
    [20, 120], 64 or 128 nodes per pore, 1024 or 2048 wall nodes, otherwise
    as batch_geometry. Seed = index."""
    rng = np.random.default_rng(20_000 + index)
    M = int(rng.integers(20, 121))
    npp = int(rng.choice([64, 128]))
    no = int(rng.choice([1024, 2048]))
    return batch_geometry(index, n_pores=M, n_per_pore=npp, n_outer=no)


def batch_config4_geometry(index: int):
    """Geometry `index` (0..63) of the batched configuration's subset: pore
    count uniform in [50, 200] (the configuration states [50, 800]), nodes per
    pore in {64, 128, 256}, wall nodes in {2048, 4096, 8192}, otherwise as
    batch_geometry (pores fill ~30 % of the wall's area). Seed 40000 + index."""
    rng = np.random.default_rng(40_000 + index)
    M = int(rng.integers(50, 201))
    npp = int(rng.choice([64, 128, 256]))
    no = int(rng.choice([2048, 4096, 8192]))
    return batch_geometry(40_000 + index, n_pores=M, n_per_pore=npp, n_outer=no)


def coarse_train_geometry(index: int):
    """Training geometry `index` of the learned coarse correction: even
    indices are 1152-node pipes of the pipe10 family (seed 1 + index: 10
    pores, radii U[0.1, 0.2], 64 nodes per pore, 512 wall nodes); odd ones
    are longer pipes at the same pore density: M in {20, 30, 40, 50, 60},
    wall |x/a|^8 + |y|^8 = 1 with a = 0.4 M, centres in |x| < a - 0.8,
    |y| < 0.6, 64 nodes per pore, 64 * round(0.8 M) wall nodes."""
    if index % 2 == 0:
        return pipe10_geometry(1 + index)
    rng = np.random.default_rng(30_000 + index)
    M = 20 + 10 * int(rng.integers(0, 5))
    a = 0.4 * M
    return _build(30_000 + index, (a, 1.0, 8), 64 * int(round(0.8 * M)),
                  lambda r, m: r.uniform(0.1, 0.2, m), M, 64, 0.05, (-(a - 0.8), a - 0.8, -0.6, 0.6), False,
                  {"name": f"coarsetrain{index}"})


def coarse_eval_geometry(index: int):
    """Held-out evaluation geometry `index` (0..99): the 1152-node pipe of
    the pipe10 family with seed 10000 + index."""
    return pipe10_geometry(10_000 + index)


def mlp_initial_params(seed: int = 0, sizes=((35, 256), (256, 256), (256, 153))) -> np.ndarray:
    """Initial network parameters, float32, flat in the order W1, b1, W2, b2,
    W3, b3 (W row-major, fan_in x fan_out): W ~ N(0, 2 / fan_in) (He), b = 0."""
    rng = np.random.default_rng(777 + seed)
    parts = []
    for fi, fo in sizes:
        parts.append((rng.standard_normal(fi * fo) * math.sqrt(2.0 / fi)).astype(np.float32))
        parts.append(np.zeros(fo, dtype=np.float32))
    return np.ascontiguousarray(np.concatenate(parts))


# ---------------------------------------------------------------------------
# Boundary data (rows of f, shape (N, 2))
# ---------------------------------------------------------------------------

def _outer_half_height(geom: Geometry) -> float:
    if geom.outer_shape:
        return float(geom.outer_shape[1])
    sl = geom.comp_slice(geom.outer_comp)
    return float(np.abs(geom.nodes[sl, 1]).max())


def pipe_bc(geom: Geometry, k: float = 1.0) -> np.ndarray:
    """Pipe flow (Eq. 2): f = k (H^2 - y^2) along x on Gamma_0, zero on the
    pores. Read with H = the wall's half-height b and k = 1/H^2, i.e.
    f = (1 - (y/b)^2, 0): the parabola of the intake and outtake, extended
    smoothly along the wall (where it is nearly zero). `k` scales it."""
    f = np.zeros_like(geom.nodes)
    sl = geom.comp_slice(geom.outer_comp)
    H = _outer_half_height(geom)
    f[sl, 0] = k * (1.0 - (geom.nodes[sl, 1] / H) ** 2)
    return f


def reversed_pipe_bc(geom: Geometry) -> np.ndarray:
    return -pipe_bc(geom)


def outer_shear_bc(geom: Geometry) -> np.ndarray:
    """Linear shear u = (y, 0) on the wall, no slip on the pores."""
    f = np.zeros_like(geom.nodes)
    sl = geom.comp_slice(geom.outer_comp)
    f[sl, 0] = geom.nodes[sl, 1]
    return f


def shear_bc(geom: Geometry) -> np.ndarray:
    """Shear flow of Sec. 4.1 on every boundary: exact solution u = (y, 0)."""
    f = np.zeros_like(geom.nodes)
    f[:, 0] = geom.nodes[:, 1]
    return f


def translation_bc(geom: Geometry, U=(1.0, 0.5)) -> np.ndarray:
    """Rigid translation on every boundary: exact solution u = U."""
    return np.tile(np.asarray(U, dtype=np.float64), (geom.n_nodes, 1))


def rotation_bc(geom: Geometry, omega: float = 1.0, centre=(0.0, 0.0)) -> np.ndarray:
    """Rigid rotation on every boundary: exact solution u = omega (-(y-c_y), x-c_x)."""
    d = geom.nodes - np.asarray(centre)[None, :]
    return omega * np.stack([-d[:, 1], d[:, 0]], 1)


def stokeslet_rotlet_params(geom: Geometry, seed: int = 0):
    """Singularity data for Eq. 13: c_0 outside Omega_0 (at (0, 3b)), c_k the
    pore centres; lambda_k with N(0,1) entries, mu_k ~ N(0,1)."""
    rng = np.random.default_rng(seed + 7919)
    H = _outer_half_height(geom)
    c = np.concatenate([[[0.0, 3.0 * H]], geom.centres[: geom.n_pores]], 0)
    lam = rng.standard_normal((c.shape[0], 2))
    mu = rng.standard_normal(c.shape[0])
    return c, lam, mu


def stokeslet_rotlet_velocity(points, c, lam, mu) -> np.ndarray:
    """Closed form of Eq. 13 (no 1/(4 pi) factor, as printed):
    u(x) = sum_k (-log|x-c_k| I + (x-c_k)(x-c_k)^T/|x-c_k|^2) lambda_k
           + sum_k (x-c_k)^perp / |x-c_k|^2 mu_k,   (x, y)^perp = (y, -x)."""
    pts = np.asarray(points, dtype=np.float64)
    u = np.zeros_like(pts)
    for ck, lk, mk in zip(c, lam, mu):
        r = pts - ck[None, :]
        rho2 = (r * r).sum(1)
        rl = r @ lk
        u += -0.5 * np.log(rho2)[:, None] * lk[None, :] + (rl / rho2)[:, None] * r
        u += mk * np.stack([r[:, 1], -r[:, 0]], 1) / rho2[:, None]
    return u


def stokeslet_rotlet_bc(geom: Geometry, seed: int = 0) -> np.ndarray:
    c, lam, mu = stokeslet_rotlet_params(geom, seed)
    return stokeslet_rotlet_velocity(geom.nodes, c, lam, mu)


def random_density(geom: Geometry, seed: int = 0) -> np.ndarray:
    """Smooth-ish random density (N, 2) for operator tests: N(0,1) entries."""
    rng = np.random.default_rng(seed + 104729)
    return rng.standard_normal((geom.n_nodes, 2))


# ---------------------------------------------------------------------------
# Interior targets
# ---------------------------------------------------------------------------

def interior_targets(geom: Geometry, count: int, min_dist: float = 0.05, seed: int = 0,
                     box=None) -> np.ndarray:
    """`count` points uniform in the fluid at distance >= min_dist from every
    boundary (pores: exact circle distance; wall: distance to a 16x refined
    polygon of the wall nodes' curve, checked with the implicit function)."""
    rng = np.random.default_rng(seed + 31337)
    sl = geom.comp_slice(geom.outer_comp)
    wall = geom.nodes[sl]
    if box is None:
        box = (wall[:, 0].min(), wall[:, 0].max(), wall[:, 1].min(), wall[:, 1].max())
    if geom.outer_shape:
        a, b, p = geom.outer_shape
        fine = superellipse_curve(a, b, max(4096, 16 * wall.shape[0]), p, spacing="polar").nodes
    else:
        fine = wall
    pc, pr = geom.centres[: geom.n_pores], geom.radii[: geom.n_pores]
    out = []
    have = 0
    while have < count:
        m = 4096
        cand = np.stack([rng.uniform(box[0], box[1], m), rng.uniform(box[2], box[3], m)], 1)
        if geom.outer_shape:
            keep = superellipse_inside(cand, a, b, p) < 1.0
        else:
            keep = np.ones(m, bool)
        if pc.size:
            d = np.linalg.norm(cand[:, None, :] - pc[None], axis=2) - pr[None]
            keep &= (d >= min_dist).all(1)
        idx = np.nonzero(keep)[0]
        if idx.size:
            dw = np.full(idx.size, np.inf)
            for s in range(0, fine.shape[0], 8192):
                dd = np.linalg.norm(cand[idx, None, :] - fine[None, s:s + 8192], axis=2).min(1)
                dw = np.minimum(dw, dd)
            idx = idx[dw >= min_dist]
        out.append(cand[idx])
        have += idx.size
    return np.ascontiguousarray(np.concatenate(out, 0)[:count])


# ---------------------------------------------------------------------------
# On-disk cache (generation of the largest workload takes ~30 s)
# ---------------------------------------------------------------------------

def _source_tag() -> str:
    import hashlib
    import pathlib
    return hashlib.sha1(pathlib.Path(__file__).read_bytes()).hexdigest()[:12]


def cached_geometry(name: str, seed: int = 0, cache_dir=None) -> Geometry:
    """pipe10_geometry / pipe1000_geometry / batch_geometry /
    batch_small_geometry by name ("pipe10", "pipe1000", "batch<i>", "batchsmall<i>"), stored as .npz under `cache_dir`
    (default: <repo>/.cache) keyed by the generator's source hash."""
    import os
    import pathlib
    if cache_dir is None:
        cache_dir = pathlib.Path(__file__).resolve().parent.parent / ".cache"
    cache_dir = pathlib.Path(cache_dir)
    fn = cache_dir / f"geom_{name}_{seed}_{_source_tag()}.npz"
    if fn.exists():
        z = np.load(fn, allow_pickle=False)
        info = {"name": name, "seed": seed, "radius_scale": float(z["radius_scale"])}
        return Geometry(z["nodes"], z["normals"], z["weights"], z["curvature"], z["offsets"],
                        int(z["outer_comp"]), z["centres"], z["radii"],
                        tuple(float(v) for v in z["outer_shape"]), info)
    if name == "pipe10":
        g = pipe10_geometry(seed)
    elif name == "pipe1000":
        g = pipe1000_geometry(seed)
    elif name.startswith("batchsmall"):
        g = batch_small_geometry(int(name[10:]))
    elif name.startswith("batch"):
        g = batch_geometry(int(name[5:]))
    else:
        raise ValueError(name)
    try:
        cache_dir.mkdir(parents=True, exist_ok=True)
        tmp = fn.with_suffix(f".{os.getpid()}.tmp.npz")
        np.savez(tmp, nodes=g.nodes, normals=g.normals, weights=g.weights, curvature=g.curvature,
                 offsets=g.offsets, outer_comp=g.outer_comp, centres=g.centres, radii=g.radii,
                 outer_shape=np.asarray(g.outer_shape, dtype=np.float64),
                 radius_scale=g.info.get("radius_scale", 1.0))
        os.replace(tmp, fn)
    except OSError:
        pass
    return g
