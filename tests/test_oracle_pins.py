"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these retypes an oracle formula: each checks a closed form, an
identity, an invariant, a textbook routine or a limit that a dropped term, a
wrong sign or index or a transposed operand would break.
"""
import math

import numpy as np
import pytest

import oracle as O
import stokes_inputs as si


def _ellipse_geometry(orientation):
    c = si.superellipse_curve(1.3, 0.6, 400, p=2)
    if orientation == "cw":   # pore-like: traversal reversed, normal into the curve
        c = si.Curve(c.nodes[::-1].copy(), -c.normals[::-1].copy(), c.weights[::-1].copy(),
                     -c.curvature[::-1].copy(), c.centre, 0.0)
    return si.assemble_geometry([], c)


@pytest.mark.parametrize("orientation,sign", [("ccw", -1.0), ("cw", 1.0)])
@pytest.mark.parametrize("e", [(1.0, 0.0), (0.0, 1.0), (0.6, -0.8)])
def test_double_layer_of_constant_density(orientation, sign, e):
    """Gauss-type identity for the Stokes double layer of Sec. 2.1 with a
    constant density e: -e inside / 0 outside a curve whose normal points out
    of it, and the mean -e/2 on the curve (principal value + diagonal entry).
    Flipping the normal flips the sign."""
    g = _ellipse_geometry(orientation)
    e = np.asarray(e)
    sig = np.tile(e, (g.n_nodes, 1))
    inside = O.velocity(g, sig, np.array([[0.1, 0.05], [-0.9, 0.2], [0.0, -0.45]]))
    outside = O.velocity(g, sig, np.array([[2.0, 1.0], [0.0, 1.5], [-1.6, 0.0]]))
    assert np.abs(inside - sign * e).max() < 1e-12
    assert np.abs(outside).max() < 1e-12
    idx = np.arange(g.n_nodes)
    B = O.operator_blocks(g, idx, idx, completion=False, outer_fix=False, jump=False)
    on = np.einsum("ijab,jb->ia", B, sig)
    assert np.abs(on - sign * 0.5 * e).max() < 1e-12
    # the jump term makes the boundary value equal the limit from the
    # fluid side (outside for "cw", inside for "ccw")
    Bj = O.operator_blocks(g, idx, idx, completion=False, outer_fix=False, jump=True)
    lim = np.einsum("ijab,jb->ia", Bj, sig)
    assert np.abs(lim - (sign * e if orientation == "ccw" else 0 * e)).max() < 1e-12


def test_diagonal_entry_is_the_kernel_limit():
    """The j = i entry equals the limit of the kernel as the source slides
    along the curve onto the target (ellipse, both orientations)."""
    for orientation in ("ccw", "cw"):
        g = _ellipse_geometry(orientation)
        S = O.self_blocks(g)
        for i in (0, 37, 150):
            # exact nearby point on the ellipse (parametric), its normal from the same curve
            th = np.arctan2(g.nodes[i, 1] / 0.6, g.nodes[i, 0] / 1.3)
            for eps in (1e-3,):
                y = np.array([[1.3 * np.cos(th + eps), 0.6 * np.sin(th + eps)]])
                t = np.array([-1.3 * np.sin(th + eps), 0.6 * np.cos(th + eps)])
                n = np.array([t[1], -t[0]]) / np.linalg.norm(t)
                if orientation == "cw":
                    n = -n
                K = O.dlp_kernel(g.nodes[i:i + 1], y, n[None])[0, 0]
                assert np.abs(K * g.weights[i] - S[i]).max() < 5e-3 * np.abs(S[i]).max() + 1e-12


def test_self_term_is_needed():
    """Dropping the diagonal term breaks the on-curve identity for a
    tangential density (a planted mistake the identity test must catch)."""
    g = _ellipse_geometry("ccw")
    t = np.stack([-g.normals[:, 1], g.normals[:, 0]], 1)
    idx = np.arange(g.n_nodes)
    B = O.operator_blocks(g, idx, idx, completion=False, outer_fix=False, jump=False)
    sig = np.tile([1.0, 0.0], (g.n_nodes, 1))
    B_noself = B.copy()
    B_noself[idx, idx] = 0.0
    bad = np.einsum("ijab,jb->ia", B_noself, sig)
    assert np.abs(bad + 0.5 * sig).max() > 1e-3


def test_null_space_rank_without_completion(small_geom):
    """Sec. 2.1: the double layer has a rank-3 null space per pore (rigid
    motions); the interior problem adds a rank-1 defect on the wall. The
    completion of each pore and the wall term remove all of them."""
    g = small_geom
    sv0 = np.linalg.svd(O.assemble(g, completion=False, outer_fix=False), compute_uv=False)
    tiny = (sv0 < 1e-7 * sv0[0]).sum()
    assert tiny == 3 * g.n_pores + 1
    assert sv0[-(3 * g.n_pores + 2)] > 1e-3 * sv0[0]
    sv = np.linalg.svd(O.assemble(g), compute_uv=False)
    assert sv[-1] > 1e-3


def test_smallest_singular_value_stable_under_refinement():
    """A second-kind system: the smallest singular value does not decay as
    the mesh is refined."""
    smins = []
    for npp, no in ((16, 128), (32, 256), (64, 512)):
        g = si.pipe10_geometry(1, n_outer=no, n_pores=3, n_per_pore=npp)
        smins.append(np.linalg.svd(O.assemble(g), compute_uv=False)[-1])
    assert smins[-1] > 0.5 * smins[0]


@pytest.fixture(scope="module")
def fine_geom():
    return si.pipe10_geometry(2, n_outer=512, n_pores=4, n_per_pore=64)


@pytest.mark.parametrize("case", ["translation", "rotation", "shear"])
def test_exact_rigid_and_shear_flows(fine_geom, case):
    """Translation, rotation and the shear flow of Sec. 4.1 on every boundary
    are Stokes flows: the computed velocity must reproduce them in the
    interior, and (as Sec. 4.1 notes for shear) the pore densities vanish."""
    g = fine_geom
    f = {"translation": si.translation_bc, "rotation": si.rotation_bc, "shear": si.shear_bc}[case](g)
    s = O.solve_dense(g, f)
    T = si.interior_targets(g, 300, min_dist=0.3, seed=4)
    u = O.velocity(g, s, T)
    exact = {"translation": si.translation_bc, "rotation": si.rotation_bc, "shear": si.shear_bc}
    tmp = si.Geometry(T, T, np.ones(len(T)), np.ones(len(T)), np.array([0, len(T)]), 0,
                      np.zeros((1, 2)), np.zeros(1))
    ue = exact[case](tmp)
    assert np.abs(u - ue).max() < 1e-9 * max(1.0, np.abs(ue).max())
    pores = 2 * int(g.offsets[g.outer_comp])
    assert np.abs(s[:pores]).max() < 1e-7 * np.abs(s[pores:]).max()
    lam, xi, s0 = O.moments(g, s)
    assert abs(s0) < 1e-12


def test_stokeslet_rotlet_exact_and_spectral_convergence():
    """Eq. 13 data (Stokeslets and rotlets inside the pores and outside the
    wall) has the closed-form velocity of Eq. 13; the error decays
    geometrically under refinement (trapezoid rule on analytic curves)."""
    errs = []
    for npp, no in ((16, 128), (32, 256), (64, 512)):
        g = si.pipe10_geometry(2, n_outer=no, n_pores=4, n_per_pore=npp)
        c, lam, mu = si.stokeslet_rotlet_params(g, 0)
        s = O.solve_dense(g, si.stokeslet_rotlet_velocity(g.nodes, c, lam, mu))
        T = si.interior_targets(g, 200, min_dist=0.3, seed=5)
        ue = si.stokeslet_rotlet_velocity(T, c, lam, mu)
        errs.append(np.abs(O.velocity(g, s, T) - ue).max() / np.abs(ue).max())
        if npp == 64:
            pores = 2 * int(g.offsets[g.outer_comp])
            assert np.abs(s[:pores]).max() > 1e-2     # non-zero pore densities
    assert errs[-1] < 1e-9
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-2 * errs[1]


def test_matrix_free_rows_match_dense(small_geom):
    g = small_geom
    A = O.assemble(g)
    sig = si.random_density(g, 1)
    assert np.abs(O.matvec(g, sig) - A @ sig.reshape(-1)).max() < 1e-12 * np.abs(A).max() * g.n_nodes
    rows = np.array([0, 5, 100, g.n_nodes - 1])
    got = O.apply_rows(g, sig, rows).reshape(-1)
    idx = np.stack([2 * rows, 2 * rows + 1], 1).reshape(-1)
    assert np.allclose(got, (A @ sig.reshape(-1))[idx], rtol=0, atol=1e-12)


def test_moments_match_completion_columns(small_geom):
    """A sigma - A_nocompletion sigma equals the Stokeslet/rotlet field of the
    moments (checks the moment definitions against the assembled columns)."""
    g = small_geom
    sig = si.random_density(g, 2)
    d = (O.assemble(g) - O.assemble(g, completion=False)) @ sig.reshape(-1)
    lam, xi, _ = O.moments(g, sig)
    u = np.zeros((g.n_nodes, 2))
    for k in range(g.n_pores):
        u += np.einsum("tab,b->ta", O.stokeslet(g.nodes, g.centres[k]), lam[k])
        u += O.rotlet(g.nodes, g.centres[k]) * xi[k]
    assert np.abs(d - u.reshape(-1)).max() < 1e-12


def test_gmres_matches_dense_lu(small_geom):
    """Restarted GMRES (Sec. 4, Saad-Schultz) against LAPACK LU, with and
    without the block-diagonal preconditioner, right and left."""
    g = small_geom
    f = si.pipe_bc(g)
    sd = O.solve_dense(g, f)
    for pc in ("bd", None):
        r = O.solve_gmres(g, f, tol=1e-12, restart=20, precond=pc, side="right")
        assert r["relres"] <= 1e-12
        assert np.linalg.norm(r["x"] - sd) < 1e-10 * np.linalg.norm(sd)
    r = O.solve_gmres(g, f, tol=1e-12, restart=20, precond="bd", side="left")
    assert r["pc_relres"] <= 1e-12 and r["relres"] < 1e-10


def test_block_diagonal_is_exact_inverse_of_blocks(small_geom):
    """Each preconditioner block is the restriction of A to one component
    (Sec. 4.1 footnote), applied exactly."""
    g = small_geom
    A = O.assemble(g)
    bd = O.BlockDiagonal(g)
    v = np.random.default_rng(0).standard_normal(2 * g.n_nodes)
    z = bd.apply(v)
    for k in range(g.n_comp):
        a, b = 2 * int(g.offsets[k]), 2 * int(g.offsets[k + 1])
        assert np.allclose(A[a:b, a:b] @ z[a:b], v[a:b], rtol=0, atol=1e-11)
        assert np.array_equal(bd.blocks[k], A[a:b, a:b])


def test_bd_gmres_fewer_iterations_than_none(pipe10_geom):
    """Sec. 4.1: block-diagonal preconditioning cuts the iteration count."""
    f = si.pipe_bc(pipe10_geom)
    r_bd = O.solve_gmres(pipe10_geom, f, tol=1e-8, restart=50, precond="bd")
    r_no = O.solve_gmres(pipe10_geom, f, tol=1e-8, restart=50, precond=None)
    assert r_bd["relres"] <= 1e-8 and r_no["relres"] <= 1e-8
    assert r_bd["iters"] < 0.5 * r_no["iters"]


def test_pipe_flow_no_net_flux_around_a_pore(pipe10_geom):
    """Incompressibility and no slip (Eq. 1-2): the flux of u through any
    closed curve in the fluid that encloses one pore is zero; the flux
    through a vertical cut equals the flux leaving the wall beyond it."""
    g = pipe10_geom
    f = si.pipe_bc(g)
    s = O.solve_gmres(g, f, tol=1e-12, restart=50)["x"]
    pc, pr = g.centres[: g.n_pores], g.radii[: g.n_pores]
    for k in range(g.n_pores):
        R = pr[k] + 0.025
        others = np.delete(np.arange(g.n_pores), k)
        if (np.linalg.norm(pc[others] - pc[k], axis=1) - pr[others] < R + 0.02).any():
            continue
        th = 2 * np.pi * np.arange(256) / 256
        pts = pc[k] + R * np.stack([np.cos(th), np.sin(th)], 1)
        u = O.velocity(g, s, pts)
        flux = (u * np.stack([np.cos(th), np.sin(th)], 1)).sum() * (2 * np.pi * R / 256)
        scale = (np.abs(u).sum(1)).mean() * 2 * np.pi * R
        assert abs(flux) < 1e-9 * max(scale, 1e-3)
    # the velocity reproduces the data on the boundary from the fluid side
    # when evaluated just inside the wall near the intake centre
    x0 = np.array([[-3.9, 0.0]])
    assert abs(O.velocity(g, s, x0)[0, 0] - 1.0) < 0.05


def test_trig_interpolation_is_exact_for_band_limited_data():
    """The interpolation of the two-grid preconditioner reproduces every
    trigonometric polynomial the coarse grid resolves, and the coarse
    samples themselves."""
    for nc, nf in ((8, 32), (16, 128), (9, 27)):
        P = O.trig_interpolation(nc, nf)
        t = 2 * np.pi * np.arange(nf) / nf
        s = 2 * np.pi * np.arange(nc) / nc
        for k in range((nc + 1) // 2):
            for fn in (np.cos, np.sin):
                assert np.abs(P @ fn(k * s) - fn(k * t)).max() < 1e-13
        assert np.abs(P[:: nf // nc] - np.eye(nc)).max() < 1e-13 if nf % nc == 0 else True


def test_restriction_is_the_left_inverse_of_interpolation_up_to_nyquist():
    """R = (n_c / n_f) I^T undoes the interpolation I on every Fourier mode
    of the coarse grid except the Nyquist mode: by discrete orthogonality of
    the modes on the fine grid, (n_c / n_f) I^T I = Id - v v^T / (2 n_c) with
    v_j = (-1)^j, the Nyquist cosine split evenly between +-n_c / 2 keeping
    half its weight. A wrong restriction scale or Nyquist split fails it."""
    for nc, nf in ((8, 32), (16, 64), (8, 64), (32, 128), (128, 1024)):
        P = O.trig_interpolation(nc, nf)
        M = (nc / nf) * P.T @ P
        v = (-1.0) ** np.arange(nc)
        assert np.abs(M - (np.eye(nc) - np.outer(v, v) / (2 * nc))).max() < 1e-13


def test_coarse_geometry_is_the_trapezoid_rule_on_every_qth_node(small_geom):
    g = small_geom
    gc = O.coarse_geometry(g, 4)
    for k in range(g.n_comp):
        assert abs(gc.weights[gc.comp_slice(k)].sum() - g.weights[g.comp_slice(k)].sum()) < 1e-12
    # on each circular pore the coarse rule integrates (x - c_x)^2 exactly:
    # the integral is pi R^3
    for k in range(g.n_pores):
        sl = gc.comp_slice(k)
        val = (gc.weights[sl] * (gc.nodes[sl, 0] - g.centres[k, 0]) ** 2).sum()
        assert abs(val - math.pi * g.radii[k] ** 3) < 1e-14


def test_two_grid_fgmres_solves_the_dense_system_faster_than_block_diagonal():
    g = si.pipe10_geometry(0, n_outer=256, n_pores=6, n_per_pore=32)
    f = si.pipe_bc(g).reshape(-1)
    A = O.assemble(g)
    ref = np.linalg.solve(A, f)
    tg = O.TwoGrid(g, 4)
    r = O.fgmres(lambda v: A @ v, f, tg.apply, tol=1e-12)
    assert r["relres"] <= 1e-12 and np.linalg.norm(r["x"] - ref) < 1e-10 * np.linalg.norm(ref)
    rb = O.solve_gmres(g, f, tol=1e-12, restart=200)
    assert r["iters"] < 0.6 * rb["iters"]


def test_fgmres_tolerates_a_varying_preconditioner(small_geom):
    """Flexible GMRES (the iterate is built from the stored preconditioned
    vectors) still converges when the preconditioner changes each step."""
    g = small_geom
    f = si.pipe_bc(g).reshape(-1)
    A = O.assemble(g)
    bd = O.BlockDiagonal(g)
    rng = np.random.default_rng(3)
    noisy = lambda v: bd.apply(v) * (1.0 + 1e-3 * rng.standard_normal(v.size))
    r = O.fgmres(lambda v: A @ v, f, noisy, tol=1e-11, restart=100)
    assert r["relres"] <= 1e-11
    assert np.linalg.norm(r["x"] - np.linalg.solve(A, f)) < 1e-9 * np.linalg.norm(r["x"])


# ---------------------------------------------------------------------------
# Exact pins of the two-grid apply P^-1 r = I Ac^-1 R r + B^-1 (r - I R r)
# (wall remainder scaled by -2): three special cases in which the result
# has a closed form built only from pieces pinned above (the interpolation,
# the coarse trapezoid rule, the dense operator and its blocks).
# ---------------------------------------------------------------------------

def _high_band_residual(g, q, seed):
    """A residual with, on every component, only the fine-grid Fourier modes
    m with n_c / 2 < m <= n_f / 2 (n_c = n_f / q) in both vector components:
    by discrete orthogonality the restriction maps it to zero."""
    rng = np.random.default_rng(seed)
    r = np.zeros((g.n_nodes, 2))
    for k in range(g.n_comp):
        sl = g.comp_slice(k)
        nf = sl.stop - sl.start
        nc = nf // q
        t = 2 * np.pi * np.arange(nf) / nf
        for m in range(nc // 2 + 1, nf // 2 + 1):
            for comp in range(2):
                a, b = rng.standard_normal(2)
                r[sl, comp] += a * np.cos(m * t) + (b * np.sin(m * t) if 2 * m != nf else 0.0)
    return r.reshape(-1)


def _nyquist_free_coarse_vector(gc, seed):
    """Random coarse vector orthogonal, per component and per vector
    component, to that component's alternating vector (-1)^j."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((gc.n_nodes, 2))
    for k in range(gc.n_comp):
        sl = gc.comp_slice(k)
        v = (-1.0) ** np.arange(sl.stop - sl.start)
        c[sl] -= np.outer(v, v @ c[sl]) / (v @ v)
    return c.reshape(-1)


def _two_grid_pin_errors(tg_cls, q=4, seed=0):
    """Relative errors of the three closed-form cases for a TwoGrid class.
    (1) q = 1: I = R = Id, so the apply is A^-1 r.
    (2) R r = 0: the coarse part vanishes and the remainder is r itself, so
        the apply is B^-1 r on the pores and -2 r on the wall.
    (3) r = I c with c free of the Nyquist vectors: R I c = c, so the
        remainder vanishes and the apply is I Ac^-1 c."""
    import scipy.linalg as sla
    g = si.pipe10_geometry(0, n_outer=256, n_pores=4, n_per_pore=32)
    A = O.assemble(g)
    rng = np.random.default_rng(seed)
    errs = {}
    # (1)
    r = rng.standard_normal(2 * g.n_nodes)
    z = tg_cls(g, 1).apply(r)
    ref = np.linalg.solve(A, r)
    errs["q1"] = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    tg = tg_cls(g, q)
    # (2)
    r = _high_band_residual(g, q, seed)
    assert np.linalg.norm(tg.R @ r) < 1e-12 * np.linalg.norm(r)
    z = tg.apply(r)
    ref = np.empty_like(r)
    for k in range(g.n_comp):
        a, b = 2 * int(g.offsets[k]), 2 * int(g.offsets[k + 1])
        if k == g.outer_comp:
            ref[a:b] = -2.0 * r[a:b]
        else:
            ref[a:b] = np.linalg.solve(A[a:b, a:b], r[a:b])
    errs["kernel_of_R"] = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    # (3)
    gc = O.coarse_geometry(g, q)
    c = _nyquist_free_coarse_vector(gc, seed + 1)
    Ic = sla.block_diag(*[O.trig_interpolation((g.offsets[k + 1] - g.offsets[k]) // q,
                                               g.offsets[k + 1] - g.offsets[k]) for k in range(g.n_comp)])
    Ic = np.kron(Ic, np.eye(2))
    z = tg.apply(Ic @ c)
    ref = Ic @ np.linalg.solve(O.assemble(gc), c)
    errs["range_of_I"] = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    return errs


def test_two_grid_apply_closed_forms():
    errs = _two_grid_pin_errors(O.TwoGrid)
    assert max(errs.values()) < 1e-12, errs


class _WrongWallScale(O.TwoGrid):
    """Planted mistake: the wall remainder scaled by -1 instead of -2."""

    def apply(self, r):
        z = super().apply(r)
        h = np.asarray(r, dtype=np.float64).reshape(-1) - self.I @ (self.R @ r)
        z[self.wall] += h[self.wall]
        return z


class _WrongRestrictionScale(O.TwoGrid):
    """Planted mistake: R = I^T without the n_c / n_f factor."""

    def __init__(self, geom, q):
        super().__init__(geom, q)
        if q > 1:
            self.R = self.R * q


class _RemainderNotSplit(O.TwoGrid):
    """Planted mistake: the pore blocks act on r instead of r - I R r."""

    def apply(self, r):
        import scipy.linalg as sla
        r = np.asarray(r, dtype=np.float64).reshape(-1)
        zc = sla.lu_solve(self.lu, self.R @ r)
        zh = self.bd.apply(r)
        zh[self.wall] = -2.0 * r[self.wall]
        return self.I @ zc + zh


@pytest.mark.parametrize("cls", [_WrongWallScale, _WrongRestrictionScale, _RemainderNotSplit])
def test_two_grid_closed_forms_catch_planted_mistakes(cls):
    errs = _two_grid_pin_errors(cls)
    assert max(errs.values()) > 1e-3, errs
