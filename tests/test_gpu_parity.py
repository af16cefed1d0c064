"""GPU path (through the C ABI) against the CPU FP64 oracle.

Tolerances: the operator is evaluated in a different order on the GPU
(tiled pair sums, split over sources, FMA contraction), so results agree to
a relative L2 error of a few hundred ulps of the operator's scale; the bound
1e-12 on operator outputs leaves two decades of margin. Solutions: both
sides solve to relative residual 1e-12, so densities agree to
cond(A) * 1e-12 ~ 1e-9 at worst; the stated bound is 1e-10 (north of the
measured cond ~5e3 for the 1152-node case times the GMRES stopping error
being well below the bound in practice).
"""
import numpy as np
import pytest

import oracle as O
import stokes_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    return S


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ragged_geometry():
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    outer = si.superellipse_curve(3.0, 1.0, 203)
    return si.assemble_geometry(pores, outer, (3.0, 1.0, 8))


def _outer_only():
    return si.assemble_geometry([], si.superellipse_curve(2.0, 1.0, 130), (2.0, 1.0, 8))


GEOMS = {
    "pipe10": lambda: si.cached_geometry("pipe10", 0),
    "ragged": _ragged_geometry,
    "outer_only": _outer_only,
    "one_pore": lambda: si.pipe10_geometry(3, n_outer=96, n_pores=1, n_per_pore=40),
}


@pytest.fixture(scope="module", params=list(GEOMS))
def case(request):
    return request.param, GEOMS[request.param]()


def test_newton_reciprocal_matches_ieee_division(S, dev):
    """The FP64 pair kernel's reciprocal (hardware approximation + two
    Newton steps) against IEEE division over the squared distances the
    operator meets (1e-12 .. 1e6, log-uniform), powers of two and the
    padding sources' 1e60: within 2 ulps."""
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-12, 6, 200000), 2.0 ** np.arange(-60, 61), [1.0, 3.0, 0.1, 1e60]])
    xt = torch.tensor(x, device=dev)
    y = torch.empty_like(xt)
    S.stokes_rcp_f64(xt, y)
    torch.cuda.synchronize()
    ref = 1.0 / x
    err = np.abs(y.cpu().numpy() - ref) / ref
    assert err.max() <= 2 * 2.0 ** -53, err.max()


def test_matvec_fp64_matches_oracle(S, dev, case):
    name, g = case
    sig = si.random_density(g, 3).reshape(-1)
    ref = O.matvec(g, sig)
    with S.Geometry(g) as G:
        y = torch.empty(2 * g.n_nodes, dtype=torch.float64, device=dev)
        S.stokes_matvec(G.handle, torch.tensor(sig, device=dev), y, S.STOKES_FP64)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), ref) < 1e-12
        # host pointers give the same bits
        yh = np.empty_like(sig)
        S.stokes_matvec(G.handle, sig, yh, S.STOKES_FP64)
        assert np.array_equal(yh, y.cpu().numpy())


def test_block_diagonal_apply_matches_oracle(S, dev, case):
    name, g = case
    v = np.random.default_rng(5).standard_normal(2 * g.n_nodes)
    ref = O.BlockDiagonal(g).apply(v)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
        assert rel(z, ref) < 1e-11


def test_gmres_fp64_matches_dense_oracle(S, dev, case):
    name, g = case
    f = si.pipe_bc(g).reshape(-1) if g.n_pores else si.shear_bc(g).reshape(-1)
    ref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        sig = torch.zeros(2 * g.n_nodes, dtype=torch.float64, device=dev)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, torch.tensor(f, device=dev), sig, tol=1e-12,
                                                  restart=50, max_iter=2000)
        assert code == S.STOKES_OK and rr <= 1e-12
        assert rel(sig.cpu().numpy(), ref) < 1e-10


def test_gmres_iteration_count_matches_oracle_gmres(S, dev):
    """Same method (right block-diagonal GMRES(50), tol 1e-10) on the
    1152-node pipe problem: iteration counts within 2 (different rounding:
    CGS2 on the GPU, MGS in the oracle)."""
    g = si.cached_geometry("pipe10", 0)
    f = si.pipe_bc(g).reshape(-1)
    r_or = O.solve_gmres(g, f, tol=1e-10, restart=50, precond="bd")
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-10, restart=50)
        assert code == S.STOKES_OK and rr <= 1e-10
        assert abs(iters - r_or["iters"]) <= 2
        assert rel(sig, r_or["x"]) < 1e-8


@pytest.mark.parametrize("side", ["left", "none"])
def test_gmres_left_and_unpreconditioned(S, dev, side):
    g = si.pipe10_geometry(0, n_outer=256, n_pores=4, n_per_pore=32)
    f = si.pipe_bc(g).reshape(-1)
    ref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        if side == "left":
            S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        sig = np.zeros_like(f)
        code, iters, rr, pr = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-12, restart=40, max_iter=3000,
                                                   pc_side=S.STOKES_PC_LEFT if side == "left" else S.STOKES_PC_RIGHT)
        assert code == S.STOKES_OK
        if side == "left":
            assert pr <= 1e-12
        assert rel(sig, ref) < 1e-9


def test_velocity_matches_oracle(S, dev):
    g = si.cached_geometry("pipe10", 0)
    sig = O.solve_dense(g, si.pipe_bc(g).reshape(-1))
    T = si.interior_targets(g, 4096, min_dist=0.05, seed=11)
    ref = O.velocity(g, sig, T)
    with S.Geometry(g) as G:
        u = np.empty(T.size)
        S.stokes_eval_velocity(G.handle, sig, T.reshape(-1), u)
        assert rel(u, ref) < 1e-12


def test_exact_stokeslet_flow_through_gpu_solve(S, dev):
    """End to end against the closed form of Eq. 13 (not just the oracle)."""
    g = si.pipe10_geometry(2, n_outer=512, n_pores=4, n_per_pore=64)
    c, lam, mu = si.stokeslet_rotlet_params(g, 0)
    f = si.stokeslet_rotlet_velocity(g.nodes, c, lam, mu).reshape(-1)
    T = si.interior_targets(g, 300, min_dist=0.3, seed=5)
    ue = si.stokeslet_rotlet_velocity(T, c, lam, mu)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle)
        sig = np.zeros_like(f)
        S.stokes_gmres_solve(G.handle, f, sig, tol=1e-13, restart=50)
        u = np.empty(T.size)
        S.stokes_eval_velocity(G.handle, sig, T.reshape(-1), u)
        assert np.abs(u.reshape(-1, 2) - ue).max() / np.abs(ue).max() < 1e-9


def test_errors_are_reported(S, dev):
    g = si.pipe10_geometry(0, n_outer=64, n_pores=2, n_per_pore=16)
    bad = g.offsets.copy()
    bad[1] = bad[0] + 4                 # a component with fewer than 8 nodes
    with pytest.raises(S.StokesError) as e:
        S.stokes_geometry_create(g.nodes.reshape(-1), g.normals.reshape(-1), g.weights, g.curvature, bad,
                                 g.n_comp, g.outer_comp)
    assert e.value.code == S.STOKES_EINVAL
    nb = g.normals.copy()
    nb[3] *= 1.1
    with pytest.raises(S.StokesError):
        S.stokes_geometry_create(g.nodes.reshape(-1), nb.reshape(-1), g.weights, g.curvature, g.offsets,
                                 g.n_comp, g.outer_comp)
    with S.Geometry(g) as G:
        v = np.zeros(2 * g.n_nodes)
        with pytest.raises(S.StokesError) as e:
            S.stokes_precond_apply(G.handle, v, np.empty_like(v))
        assert e.value.code == S.STOKES_ESTATE
        f = si.pipe_bc(g).reshape(-1)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-14, restart=5, max_iter=3)
        assert code == S.STOKES_ENOTCONV and iters == 3 and rr > 1e-14
        with pytest.raises(S.StokesError):
            S.stokes_gmres_solve(G.handle, f, sig, tol=-1.0)
        # zero right-hand side: zero solution, no iterations
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, np.zeros_like(f), sig)
        assert code == S.STOKES_OK and iters == 0 and not sig.any()


@pytest.mark.parametrize("rows", [64])
def test_full_size_matvec_sampled_rows(S, dev, rows):
    """136,192-node geometry (1000 pores), launch shape as in the benchmark:
    sampled rows of A sigma against the oracle's matrix-free rows."""
    g = si.cached_geometry("pipe1000", 0)
    sig = si.random_density(g, 9).reshape(-1)
    idx = np.random.default_rng(1).choice(g.n_nodes, rows, replace=False)
    idx = np.concatenate([idx, [0, g.n_nodes - 1, int(g.offsets[g.outer_comp])]])
    ref = O.apply_rows(g, sig, idx)
    with S.Geometry(g) as G:
        y = torch.empty(2 * g.n_nodes, dtype=torch.float64, device=dev)
        S.stokes_matvec(G.handle, torch.tensor(sig, device=dev), y, S.STOKES_FP64)
        got = y.cpu().numpy().reshape(-1, 2)[idx]
        assert rel(got, ref) < 1e-12


def test_block_diagonal_large_wall_block_triangular_path(S, dev):
    """A wall block above the explicit-inverse limit (2 x 2200 rows) is
    applied by blocked triangular solves; it must match the oracle too."""
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 64), si.circle_curve((1.0, -0.2), 0.2, 64)]
    g = si.assemble_geometry(pores, si.superellipse_curve(4.0, 1.0, 2200), (4.0, 1.0, 8))
    v = np.random.default_rng(6).standard_normal(2 * g.n_nodes)
    ref = O.BlockDiagonal(g).apply(v)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
        assert rel(z, ref) < 1e-11


def test_block_diagonal_float_inverses(S, dev):
    """The float explicit inverses (including a wall block inverted by the
    blocked float triangular inversion) match the oracle to single
    precision times the blocks' conditioning (1e-4)."""
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 64), si.circle_curve((1.0, -0.2), 0.2, 64)]
    g = si.assemble_geometry(pores, si.superellipse_curve(4.0, 1.0, 2200), (4.0, 1.0, 8))
    v = np.random.default_rng(9).standard_normal(2 * g.n_nodes)
    ref = O.BlockDiagonal(g).apply(v)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle)
        z = np.empty_like(v)
        S.stokes_precond_apply_prec(G.handle, v, z, S.STOKES_FP32)
        assert rel(z, ref) < 1e-4


def test_full_size_block_diagonal_sampled_rows(S, dev):
    """136,192-node geometry: for sampled rows i of each sampled block k,
    (A_kk z_k)_i equals v_i, with A_kk's rows from the oracle."""
    g = si.cached_geometry("pipe1000", 0)
    v = np.random.default_rng(7).standard_normal(2 * g.n_nodes)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
    rng = np.random.default_rng(8)
    for k in [0, 517, g.n_pores - 1, g.outer_comp]:
        sl = g.comp_slice(k)
        cols = np.arange(sl.start, sl.stop)
        rows = np.sort(rng.choice(cols, 16, replace=False))
        B = O.operator_blocks(g, rows, cols)           # (16, n_k, 2, 2)
        Az = np.einsum("rcab,cb->ra", B, z.reshape(-1, 2)[cols])
        want = v.reshape(-1, 2)[rows]
        assert np.abs(Az - want).max() < 1e-9 * np.abs(want).max(), k


@pytest.mark.parametrize("prec,bound", [("DF64", 1e-12), ("FP32", 2e-6)])
def test_matvec_reduced_precision_matches_oracle(S, dev, case, prec, bound):
    """DF64 (double-float pair sums) meets the FP64 bound; FP32 is bounded
    by single-precision rounding of ~N-term sums (2e-6 relative)."""
    name, g = case
    sig = si.random_density(g, 4).reshape(-1)
    ref = O.matvec(g, sig)
    with S.Geometry(g) as G:
        y = np.empty_like(sig)
        S.stokes_matvec(G.handle, sig, y, getattr(S, "STOKES_" + prec))
        assert rel(y, ref) < bound


@pytest.mark.parametrize("prec,bound", [("DF64", 1e-12), ("FP32", 2e-6)])
def test_velocity_reduced_precision(S, dev, prec, bound):
    g = si.cached_geometry("pipe10", 0)
    sig = si.random_density(g, 5).reshape(-1)
    T = si.interior_targets(g, 1000, min_dist=0.05, seed=12)
    ref = O.velocity(g, sig, T)
    with S.Geometry(g) as G:
        u = np.empty(T.size)
        S.stokes_eval_velocity(G.handle, sig, T.reshape(-1), u, getattr(S, "STOKES_" + prec))
        assert rel(u, ref) < bound


@pytest.mark.parametrize("prec", ["DF64", "MIXED_IR"])
def test_gmres_reduced_precision_solves_to_fp64_accuracy(S, dev, prec):
    """DF64 GMRES and mixed-precision refinement reach a true (FP64-class)
    relative residual of 1e-11 (the double-float operator's own accuracy is
    ~1e-12 relative, so refinement stalls near there) and the dense FP64
    solution."""
    g = si.cached_geometry("pipe10", 0)
    f = si.pipe_bc(g).reshape(-1)
    ref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=50,
                                                  precision=getattr(S, "STOKES_" + prec))
        assert code == S.STOKES_OK and rr <= 1e-11
        assert rel(sig, ref) < 1e-10
        # and the oracle agrees that the residual is small
        assert np.linalg.norm(f - O.matvec(g, sig)) / np.linalg.norm(f) < 1e-11


def test_profile_records_pair_launches(S, dev):
    g = si.cached_geometry("pipe10", 0)
    f = si.pipe_bc(g).reshape(-1)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle)
        S.stokes_profile_enable(G.handle, True)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-10, restart=30, precision=S.STOKES_DF64)
        n, ms, units = S.stokes_profile_read(G.handle, S.STOKES_PROF_PAIRS_DF64)
        n32 = S.stokes_profile_read(G.handle, S.STOKES_PROF_PAIRS_FP32)[0]
        n64 = S.stokes_profile_read(G.handle, S.STOKES_PROF_PAIRS_FP64)[0]
        cycles = -(-iters // 30)
        # one pair launch per iteration (double-float, or FP32 in a cycle that
        # starts within 1e4 tol of the tolerance); one double-float launch for
        # the residual each restart starts from, except after a refinement
        # cycle that converged (straight to FP64); the FP64 kernel only
        # confirms convergence (at least once, at most once per restart);
        # flexible GMRES applies the preconditioner once per iteration
        assert iters + cycles - 1 <= n + n32 <= iters + cycles + 2
        assert 1 <= n64 <= cycles
        assert units == pytest.approx(n * g.n_nodes**2)
        assert ms > 0
        nb, msb, ub = S.stokes_profile_read(G.handle, S.STOKES_PROF_BD_APPLY)
        assert nb == iters and msb > 0
        S.stokes_profile_enable(G.handle, False)
        assert S.stokes_profile_read(G.handle, S.STOKES_PROF_PAIRS_DF64)[0] == 0


def test_mixed_refinement_with_triangular_wall_block(S, dev):
    """Refinement on a geometry whose wall block takes the persistent
    triangular-solve path (float factors in the inner solves)."""
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 64), si.circle_curve((1.0, -0.2), 0.2, 64)]
    g = si.assemble_geometry(pores, si.superellipse_curve(4.0, 1.0, 2200), (4.0, 1.0, 8))
    f = si.pipe_bc(g).reshape(-1)
    ref = O.solve_gmres(g, f, tol=1e-12, restart=100)["x"]
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle)
        for prec in (S.STOKES_MIXED_IR, S.STOKES_DF64, S.STOKES_FP64):
            sig = np.zeros_like(f)
            code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=100, precision=prec)
            assert code == S.STOKES_OK and rr <= 1e-11
            assert rel(sig, ref) < 1e-9


def test_unrestarted_gmres_long_basis(S, dev):
    """A Krylov basis longer than 1000 vectors (no restart) on the
    1152-node problem without preconditioner."""
    g = si.cached_geometry("pipe10", 0)
    f = si.pipe_bc(g).reshape(-1)
    ref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=1500, max_iter=1500)
        assert code == S.STOKES_OK and rr <= 1e-11 and iters < 1500
        assert rel(sig, ref) < 1e-9


@pytest.mark.parametrize("prec", ["FP64", "DF64", "MIXED_IR"])
def test_two_grid_solve_matches_dense_oracle(S, dev, prec):
    """Flexible GMRES with the two-grid preconditioner reaches the dense FP64
    solution, in about as many iterations as the oracle's two-grid FGMRES
    (whose coarse LU is double: the float one here may cost a few more)."""
    g = si.pipe10_geometry(0, n_outer=256, n_pores=6, n_per_pore=32)
    f = si.pipe_bc(g).reshape(-1)
    A = O.assemble(g)
    ref = np.linalg.solve(A, f)
    r_or = O.fgmres(lambda v: A @ v, f, O.TwoGrid(g, 4).apply, tol=1e-11)
    with S.Geometry(g) as G:
        S.stokes_precond_setup_twogrid(G.handle, 4)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=100,
                                                  precision=getattr(S, "STOKES_" + prec))
        assert code == S.STOKES_OK and rr <= 1e-11
        assert rel(sig, ref) < 1e-9
        if prec != "MIXED_IR":
            assert iters <= r_or["iters"] + 3


@pytest.mark.parametrize("mode", ["AUTO", "INVERSE", "LU"])
def test_two_grid_apply_matches_oracle(S, dev, mode):
    """P^-1 v against the oracle's double-precision two-grid apply: equal up
    to the float coarse factorisation (coarse condition number x 1e-7),
    with the coarse solve by the explicit inverse or by the LU factors
    (persistent triangular solves)."""
    g = si.pipe10_geometry(1, n_outer=256, n_pores=5, n_per_pore=32)
    v = np.random.default_rng(2).standard_normal(2 * g.n_nodes)
    ref = O.TwoGrid(g, 4).apply(v)
    with S.Geometry(g) as G:
        S.stokes_precond_setup_twogrid_ex(G.handle, 4, getattr(S, "STOKES_TG_COARSE_" + mode))
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
        assert rel(z, ref) < 1e-3


@pytest.mark.parametrize("panel", ["coop", "launches"])
def test_two_grid_panel_factorisation_paths(S, dev, panel, monkeypatch):
    """The coarse LU's panels factored by one cooperative launch per panel
    (one grid barrier per column) or by three launches per column: both give
    the oracle's two-grid apply and the dense solution."""
    monkeypatch.setenv("STOKES_TG_PANEL", panel)
    g = si.pipe10_geometry(1, n_outer=256, n_pores=5, n_per_pore=32)
    v = np.random.default_rng(2).standard_normal(2 * g.n_nodes)
    ref = O.TwoGrid(g, 4).apply(v)
    f = si.pipe_bc(g).reshape(-1)
    sref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        S.stokes_precond_setup_twogrid_ex(G.handle, 4, S.STOKES_TG_COARSE_LU)
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
        assert rel(z, ref) < 1e-3
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=100,
                                                  precision=S.STOKES_DF64)
        assert code == S.STOKES_OK and rel(sig, sref) < 1e-9


def test_two_grid_panel_paths_give_identical_factors(S, dev, monkeypatch):
    """On a coarse LU of 11,776 rows (128-column panels next to the
    tensor-core trailing updates) the cooperative panel kernel (one grid
    barrier per column, interchanges outside the panel applied afterwards)
    and the three launches per column pick the same pivots and do the same
    float operations, so the two LU-applied two-grid applies are equal bit
    for bit."""
    g = si.batch_geometry(3, n_pores=120, n_per_pore=64, n_outer=4096)
    v = torch.tensor(si.random_density(g, 5).reshape(-1), device=dev)
    out = {}
    for panel in ("coop", "launches"):
        monkeypatch.setenv("STOKES_TG_PANEL", panel)
        with S.Geometry(g) as G:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)
            z = torch.empty_like(v)
            S.stokes_precond_apply(G.handle, v, z)
            torch.cuda.synchronize()
            out[panel] = z
    assert torch.isfinite(out["coop"]).all()
    assert torch.equal(out["coop"], out["launches"])


def test_two_grid_lu_coarse_solve_matches_dense_oracle(S, dev):
    """The coarse LU applied by triangular solves inside the double-float
    FGMRES gives the dense FP64 solution."""
    g = si.pipe10_geometry(0, n_outer=256, n_pores=6, n_per_pore=32)
    f = si.pipe_bc(g).reshape(-1)
    ref = O.solve_dense(g, f)
    with S.Geometry(g) as G:
        S.stokes_precond_setup_twogrid_ex(G.handle, 4, S.STOKES_TG_COARSE_LU)
        sig = np.zeros_like(f)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, f, sig, tol=1e-11, restart=100,
                                                  precision=S.STOKES_DF64)
        assert code == S.STOKES_OK and rr <= 1e-11
        assert rel(sig, ref) < 1e-9
        with pytest.raises(S.StokesError):
            S.stokes_precond_setup_twogrid_ex(G.handle, 4, 7)


def test_two_grid_triangular_solve_with_more_tiles_than_ctas(S, dev):
    """The persistent triangular solve on a float coarse LU of 11,776 rows
    (184 tiles of 64 for 152 CTAs, so CTAs own several tiles): two applies
    give bit-identical results (each CTA's sums run in a fixed order, so a
    missed wait would show as a difference), and the result agrees with the
    explicit float inverse formed from the same factors to float rounding
    times the coarse operator's conditioning (both are float: 1e-2)."""
    g = si.batch_geometry(3, n_pores=120, n_per_pore=64, n_outer=4096)
    assert g.n_nodes > 152 * 64
    v = torch.tensor(si.random_density(g, 8).reshape(-1), device=dev)
    out = {}
    for mode in (S.STOKES_TG_COARSE_LU, S.STOKES_TG_COARSE_INVERSE):
        with S.Geometry(g) as G:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, mode)
            zs = []
            for _ in range(2):  # the second apply reuses the flags with a new generation
                z = torch.empty_like(v)
                S.stokes_precond_apply(G.handle, v, z)
                zs.append(z)
            torch.cuda.synchronize()
            assert torch.equal(zs[0], zs[1])
            out[mode] = zs[0].cpu().numpy()
    assert rel(out[S.STOKES_TG_COARSE_LU], out[S.STOKES_TG_COARSE_INVERSE]) < 1e-2


def test_block_diagonal_triangular_solve_many_tiles_fp64(S, dev):
    """The FP64 wall block of a 5000-node wall (10,000 rows: 157 tiles for
    152 CTAs) applied by the persistent triangular solve equals the oracle's
    LAPACK block solve."""
    g = si.assemble_geometry([], si.superellipse_curve(8.0, 1.0, 5000), (8.0, 1.0, 8))
    v = np.random.default_rng(11).standard_normal(2 * g.n_nodes)
    ref = O.BlockDiagonal(g).apply(v)
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        z = np.empty_like(v)
        S.stokes_precond_apply(G.handle, v, z)
    assert rel(z, ref) < 1e-11


def test_two_grid_tensor_core_lu_matches_cuda_core_lu(S, dev, monkeypatch):
    """The coarse LU with its trailing updates on the tensor cores (three
    TF32 products, tcgen05) against the same LU with the CUDA-core float
    GEMM, on the 1152-node pipe: the two-grid applies agree to float
    rounding times the coarse operator's conditioning (1e-3)."""
    g = si.cached_geometry("pipe10", 0)
    v = torch.tensor(si.random_density(g, 9).reshape(-1), device=dev)
    out = {}
    for gemm in ("tc", "simt"):
        if gemm == "simt":
            monkeypatch.setenv("STOKES_TG_GEMM", "simt")
        with S.Geometry(g) as G:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_INVERSE)
            z = torch.empty_like(v)
            S.stokes_precond_apply(G.handle, v, z)
            torch.cuda.synchronize()
            out[gemm] = z.cpu().numpy()
    assert np.isfinite(out["tc"]).all()
    assert rel(out["tc"], out["simt"]) < 1e-3


def test_two_grid_tensor_core_lu_unaligned_column_stride(S, dev, monkeypatch):
    """A coarse LU of 346 rows (173 coarse nodes: 1384-byte columns, not a
    multiple of 16, so the tensor-core update's epilogue loads and stores C
    itself instead of reducing into it through TMA): the two-grid applies
    with tensor-core and CUDA-core trailing updates agree to 1e-3, and both
    match the oracle's two-grid apply to the same tolerance."""
    g = si.pipe10_geometry(2, n_outer=256, n_pores=5, n_per_pore=18)
    assert (g.n_nodes // 2) % 2 == 1
    v = np.random.default_rng(4).standard_normal(2 * g.n_nodes)
    ref = O.TwoGrid(g, 2).apply(v)
    out = {}
    for gemm in ("tc", "simt"):
        if gemm == "simt":
            monkeypatch.setenv("STOKES_TG_GEMM", "simt")
        with S.Geometry(g) as G:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_INVERSE)
            z = np.empty_like(v)
            S.stokes_precond_apply(G.handle, v, z)
            out[gemm] = z
    assert rel(out["tc"], out["simt"]) < 1e-3
    assert rel(out["tc"], ref) < 1e-3


def test_two_grid_tensor_core_lu_solve_on_many_tiles(S, dev, monkeypatch):
    """On a 11,776-node geometry (coarse LU of 11,776 rows, 92 x 92 output
    tiles per early trailing update, several per CTA) the coarse operator is
    ill conditioned enough that two float LUs differ by ~1e-3 in an apply;
    what matters is the preconditioner: both two-grid FGMRES solves reach
    1e-9 and take the same number of iterations to within 10 %."""
    g = si.batch_geometry(3, n_pores=120, n_per_pore=64, n_outer=4096)
    f = torch.tensor(si.pipe_bc(g).reshape(-1), device=dev)
    its = {}
    for gemm in ("tc", "simt"):
        if gemm == "simt":
            monkeypatch.setenv("STOKES_TG_GEMM", "simt")
        with S.Geometry(g) as G:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)
            x = torch.zeros_like(f)
            code, it, rr, _ = S.stokes_gmres_solve(G.handle, f, x, tol=1e-9, restart=300, max_iter=3000,
                                                   precision=S.STOKES_DF64)
            assert code == S.STOKES_OK and rr <= 1e-9, (gemm, code, rr)
            its[gemm] = it
    assert abs(its["tc"] - its["simt"]) <= max(2, 0.1 * its["simt"]), its


def test_two_grid_rejects_bad_coarsening(S, dev):
    g = si.pipe10_geometry(0, n_outer=96, n_pores=2, n_per_pore=24)
    with S.Geometry(g) as G:
        with pytest.raises(S.StokesError) as e:
            S.stokes_precond_setup_twogrid(G.handle, 5)    # 24 not a multiple of 5
        assert e.value.code == S.STOKES_EINVAL
        with pytest.raises(S.StokesError):
            S.stokes_precond_setup_twogrid(G.handle, 4)    # 24 / 4 = 6 < 8 coarse nodes


def test_full_size_two_grid_solve_reaches_tolerance(S, dev):
    """The benchmark's solve (136,192 nodes, two-grid q = 4 with the coarse LU
    applied by triangular solves, double-float FGMRES): status OK at the 1e-8
    true residual, which the FP64 operator confirms; the residual at sampled
    nodes from the oracle's matrix-free rows agrees with the GPU residual
    there; the velocity at sampled interior points equals the oracle's
    velocity of the GPU density."""
    g = si.cached_geometry("pipe1000", 0)
    f = si.pipe_bc(g).reshape(-1)
    with S.Geometry(g) as G:
        S.stokes_precond_setup_twogrid(G.handle, 4)
        ft = torch.tensor(f, device=dev)
        sig = torch.zeros_like(ft)
        code, iters, rr, _ = S.stokes_gmres_solve(G.handle, ft, sig, tol=1e-8, restart=600, max_iter=2000,
                                                  precision=S.STOKES_DF64)
        assert code == S.STOKES_OK and rr <= 1e-8
        assert iters < 200
        y = torch.empty_like(ft)
        S.stokes_matvec(G.handle, sig, y, S.STOKES_FP64)
        res = (ft - y).cpu().numpy()
        assert np.linalg.norm(res) / np.linalg.norm(f) <= 1.0001e-8
        s_h = sig.cpu().numpy()
        idx = np.random.default_rng(4).choice(g.n_nodes, 24, replace=False)
        rows = O.apply_rows(g, s_h, idx)                        # (24, 2)
        res_or = f.reshape(-1, 2)[idx] - rows
        # the oracle confirms small residuals at those nodes; both evaluations
        # are cancellations of O(|A||sigma|) terms, so they agree to a few
        # 1e-16 |A||sigma| (|sigma| is ~1e5 times |f| on this system)
        assert np.abs(res_or).max() <= 1e-7 * np.abs(f).max()
        scale = np.abs(rows).max() + np.abs(f).max()
        assert np.abs(res_or - res.reshape(-1, 2)[idx]).max() < 1e-9 * scale
        T = si.interior_targets(g, 16, min_dist=0.05, seed=5)
        u = np.empty(T.size)
        S.stokes_eval_velocity(G.handle, sig, T.reshape(-1), u, S.STOKES_FP64)
        uref = O.velocity(g, s_h, T)
        assert rel(u, uref) < 1e-9
