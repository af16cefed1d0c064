"""Batched operator and lockstep solver over several geometries and
right-hand sides, through the C ABI, against the CPU oracle.

Geometries of uneven sizes (ragged component sizes, an outer-only domain,
the 1152-node pipe) so that the persistent kernel's work items cover tails
of target blocks and source ranges of every geometry.
"""
import numpy as np
import pytest

import oracle as O
import stokes_inputs as si


def _ragged():
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    return si.assemble_geometry(pores, si.superellipse_curve(3.0, 1.0, 203), (3.0, 1.0, 8))


def _outer_only():
    return si.assemble_geometry([], si.superellipse_curve(2.0, 1.0, 130), (2.0, 1.0, 8))


def _geoms():
    return [_ragged(), si.pipe10_geometry(1, n_outer=128, n_pores=3, n_per_pore=32), _outer_only(),
            si.cached_geometry("pipe10", 0)]


def _rhs(g, r):
    if r == 0:
        return (si.pipe_bc(g) if g.n_pores else si.shear_bc(g)).reshape(-1)
    if r == 1:
        return (si.reversed_pipe_bc(g) if g.n_pores else si.translation_bc(g)).reshape(-1)
    if r == 2:
        return si.outer_shear_bc(g).reshape(-1)
    return si.stokeslet_rotlet_bc(g, seed=r).reshape(-1)


def _rel(a, b):
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not b.LIB.exists():
        b.build()
    import paper_1609_04484_gb300 as S
    return S


def test_batch_calls_validate_arguments_without_gpu(S):
    P = S.ctypes.c_void_p
    arr = (P * 1)(None)
    assert S.lib.stokes_batch_matvec(arr, 1, 1, arr, arr, S.STOKES_FP32) == S.STOKES_EINVAL
    assert S.lib.stokes_batch_matvec(None, 1, 1, arr, arr, S.STOKES_FP32) == S.STOKES_EINVAL
    assert S.lib.stokes_batch_solve(arr, 0, 1, arr, 1e-8, 50, 100, S.STOKES_DF64, arr, None, None,
                                    None) == S.STOKES_EINVAL


@pytest.fixture(scope="module")
def gpu(S):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("prec,bound", [("FP32", 2e-6), ("DF64", 1e-12)])
@pytest.mark.parametrize("R", [1, 3, 4])
def test_batch_matvec_matches_oracle(S, gpu, prec, bound, R):
    torch = gpu
    dev = torch.device("cuda:0")
    geoms = _geoms()
    p = getattr(S, "STOKES_" + prec)
    Gs = [S.Geometry(g) for g in geoms]
    try:
        sig, ys, refs, single = [], [], [], []
        for k, g in enumerate(geoms):
            for r in range(R):
                s = si.random_density(g, 10 * k + r).reshape(-1)
                refs.append(O.matvec(g, s))
                sig.append(torch.tensor(s, device=dev))
                ys.append(torch.empty_like(sig[-1]))
                y1 = torch.empty_like(sig[-1])
                S.stokes_matvec(Gs[k].handle, sig[-1], y1, p)
                single.append(y1)
        S.stokes_batch_matvec([G.handle for G in Gs], R, sig, ys, p)
        torch.cuda.synchronize()
        for s_idx, (y, ref, y1) in enumerate(zip(ys, refs, single)):
            assert _rel(y.cpu().numpy(), ref) < bound, s_idx
            # same arithmetic as the single-geometry kernel up to the partial-sum order
            assert _rel(y.cpu().numpy(), y1.cpu().numpy()) < bound / 10, s_idx
    finally:
        for G in Gs:
            G.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["DF64", "MIXED_IR"])
def test_batch_solve_matches_dense_oracle(S, gpu, prec):
    """4 geometries x 4 right-hand sides (pipe, reversed pipe, wall shear,
    Stokeslet/rotlet data): every density equals the dense LU solution; the
    outer-only geometry runs without a preconditioner, the 1152-node pipe
    with the two-grid one, the others with their block diagonal."""
    torch = gpu
    dev = torch.device("cuda:0")
    geoms = _geoms()
    R = 4
    Gs = [S.Geometry(g) for g in geoms]
    try:
        for k, G in enumerate(Gs):
            if k == 3:
                S.stokes_precond_setup_twogrid(G.handle, 4)
            elif geoms[k].n_pores:
                S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
        fs, xs, refs = [], [], []
        for g in geoms:
            for r in range(R):
                f = _rhs(g, r)
                refs.append(O.solve_dense(g, f))
                fs.append(torch.tensor(f, device=dev))
                xs.append(torch.zeros_like(fs[-1]))
        iters, relres, status = S.stokes_batch_solve([G.handle for G in Gs], R, fs, xs, tol=1e-11, restart=40,
                                                     max_iter=3000, precision=getattr(S, "STOKES_" + prec))
        for s_idx in range(len(fs)):
            assert status[s_idx] == S.STOKES_OK, (s_idx, status, relres)
            assert relres[s_idx] <= 1e-11, (s_idx, relres[s_idx])
            assert _rel(xs[s_idx].cpu().numpy(), refs[s_idx]) < 1e-8, s_idx
            assert iters[s_idx] > 0
    finally:
        for G in Gs:
            G.close()


@pytest.mark.gpu
def test_batch_solve_agrees_with_single_solves(S, gpu):
    """Lockstep DF64 FGMRES of a batch gives each system the iteration count
    of the same solve run alone (flexible GMRES, block diagonal, restart 40)
    within 2, and starts from the given initial guess."""
    torch = gpu
    dev = torch.device("cuda:0")
    geoms = [si.cached_geometry("pipe10", 0), si.pipe10_geometry(2, n_outer=256, n_pores=5, n_per_pore=32)]
    Gs = [S.Geometry(g) for g in geoms]
    try:
        fs, xs, single = [], [], []
        for k, (g, G) in enumerate(zip(geoms, Gs)):
            S.stokes_precond_setup(G.handle, S.STOKES_PC_BLOCKDIAG)
            for r in range(2):
                f = torch.tensor(_rhs(g, r), device=dev)
                x1 = torch.zeros_like(f)
                code, it, rr, _ = S.stokes_gmres_solve(G.handle, f, x1, tol=1e-10, restart=40, max_iter=2000,
                                                       precision=S.STOKES_DF64)
                assert code == S.STOKES_OK
                single.append((it, x1))
                fs.append(f)
                xs.append(torch.zeros_like(f))
        iters, relres, status = S.stokes_batch_solve([G.handle for G in Gs], 2, fs, xs, tol=1e-10, restart=40,
                                                     max_iter=2000, precision=S.STOKES_DF64)
        for s_idx, (it, x1) in enumerate(single):
            assert status[s_idx] == S.STOKES_OK and relres[s_idx] <= 1e-10
            assert abs(iters[s_idx] - it) <= 2, (iters, [s[0] for s in single])
            assert _rel(xs[s_idx].cpu().numpy(), x1.cpu().numpy()) < 1e-8
        # warm start from the solution: converged at once, no iterations
        iters2, relres2, status2 = S.stokes_batch_solve([G.handle for G in Gs], 2, fs, xs, tol=1e-10, restart=40,
                                                        max_iter=2000, precision=S.STOKES_DF64)
        assert all(i == 0 for i in iters2) and all(st == S.STOKES_OK for st in status2)
    finally:
        for G in Gs:
            G.close()


@pytest.mark.gpu
def test_batch_rejects_host_arrays_and_mixed_streams(S, gpu):
    torch = gpu
    g = si.pipe10_geometry(0, n_outer=96, n_pores=2, n_per_pore=16)
    G = S.Geometry(g)
    st = torch.cuda.Stream()
    G2 = S.Geometry(g, stream=st.cuda_stream)
    try:
        s = np.zeros(2 * g.n_nodes)
        with pytest.raises(S.StokesError) as e:
            S.stokes_batch_matvec([G.handle], 1, [s], [np.empty_like(s)], S.STOKES_FP32)
        assert e.value.code == S.STOKES_EINVAL
        d = torch.zeros(2 * g.n_nodes, dtype=torch.float64, device="cuda:0")
        with pytest.raises(S.StokesError):
            S.stokes_batch_matvec([G.handle, G2.handle], 1, [d, d.clone()], [d.clone(), d.clone()], S.STOKES_FP32)
        with pytest.raises(S.StokesError):
            S.stokes_batch_matvec([G.handle], 5, [d] * 5, [d.clone() for _ in range(5)], S.STOKES_FP32)
        with pytest.raises(S.StokesError):
            S.stokes_batch_matvec([G.handle], 1, [d], [d.clone()], S.STOKES_FP64)
    finally:
        G.close()
        G2.close()
