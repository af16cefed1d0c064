"""The learned coarse correction on the GPU (through the C ABI) against its
CPU oracle (oracle.learned_coarse).

Tolerances:
* Y = A Z and E = Z^T W A Z: FP64 pair sums in another order, 1e-12
  relative (as the operator's parity tests).
* Features: float32 copies of FP64 values, 1e-6; neighbour lists exact.
* Network: the oracle rounds to bfloat16 where the GPU stores values and
  multiplies exactly; the GPU accumulates in float, so an activation near a
  bfloat16 rounding boundary can round the other way (one bf16 ulp, 2^-8).
  Outputs and gradients therefore agree to about 1e-3 relative (bounds below
  1e-2, stated per check), far below the 1e-1 bfloat16 effect of dropping the
  rounding (checked against the unrounded oracle).
* Adam: float moments against FP64, 1e-5.
* Solves with either coarse level reach the dense solution to 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import stokes_inputs as si
from oracle import learned_coarse as LC

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    return S


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ragged():
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    return si.assemble_geometry(pores, si.superellipse_curve(3.0, 1.0, 203), (3.0, 1.0, 8))


GEOMS = {
    "small": lambda: si.pipe10_geometry(0, n_outer=256, n_pores=6, n_per_pore=32),
    "ragged": _ragged,
    "long": lambda: si.coarse_train_geometry(1),
}


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_coarse_operator_matches_oracle(S, which):
    g = GEOMS[which]()
    A = O.assemble(g)
    Z = LC.rigid_modes(g)
    with S.Geometry(g) as G:
        Y, E = S.stokes_coarse_operator(G.handle, g.n_pores)
    assert rel(Y, A @ Z) < 1e-12
    assert rel(E, LC.coarse_operator(g, A)) < 1e-12


@pytest.mark.parametrize("which", ["small", "ragged", "long"])
def test_coarse_features_match_oracle(S, which):
    g = GEOMS[which]()
    with S.Geometry(g) as G:
        X, nb = S.stokes_coarse_features(G.handle, g.n_pores)
    assert np.array_equal(nb, LC.nearest_neighbours(g))
    assert rel(X, LC.pore_features(g)) < 1e-6


def _model(S, seed=0):
    return S.stokes_coarse_model_create(si.mlp_initial_params(seed))


def _batch(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, 35)).astype(np.float32)
    T = rng.standard_normal((rows, 153)).astype(np.float32)
    mask = (rng.uniform(size=(rows, 153)) > 0.25).astype(np.float32)
    return X, T, mask


@pytest.mark.parametrize("rows", [1, 77, 300])
def test_network_forward_matches_oracle(S, rows):
    m = _model(S)
    try:
        X, _, _ = _batch(rows, rows)
        y = np.zeros((rows, 153), dtype=np.float32)
        S.stokes_coarse_model_forward(m, X, y)
        P = si.mlp_initial_params(0).astype(np.float64)
        ref, _ = LC.forward(P, X.astype(np.float64), bf16=True)
        assert rel(y, ref) < 5e-3
        unrounded, _ = LC.forward(P, X.astype(np.float64), bf16=False)
        assert rel(y, unrounded) > 3 * rel(y, ref)  # the rounding emulation is what matches
    finally:
        S.stokes_coarse_model_destroy(m)


def test_network_gradients_match_oracle(S):
    m = _model(S, 1)
    try:
        X, T, mask = _batch(300, 5)
        g = np.zeros(S.stokes_coarse_model_num_params(), dtype=np.float32)
        loss = S.stokes_coarse_model_loss_grad(m, X, T, mask, g)
        P = si.mlp_initial_params(1).astype(np.float64)
        L_ref, g_ref = LC.loss_and_grads(P, X.astype(np.float64), T.astype(np.float64), mask.astype(np.float64),
                                         bf16=True)
        assert abs(loss - L_ref) < 1e-3 * L_ref
        offs = np.cumsum([0, 35 * 256, 256, 256 * 256, 256, 256 * 153, 153])
        for a, b in zip(offs[:-1], offs[1:]):  # each weight matrix and bias
            assert rel(g[a:b], g_ref[a:b]) < 1e-2, (a, b, rel(g[a:b], g_ref[a:b]))
        assert rel(g, g_ref) < 5e-3
    finally:
        S.stokes_coarse_model_destroy(m)


def test_adam_steps_match_oracle(S):
    m = _model(S, 2)
    try:
        n = S.stokes_coarse_model_num_params()
        rng = np.random.default_rng(9)
        P = si.mlp_initial_params(2).astype(np.float64)
        mo, vo = np.zeros(n), np.zeros(n)
        for t in (1, 2, 3):
            gr = (rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 0, n)).astype(np.float32)
            S.stokes_coarse_model_adam_step(m, gr, 1e-3)
            P, mo, vo = LC.adam_step(P, gr.astype(np.float64), mo, vo, t, 1e-3)
        got = np.zeros(n, dtype=np.float32)
        S.stokes_coarse_model_save(m, got)
        assert np.abs(got - P).max() < 1e-5 * np.abs(P).max()
    finally:
        S.stokes_coarse_model_destroy(m)


def test_exact_two_level_apply_matches_oracle(S):
    g = GEOMS["small"]()
    A = O.assemble(g)
    C = np.linalg.inv(LC.coarse_operator(g, A))
    r = si.random_density(g, 3).reshape(-1)
    ref = LC.two_level_apply(g, C, r, A, O.BlockDiagonal(g))
    with S.Geometry(g) as G:
        S.stokes_precond_setup(G.handle, S.STOKES_PC_BD_COARSE)
        z = np.zeros_like(r)
        S.stokes_precond_apply(G.handle, r, z)
    assert rel(z, ref) < 1e-11


def test_exact_two_level_solve_matches_dense_with_fewer_iterations(S):
    g = si.cached_geometry("pipe10", 0)
    f = si.pipe_bc(g).reshape(-1)
    x_ref = O.solve_dense(g, f)
    its = {}
    for name, kind in (("bd", S.STOKES_PC_BLOCKDIAG), ("coarse", S.STOKES_PC_BD_COARSE)):
        with S.Geometry(g) as G:
            S.stokes_precond_setup(G.handle, kind)
            x = np.zeros_like(f)
            code, it, rr, _ = S.stokes_gmres_solve(G.handle, f, x, tol=1e-11, restart=300, max_iter=2000)
            assert code == S.STOKES_OK and rr <= 1e-11
            assert rel(x, x_ref) < 1e-10
            its[name] = it
    assert its["coarse"] < 0.8 * its["bd"], its


def test_learned_coarse_training_and_solve(S):
    """Train on 24 geometries of the pipe10 family: the loss falls; a
    held-out solve with the learned coarse level reaches the dense solution;
    the saved and reloaded model gives the same solve."""
    m = _model(S, 3)
    m2 = None
    try:
        for i in range(24):
            with S.Geometry(si.coarse_train_geometry(2 * i)) as G:
                S.stokes_coarse_model_add_geometry(m, G.handle)
        assert S.stokes_coarse_model_num_samples(m) == 240
        l0 = S.stokes_coarse_model_train(m, 1, 1e-3)
        l1 = S.stokes_coarse_model_train(m, 300, 1e-3)
        assert l1 < 0.5 * l0, (l0, l1)
        g = si.coarse_eval_geometry(0)
        f = si.pipe_bc(g).reshape(-1)
        x_ref = O.solve_dense(g, f)
        res = []
        for model in (m, "reload"):
            if model == "reload":
                P = np.zeros(S.stokes_coarse_model_num_params(), dtype=np.float32)
                st = np.zeros(S.COARSE_STATS, dtype=np.float32)
                S.stokes_coarse_model_save(m, P, st)
                m2 = S.stokes_coarse_model_create(si.mlp_initial_params(0))
                S.stokes_coarse_model_load(m2, P, st)
                model = m2
            with S.Geometry(g) as G:
                S.stokes_precond_setup(G.handle, S.STOKES_PC_BD_LEARNED, model)
                x = np.zeros_like(f)
                code, it, rr, _ = S.stokes_gmres_solve(G.handle, f, x, tol=1e-11, restart=300, max_iter=2000)
                assert code == S.STOKES_OK and rr <= 1e-11
                assert rel(x, x_ref) < 1e-10
                res.append(it)
        assert res[0] == res[1]
    finally:
        S.stokes_coarse_model_destroy(m)
        if m2:
            S.stokes_coarse_model_destroy(m2)


def test_learned_setup_needs_a_trained_model(S):
    m = _model(S)
    try:
        with S.Geometry(GEOMS["small"]()) as G:
            with pytest.raises(S.StokesError) as e:
                S.stokes_precond_setup(G.handle, S.STOKES_PC_BD_LEARNED, m)
            assert e.value.code == S.STOKES_ESTATE
            with pytest.raises(S.StokesError):
                S.stokes_precond_setup(G.handle, S.STOKES_PC_BD_LEARNED, None)
    finally:
        S.stokes_coarse_model_destroy(m)
