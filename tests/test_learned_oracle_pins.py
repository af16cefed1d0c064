"""Pins of the learned coarse correction's CPU oracle (oracle.learned_coarse)
against closed forms, library routines and finite differences. A dropped
term, a wrong sign or scale, or a transposed operand in any of its pieces
fails one of them (the planted-mistake tests check that they would)."""
import math

import numpy as np
import pytest

import oracle as O
import stokes_inputs as si
from oracle import learned_coarse as LC


@pytest.fixture(scope="module")
def geom_A():
    g = si.pipe10_geometry(0, n_outer=256, n_pores=6, n_per_pore=32)
    return g, O.assemble(g)


def test_rigid_modes_are_orthogonal_with_perimeter_norms(geom_A):
    """Z^T W Z = diag(L_k) (x) I_3: translations and the rotation
    (x - c)^perp / r all have squared W-norm L_k = 2 pi r_k on a circle, and
    they are W-orthogonal (the trapezoid rule integrates the trigonometric
    products exactly)."""
    g, _ = geom_A
    Z = LC.rigid_modes(g)
    G = Z.T @ (LC.weight_diag(g)[:, None] * Z)
    L = np.repeat([2 * math.pi * g.radii[k] for k in LC.pore_ids(g)], 3)
    assert np.abs(G - np.diag(L)).max() < 1e-13


def test_galerkin_self_blocks_have_the_closed_form(geom_A):
    """On its own pore the jump plus the double layer of a rigid motion
    vanishes (the constant-density identity seen from the fluid side), so
    only the pore's own Stokeslet and rotlet remain: with L = 2 pi r the
    self block of E is diag((L^2 / 4 pi)(1/2 - log r), same, L^2 / 4 pi)."""
    g, A = geom_A
    E = LC.coarse_operator(g, A)
    for p, k in enumerate(LC.pore_ids(g)):
        r = g.radii[k]
        L = 2 * math.pi * r
        t = L * L / (4 * math.pi) * (0.5 - math.log(r))
        want = np.diag([t, t, L * L / (4 * math.pi)])
        assert np.abs(E[3 * p:3 * p + 3, 3 * p:3 * p + 3] - want).max() < 1e-11 * t


def test_two_level_apply_inverts_A_on_the_coarse_range_and_reduces_to_bd(geom_A):
    """With C = E^-1: P^-1 (A Z v) = Z v for every coarse v. With C = 0: the
    block-diagonal preconditioner."""
    g, A = geom_A
    E = LC.coarse_operator(g, A)
    Z = LC.rigid_modes(g)
    bd = O.BlockDiagonal(g)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(E.shape[0])
    z = LC.two_level_apply(g, np.linalg.inv(E), A @ (Z @ v), A, bd)
    assert np.linalg.norm(z - Z @ v) < 1e-11 * np.linalg.norm(Z @ v)
    r = rng.standard_normal(A.shape[0])
    assert np.abs(LC.two_level_apply(g, np.zeros_like(E), r, A, bd) - bd.apply(r)).max() < 1e-13


def test_exact_two_level_preconditioner_beats_block_diagonal(geom_A):
    g, A = geom_A
    f = si.pipe_bc(g).reshape(-1)
    bd = O.BlockDiagonal(g)
    C = np.linalg.inv(LC.coarse_operator(g, A))
    r_bd = O.gmres(lambda v: A @ v, f, tol=1e-10, restart=300, apply_M=bd.apply)
    r_2l = O.gmres(lambda v: A @ v, f, tol=1e-10, restart=300, apply_M=lambda v: LC.two_level_apply(g, C, v, A, bd))
    assert r_2l["relres"] <= 1e-10 and r_2l["iters"] < r_bd["iters"]
    assert np.linalg.norm(r_2l["x"] - np.linalg.solve(A, f)) < 1e-8 * np.linalg.norm(r_2l["x"])


def test_nearest_neighbours_match_a_kd_tree():
    """Against scipy's k-d tree (an independent library routine), on a
    geometry with more than 16 pores."""
    from scipy.spatial import cKDTree
    g = si.batch_small_geometry(0)
    nb = LC.nearest_neighbours(g)
    c = g.centres[LC.pore_ids(g)]
    d, idx = cKDTree(c).query(c, k=LC.K_NBRS + 1)
    assert np.array_equal(nb, idx[:, 1:])
    F = LC.pore_features(g)
    assert np.allclose(F[:, 3:5], c[idx[:, 1]] - c)


def test_neighbour_lists_pad_small_geometries(geom_A):
    g, _ = geom_A
    nb = LC.nearest_neighbours(g)
    M = g.n_pores
    assert (nb[:, M - 1:] == -1).all() and (nb[:, :M - 1] >= 0).all()
    T, mask = LC.coarse_targets(g)
    assert mask[:, :9 * M].all() and not mask[:, 9 * M:].any()


def test_sparse_inverse_of_the_full_pattern_is_exact(geom_A):
    """With fewer than 17 pores the pattern holds every block, so the
    targets reassemble E^-1 exactly."""
    g, A = geom_A
    Einv = np.linalg.inv(LC.coarse_operator(g, A))
    T, _ = LC.coarse_targets(g, Einv)
    assert np.abs(LC.assemble_sparse_inverse(g, T) - Einv).max() < 1e-15 * np.abs(Einv).max()


def _small_net(rng, n_in=5, hidden=8, n_out=4):
    shapes = [(n_in, hidden), (hidden, hidden), (hidden, n_out)]
    P = np.concatenate([np.concatenate([rng.standard_normal(i * j) / math.sqrt(i), 0.1 * rng.standard_normal(j)])
                        for i, j in shapes])
    return P, shapes


def _with_shapes(shapes, fn, *a, **kw):
    old = LC.layer_shapes
    LC.layer_shapes = lambda *x, **y: shapes
    try:
        return fn(*a, **kw)
    finally:
        LC.layer_shapes = old


def test_gradients_match_central_finite_differences():
    rng = np.random.default_rng(4)
    P, shapes = _small_net(rng)
    X = rng.standard_normal((7, 5))
    T = rng.standard_normal((7, 4))
    mask = (rng.uniform(size=(7, 4)) > 0.3).astype(float)
    L, g = _with_shapes(shapes, LC.loss_and_grads, P, X, T, mask)
    h = 1e-6
    fd = np.empty_like(P)
    for i in range(P.size):
        e = np.zeros_like(P)
        e[i] = h
        fd[i] = (_with_shapes(shapes, LC.loss_and_grads, P + e, X, T, mask)[0] -
                 _with_shapes(shapes, LC.loss_and_grads, P - e, X, T, mask)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_dropped_relu_mask_fails_the_finite_difference_pin():
    """Planted mistake (on a copy): the hidden layers' ReLU derivative left
    out of backpropagation."""
    rng = np.random.default_rng(4)
    P, shapes = _small_net(rng)
    X = rng.standard_normal((7, 5))
    T = rng.standard_normal((7, 4))
    mask = np.ones((7, 4))

    def wrong(params, X, T, mask):
        Y, cache = LC.forward(params, X)
        cnt = mask.sum()
        diff = (Y - T) * mask
        g = 2.0 * diff / cnt
        grads = []
        for li in range(len(cache) - 1, -1, -1):
            h, W, z = cache[li]
            grads.append((h.T @ g, g.sum(0)))
            g = g @ W.T
        return float((diff * diff).sum() / cnt), LC.pack(grads[::-1])

    _, g = _with_shapes(shapes, wrong, P, X, T, mask)
    _, g_ok = _with_shapes(shapes, LC.loss_and_grads, P, X, T, mask)
    assert np.abs(g - g_ok).max() > 1e-3


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0]])  # two ties
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(LC.bf16_round(x), want)


def test_first_adam_step_moves_each_weight_by_the_learning_rate():
    """m_hat = g and v_hat = g^2 after one step, so w -= lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    P = rng.standard_normal(50)
    g = rng.standard_normal(50)
    P1, m, v = LC.adam_step(P, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.abs(P1 - (P - 1e-3 * g / (np.abs(g) + 1e-8))).max() < 1e-15
