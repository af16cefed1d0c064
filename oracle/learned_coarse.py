"""Plain FP64 CPU oracle of the learned coarse correction (not in the paper).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module. The CUDA library
never calls it and shares no code with it; the only thing both sides use
is the seeded input generator (``stokes_inputs``), which holds no method
arithmetic (it draws the geometries and the network's initial weights).

What it computes:

* Coarse space. The completed double-layer operator (Sec. 2.1: the rank-3
  null space of each component removed by a Stokeslet and a rotlet at the
  pore centre) couples the pores through the moments lambda_k and xi_k of
  the density. The coarse space Z (2N x 3M) holds, for each pore k, the
  three rigid-motion densities on its nodes: e_x, e_y and the rotation
  (x - c_k)^perp / r_k, with (a, b)^perp = (b, -a) as in Sec. 4.2 (zero on
  every other component) and r_k = L_k / (2 pi), L_k the sum of the pore's
  quadrature weights (its perimeter; the radius for a circle). With
  W = diag(w) on both vector components, Z^T W sigma gives lambda_k and
  xi_k / r_k.
* Galerkin coarse operator E = Z^T W A Z (3M x 3M), A the dense operator of
  Eq. 6 (``stokes_oracle.assemble``).
* Two-level preconditioner (coarse level first, then the block diagonal of
  Sec. 4.1 on what remains):
      c = C Z^T W r,   z = Z c + B^-1 (r - A Z c).
  With C = E^-1 it maps A Z v to Z v exactly for every coarse v; with C = 0
  it is the block-diagonal preconditioner.
* Learned C: for each pore k a network predicts the 3 x 3 blocks C[k, l]
  for l in {k} and the 16 pores nearest to it (the sparse pattern of a
  truncated E^-1), from the features [centre of k relative to the wall's
  half-extents (2), radius of k (1), offsets c_l - c_k of the 16 nearest
  pores (32)]. Network: 35 -> 256 -> 256 -> 153, ReLU after the first two
  layers, weights rounded to bfloat16; the training target is E^-1 on the
  pattern in the scaled form L_k L_l E^-1[k, l] (perimeter-weighted, so the
  targets of small and large pores are alike), standardised per output, and
  the loss the masked mean squared error. The optimiser is Adam (Kingma and
  Ba 2015).
"""
from __future__ import annotations

import numpy as np

from . import stokes_oracle as so

K_NBRS = 16
N_FEAT = 3 + 2 * K_NBRS            # 35
N_OUT = 9 * (K_NBRS + 1)           # 153
HIDDEN = 256


# ---------------------------------------------------------------------------
# Coarse space and Galerkin operator
# ---------------------------------------------------------------------------

def pore_ids(geom):
    return [k for k in range(geom.n_comp) if k != geom.outer_comp]


def perimeters(geom):
    """L_k = sum of the quadrature weights of each pore (pore order)."""
    return np.array([geom.weights[geom.comp_slice(k)].sum() for k in pore_ids(geom)])


def rigid_modes(geom):
    """Z (2N x 3M): columns 3p, 3p+1, 3p+2 of the p-th pore are e_x, e_y and
    (x - c)^perp / r on its nodes, r = L / (2 pi)."""
    pores = pore_ids(geom)
    L = perimeters(geom)
    Z = np.zeros((2 * geom.n_nodes, 3 * len(pores)))
    for p, k in enumerate(pores):
        sl = geom.comp_slice(k)
        idx = np.arange(sl.start, sl.stop)
        d = geom.nodes[sl] - geom.centres[k][None, :]
        r = L[p] / (2.0 * np.pi)
        Z[2 * idx, 3 * p] = 1.0
        Z[2 * idx + 1, 3 * p + 1] = 1.0
        Z[2 * idx, 3 * p + 2] = d[:, 1] / r
        Z[2 * idx + 1, 3 * p + 2] = -d[:, 0] / r
    return Z


def weight_diag(geom):
    return np.repeat(geom.weights, 2)


def coarse_operator(geom, A=None):
    """E = Z^T W A Z (dense; small N)."""
    if A is None:
        A = so.assemble(geom)
    Z = rigid_modes(geom)
    return Z.T @ (weight_diag(geom)[:, None] * (A @ Z))


def two_level_apply(geom, C, r, A=None, bd=None):
    """z = Z c + B^-1 (r - A Z c), c = C Z^T W r (B^-1: the block diagonal)."""
    if A is None:
        A = so.assemble(geom)
    if bd is None:
        bd = so.BlockDiagonal(geom)
    Z = rigid_modes(geom)
    r = np.asarray(r, dtype=np.float64).reshape(-1)
    c = C @ (Z.T @ (weight_diag(geom) * r))
    Zc = Z @ c
    return Zc + bd.apply(r - A @ Zc)


# ---------------------------------------------------------------------------
# Features, neighbour lists, targets
# ---------------------------------------------------------------------------

def nearest_neighbours(geom, k=K_NBRS):
    """(M, k) pore numbers (0..M-1 in pore order) of the k nearest other
    pores by centre distance, nearest first, ties to the smaller number;
    -1 where fewer than k other pores exist."""
    pores = pore_ids(geom)
    c = geom.centres[pores]
    M = len(pores)
    out = -np.ones((M, k), dtype=np.int64)
    for p in range(M):
        d2 = ((c - c[p]) ** 2).sum(1)
        order = sorted((d2[q], q) for q in range(M) if q != p)
        for j, (_, q) in enumerate(order[:k]):
            out[p, j] = q
    return out


def wall_half_extents(geom):
    sl = geom.comp_slice(geom.outer_comp)
    w = geom.nodes[sl]
    return 0.5 * (w[:, 0].max() - w[:, 0].min()), 0.5 * (w[:, 1].max() - w[:, 1].min())


def pore_features(geom, k=K_NBRS):
    """(M, 3 + 2k): [c_x / a, c_y / b, r, (c_l - c_k) for the k nearest l
    (zeros where absent)], a and b the wall's half-extents."""
    pores = pore_ids(geom)
    c = geom.centres[pores]
    a, b = wall_half_extents(geom)
    nb = nearest_neighbours(geom, k)
    F = np.zeros((len(pores), 3 + 2 * k))
    F[:, 0] = c[:, 0] / a
    F[:, 1] = c[:, 1] / b
    F[:, 2] = perimeters(geom) / (2.0 * np.pi)
    for p in range(len(pores)):
        for j in range(k):
            q = nb[p, j]
            if q >= 0:
                F[p, 3 + 2 * j:5 + 2 * j] = c[q] - c[p]
    return F


def coarse_targets(geom, Einv=None, k=K_NBRS):
    """Scaled blocks L_p L_q E^-1[p, q] on the pattern: T (M, 9 (k + 1)) with
    block j (j = 0: the pore itself, j >= 1: its j-th nearest pore q)
    flattened row-major, and the mask (M, 9 (k + 1)) of present blocks."""
    if Einv is None:
        Einv = np.linalg.inv(coarse_operator(geom))
    L = perimeters(geom)
    nb = nearest_neighbours(geom, k)
    M = nb.shape[0]
    T = np.zeros((M, 9 * (k + 1)))
    mask = np.zeros((M, 9 * (k + 1)))
    for p in range(M):
        cols = [p] + list(nb[p])
        for j, q in enumerate(cols):
            if q < 0:
                continue
            T[p, 9 * j:9 * j + 9] = L[p] * L[q] * Einv[3 * p:3 * p + 3, 3 * q:3 * q + 3].reshape(-1)
            mask[p, 9 * j:9 * j + 9] = 1.0
    return T, mask


def assemble_sparse_inverse(geom, Y, k=K_NBRS):
    """The dense 3M x 3M matrix C with the scaled blocks Y (M, 9 (k + 1))
    unscaled (divided by L_p L_q) at the pattern's positions, zeros elsewhere."""
    L = perimeters(geom)
    nb = nearest_neighbours(geom, k)
    M = nb.shape[0]
    C = np.zeros((3 * M, 3 * M))
    for p in range(M):
        for j, q in enumerate([p] + list(nb[p])):
            if q >= 0:
                C[3 * p:3 * p + 3, 3 * q:3 * q + 3] = Y[p, 9 * j:9 * j + 9].reshape(3, 3) / (L[p] * L[q])
    return C


# ---------------------------------------------------------------------------
# The network (FP64, optionally rounding to bfloat16 where the GPU stores it)
# ---------------------------------------------------------------------------

def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even), through
    float32 (inputs here are already float32-representable or their float32
    rounding is the first step the GPU takes too)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_shapes(n_in=N_FEAT, hidden=HIDDEN, n_out=N_OUT):
    return [(n_in, hidden), (hidden, hidden), (hidden, n_out)]


def unpack(params, shapes=None):
    """Flat parameter vector -> [(W (in x out), b (out))] per layer, in the
    order W1, b1, W2, b2, W3, b3 (each W row-major, in x out)."""
    shapes = shapes or layer_shapes()
    out, o = [], 0
    for i, j in shapes:
        W = np.asarray(params[o:o + i * j], dtype=np.float64).reshape(i, j)
        o += i * j
        b = np.asarray(params[o:o + j], dtype=np.float64)
        o += j
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def forward(params, X, bf16=False):
    """Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3. With bf16=True the input,
    the weights and the hidden activations are rounded to bfloat16 where the
    GPU stores them (products are exact here; the GPU accumulates in float).
    Returns Y and the cache for backward."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(params)
    h = rnd(X)
    cache = []
    for li, (W, b) in enumerate(layers):
        Wr = rnd(W)
        z = h @ Wr + b
        cache.append((h, Wr, z))
        if li < len(layers) - 1:
            h = rnd(np.maximum(z, 0.0))
        else:
            h = z
    return h, cache


def loss_and_grads(params, X, T, mask, bf16=False):
    """Masked mean squared error L = sum mask (Y - T)^2 / sum mask and its
    gradient with respect to the flat parameters (backpropagation; with
    bf16=True the output gradient and the hidden-layer gradients are
    rounded to bfloat16 where the GPU stores them)."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    Y, cache = forward(params, X, bf16)
    cnt = mask.sum()
    diff = (Y - T) * mask
    L = float((diff * diff).sum() / cnt)
    g = rnd(2.0 * diff / cnt)
    grads = []
    for li in range(len(cache) - 1, -1, -1):
        h, Wr, z = cache[li]
        if li < len(cache) - 1:
            g = rnd(g * (z > 0.0))
        gW = h.T @ g
        gb = g.sum(0)
        grads.append((gW, gb))
        g = g @ Wr.T
    return L, pack(grads[::-1])


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) of the flat parameters; t is the
    1-based step number. Returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grads
    v = b2 * v + (1.0 - b2) * grads * grads
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
