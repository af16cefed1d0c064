"""Plain FP64 CPU oracle for the second-kind double-layer Stokes system.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. The
CUDA library and its Python binding never call it, and it shares no code
with them: the only thing both sides use is the seeded input generator
(``stokes_inputs``), which holds none of the arithmetic below.

What it computes (numbers in brackets are the paper's sections/equations):

* Problem [Sec. 2, Eq. 1-2]: Stokes flow (mu = 1) in Omega = Omega_0 minus
  M circular pores, velocity f prescribed on the boundary Gamma.
* Representation: the double-layer potential of Sec. 2.1,
      D[s](x) = (1/pi) int_Gamma (r.n / rho^2) (r r^T / rho^2) s(y) ds_y,
  r = x - y, rho = |r|, n the unit normal pointing out of the fluid. The
  paper names D and notes it gives a second-kind equation whose
  conditioning is mesh independent, and that D has a rank-three null space
  per connected component that can be removed (Sec. 2.1). It then chooses
  the single layer; the double-layer system is what this code solves.
* Discretisation [Sec. 2.2, Eq. 5-6]: collocation at the quadrature nodes
  with trapezoid weights w_j (arclength x quadrature weight), giving a dense
  2N x 2N system f = A sigma with unknowns interleaved (sigma_x, sigma_y)
  per node, pores first, outer wall last.
* Velocity at interior points [Sec. 2.2, Eq. 7 with the double-layer kernel].

Readings where the paper is silent (each is a choice the CUDA path makes
identically):

R1 Orientation: n points out of the fluid (out of Omega_0 on Gamma_0, into
   each pore). kappa is the signed curvature along the traversal for which
   n is the tangent turned clockwise (Gamma_0 counter-clockwise, pores
   clockwise): kappa > 0 on the convex wall, kappa = -1/R on a pore.
R2 Diagonal (self) term: the double-layer kernel has a finite limit as y
   approaches x along a smooth curve, -(kappa(x) / (2 pi)) t t^T with
   t = (-n_y, n_x); the trapezoid rule uses it as the j = i entry.
R3 Jump: with n out of the fluid, the boundary value from the fluid side is
   u(x_i) = -sigma_i / 2 + (principal value of D[sigma])(x_i).
R4 Completion of each pore k (removes its rank-3 null space): add
   S(x, c_k) lambda_k + R(x, c_k) xi_k with
   S(x, c) = (1/4pi)(-log rho I + r r^T / rho^2),  R(x, c) = (1/4pi) r^perp / rho^2,
   r = x - c, (a, b)^perp = (b, -a) (the perp of Sec. 4.2),
   lambda_k = sum_{j in k} w_j sigma_j,  xi_k = sum_{j in k} w_j (x_j - c_k)^perp . sigma_j,
   c_k the pore centre.
R5 Outer wall (removes its rank-1 defect): for targets i on Gamma_0 add
   n_i sum_{j in Gamma_0} w_j n_j . sigma_j. It is a boundary-equation term
   only and is not part of the velocity.
R6 Preconditioning: block diagonal (one block per component, the
   restriction of A to that component, Sec. 4.1 footnote: assembled,
   factorised and inverted exactly), applied from the RIGHT by default so
   the GMRES residual is the true residual; LEFT is available as in
   Sec. 4.1. Stopping: relative residual <= tol (Sec. 4: 1e-8).
R7 GMRES(m) [Sec. 4, Saad-Schultz]: Arnoldi with modified Gram-Schmidt,
   Givens rotations, x0 = 0, restart every m steps, true residual checked at
   each restart.
"""
from __future__ import annotations

import math

import numpy as np

INV_PI = 1.0 / math.pi
INV_4PI = 1.0 / (4.0 * math.pi)


# ---------------------------------------------------------------------------
# Kernels
# ---------------------------------------------------------------------------

def dlp_kernel(targets, src_nodes, src_normals):
    """Double-layer kernel of Sec. 2.1 without the weight:
    K(x, y) = (1/pi) (r.n_y)(r r^T) / rho^4, r = x - y.
    Returns (T, S, 2, 2). Coincident points give NaN (callers exclude them)."""
    r = targets[:, None, :] - src_nodes[None, :, :]
    rho2 = (r * r).sum(-1)
    rn = (r * src_normals[None, :, :]).sum(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        coef = INV_PI * rn / (rho2 * rho2)
    return coef[..., None, None] * r[..., :, None] * r[..., None, :]


def self_blocks(geom):
    """Diagonal entries of the discrete double layer (reading R2):
    w_i * (-(kappa_i / (2 pi)) t_i t_i^T), t_i = (-n_y, n_x). Returns (N, 2, 2)."""
    t = np.stack([-geom.normals[:, 1], geom.normals[:, 0]], 1)
    coef = -geom.curvature * geom.weights / (2.0 * math.pi)
    return coef[:, None, None] * t[:, :, None] * t[:, None, :]


def stokeslet(points, c):
    """(1/4pi)(-log rho I + r r^T / rho^2), r = x - c. Returns (T, 2, 2)."""
    r = points - c[None, :]
    rho2 = (r * r).sum(1)
    out = (r[:, :, None] * r[:, None, :]) / rho2[:, None, None]
    out[:, 0, 0] -= 0.5 * np.log(rho2)
    out[:, 1, 1] -= 0.5 * np.log(rho2)
    return INV_4PI * out


def rotlet(points, c):
    """(1/4pi) r^perp / rho^2 with (a, b)^perp = (b, -a). Returns (T, 2)."""
    r = points - c[None, :]
    rho2 = (r * r).sum(1)
    return INV_4PI * np.stack([r[:, 1], -r[:, 0]], 1) / rho2[:, None]


def _blocks_to_matrix(B):
    """(T, S, 2, 2) blocks -> (2T, 2S) matrix with interleaved unknowns."""
    T, S = B.shape[:2]
    return B.transpose(0, 2, 1, 3).reshape(2 * T, 2 * S)


# ---------------------------------------------------------------------------
# Operator A (Eq. 6 for the double-layer system)
# ---------------------------------------------------------------------------

def operator_blocks(geom, rows, cols, completion=True, outer_fix=True, jump=True):
    """Blocks A[i, j] (2x2) for node index arrays rows x cols. Returns (R, C, 2, 2)."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    x_r = geom.nodes[rows]
    B = dlp_kernel(x_r, geom.nodes[cols], geom.normals[cols]) * geom.weights[cols][None, :, None, None]
    same = rows[:, None] == cols[None, :]
    B[same] = 0.0
    ri, ci = np.nonzero(same)
    if ri.size:
        diag = self_blocks(geom)[rows[ri]]
        if jump:
            diag = diag - 0.5 * np.eye(2)[None]
        B[ri, ci] += diag
    comp = geom.comp_of_node()
    if completion:
        for k in range(geom.n_comp):
            if k == geom.outer_comp:
                continue
            in_k = comp[cols] == k
            if not in_k.any():
                continue
            ck = geom.centres[k]
            Sk = stokeslet(x_r, ck)               # (R, 2, 2)
            Rk = rotlet(x_r, ck)                  # (R, 2)
            jc = cols[in_k]
            wj = geom.weights[jc]
            d = geom.nodes[jc] - ck[None, :]
            perp = np.stack([d[:, 1], -d[:, 0]], 1) * wj[:, None]     # (Ck, 2)
            B[:, in_k] += Sk[:, None, :, :] * wj[None, :, None, None]
            B[:, in_k] += Rk[:, None, :, None] * perp[None, :, None, :]
    if outer_fix:
        k0 = geom.outer_comp
        ri = comp[rows] == k0
        cj = comp[cols] == k0
        if ri.any() and cj.any():
            n_i = geom.normals[rows[ri]]
            wn_j = geom.normals[cols[cj]] * geom.weights[cols[cj]][:, None]
            sub = n_i[:, None, :, None] * wn_j[None, :, None, :]
            idx = np.ix_(np.nonzero(ri)[0], np.nonzero(cj)[0])
            B[idx] += sub
    return B


def assemble(geom, completion=True, outer_fix=True, jump=True):
    """Dense 2N x 2N matrix A (small N only: O(N^2) memory)."""
    n = geom.n_nodes
    idx = np.arange(n)
    return _blocks_to_matrix(operator_blocks(geom, idx, idx, completion, outer_fix, jump))


def moments(geom, sigma):
    """Per-pore lambda_k (2,) and xi_k, and the wall's s0 = sum w n.sigma (R4, R5)."""
    sigma = np.asarray(sigma).reshape(-1, 2)
    lam = np.zeros((geom.n_comp, 2))
    xi = np.zeros(geom.n_comp)
    s0 = 0.0
    for k in range(geom.n_comp):
        sl = geom.comp_slice(k)
        w = geom.weights[sl]
        if k == geom.outer_comp:
            s0 = float((w[:, None] * geom.normals[sl] * sigma[sl]).sum())
            continue
        d = geom.nodes[sl] - geom.centres[k][None, :]
        lam[k] = (w[:, None] * sigma[sl]).sum(0)
        xi[k] = float((w * (d[:, 1] * sigma[sl, 0] - d[:, 0] * sigma[sl, 1])).sum())
    return lam, xi, s0


def apply_rows(geom, sigma, rows, chunk=256):
    """Matrix-free rows of A sigma at node indices `rows`: (len(rows), 2).

    Direct sums over all sources, the diagonal (self + jump) entry, the pore
    completions from the moments and the wall term; used where N is too large
    to assemble."""
    sigma = np.asarray(sigma, dtype=np.float64).reshape(-1, 2)
    rows = np.asarray(rows)
    lam, xi, s0 = moments(geom, sigma)
    comp = geom.comp_of_node()
    ws = geom.weights[:, None] * sigma
    out = np.zeros((rows.size, 2))
    for a in range(0, rows.size, chunk):
        rr = rows[a:a + chunk]
        x = geom.nodes[rr]
        r = x[:, None, :] - geom.nodes[None, :, :]
        rho2 = (r * r).sum(-1)
        rn = (r * geom.normals[None]).sum(-1)
        rs = (r * ws[None]).sum(-1)
        self_mask = rr[:, None] == np.arange(geom.n_nodes)[None, :]
        rho2[self_mask] = 1.0
        c = INV_PI * rn * rs / (rho2 * rho2)
        c[self_mask] = 0.0
        out[a:a + chunk] = (c[..., None] * r).sum(1)
    # diagonal: self term and jump
    S = self_blocks(geom)[rows]
    out += np.einsum("rab,rb->ra", S, sigma[rows]) - 0.5 * sigma[rows]
    # completion
    x = geom.nodes[rows]
    for k in range(geom.n_comp):
        if k == geom.outer_comp:
            continue
        out += np.einsum("rab,b->ra", stokeslet(x, geom.centres[k]), lam[k])
        out += rotlet(x, geom.centres[k]) * xi[k]
    on_wall = comp[rows] == geom.outer_comp
    out[on_wall] += geom.normals[rows[on_wall]] * s0
    return out


def matvec(geom, sigma):
    """A sigma as a (2N,) vector (matrix-free)."""
    return apply_rows(geom, sigma, np.arange(geom.n_nodes)).reshape(-1)


def velocity(geom, sigma, targets, chunk=256):
    """u(x) = D[sigma](x) + sum_k S(x, c_k) lambda_k + R(x, c_k) xi_k at
    interior points (Eq. 7 with the double-layer kernel; reading R4).
    Returns (T, 2)."""
    sigma = np.asarray(sigma, dtype=np.float64).reshape(-1, 2)
    targets = np.asarray(targets, dtype=np.float64)
    lam, xi, _ = moments(geom, sigma)
    ws = geom.weights[:, None] * sigma
    u = np.zeros_like(targets)
    for a in range(0, targets.shape[0], chunk):
        x = targets[a:a + chunk]
        r = x[:, None, :] - geom.nodes[None, :, :]
        rho2 = (r * r).sum(-1)
        rn = (r * geom.normals[None]).sum(-1)
        rs = (r * ws[None]).sum(-1)
        c = INV_PI * rn * rs / (rho2 * rho2)
        u[a:a + chunk] = (c[..., None] * r).sum(1)
    for k in range(geom.n_comp):
        if k == geom.outer_comp:
            continue
        u += np.einsum("tab,b->ta", stokeslet(targets, geom.centres[k]), lam[k])
        u += rotlet(targets, geom.centres[k]) * xi[k]
    return u


# ---------------------------------------------------------------------------
# Block-diagonal preconditioner (Sec. 4.1 footnote)
# ---------------------------------------------------------------------------

class BlockDiagonal:
    """Diagonal blocks A_kk (the restriction of A to component k, including
    its own completion or wall term), each LU-factorised with partial
    pivoting (LAPACK getrf through scipy)."""

    def __init__(self, geom):
        import scipy.linalg as sla
        self.geom = geom
        self.factors = []
        self.blocks = []
        for k in range(geom.n_comp):
            idx = np.arange(geom.offsets[k], geom.offsets[k + 1])
            Akk = _blocks_to_matrix(operator_blocks(geom, idx, idx))
            self.blocks.append(Akk)
            self.factors.append(sla.lu_factor(Akk))

    def apply(self, v):
        import scipy.linalg as sla
        v = np.asarray(v, dtype=np.float64).reshape(-1)
        z = np.empty_like(v)
        for k, fac in enumerate(self.factors):
            a, b = 2 * int(self.geom.offsets[k]), 2 * int(self.geom.offsets[k + 1])
            z[a:b] = sla.lu_solve(fac, v[a:b])
        return z


# ---------------------------------------------------------------------------
# GMRES(m) (Sec. 4; Saad and Schultz)
# ---------------------------------------------------------------------------

def gmres(apply_A, f, tol=1e-8, restart=50, max_iter=2000, apply_M=None, side="right", x0=None):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.

    side="right": solves A M^-1 u = f, x = M^-1 u; the Arnoldi residual is
    the true residual, and the stop is on the TRUE relative residual
    |f - A x| / |f| <= tol, recomputed at every restart and whenever the
    Arnoldi estimate drops below tol.
    side="left": solves M^-1 A x = M^-1 f and stops on the PRECONDITIONED
    relative residual, as in Sec. 4.1; the true residual is reported.
    Either way at most max_iter inner steps are taken.
    Returns dict(x, iters, relres (true), pc_relres, history).
    """
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    n = f.size
    M = apply_M if apply_M is not None else (lambda v: v)
    if side == "right":
        op = lambda v: apply_A(M(v))
        rhs = f
    elif side == "left":
        op = lambda v: M(apply_A(v))
        rhs = M(f)
    else:
        raise ValueError(side)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    u = np.zeros(n)          # right-PC variable: x = x0 + M^-1 u
    fnorm = np.linalg.norm(f)
    rhsnorm = np.linalg.norm(rhs)
    if fnorm == 0.0:
        return dict(x=np.zeros(n), iters=0, relres=0.0, pc_relres=0.0, history=[0.0])
    iters = 0
    history = []
    x_base = x.copy()

    def current_x():
        return x_base + M(u) if side == "right" else x

    while True:
        xc = current_x()
        r_true = f - apply_A(xc)
        relres = np.linalg.norm(r_true) / fnorm
        r = r_true if side == "right" else M(r_true)
        beta = np.linalg.norm(r)
        history.append(beta / rhsnorm)
        done = relres <= tol if side == "right" else beta / rhsnorm <= tol
        if done or iters >= max_iter:
            return dict(x=xc, iters=iters, relres=relres, pc_relres=beta / rhsnorm, history=history)
        m = min(restart, max_iter - iters)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(m):
            w = op(V[j])
            for i in range(j + 1):               # modified Gram-Schmidt
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            if hnext > 0.0:
                V[j + 1] = w / hnext
            for i in range(j):                   # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_done = j + 1
            history.append(abs(g[j + 1]) / rhsnorm)
            if abs(g[j + 1]) / rhsnorm <= tol or hnext == 0.0:   # converged / happy breakdown
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):       # back substitution R y = g
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        upd = V[:j_done].T @ y
        if side == "right":
            u = u + upd
        else:
            x = x + upd


def solve_dense(geom, f):
    """Direct solve of the dense system (small N): numpy LAPACK gesv."""
    A = assemble(geom)
    return np.linalg.solve(A, np.asarray(f, dtype=np.float64).reshape(-1))


def solve_gmres(geom, f, tol=1e-8, restart=50, max_iter=2000, precond="bd", side="right"):
    """GMRES on the matrix-free operator, optional block-diagonal PC."""
    if geom.n_nodes <= 4000:
        A = assemble(geom)
        apply_A = lambda v: A @ v
    else:
        apply_A = lambda v: matvec(geom, v)
    M = BlockDiagonal(geom).apply if precond == "bd" else None
    return gmres(apply_A, f, tol=tol, restart=restart, max_iter=max_iter, apply_M=M, side=side)


# ---------------------------------------------------------------------------
# Two-grid preconditioner and flexible GMRES (not in the paper: the GPU
# library's alternative to block-diagonal preconditioning, checked here)
# ---------------------------------------------------------------------------

def trig_interpolation(nc, nf):
    """(nf x nc) matrix of trigonometric interpolation from nc equispaced
    samples s_j = 2 pi j / nc of a periodic function to nf samples
    t_i = 2 pi i / nf: the real trigonometric interpolant
        P[i, j] = (1/nc) [1 + 2 sum_{k=1}^{K} cos(k (t_i - s_j)) (+ cos((nc/2)(t_i - s_j)) if nc even)],
    K = ceil(nc / 2) - 1 (the Nyquist cosine split evenly between +-nc/2)."""
    t = 2.0 * np.pi * np.arange(nf) / nf
    s = 2.0 * np.pi * np.arange(nc) / nc
    d = t[:, None] - s[None, :]
    P = np.ones((nf, nc))
    for k in range(1, (nc + 1) // 2):
        P += 2.0 * np.cos(k * d)
    if nc % 2 == 0:
        P += np.cos((nc // 2) * d)
    return P / nc


def coarse_geometry(geom, q):
    """Every q-th node of every component, weights times q (the trapezoid
    rule on a q-times coarser equispaced parameter grid)."""
    import dataclasses
    idx = np.concatenate([np.arange(geom.offsets[k], geom.offsets[k + 1], q) for k in range(geom.n_comp)])
    sizes = np.diff(geom.offsets) // q
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return dataclasses.replace(geom, nodes=geom.nodes[idx].copy(), normals=geom.normals[idx].copy(),
                               weights=geom.weights[idx] * q, curvature=geom.curvature[idx].copy(),
                               offsets=offs)


class TwoGrid:
    """P^-1 r = I Ac^-1 R r + B^-1 (r - I R r): an exact solve with the same
    operator on the q-times coarser grid, plus the pores' diagonal blocks on
    what the coarse grid cannot represent; on the wall the remainder is
    scaled by -2 (the inverse of the jump -1/2). I is trigonometric
    interpolation per component, R = (nc / nf) I^T."""

    def __init__(self, geom, q):
        import scipy.linalg as sla
        if any(int(n) % q or int(n) // q < 8 for n in np.diff(geom.offsets)):
            raise ValueError("every component needs a multiple of q nodes, at least 8 q")
        self.geom = geom
        self.gc = coarse_geometry(geom, q)
        self.lu = sla.lu_factor(assemble(self.gc))
        blocks = []
        for k in range(geom.n_comp):
            nf = int(geom.offsets[k + 1] - geom.offsets[k])
            blocks.append(trig_interpolation(nf // q, nf))
        Inode = sla.block_diag(*blocks)
        Rnode = sla.block_diag(*[B.T * (B.shape[1] / B.shape[0]) for B in blocks])
        self.I = np.kron(Inode, np.eye(2))
        self.R = np.kron(Rnode, np.eye(2))
        self.bd = BlockDiagonal(geom)
        self.wall = slice(2 * int(geom.offsets[geom.outer_comp]), 2 * int(geom.offsets[geom.outer_comp + 1]))

    def apply(self, r):
        import scipy.linalg as sla
        r = np.asarray(r, dtype=np.float64).reshape(-1)
        rc = self.R @ r
        zc = sla.lu_solve(self.lu, rc)
        h = r - self.I @ rc
        zh = self.bd.apply(h)
        zh[self.wall] = -2.0 * h[self.wall]
        return self.I @ zc + zh


def fgmres(apply_A, f, apply_M, tol=1e-8, restart=200, max_iter=2000):
    """Flexible GMRES (Saad 1993): the preconditioned vectors z_j = M(v_j)
    are kept and the iterate is x0 + Z y, so M may vary between steps
    (rounding inside it included). Stops on the true relative residual."""
    f = np.asarray(f, dtype=np.float64).reshape(-1)
    n = f.size
    x = np.zeros(n)
    fnorm = np.linalg.norm(f)
    iters = 0
    while True:
        r = f - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * fnorm or iters >= max_iter:
            return dict(x=x, iters=iters, relres=beta / fnorm)
        m = min(restart, max_iter - iters)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        jd = 0
        for j in range(m):
            Z[j] = apply_M(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            jd = j + 1
            if abs(g[j + 1]) <= tol * fnorm:
                break
        y = np.zeros(jd)
        for i in range(jd - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:jd] @ y[i + 1:]) / H[i, i]
        x = x + Z[:jd].T @ y
