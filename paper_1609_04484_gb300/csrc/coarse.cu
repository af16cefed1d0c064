// Two-level preconditioner with a coarse space of pore rigid motions, and
// the learned coarse correction (the paper has no counterpart: its
// preconditioners are the block diagonal of Sec. 4.1 and the IFMM).
//
// The completed double-layer operator couples the pores through the
// moments of the density on each pore (the Stokeslet and rotlet that remove
// each component's rank-3 null space, Sec. 2.1), and the block-diagonal
// preconditioner ignores that coupling. The coarse space Z (2N x 3M) holds
// for pore p the rigid-motion densities on its nodes: e_x, e_y and the
// rotation (x - c_p)^perp / r_p ((a, b)^perp = (b, -a), r_p = L_p / 2 pi with
// L_p = sum of the pore's weights). With W = diag(w), Y = A Z (computed at
// setup, one column per mode) and a coarse inverse C, each apply is
//   c = C Z^T W r,   z = Z c + B^-1 (r - Y c)
// (coarse level first, then the block diagonal B^-1 on what remains): no
// operator application beyond the GMRES step's own.
//
// C is either the exact inverse of the Galerkin operator E = Z^T W Y
// (STOKES_PC_BD_COARSE) or a network's prediction of it on a sparse pattern
// (STOKES_PC_BD_LEARNED): for each pore, the blocks C[p][q] of q = p and its
// 16 nearest pores, predicted from 35 features (the centre over the wall's
// half-extents, the radius, the 16 offsets c_q - c_p) in the scaled form
// L_p L_q C[p][q], standardised with the training set's means and spreads.
// The training targets are the exact E^-1 of training geometries, computed
// by the same kernels on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.cuh"

namespace stokes {

constexpr int kNbrs = 16;
constexpr int kFeat = 3 + 2 * kNbrs;       // 35
constexpr int kOut = 9 * (kNbrs + 1);      // 153
constexpr int kHidden = 256;
constexpr int kMaxCoarse = 4096;           // largest 3M the dense coarse inverse takes

struct CoarseModel {
  mlp::Net net{kFeat, kHidden, kOut};
  cudaStream_t stream = nullptr;
  // training set (float): features, scaled targets, mask
  DevBuf<float> X, T, mask, Tstd;
  int64_t rows = 0, cap = 0;
  double count = 0.0;
  // standardisation: x_mean, x_std [35], t_mean, t_std [153]
  DevBuf<float> stats;
  bool stats_ready = false;
};

namespace {

// ---------------------------------------------------------------------------
// Coarse space
// ---------------------------------------------------------------------------

// Per pore: L, r = L / 2 pi, sum w dx, sum w dy, sum w |d|^2 (d = x - c).
__global__ void __launch_bounds__(256)
k_cl_pore_stats(const int* __restrict__ pores, const int64_t* __restrict__ off, const double2* __restrict__ pos,
                const double* __restrict__ w, const double2* __restrict__ centre, double* __restrict__ stats) {
  count_launch();
  __shared__ double red[4][256];
  const int p = blockIdx.x, k = pores[p];
  const double2 c = centre[k];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int64_t j = off[k] + threadIdx.x; j < off[k + 1]; j += blockDim.x) {
    const double dx = pos[j].x - c.x, dy = pos[j].y - c.y, wj = w[j];
    a0 += wj;
    a1 += wj * dx;
    a2 += wj * dy;
    a3 += wj * (dx * dx + dy * dy);
  }
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = a1;
  red[2][threadIdx.x] = a2;
  red[3][threadIdx.x] = a3;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[5 * p] = red[0][0];
    stats[5 * p + 1] = red[0][0] / (2.0 * kPi);
    stats[5 * p + 2] = red[1][0];
    stats[5 * p + 3] = red[2][0];
    stats[5 * p + 4] = red[3][0];
  }
}

// Y = A Z: CTA (target block, pore p); each thread one target node i and the
// pore's three modes. Pair sum over the pore's nodes j != i of the
// double-layer kernel, the diagonal entry where i is on the pore, and the
// pore's completion of each mode (the wall term vanishes: Z is zero on the
// wall). Column-major, leading dimension 2N.
constexpr int kAzTile = 128;
__global__ void __launch_bounds__(kAzTile)
k_cl_az(int64_t N, const int* __restrict__ pores, const int64_t* __restrict__ off, const double2* __restrict__ pos,
        const double4_32a* __restrict__ src, const double4_32a* __restrict__ selfc, const int* __restrict__ comp,
        const double2* __restrict__ centre, const double* __restrict__ stats, double* __restrict__ Y) {
  count_launch();
  __shared__ double2 s_x[kAzTile], s_a[kAzTile], s_z[kAzTile];
  const int p = blockIdx.y, k = pores[p];
  const double2 c = centre[k];
  const double L = stats[5 * p], r = stats[5 * p + 1], Sx = stats[5 * p + 2], Sy = stats[5 * p + 3],
               S2 = stats[5 * p + 4];
  const int64_t i = blockIdx.x * (int64_t)kAzTile + threadIdx.x;
  const double2 xi = i < N ? pos[i] : make_double2(0.0, 0.0);
  double u[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  for (int64_t t0 = off[k]; t0 < off[k + 1]; t0 += kAzTile) {
    __syncthreads();
    const int64_t j = t0 + threadIdx.x;
    if (j < off[k + 1]) {
      const double4_32a sj = src[j];
      s_x[threadIdx.x] = make_double2(sj.x, sj.y);
      s_a[threadIdx.x] = make_double2(sj.z, sj.w);
      s_z[threadIdx.x] = make_double2((sj.y - c.y) / r, -(sj.x - c.x) / r);
    }
    __syncthreads();
    const int nt = (int)imin64(kAzTile, off[k + 1] - t0);
    for (int q = 0; q < nt; ++q) {
      if (t0 + q == i) continue;
      const double rx = xi.x - s_x[q].x, ry = xi.y - s_x[q].y;
      const double r2 = rx * rx + ry * ry;
      const double inv = 1.0 / r2;
      const double coef = (rx * s_a[q].x + ry * s_a[q].y) * inv * inv;
      const double q0 = coef * rx, q1 = coef * ry, q2 = coef * (rx * s_z[q].x + ry * s_z[q].y);
      u[0][0] += q0 * rx;
      u[0][1] += q0 * ry;
      u[1][0] += q1 * rx;
      u[1][1] += q1 * ry;
      u[2][0] += q2 * rx;
      u[2][1] += q2 * ry;
    }
  }
  if (i >= N) return;
  const double dxi = xi.x - c.x, dyi = xi.y - c.y;
  if (comp[i] == k) {  // diagonal entry: s t t^T - I / 2 on the modes at node i
    const double4_32a sc = selfc[i];
    const double z[3][2] = {{1.0, 0.0}, {0.0, 1.0}, {dyi / r, -dxi / r}};
    for (int a = 0; a < 3; ++a) {
      const double tz = sc.x * z[a][0] + sc.y * z[a][1];
      u[a][0] += sc.z * sc.x * tz - 0.5 * z[a][0];
      u[a][1] += sc.z * sc.y * tz - 0.5 * z[a][1];
    }
  }
  // completion: S(x, c) lambda + R(x, c) xi of each mode's moments
  const double lam[3][2] = {{L, 0.0}, {0.0, L}, {Sy / r, -Sx / r}};
  const double xim[3] = {Sy, -Sx, S2 / r};
  const double rho2 = dxi * dxi + dyi * dyi;
  const double lg = -0.5 * log(rho2), irho2 = 1.0 / rho2;
  for (int a = 0; a < 3; ++a) {
    const double rl = (dxi * lam[a][0] + dyi * lam[a][1]) * irho2;
    u[a][0] += kInv4Pi * (lg * lam[a][0] + rl * dxi + dyi * irho2 * xim[a]);
    u[a][1] += kInv4Pi * (lg * lam[a][1] + rl * dyi - dxi * irho2 * xim[a]);
    double* col = Y + (int64_t)(3 * p + a) * (2 * N);
    col[2 * i] = u[a][0];
    col[2 * i + 1] = u[a][1];
  }
}

// E = Z^T W Y (row-major m x m, m = 3M): one CTA per row (pore p, mode a).
__global__ void __launch_bounds__(256)
k_cl_galerkin(int64_t N, int m, const int* __restrict__ pores, const int64_t* __restrict__ off,
              const double2* __restrict__ pos, const double* __restrict__ w, const double2* __restrict__ centre,
              const double* __restrict__ stats, const double* __restrict__ Y, double* __restrict__ E) {
  count_launch();
  const int row = blockIdx.x, p = row / 3, a = row % 3, k = pores[p];
  const double2 c = centre[k];
  const double r = stats[5 * p + 1];
  for (int col = threadIdx.x; col < m; col += blockDim.x) {
    const double* yc = Y + (int64_t)col * (2 * N);
    double s = 0.0;
    for (int64_t i = off[k]; i < off[k + 1]; ++i) {
      const double zx = a == 0 ? 1.0 : (a == 1 ? 0.0 : (pos[i].y - c.y) / r);
      const double zy = a == 0 ? 0.0 : (a == 1 ? 1.0 : -(pos[i].x - c.x) / r);
      s += w[i] * (zx * yc[2 * i] + zy * yc[2 * i + 1]);
    }
    E[(int64_t)row * m + col] = s;
  }
}

// X = A^-1 (row-major m x m, A destroyed) by Gauss-Jordan elimination with
// partial pivoting (largest |A[r][c]|, ties to the smaller row), one CTA.
// col: m doubles of scratch. status = 1 on a zero or non-finite pivot.
__global__ void __launch_bounds__(1024)
k_gauss_jordan(double* __restrict__ A, double* __restrict__ X, double* __restrict__ col, int m,
               int* __restrict__ status) {
  count_launch();
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  __shared__ double s_inv;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nthr = blockDim.x;
  for (int64_t e = tid; e < (int64_t)m * m; e += nthr) X[e] = (e / m == e % m) ? 1.0 : 0.0;
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    double best = -1.0;
    int bi = m;
    for (int r = c + tid; r < m; r += nthr) {
      const double v = fabs(A[(int64_t)r * m + c]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[wid] = best; si[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = m;
      for (int q = 0; q < (nthr >> 5); ++q)
        if (sv[q] > b || (sv[q] == b && si[q] < p)) { b = sv[q]; p = si[q]; }
      if (p >= m) p = c;
      const double d = A[(int64_t)p * m + c];
      if (d == 0.0 || !isfinite(d)) { *status = 1; s_inv = 0.0; } else s_inv = 1.0 / d;
      s_p = p;
    }
    __syncthreads();
    const int p = s_p;
    const double iv = s_inv;
    for (int j = tid; j < m; j += nthr) {  // swap rows c and p, scale the pivot row
      const double ac = A[(int64_t)c * m + j], ap = A[(int64_t)p * m + j];
      const double xc = X[(int64_t)c * m + j], xp = X[(int64_t)p * m + j];
      A[(int64_t)p * m + j] = ac;
      X[(int64_t)p * m + j] = xc;
      A[(int64_t)c * m + j] = ap * iv;
      X[(int64_t)c * m + j] = xp * iv;
    }
    __syncthreads();
    for (int r = tid; r < m; r += nthr) col[r] = A[(int64_t)r * m + c];
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)m * m; e += nthr) {
      const int r = (int)(e / m);
      if (r == c) continue;
      const int j = (int)(e % m);
      const double f = col[r];
      A[e] -= f * A[(int64_t)c * m + j];
      X[e] -= f * X[(int64_t)c * m + j];
    }
    __syncthreads();
  }
}

// Half-extents of the wall: ab[0] = (max x - min x) / 2, ab[1] the same in y.
__global__ void k_cl_wall_extent(const double2* __restrict__ pos, int64_t j0, int64_t j1, double* __restrict__ ab) {
  count_launch();
  __shared__ double red[4][256];
  double v[4] = {1e300, -1e300, 1e300, -1e300};
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double2 x = pos[j];
    v[0] = fmin(v[0], x.x);
    v[1] = fmax(v[1], x.x);
    v[2] = fmin(v[2], x.y);
    v[3] = fmax(v[3], x.y);
  }
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      red[0][threadIdx.x] = fmin(red[0][threadIdx.x], red[0][threadIdx.x + st]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + st]);
      red[2][threadIdx.x] = fmin(red[2][threadIdx.x], red[2][threadIdx.x + st]);
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ab[0] = 0.5 * (red[1][0] - red[0][0]);
    ab[1] = 0.5 * (red[3][0] - red[2][0]);
  }
}

__device__ __forceinline__ bool knn_less(double d, int i, double e, int j) { return d < e || (d == e && i < j); }

// Per pore p: its 16 nearest other pores by centre distance (nearest first,
// ties to the smaller pore number, -1 where absent) and its 35 features.
__global__ void __launch_bounds__(128)
k_cl_features(int M, const int* __restrict__ pores, const double2* __restrict__ centre,
              const double* __restrict__ stats, const double* __restrict__ ab, int* __restrict__ nbr,
              float* __restrict__ X) {
  count_launch();
  __shared__ double2 s_c[256];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const double2 cp = p < M ? centre[pores[p]] : make_double2(0.0, 0.0);
  double bd[kNbrs];
  int bi[kNbrs];
#pragma unroll
  for (int s = 0; s < kNbrs; ++s) { bd[s] = INFINITY; bi[s] = M; }
  for (int q0 = 0; q0 < M; q0 += 256) {
    __syncthreads();
    for (int e = threadIdx.x; e < 256; e += blockDim.x)
      if (q0 + e < M) s_c[e] = centre[pores[q0 + e]];
    __syncthreads();
    const int nq = min(256, M - q0);
    for (int e = 0; e < nq; ++e) {
      const int q = q0 + e;
      if (q == p) continue;
      const double dx = s_c[e].x - cp.x, dy = s_c[e].y - cp.y;
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      if (knn_less(d2, q, bd[kNbrs - 1], bi[kNbrs - 1])) {
        bd[kNbrs - 1] = d2;
        bi[kNbrs - 1] = q;
#pragma unroll
        for (int s = kNbrs - 1; s > 0; --s)
          if (knn_less(bd[s], bi[s], bd[s - 1], bi[s - 1])) {
            const double td = bd[s]; bd[s] = bd[s - 1]; bd[s - 1] = td;
            const int ti = bi[s]; bi[s] = bi[s - 1]; bi[s - 1] = ti;
          }
      }
    }
  }
  if (p >= M) return;
  float* f = X + (int64_t)p * kFeat;
  f[0] = (float)(cp.x / ab[0]);
  f[1] = (float)(cp.y / ab[1]);
  f[2] = (float)stats[5 * p + 1];
#pragma unroll
  for (int s = 0; s < kNbrs; ++s) {
    const bool has = bi[s] < M;
    nbr[(int64_t)p * kNbrs + s] = has ? bi[s] : -1;
    double ox = 0.0, oy = 0.0;
    if (has) {
      const double2 cq = centre[pores[bi[s]]];
      ox = cq.x - cp.x;
      oy = cq.y - cp.y;
    }
    f[3 + 2 * s] = (float)ox;
    f[4 + 2 * s] = (float)oy;
  }
}

// Targets: T[p][9 j + 3 al + be] = L_p L_q Einv[3 p + al][3 q + be] for
// q = p (j = 0) and the j-th neighbour; mask 1 where q exists.
__global__ void k_cl_targets(int M, const int* __restrict__ nbr, const double* __restrict__ stats,
                             const double* __restrict__ Einv, float* __restrict__ T, float* __restrict__ mask) {
  count_launch();
  const int64_t total = (int64_t)M * kOut;
  const int m = 3 * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / kOut), o = (int)(e % kOut), j = o / 9, al = (o % 9) / 3, be = o % 3;
    const int q = j == 0 ? p : nbr[(int64_t)p * kNbrs + j - 1];
    if (q < 0) {
      T[e] = 0.f;
      mask[e] = 0.f;
    } else {
      T[e] = (float)(stats[5 * p] * stats[5 * q] * Einv[(int64_t)(3 * p + al) * m + 3 * q + be]);
      mask[e] = 1.f;
    }
  }
}

// C (row-major 3M x 3M, zeroed first) from the network's standardised
// outputs y [M][ldy]: C[3p + al][3q + be] = (mean + std y) / (L_p L_q).
__global__ void k_cl_scatter(int M, const int* __restrict__ nbr, const double* __restrict__ stats,
                             const float* __restrict__ y, int ldy, const float* __restrict__ t_mean,
                             const float* __restrict__ t_std, double* __restrict__ C) {
  count_launch();
  const int64_t total = (int64_t)M * kOut;
  const int m = 3 * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / kOut), o = (int)(e % kOut), j = o / 9, al = (o % 9) / 3, be = o % 3;
    const int q = j == 0 ? p : nbr[(int64_t)p * kNbrs + j - 1];
    if (q < 0) continue;
    const double v = (double)t_mean[o] + (double)t_std[o] * (double)y[(int64_t)p * ldy + o];
    C[(int64_t)(3 * p + al) * m + 3 * q + be] = v / (stats[5 * p] * stats[5 * q]);
  }
}

// Column means and spreads (population) of x [rows][cols], weighted by
// mask (or 1); spreads below 1e-12 become 1 (constant columns).
__global__ void k_col_stats(const float* __restrict__ x, const float* __restrict__ mask, int64_t rows, int cols,
                            float* __restrict__ mean, float* __restrict__ stdv) {
  count_launch();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0, n = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    const double mk = mask ? mask[r * cols + c] : 1.0;
    s += mk * x[r * cols + c];
    n += mk;
  }
  const double mu = n > 0 ? s / n : 0.0;
  double v = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    const double mk = mask ? mask[r * cols + c] : 1.0;
    const double d = x[r * cols + c] - mu;
    v += mk * d * d;
  }
  const double sd = n > 0 ? sqrt(v / n) : 1.0;
  mean[c] = (float)mu;
  stdv[c] = sd > 1e-12 ? (float)sd : 1.f;
}

__global__ void k_standardise(const float* __restrict__ x, int64_t rows, int cols, const float* __restrict__ mean,
                              const float* __restrict__ stdv, float* __restrict__ out) {
  count_launch();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % cols);
    out[e] = (x[e] - mean[c]) / stdv[c];
  }
}

// ---------------------------------------------------------------------------
// Apply
// ---------------------------------------------------------------------------

// rc = Z^T W r, one CTA per pore.
__global__ void __launch_bounds__(256)
k_cl_restrict(const int* __restrict__ pores, const int64_t* __restrict__ off, const double2* __restrict__ pos,
              const double* __restrict__ w, const double2* __restrict__ centre, const double* __restrict__ stats,
              const double* __restrict__ r, double* __restrict__ rc, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double red[3][256];
  const int p = blockIdx.x, k = pores[p];
  const double2 c = centre[k];
  const double rad = stats[5 * p + 1];
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = off[k] + threadIdx.x; j < off[k + 1]; j += blockDim.x) {
    const double wx = w[j] * r[2 * j], wy = w[j] * r[2 * j + 1];
    a0 += wx;
    a1 += wy;
    a2 += ((pos[j].y - c.y) * wx - (pos[j].x - c.x) * wy) / rad;
  }
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = a1;
  red[2][threadIdx.x] = a2;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rc[3 * p] = red[0][0];
    rc[3 * p + 1] = red[1][0];
    rc[3 * p + 2] = red[2][0];
  }
}

// c = C rc (row-major m x m): one warp per row.
__global__ void k_cl_coarse_gemv(const double* __restrict__ C, int m, const double* __restrict__ rc,
                                 double* __restrict__ c, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) s += C[(int64_t)row * m + j] * rc[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) c[row] = s;
}

// t = r - Y c (Y column-major, 2N rows).
__global__ void k_cl_residual(int64_t n2, int m, const double* __restrict__ Y, const double* __restrict__ c,
                              const double* __restrict__ r, double* __restrict__ t, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    double s = r[i];
    for (int j = 0; j < m; ++j) s -= Y[(int64_t)j * n2 + i] * c[j];
    t[i] = s;
  }
}

// z += Z c on the pores' nodes.
__global__ void k_cl_add_modes(int64_t N, const int* __restrict__ comp, const int* __restrict__ pore_of,
                               const double2* __restrict__ pos, const double2* __restrict__ centre,
                               const double* __restrict__ stats, const double* __restrict__ c,
                               double* __restrict__ z, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = comp[i];
    const int p = pore_of[k];
    if (p < 0) continue;
    const double2 cc = centre[k];
    const double rad = stats[5 * p + 1];
    const double c0 = c[3 * p], c1 = c[3 * p + 1], c2 = c[3 * p + 2] / rad;
    z[2 * i] += c0 + c2 * (pos[i].y - cc.y);
    z[2 * i + 1] += c1 - c2 * (pos[i].x - cc.x);
  }
}

unsigned grid1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

// Pores, their stats and Y = A Z on the handle.
static void coarse_prepare(Geom& g) {
  CoarseLevel& cl = g.cl;
  cudaStream_t s = g.stream;
  cl.pores.clear();
  std::vector<int> pore_of(g.n_comp, -1);
  for (int k = 0; k < g.n_comp; ++k)
    if (k != g.outer) {
      pore_of[k] = (int)cl.pores.size();
      cl.pores.push_back(k);
    }
  cl.M = (int)cl.pores.size();
  require(cl.M >= 1, "the coarse level needs at least one pore");
  require(3 * (int64_t)cl.M <= kMaxCoarse, "the coarse level takes at most 1365 pores");
  const int m = 3 * cl.M;
  cl.d_pores.alloc(cl.M);
  cl.pore_of.alloc(g.n_comp);
  cl.stats.alloc(5 * (size_t)cl.M);
  cl.Y.alloc((size_t)m * 2 * g.N);
  cl.C.alloc((size_t)m * m);
  cl.rc.alloc(m);
  cl.c.alloc(m);
  cl.t.alloc(2 * g.N);
  STOKES_CUDA(cudaMemcpyAsync(cl.d_pores.get(), cl.pores.data(), 4 * cl.M, cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemcpyAsync(cl.pore_of.get(), pore_of.data(), 4 * g.n_comp, cudaMemcpyHostToDevice, s));
  k_cl_pore_stats<<<cl.M, 256, 0, s>>>(cl.d_pores.get(), g.d_off.get(), g.pos.get(), g.w.get(), g.centre.get(),
                                      cl.stats.get());
  dim3 grid((unsigned)((g.N + kAzTile - 1) / kAzTile), (unsigned)cl.M);
  k_cl_az<<<grid, kAzTile, 0, s>>>(g.N, cl.d_pores.get(), g.d_off.get(), g.pos.get(), g.src.get(), g.selfc.get(),
                                   g.comp.get(), g.centre.get(), cl.stats.get(), cl.Y.get());
  STOKES_LAUNCHED();
}

// E = Z^T W Y into E (device, row-major m x m).
static void coarse_galerkin(Geom& g, double* E) {
  const int m = 3 * g.cl.M;
  k_cl_galerkin<<<m, 256, 0, g.stream>>>(g.N, m, g.cl.d_pores.get(), g.d_off.get(), g.pos.get(), g.w.get(),
                                         g.centre.get(), g.cl.stats.get(), g.cl.Y.get(), E);
  STOKES_LAUNCHED();
}

// X = A^-1 (device, row-major m x m; A destroyed). Synchronises.
static void dense_inverse(cudaStream_t s, double* A, double* X, int m) {
  DevBuf<double> col;
  DevBuf<int> st;
  col.alloc(m);
  st.alloc(1);
  STOKES_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
  k_gauss_jordan<<<1, 1024, 0, s>>>(A, X, col.get(), m, st.get());
  STOKES_LAUNCHED();
  int h = 0;
  STOKES_CUDA(cudaMemcpyAsync(&h, st.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaStreamSynchronize(s));
  require(h == 0, "coarse operator is singular (zero pivot)", STOKES_EBREAKDOWN);
}

// Features [M][35] and neighbour lists [M][16] of the handle's pores
// (needs coarse_prepare). Device outputs.
static void coarse_features(Geom& g, float* X, int* nbr) {
  cudaStream_t s = g.stream;
  DevBuf<double> ab;
  ab.alloc(2);
  k_cl_wall_extent<<<1, 256, 0, s>>>(g.pos.get(), g.off[g.outer], g.off[g.outer + 1], ab.get());
  k_cl_features<<<(unsigned)((g.cl.M + 127) / 128), 128, 0, s>>>(g.cl.M, g.cl.d_pores.get(), g.centre.get(),
                                                                  g.cl.stats.get(), ab.get(), nbr, X);
  STOKES_LAUNCHED();
  STOKES_CUDA(cudaStreamSynchronize(s));  // ab goes out of scope
}

// Exact coarse inverse C = E^-1.
static void coarse_setup_exact(Geom& g) {
  coarse_prepare(g);
  const int m = 3 * g.cl.M;
  DevBuf<double> E;
  E.alloc((size_t)m * m);
  coarse_galerkin(g, E.get());
  dense_inverse(g.stream, E.get(), g.cl.C.get(), m);
}

static void coarse_setup_learned(Geom& g, CoarseModel& mdl) {
  require(mdl.stats_ready, "coarse model has not been trained or loaded", STOKES_ESTATE);
  coarse_prepare(g);
  cudaStream_t s = g.stream;
  const int M = g.cl.M, m = 3 * M;
  DevBuf<float> X;
  DevBuf<int> nbr;
  X.alloc((size_t)M * kFeat);
  nbr.alloc((size_t)M * kNbrs);
  coarse_features(g, X.get(), nbr.get());
  const float* st = mdl.stats.get();
  mdl.net.forward(X.get(), M, st, st + kFeat, s);
  STOKES_CUDA(cudaMemsetAsync(g.cl.C.get(), 0, sizeof(double) * (size_t)m * m, s));
  k_cl_scatter<<<grid1((int64_t)M * kOut), 256, 0, s>>>(M, nbr.get(), g.cl.stats.get(), mdl.net.y.get(),
                                                         mdl.net.L.out_p, st + 2 * kFeat, st + 2 * kFeat + kOut,
                                                         g.cl.C.get());
  STOKES_LAUNCHED();
  STOKES_CUDA(cudaStreamSynchronize(s));
}

void coarse_apply(Geom& g, const double* r, double* z, const int* done, bool f32) {
  CoarseLevel& cl = g.cl;
  cudaStream_t s = g.stream;
  const int m = 3 * cl.M;
  k_cl_restrict<<<cl.M, 256, 0, s>>>(cl.d_pores.get(), g.d_off.get(), g.pos.get(), g.w.get(), g.centre.get(),
                                     cl.stats.get(), r, cl.rc.get(), done);
  k_cl_coarse_gemv<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(cl.C.get(), m, cl.rc.get(), cl.c.get(), done);
  k_cl_residual<<<grid1(2 * g.N), 256, 0, s>>>(2 * g.N, m, cl.Y.get(), cl.c.get(), r, cl.t.get(), done);
  STOKES_LAUNCHED();
  bd_apply(g, cl.t.get(), z, done, f32);
  k_cl_add_modes<<<grid1(g.N), 256, 0, s>>>(g.N, g.comp.get(), cl.pore_of.get(), g.pos.get(), g.centre.get(),
                                            cl.stats.get(), cl.c.get(), z, done);
  STOKES_LAUNCHED();
}

// Training samples of one geometry: its features, neighbour lists and the
// scaled blocks of the exact E^-1, appended to the model's set.
static void model_add_geometry(CoarseModel& mdl, Geom& g) {
  coarse_setup_exact(g);  // C = E^-1
  cudaStream_t s = g.stream;
  const int M = g.cl.M;
  DevBuf<int> nbr;
  nbr.alloc((size_t)M * kNbrs);
  if (mdl.rows + M > mdl.cap) {  // grow (copy) the training arrays
    const int64_t cap = std::max<int64_t>(2 * mdl.cap, mdl.rows + M + 1024);
    DevBuf<float> X, T, mask;
    X.alloc((size_t)cap * kFeat);
    T.alloc((size_t)cap * kOut);
    mask.alloc((size_t)cap * kOut);
    if (mdl.rows) {
      STOKES_CUDA(cudaMemcpyAsync(X.get(), mdl.X.get(), 4 * mdl.rows * kFeat, cudaMemcpyDeviceToDevice, s));
      STOKES_CUDA(cudaMemcpyAsync(T.get(), mdl.T.get(), 4 * mdl.rows * kOut, cudaMemcpyDeviceToDevice, s));
      STOKES_CUDA(cudaMemcpyAsync(mask.get(), mdl.mask.get(), 4 * mdl.rows * kOut, cudaMemcpyDeviceToDevice, s));
    }
    STOKES_CUDA(cudaStreamSynchronize(s));
    std::swap(mdl.X.p, X.p);
    std::swap(mdl.X.n, X.n);
    std::swap(mdl.T.p, T.p);
    std::swap(mdl.T.n, T.n);
    std::swap(mdl.mask.p, mask.p);
    std::swap(mdl.mask.n, mask.n);
    mdl.cap = cap;
  }
  coarse_features(g, mdl.X.get() + mdl.rows * kFeat, nbr.get());
  k_cl_targets<<<grid1((int64_t)M * kOut), 256, 0, s>>>(M, nbr.get(), g.cl.stats.get(), g.cl.C.get(),
                                                         mdl.T.get() + mdl.rows * kOut,
                                                         mdl.mask.get() + mdl.rows * kOut);
  STOKES_LAUNCHED();
  std::vector<float> hm((size_t)M * kOut);
  STOKES_CUDA(cudaMemcpyAsync(hm.data(), mdl.mask.get() + mdl.rows * kOut, 4 * hm.size(), cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaStreamSynchronize(s));
  for (float v : hm) mdl.count += v;
  mdl.rows += M;
  mdl.stats_ready = false;  // recomputed at the next training call
  g.cl.ready = false;       // the handle's coarse level was only a by-product
}

static void model_train(CoarseModel& mdl, int steps, double lr, double* loss_out) {
  require(mdl.rows > 0, "coarse model has no training samples", STOKES_ESTATE);
  cudaStream_t s = mdl.stream;
  if (!mdl.stats_ready) {
    mdl.stats.alloc(2 * kFeat + 2 * kOut);
    float* st = mdl.stats.get();
    k_col_stats<<<1, 64, 0, s>>>(mdl.X.get(), nullptr, mdl.rows, kFeat, st, st + kFeat);
    k_col_stats<<<(kOut + 63) / 64, 64, 0, s>>>(mdl.T.get(), mdl.mask.get(), mdl.rows, kOut, st + 2 * kFeat,
                                                st + 2 * kFeat + kOut);
    mdl.Tstd.alloc((size_t)mdl.rows * kOut);
    k_standardise<<<grid1(mdl.rows * kOut), 256, 0, s>>>(mdl.T.get(), mdl.rows, kOut, st + 2 * kFeat,
                                                         st + 2 * kFeat + kOut, mdl.Tstd.get());
    STOKES_LAUNCHED();
    mdl.stats_ready = true;
  }
  const float* st = mdl.stats.get();
  for (int it = 0; it < steps; ++it) {
    mdl.net.loss_and_grad(mdl.X.get(), mdl.Tstd.get(), mdl.mask.get(), mdl.rows, mdl.count, st, st + kFeat, s);
    mdl.net.adam(nullptr, lr, s);
  }
  double h = 0.0;
  if (steps > 0) {
    STOKES_CUDA(cudaMemcpyAsync(&h, mdl.net.loss.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  STOKES_CUDA(cudaStreamSynchronize(s));
  if (loss_out) *loss_out = h;
}

bool is_device_pointer(const void* p);

unsigned long long launches_coarse() { return tu_launches(); }

}  // namespace stokes

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

struct stokes_coarse_model {
  stokes::CoarseModel* m;
};

namespace {

using stokes::CoarseModel;
using stokes::DevBuf;
using stokes::Geom;
using stokes::require;

template <class F>
int run(F&& fn) {
  struct Ctx {
    F* f;
  } ctx{&fn};
  return stokes::guarded_call([](void* p) { (*static_cast<Ctx*>(p)->f)(); }, &ctx);
}

CoarseModel& model(const stokes_coarse_model* h) {
  require(h && h->m, "null coarse model");
  return *h->m;
}

Geom& geom(stokes_geom* h) {
  require(h && h->g, "null handle");
  return *h->g;
}

// A device view of a caller's float array (copied to `stage` when on the host).
template <class T>
const T* in_view(const T* p, size_t count, DevBuf<T>& stage, cudaStream_t s) {
  if (stokes::is_device_pointer(p)) return p;
  stage.alloc(count);
  STOKES_CUDA(cudaMemcpyAsync(stage.get(), p, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return stage.get();
}

// Copy `count` elements of a device array to the caller's array (host or
// device) and synchronise.
template <class T>
void out_copy(T* dst, const T* src, size_t count, cudaStream_t s) {
  STOKES_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDefault, s));
  STOKES_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int64_t stokes_coarse_model_num_params(void) {
  stokes::mlp::Net n(stokes::kFeat, stokes::kHidden, stokes::kOut);
  return n.n_params();
}

int stokes_coarse_model_create(const float* params, int64_t n_params, void* stream, stokes_coarse_model** out) {
  return run([&] {
    require(out && params, "null argument");
    auto* m = new CoarseModel();
    try {
      require(n_params == m->net.n_params(), "n_params must be stokes_coarse_model_num_params()");
      m->stream = (cudaStream_t)stream;
      std::vector<float> host(n_params);
      STOKES_CUDA(cudaMemcpyAsync(host.data(), params, 4 * n_params, cudaMemcpyDefault, m->stream));
      STOKES_CUDA(cudaStreamSynchronize(m->stream));
      m->net.init(host.data(), m->stream);
      STOKES_CUDA(cudaStreamSynchronize(m->stream));
    } catch (...) {
      delete m;
      throw;
    }
    *out = new stokes_coarse_model{m};
  });
}

int stokes_coarse_model_destroy(stokes_coarse_model* h) {
  return run([&] {
    if (!h) return;
    if (h->m) {
      cudaStreamSynchronize(h->m->stream);
      delete h->m;
    }
    delete h;
  });
}

int stokes_coarse_model_add_geometry(stokes_coarse_model* h, stokes_geom* gh) {
  return run([&] { stokes::model_add_geometry(model(h), geom(gh)); });
}

int64_t stokes_coarse_model_num_samples(const stokes_coarse_model* h) { return (h && h->m) ? h->m->rows : -1; }

int stokes_coarse_model_train(stokes_coarse_model* h, int steps, double lr, double* loss_out) {
  return run([&] {
    require(steps >= 0 && lr > 0 && std::isfinite(lr), "steps must be >= 0 and lr > 0");
    stokes::model_train(model(h), steps, lr, loss_out);
  });
}

int stokes_coarse_model_save(const stokes_coarse_model* h, float* params, float* stats) {
  return run([&] {
    CoarseModel& m = model(h);
    require(params != nullptr, "null params");
    out_copy(params, m.net.p.get(), (size_t)m.net.n_params(), m.stream);
    if (stats) {
      require(m.stats_ready, "coarse model has no standardisation yet (train first)", STOKES_ESTATE);
      out_copy(stats, m.stats.get(), (size_t)(2 * stokes::kFeat + 2 * stokes::kOut), m.stream);
    }
  });
}

int stokes_coarse_model_load(stokes_coarse_model* h, const float* params, const float* stats) {
  return run([&] {
    CoarseModel& m = model(h);
    require(params && stats, "null argument");
    DevBuf<float> sp, ss;
    const float* p = in_view(params, (size_t)m.net.n_params(), sp, m.stream);
    const int ns = 2 * stokes::kFeat + 2 * stokes::kOut;
    const float* q = in_view(stats, (size_t)ns, ss, m.stream);
    m.net.set_params(p, true, m.stream);
    m.stats.alloc(ns);
    STOKES_CUDA(cudaMemcpyAsync(m.stats.get(), q, 4 * ns, cudaMemcpyDeviceToDevice, m.stream));
    STOKES_CUDA(cudaStreamSynchronize(m.stream));
    m.stats_ready = true;
  });
}

int stokes_coarse_model_forward(stokes_coarse_model* h, const float* x, int64_t rows, float* y) {
  return run([&] {
    CoarseModel& m = model(h);
    require(x && y && rows >= 1, "bad arguments");
    DevBuf<float> sx;
    const float* xd = in_view(x, (size_t)rows * stokes::kFeat, sx, m.stream);
    m.net.forward(xd, rows, nullptr, nullptr, m.stream);
    const int ld = m.net.L.out_p;
    DevBuf<float> packed;
    packed.alloc((size_t)rows * stokes::kOut);
    STOKES_CUDA(cudaMemcpy2DAsync(packed.get(), 4 * stokes::kOut, m.net.y.get(), 4 * ld, 4 * stokes::kOut, rows,
                                  cudaMemcpyDeviceToDevice, m.stream));
    out_copy(y, packed.get(), (size_t)rows * stokes::kOut, m.stream);
  });
}

int stokes_coarse_model_loss_grad(stokes_coarse_model* h, const float* x, const float* t, const float* mask,
                                  int64_t rows, double* loss, float* grad) {
  return run([&] {
    CoarseModel& m = model(h);
    require(x && t && mask && grad && rows >= 1, "bad arguments");
    DevBuf<float> sx, st, sm;
    const float* xd = in_view(x, (size_t)rows * stokes::kFeat, sx, m.stream);
    const float* td = in_view(t, (size_t)rows * stokes::kOut, st, m.stream);
    const float* md = in_view(mask, (size_t)rows * stokes::kOut, sm, m.stream);
    std::vector<float> hm((size_t)rows * stokes::kOut);
    STOKES_CUDA(cudaMemcpyAsync(hm.data(), md, 4 * hm.size(), cudaMemcpyDefault, m.stream));
    STOKES_CUDA(cudaStreamSynchronize(m.stream));
    double cnt = 0.0;
    for (float v : hm) cnt += v;
    require(cnt > 0, "mask selects no outputs");
    m.net.loss_and_grad(xd, td, md, rows, cnt, nullptr, nullptr, m.stream);
    if (loss) out_copy(loss, m.net.loss.get(), 1, m.stream);
    out_copy(grad, m.net.grad.get(), (size_t)m.net.n_params(), m.stream);
  });
}

int stokes_coarse_model_adam_step(stokes_coarse_model* h, const float* grad, double lr) {
  return run([&] {
    CoarseModel& m = model(h);
    require(grad && lr > 0, "bad arguments");
    DevBuf<float> sg;
    const float* gd = in_view(grad, (size_t)m.net.n_params(), sg, m.stream);
    m.net.adam(gd, lr, m.stream);
    STOKES_CUDA(cudaStreamSynchronize(m.stream));
  });
}

int stokes_coarse_features(stokes_geom* gh, float* x, int* nbr) {
  return run([&] {
    Geom& g = geom(gh);
    require(x && nbr, "null argument");
    stokes::coarse_prepare(g);
    g.cl.ready = false;
    DevBuf<float> X;
    DevBuf<int> NB;
    X.alloc((size_t)g.cl.M * stokes::kFeat);
    NB.alloc((size_t)g.cl.M * stokes::kNbrs);
    stokes::coarse_features(g, X.get(), NB.get());
    out_copy(x, X.get(), (size_t)g.cl.M * stokes::kFeat, g.stream);
    out_copy(nbr, NB.get(), (size_t)g.cl.M * stokes::kNbrs, g.stream);
  });
}

int stokes_coarse_operator(stokes_geom* gh, double* y, double* e) {
  return run([&] {
    Geom& g = geom(gh);
    stokes::coarse_prepare(g);
    g.cl.ready = false;
    const int m = 3 * g.cl.M;
    if (y) out_copy(y, g.cl.Y.get(), (size_t)m * 2 * g.N, g.stream);
    if (e) {
      DevBuf<double> E;
      E.alloc((size_t)m * m);
      stokes::coarse_galerkin(g, E.get());
      out_copy(e, E.get(), (size_t)m * m, g.stream);
    }
  });
}

int stokes_precond_setup(stokes_geom* gh, int pc_kind, const stokes_coarse_model* mh) {
  return run([&] {
    Geom& g = geom(gh);
    require(pc_kind == STOKES_PC_NONE || pc_kind == STOKES_PC_BLOCKDIAG || pc_kind == STOKES_PC_BD_LEARNED ||
                pc_kind == STOKES_PC_BD_COARSE,
            "unknown pc_kind");
    require(pc_kind != STOKES_PC_BD_LEARNED || mh, "STOKES_PC_BD_LEARNED needs a coarse model");
    g.tg.ready = false;
    g.bd.ready = false;
    g.cl.ready = false;
    if (pc_kind == STOKES_PC_NONE) {
      g.bd.lu.release();
      g.bd.inv.release();
      g.tg.lu.release();
      return;
    }
    g.tg.lu.release();
    stokes::bd_setup(g);
    if (pc_kind == STOKES_PC_BD_COARSE) {
      stokes::coarse_setup_exact(g);
      g.cl.learned = false;
      g.cl.ready = true;
    } else if (pc_kind == STOKES_PC_BD_LEARNED) {
      stokes::coarse_setup_learned(g, model(mh));
      g.cl.learned = true;
      g.cl.ready = true;
    }
  });
}

}  // extern "C"
