// Block-diagonal preconditioner (Sec. 4.1 and its footnote: the diagonal
// blocks are the self-interactions of each pore and of the outer wall,
// assembled, factorised and inverted exactly).
//
// Block k is the restriction of A to component k (2 n_k unknowns), including
// its diagonal terms, its own completion (pores) or the wall term (outer).
// Storage: column-major m x m per block. Each block is LU-factorised with
// partial pivoting (FP64) and its inverse is formed from the factors:
//   m <= kSmall        one CTA per block factorises and inverts;
//   kSmall < m <= kInv blocked right-looking LU (panel of kNb columns, FP64
//                      tiled GEMM for the trailing update), inverse from the
//                      factors with many CTAs (one tile of columns each);
//   m > kInv           blocked LU, applied by a persistent triangular solve
//                      (bd_trsv.cu).
// The apply z = P^-1 v is a batched matrix-vector product with the inverses
// (memory-bound) plus the triangular solves of the largest blocks; the
// inner solves of the mixed-precision refinement use float copies of both.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int64_t kSmall = 512;
constexpr int64_t kInv = 4096;
constexpr int kNb = 64;     // panel width of the blocked LU

// ---------------------------------------------------------------------------
// Assembly
// ---------------------------------------------------------------------------
struct AsmArgs {
  const double2* pos;
  const double2* nrm;
  const double* w;
  const double4_32a* selfc;
  const double2* centre;
  const int64_t* node_off;  // per component
  const int64_t* elem_off;  // per component (n_comp + 1)
  const int64_t* rows;
  int n_comp;
  int outer;
  double* out;
};

__global__ void k_bd_assemble(int64_t total, AsmArgs a) {
  count_launch();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = a.n_comp - 1;  // block containing idx
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.elem_off[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const int64_t m = a.rows[k];
    const int64_t loc = idx - a.elem_off[k];
    const int64_t q = loc / m, r = loc - q * m;      // column-major (r, q)
    const int64_t i = a.node_off[k] + (r >> 1), j = a.node_off[k] + (q >> 1);
    const int al = (int)(r & 1), be = (int)(q & 1);
    const double2 xi = a.pos[i];
    double v = 0.0;
    if (i == j) {
      const double4_32a sc = a.selfc[i];
      const double ta = al ? sc.y : sc.x, tb = be ? sc.y : sc.x;
      v = sc.z * ta * tb - (al == be ? 0.5 : 0.0);
    } else {
      const double2 xj = a.pos[j];
      const double2 nj = a.nrm[j];
      const double rx = xi.x - xj.x, ry = xi.y - xj.y;
      const double r2 = rx * rx + ry * ry;
      const double rn = rx * nj.x + ry * nj.y;
      const double ra = al ? ry : rx, rb = be ? ry : rx;
      v = a.w[j] * kInvPi * rn * ra * rb / (r2 * r2);
    }
    const double wj = a.w[j];
    if (k != a.outer) {
      const double2 c = a.centre[k];
      const double rx = xi.x - c.x, ry = xi.y - c.y;
      const double r2 = rx * rx + ry * ry;
      const double ra = al ? ry : rx, rb = be ? ry : rx;
      double sl = ra * rb / r2;
      if (al == be) sl -= 0.5 * log(r2);
      const double2 xj = a.pos[j];
      const double dx = xj.x - c.x, dy = xj.y - c.y;
      const double perp_b = be ? -dx : dy;          // (x_j - c)^perp, component b
      const double rot_a = (al ? -rx : ry) / r2;    // r^perp / rho^2, component a
      v += kInv4Pi * wj * (sl + rot_a * perp_b);
    } else {
      const double2 ni = a.nrm[i];
      const double2 nj = a.nrm[j];
      v += (al ? ni.y : ni.x) * wj * (be ? nj.y : nj.x);
    }
    a.out[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// Block-wide argmax of |value| (ties: smallest index) for pivoting
// ---------------------------------------------------------------------------
__device__ void argmax_reduce(double& v, int64_t& ix) {
  __shared__ double sv[32];
  __shared__ int64_t si[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int64_t oi = __shfl_down_sync(0xffffffffu, ix, o);
    if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
  }
  if (lane == 0) { sv[wid] = v; si[wid] = ix; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sv[lane] : -1.0;
    ix = lane < nw ? si[lane] : INT64_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, v, o);
      const int64_t oi = __shfl_down_sync(0xffffffffu, ix, o);
      if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
    }
    if (lane == 0) { sv[0] = v; si[0] = ix; }
  }
  __syncthreads();
  v = sv[0];
  ix = si[0];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Small blocks: one CTA factorises (right-looking, partial pivoting) and
// inverts from the factors.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_lu_inv_small(const int* __restrict__ ids, const int64_t* __restrict__ rows,
               const int64_t* __restrict__ elem_off, const int64_t* __restrict__ piv_off,
               double* __restrict__ lu, double* __restrict__ inv, int* __restrict__ piv,
               int* __restrict__ status) {
  count_launch();
  const int k = ids[blockIdx.x];
  const int64_t m = rows[k];
  double* A = lu + elem_off[k];
  double* X = inv + elem_off[k];
  int* P = piv + piv_off[k];
  __shared__ int64_t s_p;
  __shared__ double s_inv;
  for (int64_t c = 0; c < m; ++c) {
    double best = -1.0;
    int64_t bi = INT64_MAX;
    for (int64_t r = c + threadIdx.x; r < m; r += blockDim.x) {
      const double v = fabs(A[c * m + r]);
      if (v > best) { best = v; bi = r; }
    }
    argmax_reduce(best, bi);
    if (threadIdx.x == 0) {
      if (bi >= m) { bi = c; atomicExch(status, 1); }  // no finite candidate (NaN column)
      s_p = bi;
      P[c] = (int)bi;
      const double pv = A[c * m + bi];
      if (pv == 0.0 || !isfinite(pv)) { atomicExch(status, 1); s_inv = 0.0; } else s_inv = 1.0 / pv;
    }
    __syncthreads();
    const int64_t p = s_p;
    if (p != c)
      for (int64_t q = threadIdx.x; q < m; q += blockDim.x) {
        const double t = A[q * m + c];
        A[q * m + c] = A[q * m + p];
        A[q * m + p] = t;
      }
    __syncthreads();
    const double iv = s_inv;
    for (int64_t r = c + 1 + threadIdx.x; r < m; r += blockDim.x) A[c * m + r] *= iv;
    __syncthreads();
    const int64_t n = m - c - 1;
    for (int64_t e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int64_t q = c + 1 + e / n, r = c + 1 + e % n;
      A[q * m + r] -= A[c * m + r] * A[q * m + c];
    }
    __syncthreads();
  }
  // X = P I: row r of P A is row perm[r] of A (interchanges applied in order)
  __shared__ int s_perm[kSmall];
  if (threadIdx.x == 0) {
    for (int64_t r = 0; r < m; ++r) s_perm[r] = (int)r;
    for (int64_t c = 0; c < m; ++c) {
      const int p = P[c];
      const int t = s_perm[c];
      s_perm[c] = s_perm[p];
      s_perm[p] = t;
    }
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int64_t q = e / m, r = e % m;
    X[e] = (s_perm[r] == q) ? 1.0 : 0.0;
  }
  __syncthreads();
  // forward: L (unit lower)
  for (int64_t c = 0; c < m; ++c) {
    const int64_t n = m - c - 1;
    for (int64_t e = threadIdx.x; e < n * m; e += blockDim.x) {
      const int64_t q = e / n, r = c + 1 + e % n;
      X[q * m + r] -= A[c * m + r] * X[q * m + c];
    }
    __syncthreads();
  }
  // backward: U
  for (int64_t c = m - 1; c >= 0; --c) {
    const double d = A[c * m + c];
    const double id = d != 0.0 ? 1.0 / d : 0.0;
    for (int64_t q = threadIdx.x; q < m; q += blockDim.x) X[q * m + c] *= id;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < c * m; e += blockDim.x) {
      const int64_t q = e / c, r = e % c;
      X[q * m + r] -= A[c * m + r] * X[q * m + c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Big blocks: blocked right-looking LU, one launch per step
// ---------------------------------------------------------------------------
// Per-CTA argmax of |A[r][c]|, r in [c, m).
__global__ void k_piv_partial(const double* __restrict__ A, int64_t m, int64_t c,
                              double* __restrict__ pv, int64_t* __restrict__ pi) {
  count_launch();
  double best = -1.0;
  int64_t bi = INT64_MAX;
  for (int64_t r = c + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(A[c * m + r]);
    if (v > best) { best = v; bi = r; }
  }
  argmax_reduce(best, bi);
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = best;
    pi[blockIdx.x] = bi;
    pv[256 + blockIdx.x] = bi < m ? A[c * m + bi] : 0.0;  // signed pivot candidate
  }
}

// Reduce the partials, record the pivot, swap rows c and p over all columns.
__global__ void k_piv_swap(double* __restrict__ A, int64_t m, int64_t c, int nparts,
                           const double* __restrict__ pv, const int64_t* __restrict__ pi,
                           int* __restrict__ piv, int* __restrict__ status, double* __restrict__ inv_out) {
  count_launch();
  __shared__ int64_t s_p;
  if (threadIdx.x == 0) {
    double best = -1.0, d = 0.0;
    int64_t bi = INT64_MAX;
    for (int b = 0; b < nparts; ++b)
      if (pv[b] > best || (pv[b] == best && pi[b] < bi)) { best = pv[b]; bi = pi[b]; d = pv[256 + b]; }
    if (bi >= m) { bi = c; d = 0.0; }  // no finite candidate (NaN column): flagged below
    s_p = bi;
    if (blockIdx.x == 0) {  // the signed pivot comes from the partials, not from A (no race with the swap)
      piv[c] = (int)bi;
      if (d == 0.0 || !isfinite(d)) { atomicExch(status, 1); *inv_out = 0.0; } else *inv_out = 1.0 / d;
    }
  }
  __syncthreads();
  const int64_t p = s_p;
  if (p != c)
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
      const double t = A[q * m + c];
      A[q * m + c] = A[q * m + p];
      A[q * m + p] = t;
    }
}

// Scale column c below the diagonal and update the panel columns (c, pend).
__global__ void k_panel_update(double* __restrict__ A, int64_t m, int64_t c, int64_t pend,
                               const double* __restrict__ inv_ptr) {
  count_launch();
  const double iv = *inv_ptr;
  for (int64_t r = c + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double l = A[c * m + r] * iv;
    A[c * m + r] = l;
    for (int64_t q = c + 1; q < pend; ++q) A[q * m + r] -= l * A[q * m + c];
  }
}

// U12 = L11^-1 A12 for columns [k0 + kb, m): one thread per column.
__global__ void k_trsm_row_panel(double* __restrict__ A, int64_t m, int64_t k0, int kb) {
  count_launch();
  const int64_t q = k0 + kb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= m) return;
  double* col = A + q * m + k0;
  double x[kNb];
#pragma unroll
  for (int c = 0; c < kNb; ++c) x[c] = c < kb ? col[c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    if (c >= kb) break;
    const double xc = x[c];
#pragma unroll
    for (int r = c + 1; r < kNb; ++r)
      if (r < kb) x[r] -= A[(k0 + c) * m + k0 + r] * xc;
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c)
    if (c < kb) col[c] = x[c];
}

// C[r][q] -= sum_c L[r][c] U[c][q] over the trailing block: 64 x 64 tile per
// CTA, 256 threads with 4 x 4 outputs each; operands staged in shared memory
// 16 columns of L / rows of U at a time.
__global__ void __launch_bounds__(256)
k_gemm_trailing(double* __restrict__ A, int64_t m, int64_t k0, int kb) {
  count_launch();
  constexpr int kK = 16;
  __shared__ double sL[kK][64 + 1];  // [c][r]
  __shared__ double sU[kK][64 + 1];  // [c][q]
  const int64_t base = k0 + kb;
  const int64_t r0 = base + blockIdx.x * 64, q0 = base + blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int cb = 0; cb < kb; cb += kK) {
    __syncthreads();
    for (int e = threadIdx.x; e < kK * 64; e += 256) {
      const int c = e / 64, rr = e % 64;
      const int64_t r = r0 + rr, q = q0 + rr;
      const bool cin = cb + c < kb;
      sL[c][rr] = (cin && r < m) ? A[(k0 + cb + c) * m + r] : 0.0;
      sU[c][rr] = (cin && q < m) ? A[q * m + k0 + cb + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kK; ++c) {
      double l[4], u[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { l[a] = sL[c][tx + 16 * a]; u[a] = sU[c][ty + 16 * a]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t q = q0 + ty + 16 * b;
    if (q >= m) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t r = r0 + tx + 16 * a;
      if (r < m) A[q * m + r] -= acc[a][b];
    }
  }
}

// Inverse of a big block from its factors: each CTA solves for a tile of 8
// columns of the identity (rows permuted by perm). The CTAs step through the
// m columns of L and U in lockstep with a block barrier per step, so narrow
// tiles (m / 8 CTAs: 128 for a 1024-row wall block) spread the FP64 work
// over more SMs than wide ones would.
constexpr int kInvCols = 8;
__global__ void __launch_bounds__(256)
k_inv_from_lu(const double* __restrict__ A, int64_t m, const int* __restrict__ perm,
              double* __restrict__ X) {
  count_launch();
  const int64_t q0 = blockIdx.x * (int64_t)kInvCols;
  const int nq = (int)imin64(kInvCols, m - q0);
  // X[:, q] = P e_q: row r holds 1 where perm[r] == q
  for (int64_t e = threadIdx.x; e < (int64_t)nq * m; e += blockDim.x) {
    const int64_t q = q0 + e / m, r = e % m;
    X[q * m + r] = (perm[r] == q) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int64_t c = 0; c < m; ++c) {
    const int64_t n = m - c - 1;
    for (int64_t e = threadIdx.x; e < n * nq; e += blockDim.x) {
      const int64_t q = q0 + e / n, r = c + 1 + e % n;
      X[q * m + r] -= A[c * m + r] * X[q * m + c];
    }
    __syncthreads();
  }
  for (int64_t c = m - 1; c >= 0; --c) {
    const double d = A[c * m + c];
    const double id = d != 0.0 ? 1.0 / d : 0.0;
    if (threadIdx.x < nq) X[(q0 + threadIdx.x) * m + c] *= id;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < c * nq; e += blockDim.x) {
      const int64_t q = q0 + e / c, r = e % c;
      X[q * m + r] -= A[c * m + r] * X[q * m + c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Apply
// ---------------------------------------------------------------------------
// z_k = X_k v_k for the blocks in `ids`; CTA (b, s) computes rows
// [64 s, 64 s + 64) of block ids[b]; the 256 threads split the columns in
// four interleaved phases and combine them in shared memory.
template <class T, bool kAcc = false>
__global__ void __launch_bounds__(256)
k_bd_gemv(const int* __restrict__ ids, const int64_t* __restrict__ rows,
          const int64_t* __restrict__ elem_off, const int64_t* __restrict__ node_off,
          const T* __restrict__ X, const double* __restrict__ v, double* __restrict__ z,
          const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int k = ids[blockIdx.x];
  const int64_t m = rows[k];
  const int64_t r0 = blockIdx.y * (int64_t)64;
  if (r0 >= m) return;
  const T* Xk = X + elem_off[k];
  const double* vk = v + 2 * node_off[k];
  extern __shared__ double sv_raw[];
  T* sv = reinterpret_cast<T*>(sv_raw);
  __shared__ T red[4][64];
  for (int64_t q = threadIdx.x; q < m; q += blockDim.x) sv[q] = (T)vk[q];
  __syncthreads();
  const int rr = threadIdx.x & 63, ph = threadIdx.x >> 6;
  const int64_t r = r0 + rr;
  T acc = 0;
  if (r < m)
    for (int64_t q = ph; q < m; q += 4) acc += Xk[q * m + r] * sv[q];
  red[ph][rr] = acc;
  __syncthreads();
  if (ph == 0 && r < m) {
    const double val = (double)((red[0][rr] + red[1][rr]) + (red[2][rr] + red[3][rr]));
    double* zp = z + 2 * node_off[k] + r;
    *zp = kAcc ? *zp + val : val;
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

}  // namespace

void bd_init_attributes() {
  static bool inited = false;
  if (inited) return;
  STOKES_CUDA(cudaFuncSetAttribute(k_bd_gemv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kInv * sizeof(double))));
  STOKES_CUDA(cudaFuncSetAttribute(k_bd_gemv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
  STOKES_CUDA(cudaFuncSetAttribute(k_bd_gemv<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kInv * sizeof(double))));
  STOKES_CUDA(cudaFuncSetAttribute(k_bd_gemv<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
  inited = true;
}

static void bd_setup_impl(Geom& g, bool skip_wall);

void bd_setup(Geom& g) { bd_setup_impl(g, false); }

// Blocks of the pores only (the wall is left out): used next to the
// two-grid coarse solve.
void bd_setup_pores(Geom& g, bool skip_wall) { bd_setup_impl(g, skip_wall); }

static void bd_setup_impl(Geom& g, bool skip_wall) {
  bd_init_attributes();
  BlockDiag& b = g.bd;
  b.ready = false;
  cudaStream_t s = g.stream;
  double flops = 0.0;  // (2/3) m^3 for the LU, + 4/3 m^3 more where inverted
  for (int k = 0; k < g.n_comp; ++k) {
    const double m = 2.0 * (double)(g.off[k + 1] - g.off[k]);
    flops += (m <= kInv ? 2.0 : 2.0 / 3.0) * m * m * m;
  }
  const int ps = g.prof.begin(kProfBdSetup, flops, s);
  const int nc = g.n_comp;
  b.rows.assign(nc, 0);
  b.elem_off.assign(nc + 1, 0);
  b.piv_off.assign(nc + 1, 0);
  b.small_ids.clear();
  b.inv_ids.clear();
  b.tri_ids.clear();
  for (int k = 0; k < nc; ++k) {
    const int64_t m = (skip_wall && k == g.outer) ? 0 : 2 * (g.off[k + 1] - g.off[k]);
    b.rows[k] = m;
    b.elem_off[k + 1] = b.elem_off[k] + m * m;
    b.piv_off[k + 1] = b.piv_off[k] + m;
    if (m == 0) continue;
    if (m <= kSmall) b.small_ids.push_back(k);
    (m <= kInv ? b.inv_ids : b.tri_ids).push_back(k);
    b.max_inv_rows = 0;
  }
  for (int k : b.inv_ids) b.max_inv_rows = std::max(b.max_inv_rows, b.rows[k]);
  const int64_t total = b.elem_off[nc];
  b.lu.alloc(std::max<int64_t>(total, 1));
  b.inv.alloc(std::max<int64_t>(total, 1));
  b.piv.alloc(b.piv_off[nc]);
  b.perm.alloc(b.piv_off[nc]);
  b.d_elem_off.alloc(nc + 1);
  b.d_rows.alloc(nc);
  b.d_node_off.alloc(nc + 1);
  b.d_piv_off.alloc(nc + 1);
  b.d_small_ids.alloc(std::max<size_t>(1, b.small_ids.size()));
  b.d_inv_ids.alloc(std::max<size_t>(1, b.inv_ids.size()));
  b.status.alloc(1);
  b.pv.alloc(512);
  b.pi.alloc(256);
  b.ivp.alloc(1);
  STOKES_CUDA(cudaMemcpyAsync(b.d_elem_off.get(), b.elem_off.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemcpyAsync(b.d_piv_off.get(), b.piv_off.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemcpyAsync(b.d_rows.get(), b.rows.data(), 8 * nc, cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemcpyAsync(b.d_node_off.get(), g.off.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, s));
  if (!b.small_ids.empty())
    STOKES_CUDA(cudaMemcpyAsync(b.d_small_ids.get(), b.small_ids.data(), 4 * b.small_ids.size(),
                                cudaMemcpyHostToDevice, s));
  if (!b.inv_ids.empty())
    STOKES_CUDA(cudaMemcpyAsync(b.d_inv_ids.get(), b.inv_ids.data(), 4 * b.inv_ids.size(),
                                cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemsetAsync(b.status.get(), 0, sizeof(int), s));

  AsmArgs a{g.pos.get(), g.nrm.get(), g.w.get(), g.selfc.get(), g.centre.get(), g.d_off.get(),
            b.d_elem_off.get(), b.d_rows.get(), nc, g.outer, b.lu.get()};
  const int64_t want = (total + 255) / 256;
  k_bd_assemble<<<(unsigned)imin64(want, 152 * 64), 256, 0, s>>>(total, a);
  STOKES_LAUNCHED();

  if (!b.small_ids.empty()) {
    k_lu_inv_small<<<(unsigned)b.small_ids.size(), 256, 0, s>>>(b.d_small_ids.get(), b.d_rows.get(),
                                                                 b.d_elem_off.get(), b.d_piv_off.get(),
                                                                 b.lu.get(), b.inv.get(), b.piv.get(),
                                                                 b.status.get());
    STOKES_LAUNCHED();
  }
  for (int k = 0; k < nc; ++k) {
    const int64_t m = b.rows[k];
    if (m <= kSmall) continue;  // (also the skipped wall, m = 0)
    double* A = b.lu.get() + b.elem_off[k];
    int* P = b.piv.get() + b.piv_off[k];
    for (int64_t k0 = 0; k0 < m; k0 += kNb) {
      const int kb = (int)imin64(kNb, m - k0);
      for (int64_t c = k0; c < k0 + kb; ++c) {
        const int parts = (int)imin64(256, (m - c + 255) / 256);
        k_piv_partial<<<parts, 256, 0, s>>>(A, m, c, b.pv.get(), b.pi.get());
        k_piv_swap<<<(unsigned)imin64(64, (m + 255) / 256), 256, 0, s>>>(
            A, m, c, parts, b.pv.get(), b.pi.get(), P, b.status.get(), b.ivp.get());
        const int64_t nr = m - c - 1;
        if (nr > 0)
          k_panel_update<<<(unsigned)std::max<int64_t>(1, imin64(1024, (nr + 127) / 128)), 128, 0, s>>>(
              A, m, c, k0 + kb, b.ivp.get());
      }
      const int64_t rest = m - k0 - kb;
      if (rest > 0) {
        k_trsm_row_panel<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(A, m, k0, kb);
        dim3 grid((unsigned)((rest + 63) / 64), (unsigned)((rest + 63) / 64));
        k_gemm_trailing<<<grid, 256, 0, s>>>(A, m, k0, kb);
      }
      STOKES_LAUNCHED();
    }
  }
  // row permutations (P A = L U) of the blocked-LU blocks, from the interchanges
  std::vector<int> hpiv(b.piv_off[nc]);
  STOKES_CUDA(cudaMemcpyAsync(hpiv.data(), b.piv.get(), 4 * hpiv.size(), cudaMemcpyDeviceToHost, s));
  int hstatus = 0;
  STOKES_CUDA(cudaMemcpyAsync(&hstatus, b.status.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaStreamSynchronize(s));
  require(hstatus == 0, "block-diagonal preconditioner: singular block (zero pivot)", STOKES_EBREAKDOWN);
  std::vector<int> hperm(b.piv_off[nc]);
  for (int k = 0; k < nc; ++k) {
    int* p = hperm.data() + b.piv_off[k];
    const int64_t m = b.rows[k];
    for (int64_t r = 0; r < m; ++r) p[r] = (int)r;
    for (int64_t c = 0; c < m; ++c) std::swap(p[c], p[hpiv[b.piv_off[k] + c]]);
  }
  STOKES_CUDA(cudaMemcpyAsync(b.perm.get(), hperm.data(), 4 * hperm.size(), cudaMemcpyHostToDevice, s));
  for (int k = 0; k < nc; ++k) {
    const int64_t m = b.rows[k];
    if (m <= kSmall || m > kInv) continue;  // m = 0 for a skipped wall
    k_inv_from_lu<<<(unsigned)((m + kInvCols - 1) / kInvCols), 256, 0, s>>>(
        b.lu.get() + b.elem_off[k], m, b.perm.get() + b.piv_off[k], b.inv.get() + b.elem_off[k]);
    STOKES_LAUNCHED();
  }
  // single-precision copies: all inverses, and the factors of the blocks
  // applied by triangular solves
  b.inv32.alloc(std::max<int64_t>(total, 1));
  if (total > 0) {
    k_to_f32<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, s>>>(b.inv.get(), b.inv32.get(),
                                                                                       total);
    STOKES_LAUNCHED();
  }
  b.lu32_off.assign(nc, -1);
  int64_t tri_total = 0, tri_max = 0;
  for (int k : b.tri_ids) {
    b.lu32_off[k] = tri_total;
    tri_total += b.rows[k] * b.rows[k];
    tri_max = std::max(tri_max, b.rows[k]);
  }
  if (tri_total) {
    b.lu32.alloc(tri_total);
    const int64_t words = lu_solve_work_words(tri_max, sizeof(double));
    b.trsv_work.alloc(words);
    STOKES_CUDA(cudaMemsetAsync(b.trsv_work.get(), 0, words * sizeof(unsigned long long), s));
    b.trsv_gen = 0;
    b.tinv_off.assign(nc, -1);
    int64_t ti_total = 0;
    for (int k : b.tri_ids) {
      b.tinv_off[k] = ti_total;
      ti_total += lu_tile_inverse_elems(b.rows[k]);
    }
    b.tinv64.alloc(ti_total);
    for (int k : b.tri_ids)
      lu_tile_inverses<double>(s, b.lu.get() + b.elem_off[k], b.rows[k], b.tinv64.get() + b.tinv_off[k]);
    for (int k : b.tri_ids) {
      const int64_t mm = b.rows[k] * b.rows[k];
      k_to_f32<<<(unsigned)std::min<int64_t>((mm + 255) / 256, 152 * 32), 256, 0, s>>>(
          b.lu.get() + b.elem_off[k], b.lu32.get() + b.lu32_off[k], mm);
      STOKES_LAUNCHED();
      // float explicit inverse for the single-precision applies
      invert_from_lu32(g, b.lu32.get() + b.lu32_off[k], b.rows[k], b.perm.get() + b.piv_off[k],
                       b.inv32.get() + b.elem_off[k]);
    }
    b.d_tri_ids.alloc(b.tri_ids.size());
    STOKES_CUDA(cudaMemcpyAsync(b.d_tri_ids.get(), b.tri_ids.data(), 4 * b.tri_ids.size(), cudaMemcpyHostToDevice, s));
    b.max_tri_rows = tri_max;
  }
  g.prof.end(ps, s);
  STOKES_CUDA(cudaStreamSynchronize(s));
  b.ready = true;
}

void bd_apply(Geom& g, const double* v, double* z, const int* done, bool f32) {
  BlockDiag& b = g.bd;
  require(b.ready, "preconditioner not set up", STOKES_ESTATE);
  cudaStream_t s = g.stream;
  // algorithmic bytes: every block's inverse or factors once, v in, z out
  const double wbytes = f32 ? 4.0 : 8.0;
  const int pb = g.prof.begin(kProfBdApply, wbytes * (double)b.elem_off[g.n_comp] + 32.0 * (double)g.N, s);
  if (!b.inv_ids.empty()) {
    dim3 grid((unsigned)b.inv_ids.size(), (unsigned)((b.max_inv_rows + 63) / 64));
    const size_t sm = b.max_inv_rows * (f32 ? sizeof(float) : sizeof(double));
    if (f32)
      k_bd_gemv<float><<<grid, 256, sm, s>>>(b.d_inv_ids.get(), b.d_rows.get(), b.d_elem_off.get(),
                                             b.d_node_off.get(), b.inv32.get(), v, z, done);
    else
      k_bd_gemv<double><<<grid, 256, sm, s>>>(b.d_inv_ids.get(), b.d_rows.get(), b.d_elem_off.get(),
                                              b.d_node_off.get(), b.inv.get(), v, z, done);
    STOKES_LAUNCHED();
  }
  if (f32 && !b.tri_ids.empty()) {
    // the largest blocks have float explicit inverses too
    dim3 grid((unsigned)b.tri_ids.size(), (unsigned)((b.max_tri_rows + 63) / 64));
    k_bd_gemv<float><<<grid, 256, b.max_tri_rows * sizeof(float), s>>>(
        b.d_tri_ids.get(), b.d_rows.get(), b.d_elem_off.get(), b.d_node_off.get(), b.inv32.get(), v, z, done);
    STOKES_LAUNCHED();
  } else {
    for (int k : b.tri_ids) {
      const int64_t m = b.rows[k];
      const int64_t o = 2 * g.off[k];
      lu_solve_persistent<double>(g, b.lu.get() + b.elem_off[k], m, b.perm.get() + b.piv_off[k],
                                  b.tinv64.get() + b.tinv_off[k], v + o, z + o, b.trsv_work.get(), b.trsv_gen,
                                  done);
    }
  }
  g.prof.end(pb, s);
}

// z += B^-1 h over the blocks that have explicit inverses (the pores, when
// the wall block was left out).
void bd_apply_pores_accumulate(Geom& g, const double* h, double* z, const int* done, bool f32) {
  BlockDiag& b = g.bd;
  if (b.inv_ids.empty()) return;
  dim3 grid((unsigned)b.inv_ids.size(), (unsigned)((b.max_inv_rows + 63) / 64));
  const size_t sm = b.max_inv_rows * (f32 ? sizeof(float) : sizeof(double));
  if (f32)
    k_bd_gemv<float, true><<<grid, 256, sm, g.stream>>>(b.d_inv_ids.get(), b.d_rows.get(), b.d_elem_off.get(),
                                                       b.d_node_off.get(), b.inv32.get(), h, z, done);
  else
    k_bd_gemv<double, true><<<grid, 256, sm, g.stream>>>(b.d_inv_ids.get(), b.d_rows.get(), b.d_elem_off.get(),
                                                        b.d_node_off.get(), b.inv.get(), h, z, done);
  STOKES_LAUNCHED();
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_bd() { return tu_launches(); }
}  // namespace stokes
