// Batched operator and solver over many geometries and right-hand sides
// (the paper has no counterpart: it solves one geometry and one right-hand
// side at a time on a CPU).
//
// Operator: y_{g,r} = A_g sigma_{g,r} for every geometry g and right-hand
// side r < R in ONE persistent launch of the pair kernel: the CTAs pull
// work items (geometry, target block, source range) from an atomic counter,
// so geometries of very different sizes share the GPU without a launch per
// geometry; within an item the R densities share the pair geometry (r,
// 1/rho^2 and r.a are formed once for all R). The moments, diagonal, jump,
// completion and wall terms are the single-geometry kernels per system.
//
// Solver: right-preconditioned flexible GMRES(m) on all systems in lockstep.
// Each step: z = P^-1 v per system (the geometry's block-diagonal or
// two-grid preconditioner, float copies), the batched operator, classical
// Gram-Schmidt twice with dot products reduced per system, Givens rotations
// with one thread per system. A restart cycle of m steps is captured once
// as a CUDA graph and replayed for every cycle; converged systems' kernels
// return at once (per-system flag), and the pair kernel returns once all
// systems have converged. True residuals at cycle ends use the native FP64
// operator. STOKES_MIXED_IR wraps FP32 inner cycles in FP64 iterative
// refinement per system.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dlp_common.cuh"

namespace stokes {

namespace {

constexpr int kMaxRhs = 4;
constexpr int kRChunk = 2048;  // vector elements per CTA in the reductions
constexpr int kMaxSystems = 1024;

// One geometry in the device table of the persistent pair kernels.
struct BGeom {
  int64_t N;          // nodes: sources and targets
  int64_t chunk;      // sources per split
  int64_t item0;      // index of this geometry's first work item
  int64_t tblocks;    // target blocks
  int splits;
  int pad;
  const float4* f32_src;  // FP32: x_hi, y_hi, a_x, a_y
  const float2* f32_lo;   // FP32: x_lo, y_lo
  const float2* df_grid;  // double-float: position on the 2^-8 grid
  const float4* df_pos;   // double-float: position remainder
  const float4* df_a;     // double-float: a = w n / pi
  const double2* tgt;     // node positions (the targets)
  const double2* sig[kMaxRhs];  // density r of column `col` at sig[r] + col * sig_stride
  int64_t sig_stride;
  double2* part;          // partial sums [splits][R][N]
};

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Work item -> geometry (binary search on item0).
__device__ __forceinline__ int find_geom(const BGeom* __restrict__ geoms, int n_geoms, int64_t item) {
  int lo = 0, hi = n_geoms - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (geoms[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// FP32 pair sums (same arithmetic as the single-geometry FP32 kernel) for R
// right-hand sides, persistent over the work items.
template <int TH, int TPT, int TILE, int R>
__global__ void __launch_bounds__(TH)
kb_pairs_f32(const BGeom* __restrict__ geoms, int n_geoms, int64_t n_items, int col,
             unsigned long long* __restrict__ counter, const int* __restrict__ all_done) {
  count_launch();
  if (all_done && *all_done) return;
  __shared__ float4 s_a[TILE];
  __shared__ float2 s_l[TILE];
  __shared__ float2 s_s[R][TILE];
  __shared__ long long s_item;
  for (;;) {
    __syncthreads();  // every thread has read s_item and the previous tiles
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) return;
    const BGeom& G = geoms[find_geom(geoms, n_geoms, item)];
    const int64_t N = G.N;
    const int64_t local = item - G.item0;
    const int64_t tb = local % G.tblocks, sp = local / G.tblocks;
    const int64_t ib = tb * (int64_t)(TPT * TH) + threadIdx.x;
    float xh[TPT], yh[TPT], xl[TPT], yl[TPT];
    double ux[TPT][R], uy[TPT][R];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
      const int64_t i = ib + t * TH;
      const double2 x = i < N ? G.tgt[i] : make_double2(0.0, 0.0);
      xh[t] = (float)x.x;
      yh[t] = (float)x.y;
      xl[t] = (float)(x.x - (double)xh[t]);
      yl[t] = (float)(x.y - (double)yh[t]);
#pragma unroll
      for (int r = 0; r < R; ++r) ux[t][r] = uy[t][r] = 0.0;
    }
    const int64_t j0 = sp * G.chunk;
    const int64_t j1 = imin64(N, j0 + G.chunk);
    for (int64_t t0 = j0; t0 < j1; t0 += TILE) {
      __syncthreads();
      for (int q = threadIdx.x; q < TILE; q += TH) {
        const int64_t j = t0 + q;
        if (j < j1) {
          s_a[q] = G.f32_src[j];
          s_l[q] = G.f32_lo[j];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double2 sg = G.sig[r][(int64_t)col * G.sig_stride + j];
            s_s[r][q] = make_float2((float)sg.x, (float)sg.y);
          }
        } else {
          s_a[q] = make_float4(1e18f, 1e18f, 0.f, 0.f);
          s_l[q] = make_float2(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < R; ++r) s_s[r][q] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      float fx[TPT][R], fy[TPT][R];
#pragma unroll
      for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) fx[t][r] = fy[t][r] = 0.f;
#pragma unroll 2
      for (int q = 0; q < TILE; ++q) {
        const float4 a = s_a[q];
        const float2 l = s_l[q];
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
          const float rx = (xh[t] - a.x) + (xl[t] - l.x);
          const float ry = (yh[t] - a.y) + (yl[t] - l.y);
          // + 1e-30: the self pair (r = 0) contributes exactly 0
          const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1e-30f));
          const float inv = rcp_approx(r2);
          const float di = fmaf(rx, a.z, ry * a.w) * inv;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 sg = s_s[r][q];
            const float c = di * (fmaf(rx, sg.x, ry * sg.y) * inv);
            fx[t][r] = fmaf(c, rx, fx[t][r]);
            fy[t][r] = fmaf(c, ry, fy[t][r]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          ux[t][r] += fx[t][r];
          uy[t][r] += fy[t][r];
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
      const int64_t i = ib + t * TH;
      if (i < N)
#pragma unroll
        for (int r = 0; r < R; ++r) G.part[(sp * R + r) * N + i] = make_double2(ux[t][r], uy[t][r]);
    }
  }
}

using dlp::df32;

__device__ __forceinline__ void acc_prod(df32& acc, df32 c, df32 r) {
  const float p = c.h * r.h;
  float pe = fmaf(c.h, r.h, -p);
  pe = fmaf(c.h, r.l, pe);
  pe = fmaf(c.l, r.h, pe);
  const df32 s = dlp::two_sum(acc.h, p);
  acc.h = s.h;
  acc.l += s.l + pe;
}

// Double-float pair sums (the arithmetic of the single-geometry double-float
// kernel) for R right-hand sides, persistent over the work items.
template <int TH, int TILE, int R>
__global__ void __launch_bounds__(TH)
kb_pairs_df64(const BGeom* __restrict__ geoms, int n_geoms, int64_t n_items, int col,
              unsigned long long* __restrict__ counter, const int* __restrict__ all_done) {
  count_launch();
  if (all_done && *all_done) return;
  __shared__ float2 s_g[TILE];
  __shared__ float4 s_p[TILE];
  __shared__ float4 s_a[TILE];
  __shared__ float4 s_s[R][TILE];  // sigma_x hi, sigma_y hi, sigma_x lo, sigma_y lo
  __shared__ long long s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) return;
    const BGeom& G = geoms[find_geom(geoms, n_geoms, item)];
    const int64_t N = G.N;
    const int64_t local = item - G.item0;
    const int64_t tb = local % G.tblocks, sp = local / G.tblocks;
    const int64_t i = tb * (int64_t)TH + threadIdx.x;
    const double2 x = i < N ? G.tgt[i] : make_double2(0.0, 0.0);
    const double gx = rint(x.x * 256.0) * (1.0 / 256.0), gy = rint(x.y * 256.0) * (1.0 / 256.0);
    const float GX = (float)gx, GY = (float)gy;
    const df32 X = dlp::df_from_double(x.x - gx), Y = dlp::df_from_double(x.y - gy);
    double ux[R], uy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ux[r] = uy[r] = 0.0;
    const int64_t j0 = sp * G.chunk;
    const int64_t j1 = imin64(N, j0 + G.chunk);
    for (int64_t t0 = j0; t0 < j1; t0 += TILE) {
      __syncthreads();
      for (int q = threadIdx.x; q < TILE; q += TH) {
        const int64_t j = t0 + q;
        if (j < j1) {
          s_g[q] = G.df_grid[j];
          s_p[q] = G.df_pos[j];
          s_a[q] = G.df_a[j];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const double2 sg = G.sig[r][(int64_t)col * G.sig_stride + j];
            const df32 sx = dlp::df_from_double(sg.x), sy = dlp::df_from_double(sg.y);
            s_s[r][q] = make_float4(sx.h, sy.h, sx.l, sy.l);
          }
        } else {
          s_g[q] = make_float2(1e18f, 1e18f);
          s_p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          s_a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int r = 0; r < R; ++r) s_s[r][q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      __syncthreads();
      df32 ax[R], ay[R];
#pragma unroll
      for (int r = 0; r < R; ++r) ax[r] = ay[r] = df32{0.f, 0.f};
      for (int q = 0; q < TILE; ++q) {
        const float2 gq = s_g[q];
        const float4 p = s_p[q];
        const float4 a = s_a[q];
        df32 lx = dlp::two_diff(X.h, p.x);
        lx.l += X.l - p.z;
        df32 ly = dlp::two_diff(Y.h, p.y);
        ly.l += Y.l - p.w;
        df32 rx = dlp::fast_two_sum(GX - gq.x, lx.h);
        rx.l += lx.l;
        df32 ry = dlp::fast_two_sum(GY - gq.y, ly.h);
        ry.l += ly.l;
        const float px = rx.h * rx.h;
        float ex = fmaf(rx.h, rx.h, -px);
        ex = fmaf(rx.h + rx.h, rx.l, ex);
        const float py = ry.h * ry.h;
        float ey = fmaf(ry.h, ry.h, -py);
        ey = fmaf(ry.h + ry.h, ry.l, ey);
        df32 r2 = dlp::two_sum(px, py);
        r2 = dlp::fast_two_sum(r2.h, r2.l + (ex + ey));
        r2.h += 1e-30f;  // the self pair contributes exactly 0
        const float y0 = __frcp_rn(r2.h);
        float tt = fmaf(-r2.h, y0, 1.0f);
        tt = fmaf(-r2.l, y0, tt);
        const df32 inv = {y0, y0 * tt};
        const df32 di = dlp::df_mul(dlp::df_dot2(rx, ry, {a.x, a.z}, {a.y, a.w}), inv);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 s = s_s[r][q];
          const df32 e = dlp::df_dot2(rx, ry, {s.x, s.z}, {s.y, s.w});
          const df32 c = dlp::df_mul(di, dlp::df_mul(e, inv));
          acc_prod(ax[r], c, rx);
          acc_prod(ay[r], c, ry);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        ux[r] += dlp::df_to_double(ax[r]);
        uy[r] += dlp::df_to_double(ay[r]);
      }
    }
    if (i < N)
#pragma unroll
      for (int r = 0; r < R; ++r) G.part[(sp * R + r) * N + i] = make_double2(ux[r], uy[r]);
  }
}

constexpr int kF32Threads = 128, kF32Tpt = 2, kF32Tile = 128;
constexpr int kDFThreads = 128, kDFTile = 64;

template <int R>
void launch_pairs_r(int precision, const BGeom* tab, int n_geoms, int64_t n_items, int col,
                    unsigned long long* counter, const int* all_done, cudaStream_t s) {
  static int occ_f32 = 0, occ_df = 0;
  if (precision == STOKES_FP32) {
    auto k = kb_pairs_f32<kF32Threads, kF32Tpt, kF32Tile, R>;
    if (!occ_f32) STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f32, k, kF32Threads, 0));
    const int64_t grid = std::min<int64_t>(n_items, 152 * (int64_t)std::max(occ_f32, 1));
    k<<<(unsigned)grid, kF32Threads, 0, s>>>(tab, n_geoms, n_items, col, counter, all_done);
  } else {
    auto k = kb_pairs_df64<kDFThreads, kDFTile, R>;
    if (!occ_df) STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_df, k, kDFThreads, 0));
    const int64_t grid = std::min<int64_t>(n_items, 152 * (int64_t)std::max(occ_df, 1));
    k<<<(unsigned)grid, kDFThreads, 0, s>>>(tab, n_geoms, n_items, col, counter, all_done);
  }
  STOKES_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Batched Krylov kernels: blockIdx.y (or the thread, for the Givens step)
// is the system; a system whose state[0] is set returns at once.
// ---------------------------------------------------------------------------
struct BSys {
  int64_t n;        // vector length 2N
  double* V;        // (m + 1) basis vectors of n
  double* Z;        // m preconditioned vectors
  double* w;        // A z_j, orthogonalised in place
  double* x;        // iterate
  double* r;        // residual
  double* H;        // (m + 1) x m, column-major
  double* cs;
  double* sn;
  double* g;        // m + 1
  double* y;        // 2 (m + 1): coefficients, then back-substitution work
  double* partial;  // nblk x (m + 1)
  double* hvec;     // m + 1
  double* normpart; // nblk
  double* scal;     // [0] 1/h_{j+1,j}, [1] beta, [2] 1/beta, [3] rhs norm, [4] estimate, [5] tol
  int* state;       // [0] done, [1] columns, [2] breakdown
};

__global__ void __launch_bounds__(256)
kb_dot_partial(const BSys* __restrict__ sys, int j, int m) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  if (S.state[0]) return;
  const int64_t i0 = blockIdx.x * (int64_t)kRChunk;
  if (i0 >= S.n) return;
  __shared__ double sw[kRChunk];
  const int cn = (int)imin64(kRChunk, S.n - i0);
  for (int e = threadIdx.x; e < cn; e += blockDim.x) sw[e] = S.w[i0 + e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = wid; k <= j; k += nw) {
    const double* v = S.V + k * S.n + i0;
    double acc = 0.0;
    for (int e = lane; e < cn; e += 32) acc = fma(v[e], sw[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) S.partial[blockIdx.x * (int64_t)(m + 1) + k] = acc;
  }
}

__global__ void kb_reduce(const BSys* __restrict__ sys, int j, int m, int pass) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  if (S.state[0]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > j) return;
  const int nblk = (int)((S.n + kRChunk - 1) / kRChunk);
  double h = 0.0;
  for (int b = 0; b < nblk; ++b) h += S.partial[(int64_t)b * (m + 1) + k];
  S.hvec[k] = h;
  double* hc = S.H + (int64_t)j * (m + 1);
  hc[k] = pass ? hc[k] + h : h;
}

__global__ void __launch_bounds__(256)
kb_orth_update(const BSys* __restrict__ sys, int j, int pass) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  if (S.state[0]) return;
  const int64_t i0 = blockIdx.x * (int64_t)kRChunk;
  if (i0 >= S.n) return;
  __shared__ double sred[32];
  const int cn = (int)imin64(kRChunk, S.n - i0);
  double sq = 0.0;
  for (int e = threadIdx.x; e < cn; e += blockDim.x) {
    const int64_t i = i0 + e;
    double acc = S.w[i];
    for (int k = 0; k <= j; ++k) acc = fma(-S.hvec[k], S.V[k * S.n + i], acc);
    S.w[i] = acc;
    sq = fma(acc, acc, sq);
  }
  if (pass) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if (lane == 0) sred[wid] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sred[q];
      S.normpart[blockIdx.x] = s;
    }
  }
}

// Completes Hessenberg column j of every live system (one thread each):
// previous rotations, the new rotation, residual estimate, convergence.
// all_done = every system done (the pair kernel then returns at once).
__global__ void kb_finish(const BSys* __restrict__ sys, int n_sys, int j, int m, int* __restrict__ all_done,
                          double* __restrict__ est_out) {
  count_launch();
  const int sidx = threadIdx.x;
  int done = 1;
  if (sidx < n_sys) {
    const BSys S = sys[sidx];
    done = S.state[0];
    if (!done) {
      const int nblk = (int)((S.n + kRChunk - 1) / kRChunk);
      double s = 0.0;
      for (int b = 0; b < nblk; ++b) s += S.normpart[b];
      const double hnext = sqrt(s);
      double* h = S.H + (int64_t)j * (m + 1);
      double colnorm = 0.0;
      for (int i = 0; i <= j; ++i) colnorm = fmax(colnorm, fabs(h[i]));
      h[j + 1] = hnext;
      for (int i = 0; i < j; ++i) {
        const double t = S.cs[i] * h[i] + S.sn[i] * h[i + 1];
        h[i + 1] = -S.sn[i] * h[i] + S.cs[i] * h[i + 1];
        h[i] = t;
      }
      const double den = hypot(h[j], hnext);
      const double c = den > 0.0 ? h[j] / den : 1.0;
      const double sv = den > 0.0 ? hnext / den : 0.0;
      S.cs[j] = c;
      S.sn[j] = sv;
      h[j] = den;
      h[j + 1] = 0.0;
      S.g[j + 1] = -sv * S.g[j];
      S.g[j] = c * S.g[j];
      S.state[1] = j + 1;
      S.scal[0] = hnext > 0.0 ? 1.0 / hnext : 0.0;
      const double est = fabs(S.g[j + 1]) / S.scal[3];
      S.scal[4] = est;
      est_out[sidx] = est;
      if (!isfinite(est) || !isfinite(hnext)) {
        S.state[2] = 1;
        S.state[0] = 1;
      } else if (est <= S.scal[5] || hnext <= 1e-14 * colnorm || j + 1 == m) {
        S.state[0] = 1;
      }
      done = S.state[0];
    }
  }
  const int all = __syncthreads_and(done);
  if (threadIdx.x == 0) *all_done = all;
}

// v_{j+1} = w / h_{j+1,j}
__global__ void kb_scale_next(const BSys* __restrict__ sys, int j) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  if (S.state[0] && S.state[1] <= j) return;  // converged earlier: nothing to write
  const double a = S.scal[0];
  double* vn = S.V + (int64_t)(j + 1) * S.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x)
    vn[i] = S.w[i] * a;
}

// r = f - t (t = A x, or none when x = 0), normpart = chunk sums of r^2
__global__ void __launch_bounds__(256)
kb_residual(const BSys* __restrict__ sys, const double* const* __restrict__ f, const double* const* __restrict__ t) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  const int64_t i0 = blockIdx.x * (int64_t)kRChunk;
  if (i0 >= S.n) return;
  __shared__ double sred[32];
  const double* fs = f[blockIdx.y];
  const double* ts = t ? t[blockIdx.y] : nullptr;
  const int cn = (int)imin64(kRChunk, S.n - i0);
  double sq = 0.0;
  for (int e = threadIdx.x; e < cn; e += blockDim.x) {
    const int64_t i = i0 + e;
    const double v = ts ? fs[i] - ts[i] : fs[i];
    S.r[i] = v;
    sq = fma(v, v, sq);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if (lane == 0) sred[wid] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sred[q];
    S.normpart[blockIdx.x] = s;
  }
}

// beta = |r| per system into norms[s]
__global__ void kb_norms(const BSys* __restrict__ sys, int n_sys, double* __restrict__ norms) {
  count_launch();
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= n_sys) return;
  const BSys S = sys[sidx];
  const int nblk = (int)((S.n + kRChunk - 1) / kRChunk);
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += S.normpart[b];
  norms[sidx] = sqrt(s);
}

// Start of a cycle: live[s] decides whether system s iterates; v_0 = r / beta.
__global__ void kb_cycle_start(const BSys* __restrict__ sys, const int* __restrict__ live, int m) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  const double beta = S.scal[1];
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.state[0] = live[blockIdx.y] ? 0 : 1;
    S.state[1] = 0;
    S.state[2] = 0;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= m; i += blockDim.x) S.g[i] = i == 0 ? beta : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x)
    S.V[i] = S.r[i] * ib;
}

// y = R^-1 g over the completed columns, then x += Z y (one CTA per system
// for the triangular solve; the update below is a separate grid).
__global__ void __launch_bounds__(256) kb_lsq(const BSys* __restrict__ sys, int m) {
  count_launch();
  const BSys S = sys[blockIdx.x];
  const int jd = S.state[1];
  double* work = S.y + (m + 1);
  for (int i = threadIdx.x; i < jd; i += blockDim.x) work[i] = S.g[i];
  __syncthreads();
  __shared__ double yi;
  for (int i = jd - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      const double d = S.H[(int64_t)i * (m + 1) + i];
      yi = d != 0.0 ? work[i] / d : 0.0;
      S.y[i] = yi;
    }
    __syncthreads();
    const double v = yi;
    for (int r = threadIdx.x; r < i; r += blockDim.x) work[r] -= S.H[(int64_t)i * (m + 1) + r] * v;
    __syncthreads();
  }
}

__global__ void kb_update(const BSys* __restrict__ sys) {
  count_launch();
  const BSys S = sys[blockIdx.y];
  const int jd = S.state[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < jd; ++k) acc = fma(S.y[k], S.Z[k * S.n + i], acc);
    S.x[i] += acc;
  }
}

// x += d
__global__ void kb_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

}  // namespace

bool is_device_pointer(const void* p);

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct Batch {
  std::vector<Geom*> gs;
  int R = 0, S = 0, m = 0;
  cudaStream_t s = nullptr;   // the handles' stream
  cudaStream_t ls = nullptr;  // stream the batched launches go to (s, or the capture stream)
  // operator
  std::vector<BGeom> tab;
  DevBuf<BGeom> d_tab;
  DevBuf<double2> part;
  std::vector<int64_t> part_off;
  int64_t n_items = 0;
  DevBuf<double4_32a> mom;  // per system: n_comp entries
  std::vector<int64_t> mom_off;
  DevBuf<unsigned long long> counter;
  DevBuf<int> all_done;
  // systems
  std::vector<BSys> sys;
  DevBuf<BSys> d_sys;
  DevBuf<double> pool;
  DevBuf<int> ipool;
  DevBuf<double> norms, est;
  DevBuf<int> live;
  DevBuf<const double*> d_f, d_t;
  std::vector<double*> t_h;  // per system A x scratch
  int64_t max_n = 0;
  cudaGraphExec_t cycle = nullptr;
  int cycle_prec = -1;
  ~Batch() {
    if (cycle) cudaGraphExecDestroy(cycle);
  }
};

namespace {

void batch_tables(Batch& b, int precision) {
  const int R = b.R;
  const int th = precision == STOKES_FP32 ? kF32Threads * kF32Tpt : kDFThreads;
  const int tile = precision == STOKES_FP32 ? kF32Tile : kDFTile;
  b.tab.assign(b.gs.size(), BGeom{});
  b.part_off.assign(b.gs.size() + 1, 0);
  int64_t items = 0;
  for (size_t k = 0; k < b.gs.size(); ++k) {
    Geom& g = *b.gs[k];
    BGeom& e = b.tab[k];
    e.N = g.N;
    e.tblocks = (g.N + th - 1) / th;
    // at most 16 source splits, each a whole number of tiles and >= 8 tiles
    int64_t chunk = std::max<int64_t>((g.N + 15) / 16, 8 * (int64_t)tile);
    chunk = (chunk + tile - 1) / tile * tile;
    e.chunk = chunk;
    e.splits = (int)((g.N + chunk - 1) / chunk);
    e.item0 = items;
    items += e.tblocks * e.splits;
    e.f32_src = g.f32_src.get();
    e.f32_lo = g.f32_lo.get();
    e.df_grid = g.df_grid.get();
    e.df_pos = g.df_pos.get();
    e.df_a = g.df_a.get();
    e.tgt = g.pos.get();
    b.part_off[k + 1] = b.part_off[k] + (int64_t)e.splits * R * g.N;
  }
  b.n_items = items;
  b.part.alloc((size_t)b.part_off.back());
  for (size_t k = 0; k < b.gs.size(); ++k) b.tab[k].part = b.part.get() + b.part_off[k];
}

void upload_table(Batch& b) {
  b.d_tab.alloc(b.tab.size());
  STOKES_CUDA(cudaMemcpyAsync(b.d_tab.get(), b.tab.data(), b.tab.size() * sizeof(BGeom), cudaMemcpyHostToDevice,
                              b.s));
}

void batch_init(Batch& b, Geom* const* geoms, int n_geoms, int R) {
  require(geoms && n_geoms >= 1, "no geometries");
  require(R >= 1 && R <= kMaxRhs, "n_rhs must be in [1, 4]");
  require((int64_t)n_geoms * R <= kMaxSystems, "at most 1024 systems (geometries x right-hand sides)");
  b.gs.assign(geoms, geoms + n_geoms);
  b.R = R;
  b.S = n_geoms * R;
  b.s = b.gs[0]->stream;
  b.ls = b.s;
  for (Geom* g : b.gs) {
    require(g != nullptr, "null handle");
    require(g->stream == b.s, "all handles of a batch must use the same stream");
    // the captured cycle holds ordinary kernel launches only
    require(!(g->tg.ready && g->tg.use_lu),
            "batched solves need the two-grid coarse solve by its explicit inverse (STOKES_TG_COARSE_INVERSE)");
  }
  b.mom_off.assign(b.S + 1, 0);
  for (int k = 0; k < n_geoms; ++k)
    for (int r = 0; r < R; ++r) b.mom_off[k * R + r + 1] = b.mom_off[k * R + r] + b.gs[k]->n_comp;
  b.mom.alloc((size_t)b.mom_off.back());
  b.counter.alloc(1);
  b.all_done.alloc(1);
}

// y_{k,r} = A_k sig_{k,r}: sig column `col` of each system's base pointer.
// done_sys[s] (may be null) skips the per-system kernels of converged systems.
void batch_apply(Batch& b, int precision, int col, const std::vector<const double*>& sig_base, int64_t sig_stride_of,
                 const std::vector<double*>& y, const std::vector<const int*>& done_sys, const int* all_done) {
  const int R = b.R;
  const int n_geoms = (int)b.gs.size();
  for (int k = 0; k < n_geoms; ++k) {
    Geom& g = *b.gs[k];
    for (int r = 0; r < R; ++r) {
      const int sidx = k * R + r;
      const double* sg = sig_base[sidx] + (sig_stride_of ? (int64_t)col * 2 * g.N : 0);
      moments_f64(g, (const double2*)sg, done_sys.empty() ? nullptr : done_sys[sidx], b.mom.get() + b.mom_off[sidx]);
    }
  }
  STOKES_CUDA(cudaMemsetAsync(b.counter.get(), 0, sizeof(unsigned long long), b.ls));
  switch (R) {
    case 1: launch_pairs_r<1>(precision, b.d_tab.get(), n_geoms, b.n_items, col, b.counter.get(), all_done, b.ls); break;
    case 2: launch_pairs_r<2>(precision, b.d_tab.get(), n_geoms, b.n_items, col, b.counter.get(), all_done, b.ls); break;
    case 3: launch_pairs_r<3>(precision, b.d_tab.get(), n_geoms, b.n_items, col, b.counter.get(), all_done, b.ls); break;
    default: launch_pairs_r<4>(precision, b.d_tab.get(), n_geoms, b.n_items, col, b.counter.get(), all_done, b.ls);
  }
  for (int k = 0; k < n_geoms; ++k) {
    Geom& g = *b.gs[k];
    const BGeom& e = b.tab[k];
    for (int r = 0; r < R; ++r) {
      const int sidx = k * R + r;
      const double* sg = sig_base[sidx] + (sig_stride_of ? (int64_t)col * 2 * g.N : 0);
      const int* dn = done_sys.empty() ? nullptr : done_sys[sidx];
      const double2* part = e.part + (int64_t)r * g.N;
      const int64_t pstride = (int64_t)R * g.N;
      const double4_32a* mom = b.mom.get() + b.mom_off[sidx];
      if (precision == STOKES_DF64 && dlp::ensure_log_table(g))
        dlp::launch_epilogue<dlp::kCompDF>(g, g.N, e.splits, true, g.pos.get(), (const double2*)sg, (double2*)y[sidx],
                                           dn, part, pstride, mom);
      else if (precision == STOKES_DF64)
        dlp::launch_epilogue<dlp::kCompF64>(g, g.N, e.splits, true, g.pos.get(), (const double2*)sg,
                                            (double2*)y[sidx], dn, part, pstride, mom);
      else
        dlp::launch_epilogue<dlp::kCompF32>(g, g.N, e.splits, true, g.pos.get(), (const double2*)sg,
                                            (double2*)y[sidx], dn, part, pstride, mom);
    }
  }
}

void set_sigma_table(Batch& b, const std::vector<const double*>& sig_base, bool strided) {
  for (size_t k = 0; k < b.gs.size(); ++k) {
    for (int r = 0; r < kMaxRhs; ++r)
      b.tab[k].sig[r] = r < b.R ? (const double2*)sig_base[k * b.R + r] : nullptr;
    b.tab[k].sig_stride = strided ? b.gs[k]->N : 0;
  }
  upload_table(b);
}

// Per-system workspaces of the lockstep solver for restart m.
void batch_krylov_alloc(Batch& b, int m, const std::vector<double*>& x) {
  b.m = m;
  b.sys.assign(b.S, BSys{});
  int64_t total = 0;
  std::vector<int64_t> need(b.S);
  b.max_n = 0;
  for (int sidx = 0; sidx < b.S; ++sidx) {
    const int64_t n = 2 * b.gs[sidx / b.R]->N;
    const int64_t nblk = (n + kRChunk - 1) / kRChunk;
    b.max_n = std::max(b.max_n, n);
    // V, Z, w, r, t + H, cs, sn, g, y, partial, hvec, normpart, scal
    need[sidx] = (int64_t)(m + 1) * n + (int64_t)m * n + 3 * n + (int64_t)(m + 1) * m + 2 * (int64_t)m +
                 (m + 1) + 2 * (int64_t)(m + 1) + nblk * (m + 1) + (m + 1) + nblk + 8;
    need[sidx] = (need[sidx] + 3) / 4 * 4;  // 32-byte alignment of every system's block
    total += need[sidx];
  }
  b.pool.alloc((size_t)total);
  b.ipool.alloc((size_t)4 * b.S);
  b.t_h.assign(b.S, nullptr);
  double* p = b.pool.get();
  for (int sidx = 0; sidx < b.S; ++sidx) {
    const int64_t n = 2 * b.gs[sidx / b.R]->N;
    const int64_t nblk = (n + kRChunk - 1) / kRChunk;
    BSys& S = b.sys[sidx];
    double* q = p;
    S.n = n;
    S.V = q; q += (int64_t)(m + 1) * n;
    S.Z = q; q += (int64_t)m * n;
    S.w = q; q += n;
    S.r = q; q += n;
    b.t_h[sidx] = q; q += n;
    S.H = q; q += (int64_t)(m + 1) * m;
    S.cs = q; q += m;
    S.sn = q; q += m;
    S.g = q; q += m + 1;
    S.y = q; q += 2 * (int64_t)(m + 1);
    S.partial = q; q += nblk * (m + 1);
    S.hvec = q; q += m + 1;
    S.normpart = q; q += nblk;
    S.scal = q;
    S.x = x[sidx];
    S.state = b.ipool.get() + 4 * sidx;
    p += need[sidx];
  }
  b.d_sys.alloc(b.S);
  STOKES_CUDA(cudaMemcpyAsync(b.d_sys.get(), b.sys.data(), b.S * sizeof(BSys), cudaMemcpyHostToDevice, b.s));
  STOKES_CUDA(cudaMemsetAsync(b.ipool.get(), 0, 4 * sizeof(int) * b.S, b.s));
  b.norms.alloc(b.S);
  b.est.alloc(b.S);
  b.live.alloc(b.S);
  b.d_f.alloc(b.S);
  b.d_t.alloc(b.S);
}

// The launches of one restart cycle (m lockstep steps), for capture.
void batch_cycle_launches(Batch& b, int precision) {
  const int m = b.m, S = b.S;
  const bool f32pc = true;  // float copies of the preconditioner (flexible GMRES absorbs them)
  const unsigned nblk = (unsigned)((b.max_n + kRChunk - 1) / kRChunk);
  std::vector<const double*> zbase(S);
  std::vector<double*> wout(S);
  std::vector<const int*> done(S);
  for (int sidx = 0; sidx < S; ++sidx) {
    zbase[sidx] = b.sys[sidx].Z;
    wout[sidx] = b.sys[sidx].w;
    done[sidx] = b.sys[sidx].state;
  }
  for (int j = 0; j < m; ++j) {
    for (int sidx = 0; sidx < S; ++sidx) {
      Geom& g = *b.gs[sidx / b.R];
      const BSys& Sy = b.sys[sidx];
      if (g.bd.ready || g.tg.ready)
        precond_apply(g, Sy.V + (int64_t)j * Sy.n, Sy.Z + (int64_t)j * Sy.n, Sy.state, f32pc);
      else
        STOKES_CUDA(cudaMemcpyAsync(Sy.Z + (int64_t)j * Sy.n, Sy.V + (int64_t)j * Sy.n, Sy.n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, b.ls));
    }
    batch_apply(b, precision, j, zbase, 1, wout, done, b.all_done.get());
    for (int pass = 0; pass < 2; ++pass) {
      kb_dot_partial<<<dim3(nblk, S), 256, 0, b.ls>>>(b.d_sys.get(), j, m);
      kb_reduce<<<dim3((unsigned)((j + 1 + 255) / 256), S), 256, 0, b.ls>>>(b.d_sys.get(), j, m, pass);
      kb_orth_update<<<dim3(nblk, S), 256, 0, b.ls>>>(b.d_sys.get(), j, pass);
    }
    kb_finish<<<1, ((S + 31) / 32) * 32, 0, b.ls>>>(b.d_sys.get(), S, j, m, b.all_done.get(), b.est.get());
    kb_scale_next<<<dim3(std::min<unsigned>(64, (unsigned)((b.max_n + 255) / 256)), S), 256, 0, b.ls>>>(
        b.d_sys.get(), j);
    STOKES_LAUNCHED();
  }
  kb_lsq<<<S, 256, 0, b.ls>>>(b.d_sys.get(), m);
  kb_update<<<dim3(std::min<unsigned>(64, (unsigned)((b.max_n + 255) / 256)), S), 256, 0, b.ls>>>(b.d_sys.get());
  STOKES_LAUNCHED();
}

// True residuals r = f - A x (FP64 operator per system) and their norms.
// Systems with active[s] == 0 keep rn[s] (their r is not needed again).
void batch_residuals(Batch& b, const std::vector<const double*>& f, bool x_zero, std::vector<double>& rn,
                     const std::vector<int>* active = nullptr) {
  const int S = b.S;
  std::vector<const double*> th(S);
  const std::vector<double> keep = rn;
  for (int sidx = 0; sidx < S; ++sidx) {
    th[sidx] = b.t_h[sidx];
    const bool act = !active || (*active)[sidx];
    if (!x_zero && act) apply_operator(*b.gs[sidx / b.R], b.sys[sidx].x, b.t_h[sidx], STOKES_FP64, nullptr);
  }
  STOKES_CUDA(cudaMemcpyAsync(b.d_f.get(), f.data(), S * sizeof(double*), cudaMemcpyHostToDevice, b.s));
  STOKES_CUDA(cudaMemcpyAsync(b.d_t.get(), th.data(), S * sizeof(double*), cudaMemcpyHostToDevice, b.s));
  const unsigned nblk = (unsigned)((b.max_n + kRChunk - 1) / kRChunk);
  kb_residual<<<dim3(nblk, S), 256, 0, b.s>>>(b.d_sys.get(), b.d_f.get(), x_zero ? nullptr : b.d_t.get());
  kb_norms<<<(S + 255) / 256, 256, 0, b.s>>>(b.d_sys.get(), S, b.norms.get());
  STOKES_LAUNCHED();
  rn.resize(S);
  STOKES_CUDA(cudaMemcpyAsync(rn.data(), b.norms.get(), S * sizeof(double), cudaMemcpyDeviceToHost, b.s));
  STOKES_CUDA(cudaStreamSynchronize(b.s));
  if (active)
    for (int sidx = 0; sidx < S; ++sidx)
      if (!(*active)[sidx] && sidx < (int)keep.size()) rn[sidx] = keep[sidx];
}

}  // namespace

// One lockstep FGMRES solve of all systems: A x_s = f_s from the current x_s
// to relative residual tol_s (|f_s| as the scale). inner: stop each system
// on its Arnoldi estimate after its first cycle that meets it (no true
// residual), as the inner solves of the refinement do.
static void batch_fgmres(Batch& b, int precision, const std::vector<const double*>& f,
                         const std::vector<double>& fnorm, const std::vector<double>& tol, int max_cycles,
                         bool inner, bool x_zero, std::vector<int>& iters, std::vector<double>& relres,
                         std::vector<int>& status) {
  const int S = b.S;
  if (b.cycle == nullptr || b.cycle_prec != precision) {
    if (b.cycle) {
      cudaGraphExecDestroy(b.cycle);
      b.cycle = nullptr;
    }
    // one cycle run eagerly first grows every workspace the launches use
    std::vector<int> zeros(S, 0);
    STOKES_CUDA(cudaMemcpyAsync(b.live.get(), zeros.data(), S * sizeof(int), cudaMemcpyHostToDevice, b.s));
    const int one = 1;
    STOKES_CUDA(cudaMemcpyAsync(b.all_done.get(), &one, sizeof(int), cudaMemcpyHostToDevice, b.s));
    kb_cycle_start<<<dim3(1, S), 256, 0, b.s>>>(b.d_sys.get(), b.live.get(), b.m);
    STOKES_LAUNCHED();
    batch_cycle_launches(b, precision);
    STOKES_CUDA(cudaStreamSynchronize(b.s));
    // The handles' stream may be the legacy default stream, which cannot be
    // captured: every launch of the cycle (the per-geometry ones included)
    // is recorded on a private stream; the graph then runs on the handles' stream.
    struct CaptureStreams {
      Batch& b;
      cudaStream_t cs = nullptr;
      explicit CaptureStreams(Batch& bb) : b(bb) {
        STOKES_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        b.ls = cs;
        for (Geom* g : b.gs) g->stream = cs;
      }
      ~CaptureStreams() {
        for (Geom* g : b.gs) g->stream = b.s;
        b.ls = b.s;
        if (cs) cudaStreamDestroy(cs);
      }
    };
    cudaGraph_t graph = nullptr;
    {
      CaptureStreams cap(b);
      STOKES_CUDA(cudaStreamBeginCapture(cap.cs, cudaStreamCaptureModeThreadLocal));
      try {
        batch_cycle_launches(b, precision);
      } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(cap.cs, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
      }
      STOKES_CUDA(cudaStreamEndCapture(cap.cs, &graph));
    }
    const cudaError_t e = cudaGraphInstantiate(&b.cycle, graph, 0);
    cudaGraphDestroy(graph);
    STOKES_CUDA(e);
    b.cycle_prec = precision;
  }
  iters.assign(S, 0);
  relres.assign(S, 0.0);
  status.assign(S, STOKES_OK);
  std::vector<double> rn, est(S, INFINITY);
  std::vector<int> live(S, 0), met(S, 0), hstate(4 * S);
  std::vector<double> scal_init(8, 0.0);
  for (int cyc = 0;; ++cyc) {
    // after the first cycle only the systems that iterated need a new residual
    batch_residuals(b, f, x_zero && cyc == 0, rn, cyc == 0 ? nullptr : &live);
    int n_live = 0;
    for (int sidx = 0; sidx < S; ++sidx) {
      relres[sidx] = fnorm[sidx] > 0 ? rn[sidx] / fnorm[sidx] : 0.0;
      if (!std::isfinite(relres[sidx])) status[sidx] = STOKES_EBREAKDOWN;
      // inner solves stop on the Arnoldi estimate of their last cycle
      const bool conv = relres[sidx] <= tol[sidx] || (inner && met[sidx]);
      live[sidx] = (!conv && status[sidx] == STOKES_OK && rn[sidx] > 0) ? 1 : 0;
      if (live[sidx] && cyc >= max_cycles) {
        status[sidx] = STOKES_ENOTCONV;
        live[sidx] = 0;
      }
      n_live += live[sidx];
      // scal: [1] beta, [2] 1/beta, [3] |f| (scale of the estimate), [5] tol
      scal_init[1] = rn[sidx];
      scal_init[2] = rn[sidx] > 0 ? 1.0 / rn[sidx] : 0.0;
      scal_init[3] = fnorm[sidx] > 0 ? fnorm[sidx] : 1.0;
      scal_init[5] = tol[sidx];
      STOKES_CUDA(cudaMemcpyAsync(b.sys[sidx].scal + 1, scal_init.data() + 1, 5 * sizeof(double),
                                  cudaMemcpyHostToDevice, b.s));
    }
    if (n_live == 0) break;
    STOKES_CUDA(cudaMemcpyAsync(b.live.get(), live.data(), S * sizeof(int), cudaMemcpyHostToDevice, b.s));
    STOKES_CUDA(cudaMemsetAsync(b.all_done.get(), 0, sizeof(int), b.s));
    kb_cycle_start<<<dim3(std::min<unsigned>(64, (unsigned)((b.max_n + 255) / 256)), S), 256, 0, b.s>>>(
        b.d_sys.get(), b.live.get(), b.m);
    STOKES_LAUNCHED();
    STOKES_CUDA(cudaGraphLaunch(b.cycle, b.s));
    STOKES_CUDA(cudaMemcpyAsync(hstate.data(), b.ipool.get(), 4 * S * sizeof(int), cudaMemcpyDeviceToHost, b.s));
    STOKES_CUDA(cudaMemcpyAsync(est.data(), b.est.get(), S * sizeof(double), cudaMemcpyDeviceToHost, b.s));
    STOKES_CUDA(cudaStreamSynchronize(b.s));
    for (int sidx = 0; sidx < S; ++sidx) {
      if (!live[sidx]) continue;
      iters[sidx] += hstate[4 * sidx + 1];
      if (hstate[4 * sidx + 2]) status[sidx] = STOKES_EBREAKDOWN;
      met[sidx] = est[sidx] <= tol[sidx] ? 1 : 0;
    }
    if (std::getenv("STOKES_TRACE")) {
      double worst = 0.0;
      for (int sidx = 0; sidx < S; ++sidx)
        if (live[sidx]) worst = std::max(worst, est[sidx]);
      std::fprintf(stderr, "[stokes] batch cycle %d: %d live systems, worst estimate %.3e\n", cyc, n_live, worst);
    }
    if (inner) {
      bool all = true;
      for (int sidx = 0; sidx < S; ++sidx)
        if (live[sidx] && status[sidx] == STOKES_OK && !met[sidx]) all = false;
      if (all) {
        for (int sidx = 0; sidx < S; ++sidx)
          if (live[sidx]) relres[sidx] = -1.0;  // not evaluated
        return;
      }
    }
  }
}

// Mixed precision: outer FP64 residuals per system, inner lockstep FP32
// cycles to max(1e-4, tol / (2 relres)) on the corrections. Each system
// has its own budget of max_iter inner iterations: one that stagnates is
// stopped (STOKES_ENOTCONV) without ending the refinement of the others.
static void batch_ir(Batch& b, const std::vector<const double*>& f, const std::vector<double>& fnorm, double tol,
                     int max_iter, std::vector<int>& iters, std::vector<double>& relres, std::vector<int>& status) {
  const int S = b.S;
  // the corrections d_s live in a separate pool; the systems' x point at them
  std::vector<double*> xs(S);
  for (int sidx = 0; sidx < S; ++sidx) xs[sidx] = b.sys[sidx].x;
  DevBuf<double> dpool, rpool;
  int64_t tot = 0;
  std::vector<int64_t> off(S + 1, 0);
  for (int sidx = 0; sidx < S; ++sidx) off[sidx + 1] = off[sidx] + b.sys[sidx].n;
  tot = off[S];
  dpool.alloc(tot);
  rpool.alloc(tot);
  iters.assign(S, 0);
  relres.assign(S, 0.0);
  status.assign(S, STOKES_OK);
  std::vector<double> rn;
  std::vector<const double*> rptr(S);
  for (int outer = 0;; ++outer) {
    // r_s = f_s - A x_s in FP64 (into the pool), norms
    for (int sidx = 0; sidx < S; ++sidx) b.sys[sidx].x = xs[sidx];
    STOKES_CUDA(cudaMemcpyAsync(b.d_sys.get(), b.sys.data(), S * sizeof(BSys), cudaMemcpyHostToDevice, b.s));
    batch_residuals(b, f, false, rn);
    std::vector<double> itol(S);
    bool any_live = false;
    double worst = 0.0;
    int minit = max_iter;  // fewest iterations used by a system still refining
    for (int sidx = 0; sidx < S; ++sidx) {
      relres[sidx] = fnorm[sidx] > 0 ? rn[sidx] / fnorm[sidx] : 0.0;
      if (!std::isfinite(relres[sidx])) status[sidx] = STOKES_EBREAKDOWN;
      if (relres[sidx] > tol && status[sidx] == STOKES_OK) {
        if (iters[sidx] >= max_iter || outer >= 30) {
          status[sidx] = STOKES_ENOTCONV;
        } else {
          any_live = true;
          minit = std::min(minit, iters[sidx]);
        }
      }
      worst = std::max(worst, relres[sidx]);
      STOKES_CUDA(cudaMemcpyAsync(rpool.get() + off[sidx], b.sys[sidx].r, b.sys[sidx].n * sizeof(double),
                                  cudaMemcpyDeviceToDevice, b.s));
      rptr[sidx] = rpool.get() + off[sidx];
    }
    if (!any_live) return;
    // inner: A d = r from d = 0; converged systems get tol 1 (no iterations)
    STOKES_CUDA(cudaMemsetAsync(dpool.get(), 0, tot * sizeof(double), b.s));
    std::vector<double> rnorm(S);
    for (int sidx = 0; sidx < S; ++sidx) {
      b.sys[sidx].x = dpool.get() + off[sidx];
      rnorm[sidx] = rn[sidx];
      // converged or stopped systems take no iterations (tolerance 2)
      itol[sidx] = (relres[sidx] <= tol || status[sidx] != STOKES_OK) ? 2.0
                                                                      : std::max(1e-4, 0.5 * tol / relres[sidx]);
    }
    STOKES_CUDA(cudaMemcpyAsync(b.d_sys.get(), b.sys.data(), S * sizeof(BSys), cudaMemcpyHostToDevice, b.s));
    std::vector<int> it_in, st_in;
    std::vector<double> rr_in;
    const int cycles = std::max(1, (max_iter - minit + b.m - 1) / b.m);
    batch_fgmres(b, STOKES_FP32, rptr, rnorm, itol, cycles, true, true, it_in, rr_in, st_in);
    if (std::getenv("STOKES_TRACE"))
      std::fprintf(stderr, "[stokes] batch refinement step %d: worst relres %.3e\n", outer, worst);
    // x_s += d_s
    for (int sidx = 0; sidx < S; ++sidx) {
      iters[sidx] += it_in[sidx];
      if (st_in[sidx] == STOKES_EBREAKDOWN) status[sidx] = STOKES_EBREAKDOWN;
      if (itol[sidx] <= 1.0)
        kb_axpy<<<(unsigned)std::min<int64_t>(152 * 8, (b.sys[sidx].n + 255) / 256), 256, 0, b.s>>>(
            xs[sidx], dpool.get() + off[sidx], b.sys[sidx].n);
    }
    STOKES_LAUNCHED();
  }
}

void batch_matvec(Geom* const* geoms, int n_geoms, int R, const double* const* sigma, double* const* y,
                  int precision) {
  require(precision == STOKES_FP32 || precision == STOKES_DF64, "batched operator: precision must be FP32 or DF64");
  Batch b;
  batch_init(b, geoms, n_geoms, R);
  batch_tables(b, precision);
  std::vector<const double*> sb(b.S);
  std::vector<double*> yo(b.S);
  for (int sidx = 0; sidx < b.S; ++sidx) {
    require(sigma[sidx] && y[sidx], "null array argument");
    require(is_device_pointer(sigma[sidx]) && is_device_pointer(y[sidx]), "batched calls take device arrays");
    sb[sidx] = sigma[sidx];
    yo[sidx] = y[sidx];
  }
  set_sigma_table(b, sb, false);
  batch_apply(b, precision, 0, sb, 0, yo, {}, nullptr);
  STOKES_CUDA(cudaStreamSynchronize(b.s));
}

void batch_solve(Geom* const* geoms, int n_geoms, int R, const double* const* f, double tol, int restart,
                 int max_iter, int precision, double* const* sigma, int* iters_out, double* relres_out,
                 int* status_out) {
  require(precision == STOKES_DF64 || precision == STOKES_MIXED_IR,
          "batched solve: precision must be DF64 or MIXED_IR");
  require(tol > 0 && std::isfinite(tol), "tol must be > 0");
  require(restart >= 1 && restart <= 1000, "restart must be in [1, 1000]");
  require(max_iter >= 1, "max_iter must be >= 1");
  Batch b;
  batch_init(b, geoms, n_geoms, R);
  const int S = b.S;
  std::vector<const double*> fv(S);
  std::vector<double*> xv(S);
  for (int sidx = 0; sidx < S; ++sidx) {
    require(f[sidx] && sigma[sidx] && f[sidx] != sigma[sidx], "bad array arguments");
    require(is_device_pointer(f[sidx]) && is_device_pointer(sigma[sidx]), "batched calls take device arrays");
    fv[sidx] = f[sidx];
    xv[sidx] = sigma[sidx];
  }
  const int op_prec = precision == STOKES_MIXED_IR ? STOKES_FP32 : STOKES_DF64;
  batch_tables(b, op_prec);
  batch_krylov_alloc(b, restart, xv);
  std::vector<const double*> zbase(S);
  for (int sidx = 0; sidx < S; ++sidx) zbase[sidx] = b.sys[sidx].Z;
  set_sigma_table(b, zbase, true);
  // profiling events cannot be captured: off for the duration of the solve
  std::vector<bool> prof(b.gs.size());
  for (size_t k = 0; k < b.gs.size(); ++k) {
    prof[k] = b.gs[k]->prof.on;
    b.gs[k]->prof.on = false;
    if (op_prec == STOKES_DF64) dlp::ensure_log_table(*b.gs[k]);
  }
  std::vector<int> iters, status;
  std::vector<double> relres;
  try {
    // |f_s|
    std::vector<double> fnorm;
    batch_residuals(b, fv, true, fnorm);
    if (precision == STOKES_MIXED_IR) {
      batch_ir(b, fv, fnorm, tol, max_iter, iters, relres, status);
    } else {
      std::vector<double> tv(S, tol);
      // a zero start is not assumed: sigma holds the initial guess
      batch_fgmres(b, STOKES_DF64, fv, fnorm, tv, std::max(1, (max_iter + restart - 1) / restart), false, false,
                   iters, relres, status);
    }
  } catch (...) {
    for (size_t k = 0; k < b.gs.size(); ++k) b.gs[k]->prof.on = prof[k];
    throw;
  }
  for (size_t k = 0; k < b.gs.size(); ++k) b.gs[k]->prof.on = prof[k];
  for (int sidx = 0; sidx < S; ++sidx) {
    if (iters_out) iters_out[sidx] = iters[sidx];
    if (relres_out) relres_out[sidx] = relres[sidx];
    if (status_out) status_out[sidx] = status[sidx];
  }
}

unsigned long long launches_batch() { return tu_launches(); }

}  // namespace stokes
