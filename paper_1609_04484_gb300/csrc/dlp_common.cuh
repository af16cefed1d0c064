// Shared pieces of the double-layer operator kernels: the launch shape of
// the pair kernels, the double-float (unevaluated float pair) primitives and
// the epilogue that turns pair partial sums into A sigma or a velocity.
#pragma once

#include <algorithm>

#include "internal.cuh"

namespace stokes {
namespace dlp {

constexpr int kEpiPores = 256;

// Split the sources so that the grid has ~ctas_per_sm CTAs per SM (152 SMs);
// each split covers a whole number of `tile`-sized source tiles.
inline void pair_launch_shape(int64_t N, int64_t T, int tb, int tile, int& splits, int64_t& chunk,
                              int ctas_per_sm = 4) {
  const int64_t tblocks = (T + tb - 1) / tb;
  int64_t want = ((int64_t)ctas_per_sm * 152 + tblocks - 1) / tblocks;
  const int64_t max_split = (N + tile - 1) / tile;
  if (want > max_split) want = max_split;
  if (want < 1) want = 1;
  chunk = ((N + want - 1) / want + tile - 1) / tile * tile;
  splits = (int)((N + chunk - 1) / chunk);
}

// Reciprocal of a positive double by Newton-Raphson iteration
// y <- y + y (1 - a y), each step squaring the relative error, from the
// hardware's approximate double reciprocal (PTX rcp.approx.ftz.f64, about
// single-precision accurate): two steps bring it within about one ulp of
// 1 / a. Four FP64 FMAs and one special-function op replace the FP64
// division's longer sequence on the FP64 pipe. a = +inf (and anything the
// approximation maps to 0) gives 0; a = 0 gives a non-finite value.
__device__ __forceinline__ double rcp_newton(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  double e = fma(-a, y, 1.0);
  y = fma(y, e, y);
  e = fma(-a, y, 1.0);
  return fma(y, e, y);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) (up to a
// few ulps where normalisation is skipped). Error-free transformations:
// TwoSum (Knuth), FastTwoSum (Dekker), TwoProduct via FMA.
// ---------------------------------------------------------------------------
struct df32 {
  float h, l;
};

__device__ __forceinline__ df32 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ df32 two_diff(float a, float b) {
  const float s = a - b;
  const float bb = s - a;
  const float e = (a - (s - bb)) - (b + bb);
  return {s, e};
}

__device__ __forceinline__ df32 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}

// a * b for double-floats, low-order product dropped, normalised.
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// a.x * b.x + a.y * b.y for double-float 2-vectors, normalised.
__device__ __forceinline__ df32 df_dot2(df32 ax, df32 ay, df32 bx, df32 by) {
  const float p1 = ax.h * bx.h;
  float e1 = fmaf(ax.h, bx.h, -p1);
  e1 = fmaf(ax.h, bx.l, e1);
  e1 = fmaf(ax.l, bx.h, e1);
  const float p2 = ay.h * by.h;
  float e2 = fmaf(ay.h, by.h, -p2);
  e2 = fmaf(ay.h, by.l, e2);
  e2 = fmaf(ay.l, by.h, e2);
  const df32 s = two_sum(p1, p2);
  return fast_two_sum(s.h, s.l + (e1 + e2));
}

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df32 df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// ---------------------------------------------------------------------------
// Epilogue
// ---------------------------------------------------------------------------
// y_i = sum_s part[s][i]
//       + (boundary) w_i (-kappa_i / 2pi) t_i (t_i . sigma_i) - sigma_i / 2
//       + (boundary, i on the wall) n_i s0
//       + sum_pores (1/4pi) [(-log rho I + r r^T / rho^2) lambda_k + r^perp xi_k / rho^2]
// The diagonal and wall terms are O(N) and always FP64. The completion is
//   kCompF64: double precision;
//   kCompF32: single precision with r = (x_hi - c_hi) + (x_lo - c_lo);
//   kCompDF:  double-float, log(rho^2) read from a per-geometry table
//             (targets must be the nodes).
enum CompMode { kCompF64 = 0, kCompF32 = 1, kCompDF = 2 };

// v = grid + rem with grid on multiples of 2^-8 (exact float differences)
__device__ __forceinline__ void grid_split(double v, float& gridv, df32& rem) {
  const double gv = rint(v * 256.0) * (1.0 / 256.0);
  gridv = (float)gv;
  rem = df_from_double(v - gv);
}

// r = a - b for points given as grid + remainder, exact to ~2^-48 |r|
__device__ __forceinline__ df32 df_sub_point(float ga, df32 ra, float gb, df32 rb) {
  df32 l = two_diff(ra.h, rb.h);
  l.l += ra.l - rb.l;
  // the grid difference is a multiple of 2^-8 and |l.h| <= 2^-8, so either
  // it is zero or it dominates: FastTwoSum is exact
  df32 r = fast_two_sum(ga - gb, l.h);
  r.l += l.l;
  return r;
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  const df32 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}

// 1 / a by one Newton step from the correctly rounded float reciprocal
__device__ __forceinline__ df32 df_rcp(df32 a) {
  const float y0 = __frcp_rn(a.h);
  float t = fmaf(-a.h, y0, 1.0f);
  t = fmaf(-a.l, y0, t);
  return {y0, y0 * t};
}

struct PoreF32 {
  float chx, chy, clx, cly, lx, ly, xi, pad;
};
struct PoreDF {
  float gx, gy;       // centre on the 2^-8 grid
  df32 rx, ry;        // centre remainder
  df32 lx, ly, xi;    // moments
};

template <int kMode>
__global__ void __launch_bounds__(256)
k_epilogue(int64_t T, int S, const double2* __restrict__ part, int64_t pstride, int boundary,
           const double2* __restrict__ tgt,
           const double4_32a* __restrict__ selfc, const double2* __restrict__ sig, const int* __restrict__ comp,
           int outer, const double2* __restrict__ nrm, int M, const int* __restrict__ pore_ids,
           const double2* __restrict__ centre, const double4_32a* __restrict__ mom,
           const float2* __restrict__ logtab, double2* __restrict__ y, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double2 s_c[kEpiPores];
  __shared__ double4_32a s_m[kEpiPores];
  __shared__ PoreF32 s_f[kMode == kCompF32 ? kEpiPores : 1];
  __shared__ PoreDF s_d[kMode == kCompDF ? kEpiPores : 1];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = i < T;
  double ax = 0.0, ay = 0.0;
  double2 x = make_double2(0.0, 0.0);
  if (live) {
    for (int s = 0; s < S; ++s) {
      const double2 p = part[s * pstride + i];
      ax += p.x;
      ay += p.y;
    }
    x = tgt[i];
    if (boundary) {
      const double4_32a sc = selfc[i];
      const double2 sg = sig[i];
      const double ts = sc.x * sg.x + sc.y * sg.y;
      ax += sc.z * ts * sc.x - 0.5 * sg.x;
      ay += sc.z * ts * sc.y - 0.5 * sg.y;
      if (comp[i] == outer) {
        const double s0 = mom[outer].w;
        const double2 n = nrm[i];
        ax += n.x * s0;
        ay += n.y * s0;
      }
    }
  }
  // per-target split of the position
  const float xh = (float)x.x, yh = (float)x.y;
  const float xl = (float)(x.x - (double)xh), yl = (float)(x.y - (double)yh);
  float tgx = 0.f, tgy = 0.f;
  df32 trx = {0.f, 0.f}, try_ = {0.f, 0.f};
  if (kMode == kCompDF) {
    grid_split(x.x, tgx, trx);
    grid_split(x.y, tgy, try_);
  }
  double cx = 0.0, cy = 0.0;
  for (int k0 = 0; k0 < M; k0 += kEpiPores) {
    __syncthreads();
    for (int q = threadIdx.x; q < kEpiPores && k0 + q < M; q += blockDim.x) {
      const int k = pore_ids[k0 + q];
      const double2 c = centre[k];
      const double4_32a m = mom[k];
      if (kMode == kCompF64) {
        s_c[q] = c;
        s_m[q] = m;
      } else if (kMode == kCompF32) {
        const float chx = (float)c.x, chy = (float)c.y;
        s_f[q] = {chx, chy, (float)(c.x - (double)chx), (float)(c.y - (double)chy), (float)m.x, (float)m.y,
                  (float)m.z, 0.f};
      } else {
        PoreDF p;
        grid_split(c.x, p.gx, p.rx);
        grid_split(c.y, p.gy, p.ry);
        p.lx = df_from_double(m.x);
        p.ly = df_from_double(m.y);
        p.xi = df_from_double(m.z);
        s_d[q] = p;
      }
    }
    __syncthreads();
    const int nq = (int)imin64(kEpiPores, M - k0);
    if (!live) continue;
    if (kMode == kCompF32) {
      float fx = 0.f, fy = 0.f;
      for (int q = 0; q < nq; ++q) {
        const PoreF32 p = s_f[q];
        const float rx = (xh - p.chx) + (xl - p.clx);
        const float ry = (yh - p.chy) + (yl - p.cly);
        const float r2 = fmaf(rx, rx, ry * ry);
        const float inv = __frcp_rn(r2);
        const float lg = -0.5f * __logf(r2);
        const float rl = fmaf(rx, p.lx, ry * p.ly) * inv;
        const float xr = p.xi * inv;
        fx += lg * p.lx + rl * rx + xr * ry;
        fy += lg * p.ly + rl * ry - xr * rx;
      }
      cx += fx;
      cy += fy;
    } else if (kMode == kCompDF) {
      df32 fx = {0.f, 0.f}, fy = {0.f, 0.f};
      for (int q = 0; q < nq; ++q) {
        const PoreDF p = s_d[q];
        const df32 rx = df_sub_point(tgx, trx, p.gx, p.rx);
        const df32 ry = df_sub_point(tgy, try_, p.gy, p.ry);
        const df32 r2 = df_dot2(rx, ry, rx, ry);
        const df32 inv = df_rcp(r2);
        const float2 lt = logtab[(int64_t)(k0 + q) * T + i];
        const df32 lg = {-0.5f * lt.x, -0.5f * lt.y};
        const df32 rl = df_mul(df_dot2(rx, ry, p.lx, p.ly), inv);
        const df32 xr = df_mul(p.xi, inv);
        // fx += lg lx + rl rx + xr ry ; fy += lg ly + rl ry - xr rx
        fx = df_add(fx, df_add(df_mul(lg, p.lx), df_add(df_mul(rl, rx), df_mul(xr, ry))));
        const df32 nxr = {-xr.h, -xr.l};
        fy = df_add(fy, df_add(df_mul(lg, p.ly), df_add(df_mul(rl, ry), df_mul(nxr, rx))));
      }
      cx += df_to_double(fx);
      cy += df_to_double(fy);
    } else {
      for (int q = 0; q < nq; ++q) {
        const double2 c = s_c[q];
        const double4_32a m = s_m[q];
        const double rx = x.x - c.x, ry = x.y - c.y;
        const double r2 = fma(rx, rx, ry * ry);
        const double inv = 1.0 / r2;
        const double lg = -0.5 * log(r2);
        const double rl = fma(rx, m.x, ry * m.y) * inv;
        const double xr = m.z * inv;
        cx += lg * m.x + rl * rx + xr * ry;
        cy += lg * m.y + rl * ry - xr * rx;
      }
    }
  }
  if (live) y[i] = make_double2(ax + kInv4Pi * cx, ay + kInv4Pi * cy);
}

// log(|x_i - c_k|^2) for every node i and pore k, as a float pair, layout [k][i].
static __global__ void k_log_table(int64_t N, int M, const double2* __restrict__ pos, const int* __restrict__ pore_ids,
                            const double2* __restrict__ centre, float2* __restrict__ tab) {
  count_launch();
  const int k = blockIdx.y;
  const double2 c = centre[pore_ids[k]];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 p = pos[i];
    const double rx = p.x - c.x, ry = p.y - c.y;
    const df32 v = df_from_double(log(rx * rx + ry * ry));
    tab[(int64_t)k * N + i] = make_float2(v.h, v.l);
  }
}

// Table of log rho^2 for the double-float completion; false if it would be
// too large (then the FP64 completion is used).
inline bool ensure_log_table(Geom& g) {
  if (g.logtab_ready) return true;
  const double bytes = 8.0 * (double)g.N * (double)g.M;
  if (g.M == 0 || bytes > 4.0e9) return false;
  g.logtab.alloc((size_t)g.N * g.M);
  dim3 grid((unsigned)std::min<int64_t>((g.N + 255) / 256, 64), (unsigned)g.M);
  k_log_table<<<grid, 256, 0, g.stream>>>(g.N, g.M, g.pos.get(), g.pore_ids.get(), g.centre.get(), g.logtab.get());
  STOKES_LAUNCHED();
  g.logtab_ready = true;
  return true;
}

// part: split partial sums, split s of target i at part[s * pstride + i];
// mom: the component moments of sigma.
template <int kMode>
inline void launch_epilogue(Geom& g, int64_t T, int splits, bool boundary, const double2* targets,
                            const double2* sigma, double2* y, const int* done, const double2* part = nullptr,
                            int64_t pstride = -1, const double4_32a* mom = nullptr) {
  k_epilogue<kMode><<<(unsigned)((T + 255) / 256), 256, 0, g.stream>>>(
      T, splits, part ? part : g.part.get(), pstride >= 0 ? pstride : T, boundary ? 1 : 0, targets, g.selfc.get(),
      sigma, g.comp.get(), g.outer, g.nrm.get(), g.M, g.pore_ids.get(), g.centre.get(), mom ? mom : g.mom.get(),
      g.logtab.get(), y, done);
  STOKES_LAUNCHED();
}

}  // namespace dlp
}  // namespace stokes
