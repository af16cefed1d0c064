// Shared pieces of the double-layer operator kernels: the launch shape of
// the pair kernels, the double-float (unevaluated float pair) primitives and
// the epilogue that turns pair partial sums into A sigma or a velocity.
#pragma once

#include "internal.cuh"

namespace stokes {
namespace dlp {

constexpr int kEpiPores = 256;

// Split the sources so that the grid has ~4 CTAs per SM; each split covers
// a whole number of `tile`-sized source tiles.
inline void pair_launch_shape(int64_t N, int64_t T, int tb, int tile, int& splits, int64_t& chunk) {
  const int64_t tblocks = (T + tb - 1) / tb;
  int64_t want = (4 * 152 + tblocks - 1) / tblocks;
  const int64_t max_split = (N + tile - 1) / tile;
  if (want > max_split) want = max_split;
  if (want < 1) want = 1;
  chunk = ((N + want - 1) / want + tile - 1) / tile * tile;
  splits = (int)((N + chunk - 1) / chunk);
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
// The diagonal and wall terms are O(N) and always FP64; the completion is
// FP64 (kCompF32 = false) or FP32 with r = (x_hi - c_hi) + (x_lo - c_lo).
template <bool kCompF32>
__global__ void __launch_bounds__(256)
k_epilogue(int64_t T, int S, const double2* __restrict__ part, int boundary, const double2* __restrict__ tgt,
           const double4_32a* __restrict__ selfc, const double2* __restrict__ sig, const int* __restrict__ comp,
           int outer, const double2* __restrict__ nrm, int M, const int* __restrict__ pore_ids,
           const double2* __restrict__ centre, const double4_32a* __restrict__ mom, double2* __restrict__ y,
           const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double2 s_c[kEpiPores];
  __shared__ double4_32a s_m[kEpiPores];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = i < T;
  double ax = 0.0, ay = 0.0;
  double2 x = make_double2(0.0, 0.0);
  if (live) {
    for (int s = 0; s < S; ++s) {
      const double2 p = part[s * T + i];
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
  const float xh = (float)x.x, yh = (float)x.y;
  const float xl = (float)(x.x - (double)xh), yl = (float)(x.y - (double)yh);
  double cx = 0.0, cy = 0.0;
  for (int k0 = 0; k0 < M; k0 += kEpiPores) {
    __syncthreads();
    for (int q = threadIdx.x; q < kEpiPores && k0 + q < M; q += blockDim.x) {
      const int k = pore_ids[k0 + q];
      s_c[q] = centre[k];
      s_m[q] = mom[k];
    }
    __syncthreads();
    const int nq = (int)imin64(kEpiPores, M - k0);
    if (live) {
      if (kCompF32) {
        float fx = 0.f, fy = 0.f;
        for (int q = 0; q < nq; ++q) {
          const double2 c = s_c[q];
          const double4_32a m = s_m[q];
          const float chx = (float)c.x, chy = (float)c.y;
          const float rx = (xh - chx) + (xl - (float)(c.x - (double)chx));
          const float ry = (yh - chy) + (yl - (float)(c.y - (double)chy));
          const float r2 = fmaf(rx, rx, ry * ry);
          const float inv = __frcp_rn(r2);
          const float lg = -0.5f * __logf(r2);
          const float mx = (float)m.x, my = (float)m.y, mz = (float)m.z;
          const float rl = fmaf(rx, mx, ry * my) * inv;
          const float xr = mz * inv;
          fx += lg * mx + rl * rx + xr * ry;
          fy += lg * my + rl * ry - xr * rx;
        }
        cx += fx;
        cy += fy;
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
  }
  if (live) y[i] = make_double2(ax + kInv4Pi * cx, ay + kInv4Pi * cy);
}

template <bool kCompF32>
inline void launch_epilogue(Geom& g, int64_t T, int splits, bool boundary, const double2* targets,
                            const double2* sigma, double2* y, const int* done) {
  k_epilogue<kCompF32><<<(unsigned)((T + 255) / 256), 256, 0, g.stream>>>(
      T, splits, g.part.get(), boundary ? 1 : 0, targets, g.selfc.get(), sigma, g.comp.get(), g.outer,
      g.nrm.get(), g.M, g.pore_ids.get(), g.centre.get(), g.mom.get(), y, done);
  STOKES_LAUNCHED();
}

}  // namespace dlp
}  // namespace stokes
