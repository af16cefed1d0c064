// FP64 double-layer operator: the all-pairs sum of the double-layer kernel
// (Sec. 2.1, discretised by the trapezoid rule of Sec. 2.2) as a tiled
// N-body kernel, and an epilogue adding the diagonal curvature term, the
// -1/2 jump, the pore completions and the wall term.
#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kTile = 128;  // sources staged per shared-memory tile

// Pair sum for targets [blockIdx.x * blockDim.x, ...) over the source range
// [blockIdx.y * chunk, ...); writes one partial per (split, target).
//   u_i += (r.a_j)(r.sigma_j) r / rho^4, r = x_i - x_j, a_j = w_j n_j / pi
// The j = i pair is skipped when self_skip (targets are the nodes).
__global__ void __launch_bounds__(128)
k_dlp_pairs_f64(int64_t N, const double4_32a* __restrict__ src, const double2* __restrict__ sig,
                int64_t T, const double2* __restrict__ tgt, int64_t chunk, int self_skip,
                double2* __restrict__ part, const int* __restrict__ done) {
  if (done && *done) return;
  __shared__ double4_32a s_src[kTile];
  __shared__ double2 s_sig[kTile];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double2 x = make_double2(0.0, 0.0);
  if (i < T) x = tgt[i];
  const int64_t j0 = blockIdx.y * chunk;
  const int64_t j1 = min(N, j0 + chunk);
  const int64_t iself = self_skip ? i : -1;
  double ux = 0.0, uy = 0.0;
  for (int64_t t0 = j0; t0 < j1; t0 += kTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kTile; q += blockDim.x) {
      const int64_t j = t0 + q;
      if (j < j1) {
        s_src[q] = src[j];
        s_sig[q] = sig[j];
      } else {  // padding: far away, zero weight and density -> exact zero
        s_src[q] = make_double4_32a(1e30, 1e30, 0.0, 0.0);
        s_sig[q] = make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    const int64_t jb = t0 - iself;  // q == jb  <=>  source is the target itself
#pragma unroll 4
    for (int q = 0; q < kTile; ++q) {
      const double4_32a s = s_src[q];
      const double2 sg = s_sig[q];
      const double rx = x.x - s.x, ry = x.y - s.y;
      double r2 = fma(rx, rx, ry * ry);
      r2 = (q + jb == 0) ? 1.0 : r2;  // r = 0 there, so the pair contributes 0
      const double inv = 1.0 / r2;
      const double d = fma(rx, s.z, ry * s.w);
      const double e = fma(rx, sg.x, ry * sg.y);
      const double c = (d * inv) * (e * inv);
      ux = fma(c, rx, ux);
      uy = fma(c, ry, uy);
    }
  }
  if (i < T) part[blockIdx.y * T + i] = make_double2(ux, uy);
}

constexpr int kEpiPores = 256;

// y_i = sum_s part[s][i] + (boundary: self term - sigma_i/2 + wall term)
//       + sum_pores S(x_i, c_k) lambda_k + R(x_i, c_k) xi_k
__global__ void __launch_bounds__(256)
k_dlp_epilogue_f64(int64_t T, int S, const double2* __restrict__ part, int boundary,
                   const double2* __restrict__ tgt, const double4_32a* __restrict__ selfc,
                   const double2* __restrict__ sig, const int* __restrict__ comp, int outer,
                   const double2* __restrict__ nrm, int M, const int* __restrict__ pore_ids,
                   const double2* __restrict__ centre, const double4_32a* __restrict__ mom,
                   double2* __restrict__ y, const int* __restrict__ done) {
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
  double cx = 0.0, cy = 0.0;
  for (int k0 = 0; k0 < M; k0 += kEpiPores) {
    __syncthreads();
    for (int q = threadIdx.x; q < kEpiPores && k0 + q < M; q += blockDim.x) {
      const int k = pore_ids[k0 + q];
      s_c[q] = centre[k];
      s_m[q] = mom[k];
    }
    __syncthreads();
    const int nq = min(kEpiPores, M - k0);
    if (live) {
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

}  // namespace

// Launch geometry of the pair kernel: enough CTAs to cover the GPU.
static void pair_launch_shape(int64_t N, int64_t T, int& splits, int64_t& chunk) {
  const int64_t tblocks = (T + 127) / 128;
  int64_t want = (4 * 152 + tblocks - 1) / tblocks;          // ~4 CTAs per SM
  const int64_t max_split = (N + kTile - 1) / kTile;         // >= one tile per split
  if (want > max_split) want = max_split;
  if (want < 1) want = 1;
  chunk = ((N + want - 1) / want + kTile - 1) / kTile * kTile;
  splits = (int)((N + chunk - 1) / chunk);
}

void dlp_apply_f64(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets,
                   int64_t T, const int* done) {
  if (T == 0) return;
  cudaStream_t s = g.stream;
  moments_f64(g, sigma, done);
  int splits;
  int64_t chunk;
  pair_launch_shape(g.N, T, splits, chunk);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + 127) / 128), (unsigned)splits);
  k_dlp_pairs_f64<<<grid, 128, 0, s>>>(g.N, g.src.get(), sigma, T, targets, chunk, boundary ? 1 : 0,
                                        g.part.get(), done);
  STOKES_LAUNCHED();
  k_dlp_epilogue_f64<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(
      T, splits, g.part.get(), boundary ? 1 : 0, targets, g.selfc.get(), sigma, g.comp.get(), g.outer,
      g.nrm.get(), g.M, g.pore_ids.get(), g.centre.get(), g.mom.get(), y, done);
  STOKES_LAUNCHED();
}

}  // namespace stokes
