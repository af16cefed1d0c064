// FP64 double-layer operator: the all-pairs sum of the double-layer kernel
// (Sec. 2.1, discretised by the trapezoid rule of Sec. 2.2) as a tiled
// N-body kernel, then the shared epilogue (diagonal curvature term, -1/2
// jump, pore completions, wall term).
#include "dlp_common.cuh"

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
  count_launch();
  if (done && *done) return;
  __shared__ double4_32a s_src[kTile];
  __shared__ double2 s_sig[kTile];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double2 x = make_double2(0.0, 0.0);
  if (i < T) x = tgt[i];
  const int64_t j0 = blockIdx.y * chunk;
  const int64_t j1 = imin64(N, j0 + chunk);
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
    const int64_t jb = t0 - iself;  // q + jb == 0  <=>  source is the target itself
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

}  // namespace

void dlp_apply_f64(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets,
                   int64_t T, const int* done) {
  if (T == 0) return;
  moments_f64(g, sigma, done);
  int splits;
  int64_t chunk;
  dlp::pair_launch_shape(g.N, T, 128, kTile, splits, chunk);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + 127) / 128), (unsigned)splits);
  const int pe = g.prof.begin(kProfPairsF64, (double)g.N * (double)T, g.stream);
  k_dlp_pairs_f64<<<grid, 128, 0, g.stream>>>(g.N, g.src.get(), sigma, T, targets, chunk, boundary ? 1 : 0,
                                               g.part.get(), done);
  STOKES_LAUNCHED();
  g.prof.end(pe, g.stream);
  const int pq = g.prof.begin(kProfEpilogue, (double)g.M * (double)T, g.stream);
  dlp::launch_epilogue<dlp::kCompF64>(g, T, splits, boundary, targets, sigma, y, done);
  g.prof.end(pq, g.stream);
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_dlp_f64() { return tu_launches(); }
}  // namespace stokes
