// FP64 double-layer operator: the all-pairs sum of the double-layer kernel
// (Sec. 2.1, discretised by the trapezoid rule of Sec. 2.2) as a tiled
// N-body kernel, then the shared epilogue (diagonal curvature term, -1/2
// jump, pore completions, wall term).
#include "dlp_common.cuh"

namespace stokes {

namespace {

// Pair sum for TPT targets per thread (i, i + TH, ...) of the CTA's
// TPT * TH targets over the source range [blockIdx.y * chunk, ...), TILE
// sources per shared-memory tile; writes one partial per (split, target).
//   u_i += (r.a_j)(r.sigma_j) r / rho^4, r = x_i - x_j, a_j = w_j n_j / pi
// The j = i pair is skipped when self_skip (targets are the nodes).
template <int TH, int TPT, int TILE>
__global__ void __launch_bounds__(TH)
k_dlp_pairs_f64(int64_t N, const double4_32a* __restrict__ src, const double2* __restrict__ sig,
                int64_t T, const double2* __restrict__ tgt, int64_t chunk, int self_skip,
                double2* __restrict__ part, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double4_32a s_src[TILE];
  __shared__ double2 s_sig[TILE];
  const int64_t ib = blockIdx.x * (int64_t)(TPT * TH) + threadIdx.x;
  double2 x[TPT];
  double ux[TPT], uy[TPT];
  int64_t iself[TPT];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    x[t] = i < T ? tgt[i] : make_double2(0.0, 0.0);
    iself[t] = self_skip ? i : -1;
    ux[t] = 0.0;
    uy[t] = 0.0;
  }
  const int64_t j0 = blockIdx.y * chunk;
  const int64_t j1 = imin64(N, j0 + chunk);
  for (int64_t t0 = j0; t0 < j1; t0 += TILE) {
    __syncthreads();
    for (int q = threadIdx.x; q < TILE; q += TH) {
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
#pragma unroll 4
    for (int q = 0; q < TILE; ++q) {
      const double4_32a s = s_src[q];
      const double2 sg = s_sig[q];
#pragma unroll
      for (int t = 0; t < TPT; ++t) {
        const double rx = x[t].x - s.x, ry = x[t].y - s.y;
        double r2 = fma(rx, rx, ry * ry);
        r2 = (t0 + q == iself[t]) ? 1.0 : r2;  // r = 0 there, so the pair contributes 0
        const double inv = dlp::rcp_newton(r2);
        const double d = fma(rx, s.z, ry * s.w);
        const double e = fma(rx, sg.x, ry * sg.y);
        const double c = (d * inv) * (e * inv);
        ux[t] = fma(c, rx, ux[t]);
        uy[t] = fma(c, ry, uy[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    if (i < T) part[blockIdx.y * T + i] = make_double2(ux[t], uy[t]);
  }
}

using PairKernelF64 = void (*)(int64_t, const double4_32a*, const double2*, int64_t, const double2*, int64_t, int,
                               double2*, const int*);
struct VariantF64 {
  PairVariant info;
  PairKernelF64 kernel;
};
// entry 0 is the default shape
const VariantF64 kVariants[] = {
    {{128, 1, 128}, k_dlp_pairs_f64<128, 1, 128>},
    {{64, 1, 64}, k_dlp_pairs_f64<64, 1, 64>},
    {{256, 1, 256}, k_dlp_pairs_f64<256, 1, 256>},
    {{128, 2, 128}, k_dlp_pairs_f64<128, 2, 128>},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

}  // namespace

int pair_variants_f64(PairVariant* out, int cap) {
  for (int v = 0; v < kNumVariants && v < cap; ++v) out[v] = kVariants[v].info;
  return kNumVariants;
}

int pairs_f64(Geom& g, const double2* sigma, const double2* targets, int64_t T, bool boundary, PairShape sh,
              const int* done) {
  require(sh.variant >= 0 && sh.variant < kNumVariants, "FP64 pair kernel: unknown shape variant");
  const VariantF64& v = kVariants[sh.variant];
  const int tb = v.info.threads * v.info.tpt;
  int splits;
  int64_t chunk;
  dlp::pair_launch_shape(g.N, T, tb, v.info.tile, splits, chunk, sh.ctas_per_sm);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + tb - 1) / tb), (unsigned)splits);
  const int pe = g.prof.begin(kProfPairsF64, (double)g.N * (double)T, g.stream);
  v.kernel<<<grid, v.info.threads, 0, g.stream>>>(g.N, g.src.get(), sigma, T, targets, chunk, boundary ? 1 : 0,
                                                  g.part.get(), done);
  STOKES_LAUNCHED();
  g.prof.end(pe, g.stream);
  return splits;
}

void dlp_apply_f64(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets,
                   int64_t T, const int* done) {
  if (T == 0) return;
  moments_f64(g, sigma, done);
  const int splits = pairs_f64(g, sigma, targets, T, boundary, pair_shape(g, STOKES_FP64, T), done);
  const int pq = g.prof.begin(kProfEpilogue, (double)g.M * (double)T, g.stream);
  dlp::launch_epilogue<dlp::kCompF64>(g, T, splits, boundary, targets, sigma, y, done);
  g.prof.end(pq, g.stream);
}

namespace {
__global__ void k_rcp_newton(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = dlp::rcp_newton(x[i]);
}
}  // namespace

void rcp_newton_apply(const double* x, double* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_rcp_newton<<<(unsigned)imin64((n + 255) / 256, 152 * 8), 256, 0, s>>>(x, y, n);
  STOKES_LAUNCHED();
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_dlp_f64() { return tu_launches(); }
}  // namespace stokes
