// FP32 double-layer operator (inner solves of the mixed-precision
// refinement). The pair sum runs in single precision; each node position is
// stored as hi = fl32(x) plus lo = fl32(x - hi), and r = (x_i,hi - x_j,hi) +
// (x_i,lo - x_j,lo) keeps the difference of nearby nodes accurate to single
// precision relative to |r| (a plain float subtraction would lose up to
// |x| / |r| of it). Per-tile float sums are accumulated in double; the
// diagonal, jump and wall terms stay FP64, the completion runs in FP32.
#include "dlp_common.cuh"

namespace stokes {

namespace {

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// CTA of TH threads, each accumulating TPT targets (i, i + TH, ...), so each
// staged source (two shared-memory loads) feeds TPT pair evaluations;
// TILE sources per shared-memory tile.
template <int TH, int TPT, int TILE>
__global__ void __launch_bounds__(TH)
k_dlp_pairs_f32(int64_t N, const float4* __restrict__ src, const float2* __restrict__ lo,
                const double2* __restrict__ sig, int64_t T, const double2* __restrict__ tgt, int64_t chunk,
                double2* __restrict__ part, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ float4 s_a[TILE];  // x_hi, y_hi, a_x, a_y
  __shared__ float4 s_b[TILE];  // x_lo, y_lo, sigma_x, sigma_y
  const int64_t ib = blockIdx.x * (int64_t)(TPT * TH) + threadIdx.x;
  float xh[TPT], yh[TPT], xl[TPT], yl[TPT];
  double ux[TPT], uy[TPT];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    const double2 x = i < T ? tgt[i] : make_double2(0.0, 0.0);
    xh[t] = (float)x.x;
    yh[t] = (float)x.y;
    xl[t] = (float)(x.x - (double)xh[t]);
    yl[t] = (float)(x.y - (double)yh[t]);
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
        const float2 l = lo[j];
        const double2 sg = sig[j];
        s_a[q] = src[j];
        s_b[q] = make_float4(l.x, l.y, (float)sg.x, (float)sg.y);
      } else {
        s_a[q] = make_float4(1e18f, 1e18f, 0.f, 0.f);
        s_b[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    float fx[TPT], fy[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) fx[t] = fy[t] = 0.f;
#pragma unroll 4
    for (int q = 0; q < TILE; ++q) {
      const float4 a = s_a[q];
      const float4 b = s_b[q];
#pragma unroll
      for (int t = 0; t < TPT; ++t) {
        const float rx = (xh[t] - a.x) + (xl[t] - b.x);
        const float ry = (yh[t] - a.y) + (yl[t] - b.y);
        // + 1e-30: the self pair (r = 0, so d = e = 0) gives a finite inverse
        // and contributes exactly 0; for any other pair rho^2 >> 1e-30
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1e-30f));
        const float inv = rcp_approx(r2);
        const float d = fmaf(rx, a.z, ry * a.w);
        const float e = fmaf(rx, b.z, ry * b.w);
        const float c = (d * inv) * (e * inv);
        fx[t] = fmaf(c, rx, fx[t]);
        fy[t] = fmaf(c, ry, fy[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
      ux[t] += fx[t];
      uy[t] += fy[t];
    }
  }
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    if (i < T) part[blockIdx.y * T + i] = make_double2(ux[t], uy[t]);
  }
}

using PairKernelF32 = void (*)(int64_t, const float4*, const float2*, const double2*, int64_t, const double2*, int64_t,
                               double2*, const int*);
struct VariantF32 {
  PairVariant info;
  PairKernelF32 kernel;
};
// entry 0 is the default shape
const VariantF32 kVariants[] = {
    {{256, 2, 256}, k_dlp_pairs_f32<256, 2, 256>}, {{128, 2, 128}, k_dlp_pairs_f32<128, 2, 128>},
    {{256, 1, 256}, k_dlp_pairs_f32<256, 1, 256>}, {{128, 4, 128}, k_dlp_pairs_f32<128, 4, 128>},
    {{256, 4, 256}, k_dlp_pairs_f32<256, 4, 256>}, {{64, 4, 128}, k_dlp_pairs_f32<64, 4, 128>},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

}  // namespace

int pair_variants_f32(PairVariant* out, int cap) {
  for (int v = 0; v < kNumVariants && v < cap; ++v) out[v] = kVariants[v].info;
  return kNumVariants;
}

int pairs_f32(Geom& g, const double2* sigma, const double2* targets, int64_t T, PairShape sh, const int* done) {
  require(sh.variant >= 0 && sh.variant < kNumVariants, "FP32 pair kernel: unknown shape variant");
  const VariantF32& v = kVariants[sh.variant];
  int splits;
  int64_t chunk;
  dlp::pair_launch_shape(g.N, T, v.info.threads * v.info.tpt, v.info.tile, splits, chunk, sh.ctas_per_sm);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + v.info.threads * v.info.tpt - 1) / (v.info.threads * v.info.tpt)), (unsigned)splits);
  const int pe = g.prof.begin(kProfPairsF32, (double)g.N * (double)T, g.stream);
  v.kernel<<<grid, v.info.threads, 0, g.stream>>>(g.N, g.f32_src.get(), g.f32_lo.get(), sigma, T, targets, chunk,
                                                  g.part.get(), done);
  STOKES_LAUNCHED();
  g.prof.end(pe, g.stream);
  return splits;
}

void dlp_apply_f32(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets, int64_t T,
                   const int* done) {
  if (T == 0) return;
  moments_f64(g, sigma, done);
  const int splits = pairs_f32(g, sigma, targets, T, pair_shape(g, STOKES_FP32, T), done);
  const int pq = g.prof.begin(kProfEpilogue, (double)g.M * (double)T, g.stream);
  dlp::launch_epilogue<dlp::kCompF32>(g, T, splits, boundary, targets, sigma, y, done);
  g.prof.end(pq, g.stream);
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_dlp_f32() { return tu_launches(); }
}  // namespace stokes
