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

constexpr int kTile = 256;
constexpr int kThreads = 256;

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Each thread accumulates two targets, i and i + kThreads, so each staged
// source (two shared-memory loads) feeds two pair evaluations.
__global__ void __launch_bounds__(kThreads)
k_dlp_pairs_f32(int64_t N, const float4* __restrict__ src, const float2* __restrict__ lo,
                const double2* __restrict__ sig, int64_t T, const double2* __restrict__ tgt, int64_t chunk,
                double2* __restrict__ part, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ float4 s_a[kTile];  // x_hi, y_hi, a_x, a_y
  __shared__ float4 s_b[kTile];  // x_lo, y_lo, sigma_x, sigma_y
  const int64_t i0 = blockIdx.x * (int64_t)(2 * kThreads) + threadIdx.x;
  const int64_t i1 = i0 + kThreads;
  const double2 x0 = i0 < T ? tgt[i0] : make_double2(0.0, 0.0);
  const double2 x1 = i1 < T ? tgt[i1] : make_double2(0.0, 0.0);
  const float xh0 = (float)x0.x, yh0 = (float)x0.y;
  const float xl0 = (float)(x0.x - (double)xh0), yl0 = (float)(x0.y - (double)yh0);
  const float xh1 = (float)x1.x, yh1 = (float)x1.y;
  const float xl1 = (float)(x1.x - (double)xh1), yl1 = (float)(x1.y - (double)yh1);
  const int64_t j0 = blockIdx.y * chunk;
  const int64_t j1 = imin64(N, j0 + chunk);
  double ux0 = 0.0, uy0 = 0.0, ux1 = 0.0, uy1 = 0.0;
  for (int64_t t0 = j0; t0 < j1; t0 += kTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kTile; q += blockDim.x) {
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
    float fx0 = 0.f, fy0 = 0.f, fx1 = 0.f, fy1 = 0.f;
#pragma unroll 4
    for (int q = 0; q < kTile; ++q) {
      const float4 a = s_a[q];
      const float4 b = s_b[q];
      {
        const float rx = (xh0 - a.x) + (xl0 - b.x);
        const float ry = (yh0 - a.y) + (yl0 - b.y);
        // + 1e-30: the self pair (r = 0, so d = e = 0) gives a finite inverse
        // and contributes exactly 0; for any other pair rho^2 >> 1e-30
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1e-30f));
        const float inv = rcp_approx(r2);
        const float d = fmaf(rx, a.z, ry * a.w);
        const float e = fmaf(rx, b.z, ry * b.w);
        const float c = (d * inv) * (e * inv);
        fx0 = fmaf(c, rx, fx0);
        fy0 = fmaf(c, ry, fy0);
      }
      {
        const float rx = (xh1 - a.x) + (xl1 - b.x);
        const float ry = (yh1 - a.y) + (yl1 - b.y);
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1e-30f));
        const float inv = rcp_approx(r2);
        const float d = fmaf(rx, a.z, ry * a.w);
        const float e = fmaf(rx, b.z, ry * b.w);
        const float c = (d * inv) * (e * inv);
        fx1 = fmaf(c, rx, fx1);
        fy1 = fmaf(c, ry, fy1);
      }
    }
    ux0 += fx0;
    uy0 += fy0;
    ux1 += fx1;
    uy1 += fy1;
  }
  if (i0 < T) part[blockIdx.y * T + i0] = make_double2(ux0, uy0);
  if (i1 < T) part[blockIdx.y * T + i1] = make_double2(ux1, uy1);
}

}  // namespace

void dlp_apply_f32(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets, int64_t T,
                   const int* done) {
  if (T == 0) return;
  moments_f64(g, sigma, done);
  int splits;
  int64_t chunk;
  dlp::pair_launch_shape(g.N, T, 2 * kThreads, kTile, splits, chunk);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + 2 * kThreads - 1) / (2 * kThreads)), (unsigned)splits);
  const int pe = g.prof.begin(kProfPairsF32, (double)g.N * (double)T, g.stream);
  k_dlp_pairs_f32<<<grid, kThreads, 0, g.stream>>>(g.N, g.f32_src.get(), g.f32_lo.get(), sigma, T, targets, chunk,
                                                    g.part.get(), done);
  STOKES_LAUNCHED();
  g.prof.end(pe, g.stream);
  const int pq = g.prof.begin(kProfEpilogue, (double)g.M * (double)T, g.stream);
  dlp::launch_epilogue<dlp::kCompF32>(g, T, splits, boundary, targets, sigma, y, done);
  g.prof.end(pq, g.stream);
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_dlp_f32() { return tu_launches(); }
}  // namespace stokes
