// Double-float double-layer operator: FP64-class accuracy on the FP32 pipes.
//
// On this GPU double precision issues at 1/64 of the single-precision rate,
// so the pair sum is evaluated with unevaluated sums of two floats
// (Dekker's double-length arithmetic: TwoSum, FastTwoSum and an FMA-based
// TwoProduct). Each position is a float on a 2^-8 grid (differences of grid
// values are exact) plus a float-pair remainder, which keeps ~2^-57 absolute
// precision, finer than the double input itself; r = (grid difference) +
// (remainder difference) is then exact to ~2^-48 |r|. The weighted normals
// and the density are split hi + lo; rho^2, r.a and r.sigma are formed with
// error-free transformations, 1/rho^2 by one Newton step on a correctly rounded float
// reciprocal, and the running sum keeps its rounding errors in a second float
// (the compensated summation of Ogita, Rump and Oishi) over kFlush pairs, then
// moves to a double accumulator: the error of the float-pair sum grows with
// the number of terms it holds, and 16 pairs instead of a whole 256-source
// tile cut the operator's error at an ill-conditioned system's solution ten
// times for 2 % of the time. The diagonal, jump, wall and completion terms
// are FP64.
#include "dlp_common.cuh"

namespace stokes {

namespace {

using dlp::df32;

constexpr int kFlush = 16;  // pairs summed in double-float before the double accumulator

__device__ __forceinline__ void acc_prod(df32& acc, df32 c, df32 r) {
  const float p = c.h * r.h;
  float pe = fmaf(c.h, r.h, -p);
  pe = fmaf(c.h, r.l, pe);
  pe = fmaf(c.l, r.h, pe);
  const df32 s = dlp::two_sum(acc.h, p);
  acc.h = s.h;
  acc.l += s.l + pe;
}

// One pair in double-float arithmetic: adds the pair's term to (ax, ay).
__device__ __forceinline__ void df_pair(float GX, float GY, df32 X, df32 Y, float2 gq, float4 p, float4 a, float4 s,
                                        df32& ax, df32& ay) {
  // r = (grid difference, exact) + (remainder difference as a float pair)
  df32 lx = dlp::two_diff(X.h, p.x);
  lx.l += X.l - p.z;
  df32 ly = dlp::two_diff(Y.h, p.y);
  ly.l += Y.l - p.w;
  // the grid difference is zero or dominates |lx.h| <= 2^-8: FastTwoSum is exact
  df32 rx = dlp::fast_two_sum(GX - gq.x, lx.h);
  rx.l += lx.l;
  df32 ry = dlp::fast_two_sum(GY - gq.y, ly.h);
  ry.l += ly.l;
  // rho^2 = rx^2 + ry^2
  const float px = rx.h * rx.h;
  float ex = fmaf(rx.h, rx.h, -px);
  ex = fmaf(rx.h + rx.h, rx.l, ex);
  const float py = ry.h * ry.h;
  float ey = fmaf(ry.h, ry.h, -py);
  ey = fmaf(ry.h + ry.h, ry.l, ey);
  df32 r2 = dlp::two_sum(px, py);
  r2 = dlp::fast_two_sum(r2.h, r2.l + (ex + ey));
  // + 1e-30 after normalisation: the self pair (r = 0, so r.a = r.sigma
  // = 0) gets a finite reciprocal and contributes exactly 0; for any other
  // pair rho^2 >> 1e-30 and the addition rounds away
  r2.h += 1e-30f;
  // 1 / rho^2: one Newton step from the correctly rounded reciprocal
  const float y0 = __frcp_rn(r2.h);
  float t = fmaf(-r2.h, y0, 1.0f);
  t = fmaf(-r2.l, y0, t);
  const df32 inv = {y0, y0 * t};
  const df32 d = dlp::df_dot2(rx, ry, {a.x, a.z}, {a.y, a.w});
  const df32 e = dlp::df_dot2(rx, ry, {s.x, s.z}, {s.y, s.w});
  const df32 c = dlp::df_mul(dlp::df_mul(d, inv), dlp::df_mul(e, inv));
  acc_prod(ax, c, rx);
  acc_prod(ay, c, ry);
}

// CTA of TH threads, TPT targets per thread (i, i + TH, ...), TILE sources
// per shared-memory tile.
template <int TH, int TPT, int TILE>
__global__ void __launch_bounds__(TH)
k_dlp_pairs_df64(int64_t N, const float2* __restrict__ grid, const float4* __restrict__ pos,
                 const float4* __restrict__ aw, const double2* __restrict__ sig, int64_t T,
                 const double2* __restrict__ tgt, int64_t chunk, double2* __restrict__ part,
                 const int* __restrict__ done) {
  static_assert(TILE % kFlush == 0, "the tile is summed in groups of kFlush pairs");
  count_launch();
  if (done && *done) return;
  __shared__ float2 s_g[TILE];  // x, y on the 2^-8 grid
  __shared__ float4 s_p[TILE];  // remainder: x_hi, y_hi, x_lo, y_lo
  __shared__ float4 s_a[TILE];  // a_x hi, a_y hi, a_x lo, a_y lo
  __shared__ float4 s_s[TILE];  // sigma_x hi, sigma_y hi, sigma_x lo, sigma_y lo
  const int64_t ib = blockIdx.x * (int64_t)(TPT * TH) + threadIdx.x;
  float GX[TPT], GY[TPT];
  df32 X[TPT], Y[TPT];
  double ux[TPT], uy[TPT];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    const double2 x = i < T ? tgt[i] : make_double2(0.0, 0.0);
    const double gx = rint(x.x * 256.0) * (1.0 / 256.0), gy = rint(x.y * 256.0) * (1.0 / 256.0);
    GX[t] = (float)gx;
    GY[t] = (float)gy;
    X[t] = dlp::df_from_double(x.x - gx);
    Y[t] = dlp::df_from_double(x.y - gy);
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
        const double2 sg = sig[j];
        const df32 sx = dlp::df_from_double(sg.x), sy = dlp::df_from_double(sg.y);
        s_g[q] = grid[j];
        s_p[q] = pos[j];
        s_a[q] = aw[j];
        s_s[q] = make_float4(sx.h, sy.h, sx.l, sy.l);
      } else {
        s_g[q] = make_float2(1e18f, 1e18f);
        s_p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    for (int q0 = 0; q0 < TILE; q0 += kFlush) {
      df32 ax[TPT], ay[TPT];
#pragma unroll
      for (int t = 0; t < TPT; ++t) ax[t] = ay[t] = df32{0.f, 0.f};
#pragma unroll 2
      for (int q = q0; q < q0 + kFlush; ++q) {
        const float2 gq = s_g[q];
        const float4 p = s_p[q];
        const float4 a = s_a[q];
        const float4 s = s_s[q];
#pragma unroll
        for (int t = 0; t < TPT; ++t) df_pair(GX[t], GY[t], X[t], Y[t], gq, p, a, s, ax[t], ay[t]);
      }
#pragma unroll
      for (int t = 0; t < TPT; ++t) {
        ux[t] += dlp::df_to_double(ax[t]);
        uy[t] += dlp::df_to_double(ay[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int64_t i = ib + t * TH;
    if (i < T) part[blockIdx.y * T + i] = make_double2(ux[t], uy[t]);
  }
}

using PairKernelDF = void (*)(int64_t, const float2*, const float4*, const float4*, const double2*, int64_t,
                              const double2*, int64_t, double2*, const int*);
struct VariantDF {
  PairVariant info;
  PairKernelDF kernel;
};
// entry 0 is the default shape
const VariantDF kVariants[] = {
    {{128, 1, 128}, k_dlp_pairs_df64<128, 1, 128>}, {{64, 1, 64}, k_dlp_pairs_df64<64, 1, 64>},
    {{256, 1, 256}, k_dlp_pairs_df64<256, 1, 256>}, {{128, 2, 128}, k_dlp_pairs_df64<128, 2, 128>},
    {{64, 2, 128}, k_dlp_pairs_df64<64, 2, 128>},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

}  // namespace

int pair_variants_df64(PairVariant* out, int cap) {
  for (int v = 0; v < kNumVariants && v < cap; ++v) out[v] = kVariants[v].info;
  return kNumVariants;
}

int pairs_df64(Geom& g, const double2* sigma, const double2* targets, int64_t T, PairShape sh, const int* done) {
  require(sh.variant >= 0 && sh.variant < kNumVariants, "double-float pair kernel: unknown shape variant");
  const VariantDF& v = kVariants[sh.variant];
  const int tb = v.info.threads * v.info.tpt;
  int splits;
  int64_t chunk;
  dlp::pair_launch_shape(g.N, T, tb, v.info.tile, splits, chunk, sh.ctas_per_sm);
  g.part.alloc((size_t)splits * T);
  dim3 grid((unsigned)((T + tb - 1) / tb), (unsigned)splits);
  const int pe = g.prof.begin(kProfPairsDF64, (double)g.N * (double)T, g.stream);
  v.kernel<<<grid, v.info.threads, 0, g.stream>>>(g.N, g.df_grid.get(), g.df_pos.get(), g.df_a.get(), sigma, T,
                                                  targets, chunk, g.part.get(), done);
  STOKES_LAUNCHED();
  g.prof.end(pe, g.stream);
  return splits;
}

void dlp_apply_df64(Geom& g, const double2* sigma, double2* y, bool boundary, const double2* targets, int64_t T,
                    const int* done) {
  if (T == 0) return;
  moments_f64(g, sigma, done);
  const int splits = pairs_df64(g, sigma, targets, T, pair_shape(g, STOKES_DF64, T), done);
  const int pq = g.prof.begin(kProfEpilogue, (double)g.M * (double)T, g.stream);
  if (boundary && dlp::ensure_log_table(g))
    dlp::launch_epilogue<dlp::kCompDF>(g, T, splits, boundary, targets, sigma, y, done);
  else
    dlp::launch_epilogue<dlp::kCompF64>(g, T, splits, boundary, targets, sigma, y, done);
  g.prof.end(pq, g.stream);
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_dlp_df64() { return tu_launches(); }
}  // namespace stokes
