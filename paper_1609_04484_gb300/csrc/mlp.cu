// The learned coarse correction's network on the tensor cores: bfloat16
// GEMMs with float accumulation (mma.sync m16n8k16, operands staged in
// shared memory by cp.async and loaded with ldmatrix), the masked squared
// error and its gradient, bias-gradient column sums and the Adam update.
//
// Network (the paper has no counterpart): Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3
// with X [B x 35] (padded to 48 columns), W1 [35 x 256], W2 [256 x 256],
// W3 [256 x 153] (padded to 160 columns); every matrix is row-major. The
// master parameters are float, in the order W1, b1, W2, b2, W3, b3 (the
// oracle's layout); the GEMMs read bfloat16 copies padded with zeros.
//
// One GEMM kernel covers the three products of training:
//   forward   C = A B      A [m][k] (activations), B [k][n] (weights)
//   dX        C = A B^T    A [m][k] (output gradient), B [n][k] (weights)
//   dW        C = A^T B    A [k][m] (activations), B [k][n] (gradient)
// Shared-memory tiles keep each operand in its global layout; ldmatrix
// (.trans where the layout is [k][...]) turns them into mma fragments.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mlp.cuh"

namespace stokes {
namespace mlp {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32, kThreads = 128;
constexpr int kPadMK = kBK + 8;  // row length of a [64][32] tile (80 B rows: ldmatrix without bank conflicts)
constexpr int kPadKM = kBM + 8;  // row length of a [32][64] tile (144 B rows)
constexpr int kTileElems = 64 * kPadMK;  // >= 32 * kPadKM

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16 bytes global -> shared; src_bytes = 0 fills zeros (out-of-range chunks)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Epilogues: what is stored at C[m][n] for m < m_store, n < n_store.
enum Epi {
  kBiasReluBf16 = 0,  // bf16(relu(acc + bias[n]))
  kBiasF32 = 1,       // acc + bias[n]
  kF32 = 2,           // acc
  kMaskBf16 = 3       // bf16(aux[m][n] > 0 ? acc : 0), aux bf16 with leading dimension ldc
};

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  void* C;
  const float* bias;
  const __nv_bfloat16* aux;
  int64_t M, N, K;          // product sizes (multiples of 8)
  int64_t lda, ldb, ldc;    // leading dimensions (elements, multiples of 8)
  int64_t m_store, n_store; // stored part of C
};

// A_KM: A stored [k][m] (use A^T); B_NK: B stored [n][k] (use B^T).
template <bool A_KM, bool B_NK, int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm_bf16(GemmArgs g) {
  count_launch();
  __shared__ __align__(16) __nv_bfloat16 sA[2][kTileElems];
  __shared__ __align__(16) __nv_bfloat16 sB[2][kTileElems];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m0 = blockIdx.x * (int64_t)kBM, n0 = blockIdx.y * (int64_t)kBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

  auto load = [&](int buf, int64_t k0) {
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int c = tid + rep * kThreads;  // 256 chunks of 8 elements per operand tile
      // A
      if (!A_KM) {  // [64 m][32 k]
        const int row = c >> 2, col = (c & 3) * 8;
        const int64_t gm = m0 + row, gk = k0 + col;
        const bool ok = gm < g.M && gk < g.K;
        cp_async16(&sA[buf][row * kPadMK + col], ok ? (const void*)(g.A + gm * g.lda + gk) : (const void*)g.A,
                   ok ? 16 : 0);
      } else {      // [32 k][64 m]
        const int row = c >> 3, col = (c & 7) * 8;
        const int64_t gk = k0 + row, gm = m0 + col;
        const bool ok = gm < g.M && gk < g.K;
        cp_async16(&sA[buf][row * kPadKM + col], ok ? (const void*)(g.A + gk * g.lda + gm) : (const void*)g.A,
                   ok ? 16 : 0);
      }
      // B
      if (B_NK) {   // [64 n][32 k]
        const int row = c >> 2, col = (c & 3) * 8;
        const int64_t gn = n0 + row, gk = k0 + col;
        const bool ok = gn < g.N && gk < g.K;
        cp_async16(&sB[buf][row * kPadMK + col], ok ? (const void*)(g.B + gn * g.ldb + gk) : (const void*)g.B,
                   ok ? 16 : 0);
      } else {      // [32 k][64 n]
        const int row = c >> 3, col = (c & 7) * 8;
        const int64_t gk = k0 + row, gn = n0 + col;
        const bool ok = gn < g.N && gk < g.K;
        cp_async16(&sB[buf][row * kPadKM + col], ok ? (const void*)(g.B + gk * g.ldb + gn) : (const void*)g.B,
                   ok ? 16 : 0);
      }
    }
    cp_async_commit();
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  const int64_t nk = (g.K + kBK - 1) / kBK;
  load(0, 0);
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = (int)(kt & 1);
    cp_async_wait_all();
    __syncthreads();  // tile kt visible to all; everyone is done with tile kt - 1
    if (kt + 1 < nk) load(buf ^ 1, (kt + 1) * kBK);
    const __nv_bfloat16* tA = sA[buf];
    const __nv_bfloat16* tB = sB[buf];
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t af[2][4], bf[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int mb = wm + 16 * mi;
        if (!A_KM) {
          const int r = mb + (lane & 15), cidx = kk + (lane >> 4) * 8;
          ldsm_x4(af[mi], tA + r * kPadMK + cidx);
        } else {
          const int kr = kk + (lane & 7) + 8 * (lane >> 4), mc = mb + 8 * ((lane >> 3) & 1);
          ldsm_x4_t(af[mi], tA + kr * kPadKM + mc);
        }
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {  // two n8 tiles per ldmatrix.x4
        const int nb = wn + 16 * nj;
        if (B_NK) {
          const int r = nb + (lane & 7) + 8 * (lane >> 4), cidx = kk + 8 * ((lane >> 3) & 1);
          ldsm_x4(bf[nj], tB + r * kPadMK + cidx);
        } else {
          const int kr = kk + (lane & 7) + 8 * ((lane >> 3) & 1), nc = nb + 8 * (lane >> 4);
          ldsm_x4_t(bf[nj], tB + kr * kPadKM + nc);
        }
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          mma_bf16(acc[mi][ni], af[mi], bf[ni >> 1][2 * (ni & 1)], bf[ni >> 1][2 * (ni & 1) + 1]);
    }
  }

  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t m = m0 + wm + 16 * mi + gq + 8 * h;
        const int64_t n = n0 + wn + 8 * ni + 2 * tq;
        if (m >= g.m_store) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int64_t nn = n + e;
          if (nn >= g.n_store) continue;
          float v = acc[mi][ni][2 * h + e];
          if (EPI == kBiasReluBf16) {
            v = fmaxf(v + g.bias[nn], 0.f);
            static_cast<__nv_bfloat16*>(g.C)[m * g.ldc + nn] = __float2bfloat16_rn(v);
          } else if (EPI == kBiasF32) {
            static_cast<float*>(g.C)[m * g.ldc + nn] = v + g.bias[nn];
          } else if (EPI == kF32) {
            static_cast<float*>(g.C)[m * g.ldc + nn] = v;
          } else {
            const bool on = __bfloat162float(g.aux[m * g.ldc + nn]) > 0.f;
            static_cast<__nv_bfloat16*>(g.C)[m * g.ldc + nn] = __float2bfloat16_rn(on ? v : 0.f);
          }
        }
      }
}

template <bool A_KM, bool B_NK, int EPI>
void launch_gemm(const GemmArgs& a, cudaStream_t s) {
  require(a.M % 8 == 0 && a.N % 8 == 0 && a.K % 8 == 0 && a.lda % 8 == 0 && a.ldb % 8 == 0,
          "bf16 GEMM: sizes and leading dimensions must be multiples of 8");
  require(((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(a.B)) & 15) == 0,
          "bf16 GEMM: operands must be 16-byte aligned");
  if (a.M <= 0 || a.N <= 0) return;
  dim3 grid((unsigned)((a.M + kBM - 1) / kBM), (unsigned)((a.N + kBN - 1) / kBN));
  k_gemm_bf16<A_KM, B_NK, EPI><<<grid, kThreads, 0, s>>>(a);
  STOKES_LAUNCHED();
}

// float -> bf16 of a [rows][cols] block into a padded [rows_p][ld] array
// (zeros outside), with optional standardisation (x - mean[c]) / std[c].
__global__ void k_to_bf16_padded(const float* __restrict__ x, int64_t rows, int cols, int64_t ldx,
                                 const float* __restrict__ mean, const float* __restrict__ stdv,
                                 __nv_bfloat16* __restrict__ out, int64_t rows_p, int ld) {
  count_launch();
  const int64_t total = rows_p * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld;
    const int c = (int)(e % ld);
    float v = 0.f;
    if (r < rows && c < cols) {
      v = x[r * ldx + c];
      if (mean) v = (v - mean[c]) / stdv[c];
    }
    out[e] = __float2bfloat16_rn(v);
  }
}

// Masked squared error: per row r < rows and output o < n_out,
// d = mask (y - t); dY = bf16(2 d / count) (zero in the padding), and the
// per-CTA partial sums of d^2 (deterministic order) into part[blockIdx.x].
__global__ void __launch_bounds__(256)
k_loss_grad(const float* __restrict__ y, int ldy, const float* __restrict__ t, const float* __restrict__ mask,
            int64_t rows, int n_out, int64_t rows_p, int ldd, double inv_count, __nv_bfloat16* __restrict__ dy,
            double* __restrict__ part) {
  count_launch();
  __shared__ double red[256];
  double acc = 0.0;
  const int64_t total = rows_p * ldd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldd;
    const int o = (int)(e % ldd);
    float g = 0.f;
    if (r < rows && o < n_out) {
      const float mk = mask[r * n_out + o];
      const float d = mk * (y[r * ldy + o] - t[r * n_out + o]);
      acc += (double)d * (double)d;
      g = (float)(2.0 * (double)d * inv_count);
    }
    dy[e] = __float2bfloat16_rn(g);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  count_launch();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}

// out[c] = sum_r x[r][c] (bf16 input, c < cols), one thread per column.
__global__ void k_colsum_bf16(const __nv_bfloat16* __restrict__ x, int64_t rows, int cols, int ld,
                              float* __restrict__ out) {
  count_launch();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int64_t r = 0; r < rows; ++r) s += __bfloat162float(x[r * ld + c]);
  out[c] = s;
}

// Adam (Kingma and Ba 2015) on the float master parameters p with
// gradient g: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 copies of the weights in the GEMMs' padded layouts and float padded
// biases, from the flat master parameters.

__global__ void k_pack_weights(const float* __restrict__ p, Layout L, __nv_bfloat16* __restrict__ w1,
                               __nv_bfloat16* __restrict__ w2, __nv_bfloat16* __restrict__ w3,
                               float* __restrict__ b1, float* __restrict__ b2, float* __restrict__ b3) {
  count_launch();
  const int64_t n1 = (int64_t)L.in_p * L.hidden, n2 = (int64_t)L.hidden * L.hidden, n3 = (int64_t)L.hidden * L.out_p;
  const int64_t total = n1 + n2 + n3 + L.hidden + L.hidden + L.out_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = e;
    if (q < n1) {
      const int64_t r = q / L.hidden, c = q % L.hidden;
      w1[q] = __float2bfloat16_rn(r < L.n_in ? p[L.oW1 + r * L.hidden + c] : 0.f);
      continue;
    }
    q -= n1;
    if (q < n2) {
      w2[q] = __float2bfloat16_rn(p[L.oW2 + q]);
      continue;
    }
    q -= n2;
    if (q < n3) {
      const int64_t r = q / L.out_p, c = q % L.out_p;
      w3[q] = __float2bfloat16_rn(c < L.n_out ? p[L.oW3 + r * L.n_out + c] : 0.f);
      continue;
    }
    q -= n3;
    if (q < L.hidden) { b1[q] = p[L.ob1 + q]; continue; }
    q -= L.hidden;
    if (q < L.hidden) { b2[q] = p[L.ob2 + q]; continue; }
    q -= L.hidden;
    b3[q] = q < L.n_out ? p[L.ob3 + q] : 0.f;
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

Net::Net(int n_in, int hidden, int n_out) {
  L.n_in = n_in;
  L.hidden = hidden;
  L.n_out = n_out;
  L.in_p = (n_in + 15) / 16 * 16;
  L.out_p = (n_out + 15) / 16 * 16;
  L.oW1 = 0;
  L.ob1 = L.oW1 + (int64_t)n_in * hidden;
  L.oW2 = L.ob1 + hidden;
  L.ob2 = L.oW2 + (int64_t)hidden * hidden;
  L.oW3 = L.ob2 + hidden;
  L.ob3 = L.oW3 + (int64_t)hidden * n_out;
  L.total = L.ob3 + n_out;
}

int64_t Net::n_params() const { return L.total; }

void Net::init(const float* host_params, cudaStream_t s) {
  p.alloc(L.total);
  m.alloc(L.total);
  v.alloc(L.total);
  grad.alloc(L.total);
  w1.alloc((size_t)L.in_p * L.hidden);
  w2.alloc((size_t)L.hidden * L.hidden);
  w3.alloc((size_t)L.hidden * L.out_p);
  b1.alloc(L.hidden);
  b2.alloc(L.hidden);
  b3.alloc(L.out_p);
  STOKES_CUDA(cudaMemcpyAsync(p.get(), host_params, 4 * L.total, cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemsetAsync(m.get(), 0, 4 * L.total, s));
  STOKES_CUDA(cudaMemsetAsync(v.get(), 0, 4 * L.total, s));
  step = 0;
  pack(s);
}

void Net::set_params(const float* params, bool device, cudaStream_t s) {
  STOKES_CUDA(cudaMemcpyAsync(p.get(), params, 4 * L.total, device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s));
  pack(s);
}

void Net::pack(cudaStream_t s) {
  const int64_t total = (int64_t)L.in_p * L.hidden + (int64_t)L.hidden * L.hidden + (int64_t)L.hidden * L.out_p +
                        2 * L.hidden + L.out_p;
  k_pack_weights<<<grid_for(total), 256, 0, s>>>(p.get(), L, w1.get(), w2.get(), w3.get(), b1.get(), b2.get(),
                                                   b3.get());
  STOKES_LAUNCHED();
}

void Net::reserve(int64_t rows) {
  const int64_t rp = (rows + 63) / 64 * 64;
  if (rp <= rows_p && xb.get()) return;
  rows_p = rp;
  xb.alloc((size_t)rp * L.in_p);
  h1.alloc((size_t)rp * L.hidden);
  h2.alloc((size_t)rp * L.hidden);
  y.alloc((size_t)rp * L.out_p);
  dy.alloc((size_t)rp * L.out_p);
  dh1.alloc((size_t)rp * L.hidden);
  dh2.alloc((size_t)rp * L.hidden);
  part.alloc(1024);
  loss.alloc(1);
}

void Net::forward(const float* x, int64_t rows, const float* mean, const float* stdv, cudaStream_t s) {
  reserve(rows);
  k_to_bf16_padded<<<grid_for(rows_p * L.in_p), 256, 0, s>>>(x, rows, L.n_in, L.n_in, mean, stdv, xb.get(), rows_p,
                                                             L.in_p);
  STOKES_LAUNCHED();
  GemmArgs a{};
  // H1 = relu(X W1 + b1)
  a = GemmArgs{xb.get(), w1.get(), h1.get(), b1.get(), nullptr, rows_p, L.hidden, L.in_p, L.in_p, L.hidden, L.hidden,
               rows_p, L.hidden};
  launch_gemm<false, false, kBiasReluBf16>(a, s);
  // H2 = relu(H1 W2 + b2)
  a = GemmArgs{h1.get(), w2.get(), h2.get(), b2.get(), nullptr, rows_p, L.hidden, L.hidden, L.hidden, L.hidden,
               L.hidden, rows_p, L.hidden};
  launch_gemm<false, false, kBiasReluBf16>(a, s);
  // Y = H2 W3 + b3
  a = GemmArgs{h2.get(), w3.get(), y.get(), b3.get(), nullptr, rows_p, L.out_p, L.hidden, L.hidden, L.out_p, L.out_p,
               rows_p, L.out_p};
  launch_gemm<false, false, kBiasF32>(a, s);
}

void Net::loss_and_grad(const float* x, const float* t, const float* mask, int64_t rows, double count,
                        const float* mean, const float* stdv, cudaStream_t s) {
  forward(x, rows, mean, stdv, s);
  const unsigned gl = std::min<unsigned>(1024, grid_for(rows_p * L.out_p));
  k_loss_grad<<<gl, 256, 0, s>>>(y.get(), L.out_p, t, mask, rows, L.n_out, rows_p, L.out_p, 1.0 / count, dy.get(),
                                 part.get());
  k_sum_partials<<<1, 32, 0, s>>>(part.get(), (int)gl, 1.0 / count, loss.get());
  STOKES_LAUNCHED();
  float* G = grad.get();
  GemmArgs a{};
  // dW3 = H2^T dY  (stored [256][153] into the flat gradient)
  a = GemmArgs{h2.get(), dy.get(), G + L.oW3, nullptr, nullptr, L.hidden, L.out_p, rows_p, L.hidden, L.out_p,
               L.n_out, L.hidden, L.n_out};
  launch_gemm<true, false, kF32>(a, s);
  k_colsum_bf16<<<(L.n_out + 127) / 128, 128, 0, s>>>(dy.get(), rows_p, L.n_out, L.out_p, G + L.ob3);
  // dH2 = (dY W3^T) * [H2 > 0]
  a = GemmArgs{dy.get(), w3.get(), dh2.get(), nullptr, h2.get(), rows_p, L.hidden, L.out_p, L.out_p, L.out_p,
               L.hidden, rows_p, L.hidden};
  launch_gemm<false, true, kMaskBf16>(a, s);
  // dW2 = H1^T dH2, db2
  a = GemmArgs{h1.get(), dh2.get(), G + L.oW2, nullptr, nullptr, L.hidden, L.hidden, rows_p, L.hidden, L.hidden,
               L.hidden, L.hidden, L.hidden};
  launch_gemm<true, false, kF32>(a, s);
  k_colsum_bf16<<<(L.hidden + 127) / 128, 128, 0, s>>>(dh2.get(), rows_p, L.hidden, L.hidden, G + L.ob2);
  // dH1 = (dH2 W2^T) * [H1 > 0]
  a = GemmArgs{dh2.get(), w2.get(), dh1.get(), nullptr, h1.get(), rows_p, L.hidden, L.hidden, L.hidden, L.hidden,
               L.hidden, rows_p, L.hidden};
  launch_gemm<false, true, kMaskBf16>(a, s);
  // dW1 = X^T dH1 (rows of W1 beyond n_in are not stored), db1
  a = GemmArgs{xb.get(), dh1.get(), G + L.oW1, nullptr, nullptr, L.in_p, L.hidden, rows_p, L.in_p, L.hidden,
               L.hidden, L.n_in, L.hidden};
  launch_gemm<true, false, kF32>(a, s);
  k_colsum_bf16<<<(L.hidden + 127) / 128, 128, 0, s>>>(dh1.get(), rows_p, L.hidden, L.hidden, G + L.ob1);
  STOKES_LAUNCHED();
}

void Net::adam(const float* g, double lr, cudaStream_t s) {
  ++step;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
  k_adam<<<grid_for(L.total), 256, 0, s>>>(p.get(), g ? g : grad.get(), m.get(), v.get(), L.total, (float)lr,
                                           (float)b1, (float)b2, 1e-8f, c1, c2);
  STOKES_LAUNCHED();
  pack(s);
}

}  // namespace mlp

unsigned long long launches_mlp() { return tu_launches(); }

}  // namespace stokes
