// Single-precision explicit inverse of the largest preconditioner blocks.
//
// The double-float and mixed-precision solves apply the block-diagonal
// preconditioner through float inverses: a fixed linear operator, so the
// converged solution is unchanged while each apply becomes a memory-bound
// matrix-vector product. For a block whose double LU (P A = L U) is too
// large to invert with the one-CTA kernels, X = A^-1 = U^-1 L^-1 P is formed
// from a float copy of the factors by blocked triangular solves on the
// identity's columns: with tiles of kTs rows,
//   forward:  W_t = inv(L_tt) B_t,  B_u -= L_ut W_t  (u > t)
//   backward: X_t = inv(U_tt) W_t,  W_u -= U_ut X_t  (u < t)
// where the tile inverses come from small one-CTA kernels and the updates
// are float tiled GEMMs (128 x 128 output tile per CTA, 8 x 8 per thread).
#include <algorithm>
#include <cstdlib>

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kTs = 64;

// C = alpha A B + beta C for column-major float matrices. CTA: a 128 x 128
// tile of C, 256 threads, 8 x 8 outputs per thread (rows 4 tx .. 4 tx + 3 and
// 64 + 4 tx .., columns 4 ty .. and 64 + 4 ty ..), so each k step reads two
// float4 of A and two of B from shared memory for 64 FMAs. K advances by 8;
// the next step's tiles are loaded into registers while the current one is
// computed, then stored to the other shared-memory buffer (double
// buffering). kVec: leading dimensions multiples of 4 and 16-byte aligned
// bases, so interior tiles move as float4.
template <bool kVec>
__global__ void __launch_bounds__(256)
k_sgemm128(int64_t M, int64_t N, int K, float alpha, const float* __restrict__ A, int64_t lda,
           const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C, int64_t ldc) {
  count_launch();
  __shared__ __align__(16) float sA[2][8][128];  // [buffer][k][row]
  __shared__ __align__(16) float sB[2][8][128];  // [buffer][k][column]
  const int t = threadIdx.x;
  const int64_t r0 = blockIdx.x * (int64_t)128, c0 = blockIdx.y * (int64_t)128;
  const int la_k = t >> 5, la_r = (t & 31) * 4;  // A loader: one k, four rows
  const int lb_c = t >> 1, lb_k = (t & 1) * 4;   // B loader: one column, four k
  float4 ra, rb;
  auto load = [&](int k0) {
    const int64_t r = r0 + la_r;
    const int ka = k0 + la_k;
    if (kVec && ka < K && r + 3 < M) {
      ra = *reinterpret_cast<const float4*>(A + (int64_t)ka * lda + r);
    } else {
      const float* col = A + (int64_t)ka * lda;
      ra.x = (ka < K && r < M) ? col[r] : 0.f;
      ra.y = (ka < K && r + 1 < M) ? col[r + 1] : 0.f;
      ra.z = (ka < K && r + 2 < M) ? col[r + 2] : 0.f;
      ra.w = (ka < K && r + 3 < M) ? col[r + 3] : 0.f;
    }
    const int64_t c = c0 + lb_c;
    const int kb = k0 + lb_k;
    if (kVec && c < N && kb + 3 < K) {
      rb = *reinterpret_cast<const float4*>(B + c * ldb + kb);
    } else {
      const float* col = B + c * ldb;
      rb.x = (c < N && kb < K) ? col[kb] : 0.f;
      rb.y = (c < N && kb + 1 < K) ? col[kb + 1] : 0.f;
      rb.z = (c < N && kb + 2 < K) ? col[kb + 2] : 0.f;
      rb.w = (c < N && kb + 3 < K) ? col[kb + 3] : 0.f;
    }
  };
  auto store = [&](int buf) {
    *reinterpret_cast<float4*>(&sA[buf][la_k][la_r]) = ra;
    sB[buf][lb_k][lb_c] = rb.x;
    sB[buf][lb_k + 1][lb_c] = rb.y;
    sB[buf][lb_k + 2][lb_c] = rb.z;
    sB[buf][lb_k + 3][lb_c] = rb.w;
  };
  const int tx = t & 15, ty = t >> 4;
  float acc[8][8];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 8) {
    const bool more = k0 + 8 < K;
    if (more) load(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][kk][4 * tx]);
      const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][kk][64 + 4 * tx]);
      const float4 b0 = *reinterpret_cast<const float4*>(&sB[buf][kk][4 * ty]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sB[buf][kk][64 + 4 * ty]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t c = c0 + (q < 4 ? 4 * ty + q : 64 + 4 * ty + q - 4);
    if (c >= N) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = r0 + 64 * h + 4 * tx;
      float* cp = C + c * ldc + r;
      const float v[4] = {alpha * acc[4 * h][q], alpha * acc[4 * h + 1][q], alpha * acc[4 * h + 2][q],
                          alpha * acc[4 * h + 3][q]};
      if (kVec && r + 3 < M) {
        float4 o = make_float4(v[0], v[1], v[2], v[3]);
        if (beta != 0.f) {
          const float4 old = *reinterpret_cast<const float4*>(cp);
          o.x = fmaf(beta, old.x, o.x);
          o.y = fmaf(beta, old.y, o.y);
          o.z = fmaf(beta, old.z, o.z);
          o.w = fmaf(beta, old.w, o.w);
        }
        *reinterpret_cast<float4*>(cp) = o;
      } else {
        for (int i = 0; i < 4; ++i)
          if (r + i < M) cp[i] = beta == 0.f ? v[i] : fmaf(beta, cp[i], v[i]);
      }
    }
  }
}

// Inverse of each diagonal tile of L (unit lower) or U (upper), kTs x kTs,
// column-major into out[t * kTs * kTs]. One CTA per tile.
__global__ void __launch_bounds__(kTs)
k_tile_inverse(const float* __restrict__ A, int64_t m, int lower, float* __restrict__ out) {
  count_launch();
  const int64_t t = blockIdx.x;
  const int64_t r0 = t * kTs;
  const int n = (int)imin64(kTs, m - r0);
  __shared__ float sT[kTs][kTs + 1];  // [col][row]
  __shared__ float sX[kTs][kTs + 1];  // [col][row] of the inverse
  for (int e = threadIdx.x; e < kTs * kTs; e += blockDim.x) {
    const int c = e / kTs, r = e % kTs;
    sT[c][r] = (c < n && r < n) ? A[(r0 + c) * m + r0 + r] : (c == r ? 1.f : 0.f);
    sX[c][r] = c == r ? 1.f : 0.f;
  }
  __syncthreads();
  // thread q solves T x = e_q for column q of the inverse
  const int q = threadIdx.x;
  if (lower) {
    for (int c = 0; c < kTs; ++c) {
      const float xc = sX[q][c];
      for (int r = c + 1; r < kTs; ++r) sX[q][r] -= sT[c][r] * xc;
    }
  } else {
    for (int c = kTs - 1; c >= 0; --c) {
      const float xc = sX[q][c] / sT[c][c];
      sX[q][c] = xc;
      for (int r = 0; r < c; ++r) sX[q][r] -= sT[c][r] * xc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTs * kTs; e += blockDim.x) {
    const int c = e / kTs, r = e % kTs;
    out[t * kTs * kTs + (int64_t)c * kTs + r] = sX[c][r];
  }
}

// X = P I: row r holds 1 in column perm[r].
__global__ void k_perm_identity(const int* __restrict__ perm, int64_t m, float* __restrict__ X) {
  count_launch();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / m, r = e % m;
    X[e] = perm[r] == q ? 1.f : 0.f;
  }
}

__global__ void k_copy_rows(const float* __restrict__ src, int64_t lds, float* __restrict__ dst, int64_t ldd,
                            int rows, int64_t cols) {
  count_launch();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e % rows;
    dst[c * ldd + r] = src[c * lds + r];
  }
}

}  // namespace

void sgemm32(cudaStream_t s, int64_t M, int64_t N, int K, float alpha, const float* A, int64_t lda, const float* B,
             int64_t ldb, float beta, float* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + 127) / 128));
  const bool vec = ((lda | ldb | ldc) & 3) == 0 && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
                                                     reinterpret_cast<uintptr_t>(C)) & 15) == 0;
  if (vec)
    k_sgemm128<true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else
    k_sgemm128<false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  STOKES_LAUNCHED();
}

namespace {
using stokes::sgemm32;
}  // namespace

// X (m x m, column-major) = inverse of the block whose float factors are LU
// (unit-lower L below the diagonal, U on and above) with row permutation perm.
void invert_from_lu32(Geom& g, const float* LU, int64_t m, const int* perm, float* X) {
  cudaStream_t s = g.stream;
  const int64_t nt = (m + kTs - 1) / kTs;
  DevBuf<float> tinvL, tinvU, tmp;
  tinvL.alloc((size_t)nt * kTs * kTs);
  tinvU.alloc((size_t)nt * kTs * kTs);
  tmp.alloc((size_t)kTs * m);
  k_tile_inverse<<<(unsigned)nt, kTs, 0, s>>>(LU, m, 1, tinvL.get());
  k_tile_inverse<<<(unsigned)nt, kTs, 0, s>>>(LU, m, 0, tinvU.get());
  k_perm_identity<<<(unsigned)std::min<int64_t>((m * m + 255) / 256, 152 * 64), 256, 0, s>>>(perm, m, X);
  STOKES_LAUNCHED();
  // forward: rows of tile t of X become W_t = inv(L_tt) B_t; later rows -= L_ut W_t
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t r0 = t * kTs;
    const int n = (int)imin64(kTs, m - r0);
    sgemm32(s, n, m, n, 1.f, tinvL.get() + t * kTs * kTs, kTs, X + r0, m, 0.f, tmp.get(), kTs);
    k_copy_rows<<<(unsigned)std::min<int64_t>(((int64_t)n * m + 255) / 256, 152 * 16), 256, 0, s>>>(
        tmp.get(), kTs, X + r0, m, n, m);
    STOKES_LAUNCHED();
    const int64_t below = m - r0 - n;
    sgemm32(s, below, m, n, -1.f, LU + r0 * m + r0 + n, m, X + r0, m, 1.f, X + r0 + n, m);
  }
  // backward: X_t = inv(U_tt) W_t; earlier rows -= U_ut X_t
  for (int64_t t = nt - 1; t >= 0; --t) {
    const int64_t r0 = t * kTs;
    const int n = (int)imin64(kTs, m - r0);
    sgemm32(s, n, m, n, 1.f, tinvU.get() + t * kTs * kTs, kTs, X + r0, m, 0.f, tmp.get(), kTs);
    k_copy_rows<<<(unsigned)std::min<int64_t>(((int64_t)n * m + 255) / 256, 152 * 16), 256, 0, s>>>(
        tmp.get(), kTs, X + r0, m, n, m);
    STOKES_LAUNCHED();
    sgemm32(s, r0, m, n, -1.f, LU + r0 * m, m, X + r0, m, 1.f, X, m);
  }
  STOKES_CUDA(cudaStreamSynchronize(s));  // scratch buffers go out of scope
}

unsigned long long launches_bd_inv32() { return tu_launches(); }

}  // namespace stokes
