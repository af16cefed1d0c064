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

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kTs = 64;

// C = alpha A B + beta C (column-major, M x N = (M x K)(K x N)): 128 x 128
// output tile per CTA, 8 x 8 per thread, operands staged 16 deep.
__global__ void __launch_bounds__(256)
k_sgemm(int64_t M, int64_t N, int K, float alpha, const float* __restrict__ A, int64_t lda,
        const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C, int64_t ldc) {
  count_launch();
  constexpr int kK = 16, kT = 128;
  __shared__ float sA[kK][kT + 4];  // [k][row]
  __shared__ float sB[kK][kT + 4];  // [k][col]
  const int64_t r0 = blockIdx.x * (int64_t)kT, c0 = blockIdx.y * (int64_t)kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8] = {};
  for (int k0 = 0; k0 < K; k0 += kK) {
    __syncthreads();
    for (int e = threadIdx.x; e < kK * kT; e += 256) {
      const int kk = e / kT, rr = e % kT;
      const int64_t r = r0 + rr;
      sA[kk][rr] = (k0 + kk < K && r < M) ? A[(int64_t)(k0 + kk) * lda + r] : 0.f;
    }
    for (int e = threadIdx.x; e < kK * kT; e += 256) {
      const int cc = e / kK, kk = e % kK;
      const int64_t c = c0 + cc;
      sB[kk][cc] = (k0 + kk < K && c < N) ? B[c * ldb + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a[q] = sA[kk][tx + 16 * q];
        b[q] = sB[kk][ty + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t c = c0 + ty + 16 * q;
    if (c >= N) continue;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int64_t r = r0 + tx + 16 * p;
      if (r < M) {
        float* cp = C + c * ldc + r;
        *cp = beta == 0.f ? alpha * acc[p][q] : fmaf(alpha, acc[p][q], beta * *cp);
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

void sgemm(cudaStream_t s, int64_t M, int64_t N, int K, float alpha, const float* A, int64_t lda, const float* B,
           int64_t ldb, float beta, float* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + 127) / 128));
  k_sgemm<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  STOKES_LAUNCHED();
}

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
    sgemm(s, n, m, n, 1.f, tinvL.get() + t * kTs * kTs, kTs, X + r0, m, 0.f, tmp.get(), kTs);
    k_copy_rows<<<(unsigned)std::min<int64_t>(((int64_t)n * m + 255) / 256, 152 * 16), 256, 0, s>>>(
        tmp.get(), kTs, X + r0, m, n, m);
    STOKES_LAUNCHED();
    const int64_t below = m - r0 - n;
    sgemm(s, below, m, n, -1.f, LU + r0 * m + r0 + n, m, X + r0, m, 1.f, X + r0 + n, m);
  }
  // backward: X_t = inv(U_tt) W_t; earlier rows -= U_ut X_t
  for (int64_t t = nt - 1; t >= 0; --t) {
    const int64_t r0 = t * kTs;
    const int n = (int)imin64(kTs, m - r0);
    sgemm(s, n, m, n, 1.f, tinvU.get() + t * kTs * kTs, kTs, X + r0, m, 0.f, tmp.get(), kTs);
    k_copy_rows<<<(unsigned)std::min<int64_t>(((int64_t)n * m + 255) / 256, 152 * 16), 256, 0, s>>>(
        tmp.get(), kTs, X + r0, m, n, m);
    STOKES_LAUNCHED();
    sgemm(s, r0, m, n, -1.f, LU + r0 * m, m, X + r0, m, 1.f, X, m);
  }
  STOKES_CUDA(cudaStreamSynchronize(s));  // scratch buffers go out of scope
}

unsigned long long launches_bd_inv32() { return tu_launches(); }

}  // namespace stokes
