// Triangular solves with the LU factors of the largest preconditioner
// blocks (too large to invert explicitly), one persistent kernel per solve.
//
// z = U^-1 L^-1 P v for a column-major m x m block. The grid is one CTA per
// SM, launched cooperatively so all CTAs are resident; rows are cut into
// tiles of kTs and tile u belongs to CTA u mod gridDim.x. Forward sweep,
// phase t: every CTA subtracts L[u, t] z_t from each of its tiles u > t; the
// owner of tile t + 1 updates that tile first and then solves its unit
// lower diagonal block in shared memory; a grid barrier ends the phase.
// The backward sweep mirrors it from the last tile with U's diagonal.
//
// The grid barrier (grid_sync.cuh) spins with an iteration limit: on
// timeout it raises an error flag, every CTA leaves at the next check, and
// the host reports the failure instead of hanging.
#include <algorithm>

#include "grid_sync.cuh"

namespace stokes {

namespace {

constexpr int kTs = 64;
constexpr int kThreads = 256;
using gsync::Barrier;
using gsync::grid_sync;

template <class T>
__global__ void __launch_bounds__(kThreads)
k_lu_solve_persistent(const T* __restrict__ A, int64_t m, const int* __restrict__ perm,
                      const double* __restrict__ v, T* __restrict__ z, double* __restrict__ out, Barrier bar,
                      const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ T sT[kTs][kTs + 1];  // a diagonal tile, [col][row]
  __shared__ T sz[kTs];
  __shared__ T red[4][kTs];
  const int64_t nt = (m + kTs - 1) / kTs;
  const int G = gridDim.x;
  unsigned epoch = 0;
  // z = P v
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)G * blockDim.x)
    z[r] = (T)v[perm[r]];
  if (!grid_sync(bar, epoch)) return;

  // Solve the diagonal tile u in place (lower: unit; upper: divide by the diagonal).
  auto solve_tile = [&](int64_t u, bool lower) {
    const int64_t r0 = u * kTs;
    const int nt_u = (int)imin64(kTs, m - r0);
    for (int e = threadIdx.x; e < nt_u * nt_u; e += blockDim.x) {
      const int c = e / nt_u, r = e % nt_u;
      sT[c][r] = A[(r0 + c) * m + r0 + r];
    }
    if (threadIdx.x < nt_u) sz[threadIdx.x] = z[r0 + threadIdx.x];
    __syncthreads();
    const int r = threadIdx.x;
    if (lower) {
      for (int c = 0; c < nt_u; ++c) {
        if (r > c && r < nt_u) sz[r] -= sT[c][r] * sz[c];
        __syncthreads();
      }
    } else {
      for (int c = nt_u - 1; c >= 0; --c) {
        if (r == c) sz[c] /= sT[c][c];
        __syncthreads();
        if (r < c) sz[r] -= sT[c][r] * sz[c];
        __syncthreads();
      }
    }
    if (r < nt_u) z[r0 + r] = sz[r];
    __syncthreads();
  };

  // z_u -= A[u rows, t cols] z_t for one tile u (rows of u, columns of t).
  auto update_tile = [&](int64_t u, int64_t t) {
    const int64_t r0 = u * kTs, c0 = t * kTs;
    const int nr = (int)imin64(kTs, m - r0), nc = (int)imin64(kTs, m - c0);
    if (threadIdx.x < nc) sz[threadIdx.x] = z[c0 + threadIdx.x];
    __syncthreads();
    // 256 threads: 64 rows x 4 column phases
    const int rr = threadIdx.x & (kTs - 1), ph = threadIdx.x / kTs;
    T acc = 0;
    if (rr < nr)
      for (int c = ph; c < nc; c += 4) acc += A[(c0 + c) * m + r0 + rr] * sz[c];
    red[ph][rr] = acc;
    __syncthreads();
    if (ph == 0 && rr < nr) z[r0 + rr] -= (red[0][rr] + red[1][rr]) + (red[2][rr] + red[3][rr]);
    __syncthreads();
  };

  // forward sweep (unit lower L)
  if (blockIdx.x == 0) solve_tile(0, true);
  if (!grid_sync(bar, epoch)) return;
  for (int64_t t = 0; t + 1 < nt; ++t) {
    const int64_t first = t + 1;
    // this CTA's tiles u > t: u = first + ((blockIdx.x - first) mod G) + k G
    int64_t u0 = first + (((int64_t)blockIdx.x - first) % G + G) % G;
    for (int64_t u = u0; u < nt; u += G) {
      update_tile(u, t);
      if (u == first) solve_tile(u, true);
    }
    if (!grid_sync(bar, epoch)) return;
  }
  // backward sweep (upper U)
  if ((nt - 1) % G == blockIdx.x) solve_tile(nt - 1, false);
  if (!grid_sync(bar, epoch)) return;
  for (int64_t t = nt - 1; t > 0; --t) {
    const int64_t first = t - 1;
    // this CTA's tiles u < t, the one nearest the diagonal first
    int64_t u0 = first - ((first - (int64_t)blockIdx.x) % G + G) % G;
    for (int64_t u = u0; u >= 0; u -= G) {
      update_tile(u, t);
      if (u == first) solve_tile(u, false);
    }
    if (!grid_sync(bar, epoch)) return;
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)G * blockDim.x)
    out[r] = (double)z[r];
}

}  // namespace

// z (2N doubles, block rows [o, o + m)) = factors^-1 v for one block.
// T = double uses the FP64 factors, T = float a float copy of them.
template <class T>
void lu_solve_persistent(Geom& g, const T* A, int64_t m, const int* perm, const double* v, double* z, T* work,
                         const int* done) {
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, nsm = 0, per_sm = 0;
    STOKES_CUDA(cudaGetDevice(&dev));
    STOKES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_solve_persistent<T>, kThreads, 0));
    require(per_sm >= 1, "persistent triangular solve does not fit on an SM", STOKES_ECUDA);
    grid = nsm;  // one CTA per SM: all resident
  }
  BlockDiag& b = g.bd;
  if (!b.barrier.get()) {
    b.barrier.alloc(4);
    STOKES_CUDA(cudaMemsetAsync(b.barrier.get(), 0, 4 * sizeof(unsigned), g.stream));
  }
  // count and generation restart at zero; the error word (slot 2) is sticky
  STOKES_CUDA(cudaMemsetAsync(b.barrier.get(), 0, 2 * sizeof(unsigned), g.stream));
  Barrier bar{b.barrier.get(), b.barrier.get() + 1, (int*)(b.barrier.get() + 2), gsync::spin_limit()};
  void* args[] = {(void*)&A, (void*)&m, (void*)&perm, (void*)&v, (void*)&work, (void*)&z, (void*)&bar,
                  (void*)&done};
  STOKES_CUDA(cudaLaunchCooperativeKernel((const void*)k_lu_solve_persistent<T>, dim3(grid), dim3(kThreads), args,
                                          0, g.stream));
}

// Throws if a persistent solve's grid barrier ever timed out (synchronises).
void bd_check_barrier(Geom& g) {
  if (!g.bd.barrier.get()) return;
  unsigned err = 0;
  STOKES_CUDA(cudaMemcpyAsync(&err, g.bd.barrier.get() + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, g.stream));
  STOKES_CUDA(cudaStreamSynchronize(g.stream));
  require(err == 0, "block-diagonal triangular solve: grid barrier timed out", STOKES_ECUDA);
}

template void lu_solve_persistent<double>(Geom&, const double*, int64_t, const int*, const double*, double*,
                                          double*, const int*);
template void lu_solve_persistent<float>(Geom&, const float*, int64_t, const int*, const double*, double*, float*,
                                         const int*);

unsigned long long launches_bd_trsv() { return tu_launches(); }

}  // namespace stokes
