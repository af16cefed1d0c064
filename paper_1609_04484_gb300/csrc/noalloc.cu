// stokes_matvec_noalloc: y = A sigma (the FP64 double-layer operator) for
// callers that cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code running under an allocator that
// owns every byte of the device (a framework memory pool, an embedded
// runtime with a fixed arena), or on a real-time path where an
// allocation's implicit device synchronisation is not allowed. This variant
// of the operator does everything the normal one does (per-component
// moments, the tiled pair sum split over sources, the diagonal, jump,
// completion and wall terms) without a handle and without allocating: the
// arrays it needs besides the caller's inputs and outputs live in one
// file-scope device array, kScratchBytes long, that every GPU which loads the
// library keeps until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents. Every word a call reads is first written by the same call, so
// nothing is cleared; two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on it and give wrong results.
//
// Host code cannot use the array's name as a device address; the first call
// on each device looks the address up with cudaGetSymbolAddress while that
// device is current and keeps it for the life of the process (a
// cudaDeviceReset between calls is not supported). Make that first call
// before any stream capture.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "internal.cuh"

namespace {

constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr int kTile = 128;

static __device__ __align__(256) unsigned char g_matvec_scratch[kScratchBytes];

std::atomic<void*> g_scratch_addr[kMaxDevices] = {};

// Layout inside the scratch array (byte offsets, 256-aligned).
struct Layout {
  size_t off_offsets, off_centres, off_moments, off_part, total;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

Layout layout(int n_comp, int64_t N, int splits) {
  Layout L;
  L.off_offsets = 0;
  L.off_centres = align256(L.off_offsets + sizeof(int64_t) * (n_comp + 1));
  L.off_moments = align256(L.off_centres + sizeof(double2) * n_comp);
  L.off_part = align256(L.off_moments + 32 * (size_t)n_comp);
  L.total = L.off_part + sizeof(double2) * (size_t)splits * (size_t)N;
  return L;
}

__device__ int comp_of(const int64_t* off, int n_comp, int64_t i) {
  int lo = 0, hi = n_comp - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// lambda_k, xi_k (pores) and s0 (wall), one block per component.
__global__ void k_na_moments(const double2* __restrict__ pos, const double2* __restrict__ nrm,
                             const double* __restrict__ w, const double2* __restrict__ sig,
                             const int64_t* __restrict__ off, const double2* __restrict__ centre,
                             double4_32a* __restrict__ mom) {
  stokes::count_launch();
  __shared__ double red[4][256];
  const int k = blockIdx.x;
  const double2 c = centre[k];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int64_t j = off[k] + threadIdx.x; j < off[k + 1]; j += blockDim.x) {
    const double sx = w[j] * sig[j].x, sy = w[j] * sig[j].y;
    const double dx = pos[j].x - c.x, dy = pos[j].y - c.y;
    a0 += sx;
    a1 += sy;
    a2 += dy * sx - dx * sy;
    a3 += nrm[j].x * sx + nrm[j].y * sy;
  }
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = a1;
  red[2][threadIdx.x] = a2;
  red[3][threadIdx.x] = a3;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) mom[k] = make_double4_32a(red[0][0], red[1][0], red[2][0], red[3][0]);
}

// Pair sums over the source range of blockIdx.y, reading the caller's arrays.
__global__ void __launch_bounds__(kTile)
k_na_pairs(int64_t N, const double2* __restrict__ pos, const double2* __restrict__ nrm, const double* __restrict__ w,
           const double2* __restrict__ sig, int64_t chunk, double2* __restrict__ part) {
  stokes::count_launch();
  __shared__ double4_32a s_src[kTile];
  __shared__ double2 s_sig[kTile];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double2 x = i < N ? pos[i] : make_double2(0.0, 0.0);
  const int64_t j0 = blockIdx.y * chunk, j1 = stokes::imin64(N, j0 + chunk);
  double ux = 0.0, uy = 0.0;
  for (int64_t t0 = j0; t0 < j1; t0 += kTile) {
    __syncthreads();
    const int64_t j = t0 + threadIdx.x;
    if (j < j1) {
      const double a = w[j] * stokes::kInvPi;
      s_src[threadIdx.x] = make_double4_32a(pos[j].x, pos[j].y, a * nrm[j].x, a * nrm[j].y);
      s_sig[threadIdx.x] = sig[j];
    } else {
      s_src[threadIdx.x] = make_double4_32a(1e30, 1e30, 0.0, 0.0);
      s_sig[threadIdx.x] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int q = 0; q < kTile; ++q) {
      const double4_32a s = s_src[q];
      const double rx = x.x - s.x, ry = x.y - s.y;
      double r2 = fma(rx, rx, ry * ry);
      r2 = (t0 + q == i) ? 1.0 : r2;  // the node itself: r = 0, contributes 0
      const double inv = 1.0 / r2;
      const double d = fma(rx, s.z, ry * s.w);
      const double e = fma(rx, s_sig[q].x, ry * s_sig[q].y);
      const double c = (d * inv) * (e * inv);
      ux = fma(c, rx, ux);
      uy = fma(c, ry, uy);
    }
  }
  if (i < N) part[blockIdx.y * N + i] = make_double2(ux, uy);
}

__global__ void k_na_epilogue(int64_t N, int splits, const double2* __restrict__ pos, const double2* __restrict__ nrm,
                              const double* __restrict__ w, const double* __restrict__ kappa,
                              const double2* __restrict__ sig, const int64_t* __restrict__ off, int n_comp, int outer,
                              const double2* __restrict__ centre, const double4_32a* __restrict__ mom,
                              const double2* __restrict__ part, double2* __restrict__ y) {
  stokes::count_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ax = 0.0, ay = 0.0;
  for (int s = 0; s < splits; ++s) {
    ax += part[s * N + i].x;
    ay += part[s * N + i].y;
  }
  const double2 x = pos[i], n = nrm[i], sg = sig[i];
  const double tx = -n.y, ty = n.x;
  const double sc = -kappa[i] * w[i] / (2.0 * stokes::kPi);
  const double ts = tx * sg.x + ty * sg.y;
  ax += sc * ts * tx - 0.5 * sg.x;
  ay += sc * ts * ty - 0.5 * sg.y;
  if (comp_of(off, n_comp, i) == outer) {
    const double s0 = mom[outer].w;
    ax += n.x * s0;
    ay += n.y * s0;
  }
  double cx = 0.0, cy = 0.0;
  for (int k = 0; k < n_comp; ++k) {
    if (k == outer) continue;
    const double2 c = centre[k];
    const double4_32a m = mom[k];
    const double rx = x.x - c.x, ry = x.y - c.y;
    const double r2 = rx * rx + ry * ry;
    const double inv = 1.0 / r2;
    const double lg = -0.5 * log(r2);
    const double rl = (rx * m.x + ry * m.y) * inv;
    cx += lg * m.x + rl * rx + m.z * inv * ry;
    cy += lg * m.y + rl * ry - m.z * inv * rx;
  }
  y[i] = make_double2(ax + stokes::kInv4Pi * cx, ay + stokes::kInv4Pi * cy);
}

// Device memory (or managed) of the current device only: the kernels
// dereference the pointers, and another GPU's memory is not reachable
// without peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

int stokes_matvec_noalloc(const double* nodes, const double* normals, const double* weights, const double* curvature,
                          const int64_t* offsets, int n_comp, int outer_comp, const double* centres,
                          const double* sigma, double* y, void* stream) {
  if (!nodes || !normals || !weights || !curvature || !offsets || !centres || !sigma || !y) return STOKES_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return STOKES_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return STOKES_EINVAL;
  if (!on_device(nodes, dev) || !on_device(normals, dev) || !on_device(weights, dev) ||
      !on_device(curvature, dev) || !on_device(sigma, dev) || !on_device(y, dev))
    return STOKES_EINVAL;
  if (n_comp < 1 || outer_comp < 0 || outer_comp >= n_comp) return STOKES_EINVAL;
  if (offsets[0] != 0) return STOKES_EINVAL;
  for (int c = 0; c < n_comp; ++c)
    if (offsets[c + 1] - offsets[c] < 8) return STOKES_EINVAL;
  const int64_t N = offsets[n_comp];
  // split the sources so the grid holds about four CTAs per SM (152 SMs);
  // from 77,824 nodes on one split already fills the GPU
  const int64_t tblocks = (N + kTile - 1) / kTile;
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + tblocks - 1) / tblocks, tblocks));
  const int64_t chunk = ((N + want - 1) / want + kTile - 1) / kTile * kTile;
  const int64_t splits = (N + chunk - 1) / chunk;
  const Layout L = layout(n_comp, N, (int)splits);
  if (L.total > kScratchBytes) return STOKES_EINVAL;  // beyond the fixed scratch array
  void* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    e = cudaGetSymbolAddress(&addr, g_matvec_scratch);
    if (e != cudaSuccess) return STOKES_ECUDA;
    g_scratch_addr[dev].store(addr, std::memory_order_release);  // concurrent first calls store the same value
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  auto* d_off = reinterpret_cast<int64_t*>(base + L.off_offsets);
  auto* d_cen = reinterpret_cast<double2*>(base + L.off_centres);
  auto* d_mom = reinterpret_cast<double4_32a*>(base + L.off_moments);
  auto* d_part = reinterpret_cast<double2*>(base + L.off_part);
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * (n_comp + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cen, centres, sizeof(double2) * n_comp, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return STOKES_ECUDA;
  const auto* pos = reinterpret_cast<const double2*>(nodes);
  const auto* nrm = reinterpret_cast<const double2*>(normals);
  const auto* sg = reinterpret_cast<const double2*>(sigma);
  k_na_moments<<<n_comp, 256, 0, s>>>(pos, nrm, weights, sg, d_off, d_cen, d_mom);
  k_na_pairs<<<dim3((unsigned)tblocks, (unsigned)splits), kTile, 0, s>>>(N, pos, nrm, weights, sg, chunk, d_part);
  k_na_epilogue<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, (int)splits, pos, nrm, weights, curvature, sg, d_off,
                                                            n_comp, outer_comp, d_cen, d_mom, d_part,
                                                            reinterpret_cast<double2*>(y));
  return cudaGetLastError() == cudaSuccess ? STOKES_OK : STOKES_ECUDA;
}

}  // extern "C"

namespace stokes {
unsigned long long launches_noalloc() { return tu_launches(); }
}  // namespace stokes
