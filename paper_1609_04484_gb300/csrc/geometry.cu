// Geometry handle: validation, device copies of the node data and the
// per-component moments of a density (the completion's lambda_k, xi_k and the
// wall term's s0).
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace stokes {

namespace {

// Block-wide sum of four doubles in a fixed order (deterministic).
__device__ double4_32a block_sum4(double4_32a v) {
  __shared__ double4_32a sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    v.z += __shfl_down_sync(0xffffffffu, v.z, o);
    v.w += __shfl_down_sync(0xffffffffu, v.w, o);
  }
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (wid == 0) {
    v = lane < nw ? sh[lane] : make_double4_32a(0, 0, 0, 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
      v.z += __shfl_down_sync(0xffffffffu, v.z, o);
      v.w += __shfl_down_sync(0xffffffffu, v.w, o);
    }
  }
  return v;
}

// One block per component: lambda = sum w sigma, xi = sum w (x - c)^perp . sigma,
// s0 = sum w n . sigma.
__global__ void k_moments_f64(const double2* __restrict__ pos, const double2* __restrict__ nrm,
                              const double* __restrict__ w, const int64_t* __restrict__ off,
                              const double2* __restrict__ centre, const double2* __restrict__ sig,
                              double4_32a* __restrict__ mom, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int k = blockIdx.x;
  const int64_t a = off[k], b = off[k + 1];
  const double2 c = centre[k];
  double4_32a acc = make_double4_32a(0, 0, 0, 0);
  for (int64_t j = a + threadIdx.x; j < b; j += blockDim.x) {
    const double wj = w[j];
    const double2 s = sig[j];
    const double2 p = pos[j];
    const double2 n = nrm[j];
    const double sx = wj * s.x, sy = wj * s.y;
    const double dx = p.x - c.x, dy = p.y - c.y;
    acc.x += sx;
    acc.y += sy;
    acc.z += dy * sx - dx * sy;
    acc.w += n.x * sx + n.y * sy;
  }
  acc = block_sum4(acc);
  if (threadIdx.x == 0) mom[k] = acc;
}

__device__ __forceinline__ float2 split_f(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// v = grid + rem: grid is v rounded to a multiple of 2^-8 (exact in float
// for |v| < 2^15, and so are differences of grid values); |rem| <= 2^-9.
__device__ __forceinline__ double grid_part(double v) { return rint(v * 256.0) * (1.0 / 256.0); }

__global__ void k_prep_nodes(int64_t N, const double2* __restrict__ pos, const double2* __restrict__ nrm,
                             const double* __restrict__ w, const double* __restrict__ kappa,
                             double4_32a* __restrict__ src, double4_32a* __restrict__ selfc,
                             float4* __restrict__ f32_src, float2* __restrict__ f32_lo,
                             float2* __restrict__ df_grid, float4* __restrict__ df_pos, float4* __restrict__ df_a) {
  count_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double2 p = pos[i], n = nrm[i];
  const double wi = w[i];
  const double ax = wi * n.x * kInvPi, ay = wi * n.y * kInvPi;
  src[i] = make_double4_32a(p.x, p.y, ax, ay);
  selfc[i] = make_double4_32a(-n.y, n.x, -kappa[i] * wi / (2.0 * kPi), wi);
  const float2 sx = split_f(p.x), sy = split_f(p.y), sax = split_f(ax), say = split_f(ay);
  f32_src[i] = make_float4(sx.x, sy.x, sax.x, say.x);
  f32_lo[i] = make_float2(sx.y, sy.y);
  const double gx = grid_part(p.x), gy = grid_part(p.y);
  const float2 rx = split_f(p.x - gx), ry = split_f(p.y - gy);
  df_grid[i] = make_float2((float)gx, (float)gy);
  df_pos[i] = make_float4(rx.x, ry.x, rx.y, ry.y);
  df_a[i] = make_float4(sax.x, say.x, sax.y, say.y);
}

}  // namespace

void moments_f64(Geom& g, const double2* sigma, const int* done, double4_32a* out) {
  k_moments_f64<<<g.n_comp, 256, 0, g.stream>>>(g.pos.get(), g.nrm.get(), g.w.get(), g.d_off.get(),
                                                g.centre.get(), sigma, out ? out : g.mom.get(), done);
  STOKES_LAUNCHED();
}

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from a host-or-device pointer into device memory `dst`.
void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  STOKES_CUDA(cudaMemcpyAsync(dst, src, bytes,
                              is_device_pointer(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

Geom* geometry_create(const double* nodes, const double* normals, const double* weights,
                      const double* curvature, const int64_t* offsets, int n_comp, int outer_comp,
                      const double* centres, void* stream) {
  require(nodes && normals && weights && curvature && offsets, "null array argument");
  require(n_comp >= 1, "n_comp must be >= 1");
  require(outer_comp >= 0 && outer_comp < n_comp, "outer_comp out of range");
  require(!is_device_pointer(offsets), "offsets must be a host pointer");
  require(offsets[0] == 0, "offsets[0] must be 0");
  for (int c = 0; c < n_comp; ++c)
    require(offsets[c + 1] - offsets[c] >= 8, "each component needs at least 8 nodes");
  const int64_t N = offsets[n_comp];
  require(N <= (int64_t)1 << 28, "too many nodes");


  Geom* g = new Geom();
  try {
    g->N = N;
    g->n_comp = n_comp;
    g->outer = outer_comp;
    g->M = n_comp - 1;
    g->stream = (cudaStream_t)stream;
    g->off.assign(offsets, offsets + n_comp + 1);
    cudaStream_t s = g->stream;

    // host copies for validation and centroids
    std::vector<double> hx(2 * N), hn(2 * N), hw(N), hk(N);
    auto fetch = [&](void* dst, const void* src, size_t bytes) {
      STOKES_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    };
    fetch(hx.data(), nodes, 16 * N);
    fetch(hn.data(), normals, 16 * N);
    fetch(hw.data(), weights, 8 * N);
    fetch(hk.data(), curvature, 8 * N);
    STOKES_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < N; ++i) {
      require(std::isfinite(hx[2 * i]) && std::isfinite(hx[2 * i + 1]), "non-finite node");
      require(std::fabs(hx[2 * i]) < 16384.0 && std::fabs(hx[2 * i + 1]) < 16384.0,
              "node coordinates must be below 2^14 in magnitude");
      require(std::isfinite(hw[i]) && hw[i] > 0, "weights must be finite and > 0");
      require(std::isfinite(hk[i]), "non-finite curvature");
      const double nn = std::hypot(hn[2 * i], hn[2 * i + 1]);
      require(std::fabs(nn - 1.0) <= 1e-6, "normals must be unit vectors");
    }
    g->centre_h.assign(2 * n_comp, 0.0);
    for (int c = 0; c < n_comp; ++c) {
      if (centres && c != outer_comp) {
        g->centre_h[2 * c] = centres[2 * c];
        g->centre_h[2 * c + 1] = centres[2 * c + 1];
        require(std::isfinite(centres[2 * c]) && std::isfinite(centres[2 * c + 1]), "non-finite centre");
      } else {
        double sw = 0, sx = 0, sy = 0;
        for (int64_t j = offsets[c]; j < offsets[c + 1]; ++j) {
          sw += hw[j];
          sx += hw[j] * hx[2 * j];
          sy += hw[j] * hx[2 * j + 1];
        }
        g->centre_h[2 * c] = sx / sw;
        g->centre_h[2 * c + 1] = sy / sw;
      }
    }
    std::vector<int> hcomp(N);
    for (int c = 0; c < n_comp; ++c)
      for (int64_t j = offsets[c]; j < offsets[c + 1]; ++j) hcomp[j] = c;
    std::vector<int> pores;
    for (int c = 0; c < n_comp; ++c)
      if (c != outer_comp) pores.push_back(c);

    g->pos.alloc(N);
    g->nrm.alloc(N);
    g->w.alloc(N);
    DevBuf<double> kap;
    kap.alloc(N);
    g->src.alloc(N);
    g->selfc.alloc(N);
    g->f32_src.alloc(N);
    g->f32_lo.alloc(N);
    g->df_grid.alloc(N);
    g->df_pos.alloc(N);
    g->df_a.alloc(N);
    g->comp.alloc(N);
    g->d_off.alloc(n_comp + 1);
    g->centre.alloc(n_comp);
    g->pore_ids.alloc(pores.size() ? pores.size() : 1);
    g->mom.alloc(n_comp);
    STOKES_CUDA(cudaMemcpyAsync(g->pos.get(), hx.data(), 16 * N, cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(g->nrm.get(), hn.data(), 16 * N, cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(g->w.get(), hw.data(), 8 * N, cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(kap.get(), hk.data(), 8 * N, cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(g->comp.get(), hcomp.data(), 4 * N, cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(g->d_off.get(), offsets, 8 * (n_comp + 1), cudaMemcpyHostToDevice, s));
    STOKES_CUDA(cudaMemcpyAsync(g->centre.get(), g->centre_h.data(), 16 * n_comp, cudaMemcpyHostToDevice, s));
    if (!pores.empty())
      STOKES_CUDA(cudaMemcpyAsync(g->pore_ids.get(), pores.data(), 4 * pores.size(), cudaMemcpyHostToDevice, s));
    const int tb = 256;
    k_prep_nodes<<<(unsigned)((N + tb - 1) / tb), tb, 0, s>>>(N, g->pos.get(), g->nrm.get(), g->w.get(),
                                                             kap.get(), g->src.get(), g->selfc.get(),
                                                             g->f32_src.get(), g->f32_lo.get(), g->df_grid.get(),
                                                             g->df_pos.get(), g->df_a.get());
    STOKES_LAUNCHED();
    STOKES_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  } catch (...) {
    delete g;
    throw;
  }
  return g;
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_geometry() { return tu_launches(); }
}  // namespace stokes
