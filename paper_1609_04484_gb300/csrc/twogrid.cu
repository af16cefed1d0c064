// Two-grid preconditioner (not in the paper: a GPU-native alternative to its
// block-diagonal baseline).
//
//   P^-1 r = I Ac^-1 R r + B^-1 (r - I R r)
//
// Ac is the same completed double-layer operator on the coarse grid made of
// every q-th node of every component (weights times q: the trapezoid rule
// on the q-times coarser equispaced parameter grid), assembled densely and
// LU-factorised with partial pivoting in single precision. I interpolates
// each component's coarse samples trigonometrically (the real interpolant,
// Nyquist cosine split evenly), R = (n_c / n_f) I^T. B^-1 is the pores'
// diagonal blocks; on the wall the remainder is multiplied by -2, the inverse
// of the -1/2 jump (the wall block is not needed next to the coarse solve).
// The coarse solve rounds its input to float, so the solver runs flexible
// GMRES, which tolerates a preconditioner that is not exactly linear.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <ctime>
#include <map>
#include <string>

#include "grid_sync.cuh"

namespace stokes {

void bd_setup_pores(Geom& g, bool skip_wall);
void bd_apply_pores_accumulate(Geom& g, const double* h, double* z, const int* done, bool f32);

namespace {

constexpr int kNb = 64;      // panel width of the coarse LU (CUDA-core trailing updates)
constexpr int kNbTc = 128;   // panel width with tensor-core trailing updates (half the trailing traffic)
constexpr int kNbMax = 128;
constexpr int kChunk = 32;       // panel columns a thread moves per pass in the panel kernel
constexpr int kRedPerLane = 8;   // pivot candidates a lane loads per pass (covers 256 CTAs)
constexpr int kSubR = 3;         // row slots per thread of the shared-memory panel kernel (64 KB each)
constexpr int64_t kMaxExplicitCoarse = 40960;  // coarse unknowns up to which the inverse is formed

__global__ void k_coarse_gather(int64_t Nc, int q, const int64_t* __restrict__ off, const int64_t* __restrict__ off_c,
                                int n_comp, const double2* __restrict__ pos, const double2* __restrict__ nrm,
                                const double* __restrict__ w, const double4_32a* __restrict__ selfc,
                                double2* __restrict__ pos_c, double2* __restrict__ nrm_c, double* __restrict__ w_c,
                                double4_32a* __restrict__ selfc_c, int* __restrict__ comp_c) {
  count_launch();
  const int64_t ic = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ic >= Nc) return;
  int lo = 0, hi = n_comp - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off_c[mid] <= ic) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  const int64_t i = off[k] + (int64_t)q * (ic - off_c[k]);
  pos_c[ic] = pos[i];
  nrm_c[ic] = nrm[i];
  w_c[ic] = q * w[i];
  const double4_32a sc = selfc[i];
  selfc_c[ic] = make_double4_32a(sc.x, sc.y, q * sc.z, q * sc.w);
  comp_c[ic] = k;
}

// Float copies of the coarse nodes for the assembly (conversions from
// double run at the FP64 rate, so they are done once per node here):
// p = (x_hi, y_hi, x_lo, y_lo), q = (n_x, n_y, w, comp), d = diagonal block.
__global__ void k_coarse_floats(int64_t Nc, const double2* __restrict__ pos, const double2* __restrict__ nrm,
                                const double* __restrict__ w, const double4_32a* __restrict__ selfc,
                                const int* __restrict__ comp, float4* __restrict__ p, float4* __restrict__ qv,
                                float4* __restrict__ d) {
  count_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Nc) return;
  const double2 x = pos[i];
  const float xh = (float)x.x, yh = (float)x.y;
  p[i] = make_float4(xh, yh, (float)(x.x - (double)xh), (float)(x.y - (double)yh));
  const double2 n = nrm[i];
  qv[i] = make_float4((float)n.x, (float)n.y, (float)w[i], __int_as_float(comp[i]));
  const double4_32a sc = selfc[i];
  d[i] = make_float4((float)(sc.z * sc.x * sc.x - 0.5), (float)(sc.z * sc.x * sc.y), (float)(sc.z * sc.y * sc.y - 0.5),
                     0.f);
}

// Completion centres of all components split into float hi + lo.
__global__ void k_centre_floats(int n_comp, const double2* __restrict__ centre, float4* __restrict__ c) {
  count_launch();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_comp) return;
  const double2 v = centre[k];
  const float hx = (float)v.x, hy = (float)v.y;
  c[k] = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

// Dense coarse operator (column-major, leading dimension 2 Nc), one thread
// per (row node i, column node j) writing the 2 x 2 block A_ij. The result
// is stored and factorised in float, so it is evaluated in float too, with
// differences of positions formed from float hi + lo parts (accurate to
// float precision relative to the distance).
__global__ void __launch_bounds__(256)
k_coarse_assemble(int64_t Nc, const float4* __restrict__ P, const float4* __restrict__ Q,
                  const float4* __restrict__ D, const float4* __restrict__ C, int outer, float* __restrict__ A) {
  count_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Nc) return;
  const int64_t ld = 2 * Nc;
  const float4 pi = P[i];
  const float4 qi = Q[i];
  const int ci = __float_as_int(qi.w);
  const float k4 = (float)kInv4Pi, kp = (float)kInvPi;
  for (int64_t j = blockIdx.y; j < Nc; j += gridDim.y) {
    const float4 pj = P[j];
    const float4 qj = Q[j];
    const int cj = __float_as_int(qj.w);
    const float wj = qj.z;
    float b00, b01, b10, b11;
    if (i == j) {
      const float4 d = D[i];
      b00 = d.x;
      b01 = d.y;
      b10 = d.y;
      b11 = d.z;
    } else {
      const float rx = (pi.x - pj.x) + (pi.z - pj.z), ry = (pi.y - pj.y) + (pi.w - pj.w);
      const float r2 = fmaf(rx, rx, ry * ry);
      const float inv = __frcp_rn(r2);
      const float c = wj * kp * fmaf(rx, qj.x, ry * qj.y) * inv * inv;
      b00 = c * rx * rx;
      b01 = c * rx * ry;
      b10 = b01;
      b11 = c * ry * ry;
    }
    if (cj != outer) {
      const float4 cc = C[cj];
      const float rx = (pi.x - cc.x) + (pi.z - cc.z), ry = (pi.y - cc.y) + (pi.w - cc.w);
      const float r2 = fmaf(rx, rx, ry * ry);
      const float inv = __frcp_rn(r2);
      const float lg = -0.5f * __logf(r2);
      const float px = ((pj.y - cc.y) + (pj.w - cc.w)) * wj, py = -((pj.x - cc.x) + (pj.z - cc.z)) * wj;
      const float ra = ry * inv, rb = -rx * inv;
      b00 += k4 * (wj * (lg + rx * rx * inv) + ra * px);
      b01 += k4 * (wj * (rx * ry * inv) + ra * py);
      b10 += k4 * (wj * (rx * ry * inv) + rb * px);
      b11 += k4 * (wj * (lg + ry * ry * inv) + rb * py);
    } else if (ci == outer) {
      b00 += qi.x * wj * qj.x;
      b01 += qi.x * wj * qj.y;
      b10 += qi.y * wj * qj.x;
      b11 += qi.y * wj * qj.y;
    }
    float* col0 = A + (2 * j) * ld + 2 * i;
    float* col1 = col0 + ld;
    col0[0] = b00;
    col0[1] = b10;
    col1[0] = b01;
    col1[1] = b11;
  }
}

// y = X x for a dense column-major float m x m matrix, in two passes.
// Pass 1: CTA (b, c) covers rows [1024 b, 1024 b + 1024) (four consecutive
// rows per thread, one float4 per column: each warp reads 512 contiguous
// bytes of a column) and the column range [c w, c w + w); its partial sums go
// to part[c][rows]. A grid of (m / 1024) x kGemvSplits CTAs keeps several
// CTAs per SM streaming the matrix. Pass 2 adds the kGemvSplits partials in a
// fixed order (deterministic) and writes y in double.
constexpr int kGemvSplits = 32;

__global__ void __launch_bounds__(256)
k_dense_gemv32_part(const float* __restrict__ X, int64_t m, const float* __restrict__ x, float* __restrict__ part,
                    const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int64_t r = blockIdx.x * (int64_t)1024 + 4 * (int64_t)threadIdx.x;
  const int64_t w = (m + kGemvSplits - 1) / kGemvSplits;
  const int64_t q0 = blockIdx.y * w, q1 = imin64(m, q0 + w);
  float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
  if ((m & 3) == 0 && r + 3 < m) {  // float4 loads need 16-byte aligned columns
    int64_t q = q0;
    for (; q + 1 < q1; q += 2) {
      const float4 u = *reinterpret_cast<const float4*>(X + q * m + r);
      const float4 v = *reinterpret_cast<const float4*>(X + (q + 1) * m + r);
      const float xu = x[q], xv = x[q + 1];
      a0.x = fmaf(u.x, xu, a0.x); a0.y = fmaf(u.y, xu, a0.y); a0.z = fmaf(u.z, xu, a0.z); a0.w = fmaf(u.w, xu, a0.w);
      a1.x = fmaf(v.x, xv, a1.x); a1.y = fmaf(v.y, xv, a1.y); a1.z = fmaf(v.z, xv, a1.z); a1.w = fmaf(v.w, xv, a1.w);
    }
    if (q < q1) {
      const float4 u = *reinterpret_cast<const float4*>(X + q * m + r);
      const float xu = x[q];
      a0.x = fmaf(u.x, xu, a0.x); a0.y = fmaf(u.y, xu, a0.y); a0.z = fmaf(u.z, xu, a0.z); a0.w = fmaf(u.w, xu, a0.w);
    }
  } else if (r < m) {
    for (int64_t q = q0; q < q1; ++q) {
      const float xu = x[q];
      const float* col = X + q * m + r;
      a0.x = fmaf(col[0], xu, a0.x);
      if (r + 1 < m) a0.y = fmaf(col[1], xu, a0.y);
      if (r + 2 < m) a0.z = fmaf(col[2], xu, a0.z);
      if (r + 3 < m) a0.w = fmaf(col[3], xu, a0.w);
    }
  }
  float* out = part + blockIdx.y * m;
  const float o[4] = {a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w};
  for (int c = 0; c < 4; ++c)
    if (r + c < m) out[r + c] = o[c];
}

__global__ void k_dense_gemv32_sum(const float* __restrict__ part, int64_t m, double* __restrict__ y,
                                   const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < kGemvSplits; ++c) s += part[c * m + i];
    y[i] = (double)s;
  }
}

// ---- float blocked LU (right-looking, partial pivoting) ----
__device__ void argmax_reduce_f(float& v, int64_t& ix) {
  __shared__ float sv[32];
  __shared__ int64_t si[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, v, o);
    const int64_t oi = __shfl_down_sync(0xffffffffu, ix, o);
    if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
  }
  if (lane == 0) { sv[wid] = v; si[wid] = ix; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sv[lane] : -1.f;
    ix = lane < nw ? si[lane] : INT64_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_down_sync(0xffffffffu, v, o);
      const int64_t oi = __shfl_down_sync(0xffffffffu, ix, o);
      if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
    }
    if (lane == 0) { sv[0] = v; si[0] = ix; }
  }
  __syncthreads();
  v = sv[0];
  ix = si[0];
  __syncthreads();
}

__global__ void k_piv_partial32(const float* __restrict__ A, int64_t m, int64_t c, float* __restrict__ pv,
                                int64_t* __restrict__ pi) {
  count_launch();
  float best = -1.f;
  int64_t bi = INT64_MAX;
  for (int64_t r = c + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    const float v = fabsf(A[c * m + r]);
    if (v > best) { best = v; bi = r; }
  }
  argmax_reduce_f(best, bi);
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = best;
    pi[blockIdx.x] = bi;
    pv[256 + blockIdx.x] = bi < m ? A[c * m + bi] : 0.f;
  }
}

__global__ void k_piv_swap32(float* __restrict__ A, int64_t m, int64_t c, int nparts, const float* __restrict__ pv,
                             const int64_t* __restrict__ pi, int* __restrict__ piv, int* __restrict__ status,
                             float* __restrict__ inv_out) {
  count_launch();
  __shared__ int64_t s_p;
  if (threadIdx.x == 0) {
    float best = -1.f, d = 0.f;
    int64_t bi = INT64_MAX;
    for (int b = 0; b < nparts; ++b)
      if (pv[b] > best || (pv[b] == best && pi[b] < bi)) { best = pv[b]; bi = pi[b]; d = pv[256 + b]; }
    if (bi >= m) { bi = c; d = 0.f; }
    s_p = bi;
    if (blockIdx.x == 0) {
      piv[c] = (int)bi;
      if (d == 0.f || !isfinite(d)) { atomicExch(status, 1); *inv_out = 0.f; } else *inv_out = 1.f / d;
    }
  }
  __syncthreads();
  const int64_t p = s_p;
  if (p != c)
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
      const float t = A[q * m + c];
      A[q * m + c] = A[q * m + p];
      A[q * m + p] = t;
    }
}

__global__ void k_panel_update32(float* __restrict__ A, int64_t m, int64_t c, int64_t pend,
                                 const float* __restrict__ inv_ptr) {
  count_launch();
  const float iv = *inv_ptr;
  for (int64_t r = c + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const float l = A[c * m + r] * iv;
    A[c * m + r] = l;
    for (int64_t q = c + 1; q < pend; ++q) A[q * m + r] -= l * A[q * m + c];
  }
}

// One panel [k0, k0 + kb) of the blocked LU in a single cooperative launch
// (every CTA resident) with ONE grid barrier per column. Thread tid owns the
// rows k0 + tid + i * stride for the whole panel. For column c:
//   1. (before the barrier) each CTA's largest |A[r][c]| over its rows
//      r >= c (ties: smallest row), and that candidate row's panel values
//      A[r][c .. pend) staged in global memory (double-buffered by the
//      column's parity, as are the partials, so that a CTA one column ahead
//      never overwrites what a slower one still reads);
//   2. grid barrier; every CTA reduces the partials in the same order
//      (largest value, ties to the smallest row), takes the winner's staged
//      row as the pivot row and records the pivot;
//   3. the thread owning the pivot row p exchanges rows c and p across the
//      panel (the multipliers of the earlier panel columns directly; from
//      column c on, row c receives the staged pivot row and row p the old
//      row c); every thread then scales and updates its rows r > c with the
//      pivot row held in shared memory, and takes step 1 of column c + 1 on
//      them.
// The interchanges of the columns outside the panel are applied afterwards
// (k_laswp32), so factors and pivots equal those of the per-column kernels.
// pv: [2][2 G] (|value|, signed value), pi: [2][G], stage: [2][G][kNbMax].
__global__ void __launch_bounds__(256)
k_panel_lu32(float* __restrict__ A, int64_t m, int64_t k0, int kb, float* __restrict__ pv,
             int64_t* __restrict__ pi, float* __restrict__ stage, int* __restrict__ piv, int* __restrict__ status,
             gsync::Barrier bar) {
  count_launch();
  const int G = gridDim.x;
  const int64_t stride = (int64_t)G * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t pend = k0 + kb;
  unsigned epoch = 0;
  __shared__ float s_row[kNbMax];
  __shared__ int64_t s_p;
  __shared__ float s_inv;
  __shared__ int s_w;

  // step 1 of column c on this CTA's rows, given its threads' (best, bi)
  auto partials = [&](float best, int64_t bi, int64_t c, int par) {
    argmax_reduce_f(best, bi);  // every thread receives the CTA's result
    if (threadIdx.x == 0) {
      pv[par * 2 * G + blockIdx.x] = best;
      pv[par * 2 * G + G + blockIdx.x] = bi < m ? A[c * m + bi] : 0.f;
      pi[par * G + blockIdx.x] = bi;
    }
    if (bi < m)
      for (int64_t q = c + threadIdx.x; q < pend; q += blockDim.x)
        stage[((int64_t)par * G + blockIdx.x) * kNbMax + (q - k0)] = A[q * m + bi];
  };

  {
    float best = -1.f;
    int64_t bi = INT64_MAX;
    for (int64_t r = k0 + tid; r < m; r += stride) {
      const float v = fabsf(A[k0 * m + r]);
      if (v > best) { best = v; bi = r; }
    }
    partials(best, bi, k0, 0);
  }
  for (int64_t c = k0; c < pend; ++c) {
    const int par = (int)((c - k0) & 1);
    if (!gsync::grid_sync(bar, epoch)) return;  // partials and staged rows of column c complete
    if (threadIdx.x < 32) {
      // warp 0 reduces the G partials (largest value, ties to the smallest
      // row); each lane issues all its loads before comparing
      const int lane = threadIdx.x;
      float b = -1.f, d = 0.f;
      int64_t p = INT64_MAX;
      int w = 0;
      for (int q0 = 0; q0 < G; q0 += 32 * kRedPerLane) {
        float vv[kRedPerLane], dd[kRedPerLane];
        int64_t ii[kRedPerLane];
#pragma unroll
        for (int j = 0; j < kRedPerLane; ++j) {
          const int q = q0 + lane + 32 * j;
          if (q < G) {
            vv[j] = __ldcg(pv + par * 2 * G + q);
            dd[j] = __ldcg(pv + par * 2 * G + G + q);
            ii[j] = __ldcg(reinterpret_cast<const long long*>(pi) + par * G + q);
          }
        }
#pragma unroll
        for (int j = 0; j < kRedPerLane; ++j) {
          const int q = q0 + lane + 32 * j;
          if (q < G && (vv[j] > b || (vv[j] == b && ii[j] < p))) { b = vv[j]; p = ii[j]; d = dd[j]; w = q; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, b, o);
        const int64_t op = __shfl_down_sync(0xffffffffu, p, o);
        const float od = __shfl_down_sync(0xffffffffu, d, o);
        const int ow = __shfl_down_sync(0xffffffffu, w, o);
        if (ob > b || (ob == b && op < p)) { b = ob; p = op; d = od; w = ow; }
      }
      if (lane == 0) {
        if (p >= m) { p = c; d = 0.f; }
        s_p = p;
        s_w = w;
        const bool bad = d == 0.f || !isfinite(d);
        s_inv = bad ? 0.f : 1.f / d;
        if (blockIdx.x == 0) {
          piv[c] = (int)p;
          if (bad) atomicExch(status, 1);
        }
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const float iv = s_inv;
    // the pivot row's panel values: row c's own if p == c, else the winner's staged copy
    for (int64_t q = c + threadIdx.x; q < pend; q += blockDim.x)
      s_row[q - k0] = p == c ? __ldcg(A + q * m + c) : __ldcg(stage + ((int64_t)par * G + s_w) * kNbMax + (q - k0));
    __syncthreads();
    const bool next = c + 1 < pend;
    float best = -1.f;
    int64_t bi = INT64_MAX;
    // Rows are moved kChunk columns at a time, all loads of a pass issued
    // before its stores (one L2 round trip per pass, not per column).
    for (int64_t r = k0 + tid; r < m; r += stride) {
      if (r <= c) continue;
      if (r == p) {  // rows c and p change places across the panel
        for (int64_t qb = k0; qb < pend; qb += kChunk) {
          float oc[kChunk], op[kChunk];
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            const int64_t q = qb + j;
            if (q < pend) {
              oc[j] = __ldcg(A + q * m + c);
              // the multipliers of the earlier columns from row p itself,
              // from column c on the staged pivot row
              op[j] = q < c ? A[q * m + p] : s_row[q - k0];
            }
          }
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            const int64_t q = qb + j;
            if (q < pend) {
              A[q * m + c] = op[j];
              A[q * m + p] = oc[j];
            }
          }
        }
      }
      // l = A[r][c] / pivot, A[r][q] -= l A[c][q] for q in (c, pend)
      float l = 0.f;
      for (int64_t qb = c; qb < pend; qb += kChunk) {
        float v[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
          if (qb + j < pend) v[j] = A[(qb + j) * m + r];
        if (qb == c) {
          l = v[0] * iv;
          v[0] = l;
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int64_t q = qb + j;
          if (q > c && q < pend) v[j] -= l * s_row[q - k0];
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
          if (qb + j < pend) A[(qb + j) * m + r] = v[j];
        if (qb == c && next) {  // the next column's candidate (q = c + 1 is in this pass)
          const float a = fabsf(v[1]);
          if (a > best) { best = a; bi = r; }
        }
      }
    }
    if (next) partials(best, bi, c + 1, par ^ 1);
  }
}

// A sub-panel [k0, k0 + kb), kb <= kNb, factored in one cooperative launch
// with its rows held in shared memory: thread t of CTA b owns the rows
// k0 + 256 b + t + i stride (i < R, stride = 256 G), stored at
// s_rows[(i kNb + q) 256 + t] for column k0 + q. Per column c:
//   1. (before the barrier) the CTA's candidate (largest |a[r][c]|, r >= c,
//      ties to the smallest row) with its whole sub-panel row staged in
//      global memory, and row c's owner stages row c (both double-buffered
//      by the column's parity);
//   2. grid barrier; every CTA reduces the candidates in the same order and
//      takes the winner's staged row (or row c's, if p == c) as the pivot
//      row; row c's owner writes the pivot row into row c's slot and row p's
//      owner writes the old row c into row p's slot;
//   3. every thread scales and updates its rows r > c in shared memory and
//      takes step 1 of column c + 1.
// The rows go back to global memory at the end; the interchanges of the
// other columns follow (k_laswp32). Each entry sees the same operations as
// in the per-column kernels, so the factors are the same bit for bit.
// pv: [2][2 G], pi: [2][G], stage: [2][G][kNb], rowc: [2][kNb].
__global__ void __launch_bounds__(256)
k_panel_lu32_smem(float* __restrict__ A, int64_t m, int64_t k0, int kb, int R, float* __restrict__ pv,
                  int64_t* __restrict__ pi, float* __restrict__ stage, float* __restrict__ rowc,
                  int* __restrict__ piv, int* __restrict__ status, gsync::Barrier bar) {
  count_launch();
  extern __shared__ float s_rows[];  // [R][kNb][256]
  __shared__ float s_piv[kNb];
  __shared__ int64_t s_p;
  __shared__ float s_inv;
  __shared__ int s_w;
  const int G = gridDim.x;
  const int t = threadIdx.x;
  const int64_t stride = (int64_t)G * 256;
  const int64_t rbase = k0 + (int64_t)blockIdx.x * 256 + t;  // this thread's row in slot i: rbase + i stride
  const int64_t pend = k0 + kb;
  unsigned epoch = 0;
  auto at = [&](int i, int q, int tt) -> float& { return s_rows[((int64_t)i * kNb + q) * 256 + tt]; };
  // slot (i, CTA, thread) of row r >= k0
  auto slot = [&](int64_t r, int& i, int& cta, int& tt) {
    const int64_t off = r - k0;
    i = (int)(off / stride);
    const int64_t rem = off - (int64_t)i * stride;
    cta = (int)(rem / 256);
    tt = (int)(rem - (int64_t)cta * 256);
  };

  for (int i = 0; i < R; ++i) {
    const int64_t r = rbase + i * stride;
    for (int q = 0; q < kb; ++q) at(i, q, t) = r < m ? A[(k0 + q) * m + r] : 0.f;
  }
  __syncthreads();

  // step 1 of column c (local cc) from the threads' (best, bi)
  auto candidates = [&](float best, int64_t bi, int64_t c, int par) {
    argmax_reduce_f(best, bi);  // every thread receives the CTA's result (and the block is in step)
    const int cc = (int)(c - k0);
    if (bi < m) {
      int ib, cb, tb;
      slot(bi, ib, cb, tb);
      if (t == 0) {
        pv[par * 2 * G + blockIdx.x] = best;
        pv[par * 2 * G + G + blockIdx.x] = at(ib, cc, tb);
        pi[par * G + blockIdx.x] = bi;
      }
      if (t < kb) stage[((int64_t)par * G + blockIdx.x) * kNb + t] = at(ib, t, tb);
    } else if (t == 0) {
      pv[par * 2 * G + blockIdx.x] = -1.f;
      pv[par * 2 * G + G + blockIdx.x] = 0.f;
      pi[par * G + blockIdx.x] = INT64_MAX;
    }
    int ic, cc_cta, tc;
    slot(c, ic, cc_cta, tc);
    if (cc_cta == (int)blockIdx.x && t < kb) rowc[par * kNb + t] = at(ic, t, tc);
  };

  {
    float best = -1.f;
    int64_t bi = INT64_MAX;
    for (int i = 0; i < R; ++i) {
      const int64_t r = rbase + i * stride;
      if (r < m) {
        const float v = fabsf(at(i, 0, t));
        if (v > best) { best = v; bi = r; }
      }
    }
    candidates(best, bi, k0, 0);
  }
  for (int64_t c = k0; c < pend; ++c) {
    const int cc = (int)(c - k0);
    const int par = cc & 1;
    if (!gsync::grid_sync(bar, epoch)) return;  // candidates, staged rows and row c complete
    if (t < 32) {
      const int lane = t;
      float b = -1.f, d = 0.f;
      int64_t p = INT64_MAX;
      int w = 0;
      for (int q0 = 0; q0 < G; q0 += 32 * kRedPerLane) {
        float vv[kRedPerLane], dd[kRedPerLane];
        int64_t ii[kRedPerLane];
#pragma unroll
        for (int j = 0; j < kRedPerLane; ++j) {
          const int q = q0 + lane + 32 * j;
          if (q < G) {
            vv[j] = __ldcg(pv + par * 2 * G + q);
            dd[j] = __ldcg(pv + par * 2 * G + G + q);
            ii[j] = __ldcg(reinterpret_cast<const long long*>(pi) + par * G + q);
          }
        }
#pragma unroll
        for (int j = 0; j < kRedPerLane; ++j) {
          const int q = q0 + lane + 32 * j;
          if (q < G && (vv[j] > b || (vv[j] == b && ii[j] < p))) { b = vv[j]; p = ii[j]; d = dd[j]; w = q; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, b, o);
        const int64_t op = __shfl_down_sync(0xffffffffu, p, o);
        const float od = __shfl_down_sync(0xffffffffu, d, o);
        const int ow = __shfl_down_sync(0xffffffffu, w, o);
        if (ob > b || (ob == b && op < p)) { b = ob; p = op; d = od; w = ow; }
      }
      if (lane == 0) {
        if (p >= m) { p = c; d = 0.f; }
        s_p = p;
        s_w = w;
        const bool bad = d == 0.f || !isfinite(d);
        s_inv = bad ? 0.f : 1.f / d;
        if (blockIdx.x == 0) {
          piv[c] = (int)p;
          if (bad) atomicExch(status, 1);
        }
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const float iv = s_inv;
    if (t < kb) {
      const float oc = __ldcg(rowc + par * kNb + t);  // row c before the exchange
      const float pr = p == c ? oc : __ldcg(stage + ((int64_t)par * G + s_w) * kNb + t);
      s_piv[t] = pr;
      if (p != c) {
        int i1, b1, t1;
        slot(c, i1, b1, t1);
        if (b1 == (int)blockIdx.x) at(i1, t, t1) = pr;  // row c becomes the pivot row
        slot(p, i1, b1, t1);
        if (b1 == (int)blockIdx.x) at(i1, t, t1) = oc;  // row p takes the old row c
      }
    }
    __syncthreads();
    const bool next = c + 1 < pend;
    float best = -1.f;
    int64_t bi = INT64_MAX;
    for (int i = 0; i < R; ++i) {
      const int64_t r = rbase + i * stride;
      if (r <= c || r >= m) continue;
      const float l = at(i, cc, t) * iv;
      at(i, cc, t) = l;
      // kChunk columns per pass: loads of a pass before its stores
      for (int qb = cc + 1; qb < kb; qb += kChunk) {
        float v[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
          if (qb + j < kb) v[j] = at(i, qb + j, t);
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
          if (qb + j < kb) at(i, qb + j, t) = v[j] - l * s_piv[qb + j];
      }
      if (next) {
        const float a = fabsf(at(i, cc + 1, t));
        if (a > best) { best = a; bi = r; }
      }
    }
    if (next) candidates(best, bi, c + 1, par ^ 1);
  }
  __syncthreads();
  for (int i = 0; i < R; ++i) {
    const int64_t r = rbase + i * stride;
    if (r < m)
      for (int q = 0; q < kb; ++q) A[(k0 + q) * m + r] = at(i, q, t);
  }
}

// The interchanges piv[k0 .. k0 + kb) applied, in order, to every column
// outside the panel (one thread per column). After a panel that gave up at
// a grid barrier (*err set) its later pivots were never written, so nothing
// is swapped; a pivot outside (c, m) is skipped as well (the buffer is
// filled with -1 before the factorisation).
__global__ void k_laswp32(float* __restrict__ A, int64_t m, int64_t k0, int kb, const int* __restrict__ piv,
                          const int* __restrict__ err) {
  count_launch();
  if (*(volatile const int*)err) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m - kb; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = j < k0 ? j : j + kb;
    float* col = A + q * m;
    for (int64_t c = k0; c < k0 + kb; ++c) {
      const int64_t p = piv[c];
      if (p > c && p < m) {
        const float t = col[c];
        col[c] = col[p];
        col[p] = t;
      }
    }
  }
}

// U12 rows [k0, k0 + kb) (kb <= kNb) of the columns q0 <= q < q1: the
// forward substitution L11 x = A[k0 .. k0 + kb)[q] per column. A CTA takes 32
// columns: L11 and the 32 column segments are loaded into shared memory with
// coalesced accesses (each column segment is kb contiguous floats), four
// lanes solve one column (rows r = sub, sub + 4, ...; a warp sync per step),
// and the results are stored back the same way. Each entry sees the same
// operations in the same order as a column-at-a-time substitution.
constexpr int kTrsmCols = 32;
__global__ void __launch_bounds__(128)
k_trsm_row_panel32(float* __restrict__ A, int64_t m, int64_t k0, int kb, int64_t q0, int64_t q1) {
  count_launch();
  __shared__ float sL[kNb][kNb + 1];        // [c][r] = L11[r][c]
  __shared__ float sX[kTrsmCols][kNb + 1];  // [j][r]
  const int64_t qb = q0 + (int64_t)blockIdx.x * kTrsmCols;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int c = e / kb, r = e - c * kb;
    sL[c][r] = A[(k0 + c) * m + k0 + r];
  }
  for (int e = threadIdx.x; e < kTrsmCols * kb; e += blockDim.x) {
    const int j = e / kb, r = e - j * kb;
    const int64_t q = qb + j;
    sX[j][r] = q < q1 ? A[q * m + k0 + r] : 0.f;
  }
  __syncthreads();
  const int j = threadIdx.x >> 2, sub = threadIdx.x & 3;  // column j of the CTA, rows sub + 4 i
  for (int c = 0; c < kb; ++c) {
    const float xc = sX[j][c];
    for (int r = c + 1 + ((sub - (c + 1)) & 3); r < kb; r += 4) sX[j][r] -= sL[c][r] * xc;
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTrsmCols * kb; e += blockDim.x) {
    const int jj = e / kb, r = e - jj * kb;
    const int64_t q = qb + jj;
    if (q < q1) A[q * m + k0 + r] = sX[jj][r];
  }
}

// rc = R r per component (x and y): rc_j = (n_c / n_f) sum_i P[i][j] r_i.
// Transfers run in single precision (a preconditioner: flexible GMRES
// absorbs the rounding). Pass 1: CTA (c, k) takes rows [kRc c, kRc c + kRc)
// of component k (its r in shared memory) against all n_c columns
// (coalesced reads of P's rows) and writes partial sums part[c][j]; pass 2
// adds the chunks of each coarse node in a fixed order.
constexpr int kRc = 256;

__global__ void __launch_bounds__(128)
k_restrict_part(const int64_t* __restrict__ off, const int64_t* __restrict__ off_c, const int64_t* __restrict__ ioff,
                const float* __restrict__ P, const double* __restrict__ r, int64_t Nc, float2* __restrict__ part,
                const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int k = blockIdx.y;
  const int64_t nf = off[k + 1] - off[k], nc = off_c[k + 1] - off_c[k];
  const int64_t i0 = blockIdx.x * (int64_t)kRc;
  if (i0 >= nf) return;
  const int ni = (int)imin64(kRc, nf - i0);
  __shared__ float2 sr[kRc];
  const double2* rk = reinterpret_cast<const double2*>(r) + off[k] + i0;
  for (int e = threadIdx.x; e < ni; e += blockDim.x) {
    const double2 v = rk[e];
    sr[e] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const float* Pk = P + ioff[k] + i0 * nc;
  for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
    float ax = 0.f, ay = 0.f;
    for (int i = 0; i < ni; ++i) {
      const float pv = Pk[i * nc + j];
      ax = fmaf(pv, sr[i].x, ax);
      ay = fmaf(pv, sr[i].y, ay);
    }
    part[blockIdx.x * Nc + off_c[k] + j] = make_float2(ax, ay);
  }
}

__global__ void k_restrict_sum(int64_t Nc, const int* __restrict__ comp_c, const int64_t* __restrict__ off,
                               const int64_t* __restrict__ off_c, const float2* __restrict__ part,
                               double* __restrict__ rc, float* __restrict__ rc32, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  for (int64_t jj = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jj < Nc; jj += (int64_t)gridDim.x * blockDim.x) {
    const int k = comp_c[jj];
    const int64_t nf = off[k + 1] - off[k], nc = off_c[k + 1] - off_c[k];
    const int64_t chunks = (nf + kRc - 1) / kRc;
    float ax = 0.f, ay = 0.f;
    for (int64_t c = 0; c < chunks; ++c) {
      const float2 v = part[c * Nc + jj];
      ax += v.x;
      ay += v.y;
    }
    const float scale = (float)nc / (float)nf;
    rc[2 * jj] = (double)(scale * ax);
    rc[2 * jj + 1] = (double)(scale * ay);
    rc32[2 * jj] = scale * ax;
    rc32[2 * jj + 1] = scale * ay;
  }
}

// z = I zc (+ -2 h on the wall), h = r - I rc. One warp per fine node: the
// lanes read the node's row of P (coalesced) and reduce by shuffles.
__global__ void __launch_bounds__(256)
k_prolong(int64_t N, int outer, const int* __restrict__ comp, const int64_t* __restrict__ off,
          const int64_t* __restrict__ off_c, const int64_t* __restrict__ ioff, const float* __restrict__ P,
          const double* __restrict__ r, const double* __restrict__ rc, const double* __restrict__ zc,
          double* __restrict__ z, double* __restrict__ h, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t gi = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); gi < N; gi += warps) {
    const int k = comp[gi];
    const int64_t i = gi - off[k];
    const int64_t nc = off_c[k + 1] - off_c[k];
    const float* row = P + ioff[k] + i * nc;
    const double2* rck = reinterpret_cast<const double2*>(rc) + off_c[k];
    const double2* zck = reinterpret_cast<const double2*>(zc) + off_c[k];
    float ux = 0.f, uy = 0.f, vx = 0.f, vy = 0.f;
    for (int64_t j = lane; j < nc; j += 32) {
      const float pv = row[j];
      const double2 zv = zck[j], rv = rck[j];
      ux = fmaf(pv, (float)zv.x, ux);
      uy = fmaf(pv, (float)zv.y, uy);
      vx = fmaf(pv, (float)rv.x, vx);
      vy = fmaf(pv, (float)rv.y, vy);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ux += __shfl_xor_sync(0xffffffffu, ux, o);
      uy += __shfl_xor_sync(0xffffffffu, uy, o);
      vx += __shfl_xor_sync(0xffffffffu, vx, o);
      vy += __shfl_xor_sync(0xffffffffu, vy, o);
    }
    if (lane == 0) {
      const int64_t o2 = 2 * gi;
      const double hx = r[o2] - vx, hy = r[o2 + 1] - vy;
      h[o2] = hx;
      h[o2 + 1] = hy;
      if (k == outer) {
        z[o2] = ux - 2.0 * hx;
        z[o2 + 1] = uy - 2.0 * hy;
      } else {
        z[o2] = ux;
        z[o2 + 1] = uy;
      }
    }
  }
}

// Real trigonometric interpolation matrix nf x nc (row-major), see the top,
// from the closed form of the band-limited (periodic sinc) interpolant:
//   S(d) = sin(nc d / 2) cot(d / 2) / nc   (nc even),
//   S(d) = sin(nc d / 2) / (nc sin(d / 2)) (nc odd),  S(0) = 1.
// Weight of coarse sample j at fine node i of the trigonometric interpolant
// from nc to nf = q nc equispaced samples: a function of the angle
// d = 2 pi (i / nf - j / nc) = 2 pi delta / nf, delta = (i - q j) mod nf
// (the weight is 2 pi-periodic in d), so one row of nf values, V[delta],
// gives the whole nf x nc matrix.
std::vector<float> trig_interp_row(int64_t nc, int64_t nf) {
  std::vector<float> V((size_t)nf);
  for (int64_t delta = 0; delta < nf; ++delta) {
    const double d = 2.0 * kPi * (double)delta / (double)nf;
    const double sh = std::sin(0.5 * d);
    double v;
    if (delta == 0) {
      v = 1.0;  // the sample itself
    } else if (nc % 2 == 0) {
      v = std::sin(0.5 * (double)nc * d) * std::cos(0.5 * d) / (sh * (double)nc);
    } else {
      v = std::sin(0.5 * (double)nc * d) / (sh * (double)nc);
    }
    V[(size_t)delta] = (float)v;
  }
  return V;
}

// P[i][j] = V[(i - q j) mod nf] for the row-major nf x nc matrix P.
__global__ void k_fill_interp(const float* __restrict__ V, int64_t nf, int64_t nc, int q, float* __restrict__ P) {
  count_launch();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nf * nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nc, j = e - i * nc;
    int64_t d = (i - (int64_t)q * j) % nf;
    if (d < 0) d += nf;
    P[e] = V[d];
  }
}

}  // namespace

struct SetupTimer {
  bool on;
  cudaStream_t s;
  double t0;
  static double now() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
  }
  void lap(const char* what) {
    if (!on) return;
    cudaStreamSynchronize(s);
    const double t1 = now();
    std::fprintf(stderr, "[stokes] two-grid setup: %s %.3f s\n", what, t1 - t0);
    t0 = t1;
  }
};

void twogrid_setup(Geom& g, int q, int coarse_mode) {
  SetupTimer tm{std::getenv("STOKES_TRACE") != nullptr, g.stream, SetupTimer::now()};
  TwoGrid& t = g.tg;
  t.ready = false;
  require(q >= 2, "coarsening factor must be >= 2");
  const int nc = g.n_comp;
  cudaStream_t s = g.stream;
  t.q = q;
  t.off_c.assign(nc + 1, 0);
  for (int k = 0; k < nc; ++k) {
    const int64_t n = g.off[k + 1] - g.off[k];
    require(n % q == 0 && n / q >= 8, "two-grid: every component needs a multiple of q nodes, at least 8 q");
    t.off_c[k + 1] = t.off_c[k] + n / q;
  }
  const int64_t Nc = t.off_c[nc];
  t.Nc = Nc;
  const int64_t m = 2 * Nc;
  require((double)m * (double)m * 4.0 < 64e9, "two-grid: coarse operator too large (reduce with a larger q)");
  // interpolation matrices, one per distinct (n_f, n_c), filled on the GPU
  // from one row of weights each
  std::map<std::pair<int64_t, int64_t>, int64_t> seen;
  std::vector<float> vpool;
  std::vector<std::array<int64_t, 4>> fills;  // n_f, n_c, offset of P, offset of its row V
  int64_t ptotal = 0;
  std::vector<int64_t> ioff(nc);
  for (int k = 0; k < nc; ++k) {
    const int64_t nf = g.off[k + 1] - g.off[k], ncc = nf / q;
    auto key = std::make_pair(nf, ncc);
    auto it = seen.find(key);
    if (it == seen.end()) {
      const std::vector<float> V = trig_interp_row(ncc, nf);
      seen[key] = ptotal;
      ioff[k] = ptotal;
      fills.push_back({nf, ncc, ptotal, (int64_t)vpool.size()});
      vpool.insert(vpool.end(), V.begin(), V.end());
      ptotal += nf * ncc;
    } else {
      ioff[k] = it->second;
    }
  }
  t.interp.alloc(ptotal);
  t.d_ioff.alloc(nc);
  t.d_off_c.alloc(nc + 1);
  DevBuf<float> vrows;  // freed at the end of the setup, after its uses
  vrows.alloc(vpool.size());
  STOKES_CUDA(cudaMemcpyAsync(vrows.get(), vpool.data(), 4 * vpool.size(), cudaMemcpyHostToDevice, s));
  for (const auto& fl : fills)
    k_fill_interp<<<(unsigned)std::min<int64_t>((fl[0] * fl[1] + 255) / 256, 152 * 16), 256, 0, s>>>(
        vrows.get() + fl[3], fl[0], fl[1], q, t.interp.get() + fl[2]);
  STOKES_LAUNCHED();
  STOKES_CUDA(cudaMemcpyAsync(t.d_ioff.get(), ioff.data(), 8 * nc, cudaMemcpyHostToDevice, s));
  STOKES_CUDA(cudaMemcpyAsync(t.d_off_c.get(), t.off_c.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, s));
  // coarse nodes
  t.pos_c.alloc(Nc);
  t.nrm_c.alloc(Nc);
  t.w_c.alloc(Nc);
  t.selfc_c.alloc(Nc);
  t.comp_c.alloc(Nc);
  k_coarse_gather<<<(unsigned)((Nc + 255) / 256), 256, 0, s>>>(Nc, q, g.d_off.get(), t.d_off_c.get(), nc, g.pos.get(),
                                                              g.nrm.get(), g.w.get(), g.selfc.get(), t.pos_c.get(),
                                                              t.nrm_c.get(), t.w_c.get(), t.selfc_c.get(),
                                                              t.comp_c.get());
  STOKES_LAUNCHED();
  const int ps = g.prof.begin(kProfBdSetup, 2.0 * (double)m * m * m, s);
  // assemble and factorise the coarse operator
  t.lu.alloc((size_t)m * m);
  {
    DevBuf<float4> fp, fq, fd, fc;
    fp.alloc(Nc);
    fq.alloc(Nc);
    fd.alloc(Nc);
    fc.alloc(nc);
    k_coarse_floats<<<(unsigned)((Nc + 255) / 256), 256, 0, s>>>(Nc, t.pos_c.get(), t.nrm_c.get(), t.w_c.get(),
                                                                t.selfc_c.get(), t.comp_c.get(), fp.get(), fq.get(),
                                                                fd.get());
    k_centre_floats<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(nc, g.centre.get(), fc.get());
    dim3 ga((unsigned)((Nc + 255) / 256), (unsigned)std::min<int64_t>(Nc, 16384));
    k_coarse_assemble<<<ga, 256, 0, s>>>(Nc, fp.get(), fq.get(), fd.get(), fc.get(), g.outer, t.lu.get());
    STOKES_LAUNCHED();
    STOKES_CUDA(cudaStreamSynchronize(s));  // scratch goes out of scope
  }
  tm.lap("assembly");
  t.piv.alloc(m);
  STOKES_CUDA(cudaMemsetAsync(t.piv.get(), 0xff, 4 * m, s));  // -1 until a panel writes its pivots
  t.status.alloc(1);
  STOKES_CUDA(cudaMemsetAsync(t.status.get(), 0, sizeof(int), s));
  DevBuf<float> pv, ivp;
  DevBuf<int64_t> pi;
  // Large coarse operators factor each panel in one cooperative launch
  // (one CTA per SM); small ones (few rows per CTA) keep the per-column
  // launches. STOKES_TG_PANEL=coop or =launches overrides the choice.
  const char* panel_env = std::getenv("STOKES_TG_PANEL");
  const bool force_coop = panel_env && std::string(panel_env) == "coop";
  const bool force_launches = panel_env && std::string(panel_env) == "launches";
  int coop_grid = 0;
  if ((m >= 8192 || force_coop) && !force_launches) {
    int dev = 0, nsm = 0, per_sm = 0;
    STOKES_CUDA(cudaGetDevice(&dev));
    STOKES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_lu32, 256, 0));
    if (per_sm >= 1) coop_grid = nsm;
  }
  // the shared-memory sub-panel kernel: up to kSubR row slots of 64 KB per
  // CTA (rows below the sub-panel's first: up to kSubR * 256 * grid)
  bool smem_panel = false;
  if (coop_grid > 0) {
    const int bytes = kSubR * kNb * 256 * (int)sizeof(float);
    STOKES_CUDA(cudaFuncSetAttribute(k_panel_lu32_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int per_sm = 0;
    STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_lu32_smem, 256, bytes));
    smem_panel = per_sm >= 1;
  }
  pv.alloc(std::max(512, 4 * coop_grid));
  pi.alloc(std::max(256, 2 * coop_grid));
  DevBuf<float> stage, rowc;
  if (coop_grid > 0) {
    stage.alloc((size_t)2 * coop_grid * kNbMax);
    rowc.alloc(2 * kNb);
  }
  ivp.alloc(1);
  t.barrier.alloc(4);
  STOKES_CUDA(cudaMemsetAsync(t.barrier.get(), 0, 4 * sizeof(unsigned), s));
  float* A = t.lu.get();
  // trailing updates on the tensor cores (three TF32 products per term)
  // where the trailing block has at least 256 rows; STOKES_TG_GEMM=simt
  // keeps the CUDA-core GEMM throughout
  const bool tc = tc_trailing_enabled();
  DevBuf<float> tc_work;
  if (tc && m > 256) tc_work.alloc(tc_trailing_work_floats(m));
  // with STOKES_TRACE: time of the panel factorisations and of the trailing
  // updates, from events around each phase
  std::vector<cudaEvent_t> ev;
  auto mark = [&]() {
    if (!tm.on) return;
    cudaEvent_t e;
    STOKES_CUDA(cudaEventCreate(&e));
    STOKES_CUDA(cudaEventRecord(e, s));
    ev.push_back(e);
  };
  // 128-column panels when the trailing updates run on the tensor cores
  // (each update then moves its trailing block once per 128 columns)
  const int nb = (tc && m >= 8192) ? kNbTc : kNb;
  // One sub-panel [ks, ks + ws), ws <= kNb: pivots piv[ks .. ks + ws) and the
  // rows exchanged across all m columns. Cooperative kernels (shared-memory
  // rows where they fit, else global) plus k_laswp32 for the other columns,
  // or three launches per column; the factors are the same bit for bit.
  auto factor_subpanel = [&](int64_t ks, int ws) {
    if (coop_grid > 0) {
      gsync::Barrier bar{t.barrier.get(), t.barrier.get() + 1, (int*)(t.barrier.get() + 2), gsync::spin_limit()};
      int64_t ksv = ks;
      int wsv = ws;
      float* pvp = pv.get();
      int64_t* pip = pi.get();
      int* pivp = t.piv.get();
      int* stp = t.status.get();
      float* sgp = stage.get();
      float* rcp = rowc.get();
      const int64_t stride = (int64_t)coop_grid * 256;
      int R = (int)((m - ks + stride - 1) / stride);
      STOKES_CUDA(cudaMemsetAsync(t.barrier.get(), 0, sizeof(unsigned), s));  // arrivals restart; errors stay
      if (smem_panel && R <= kSubR) {
        void* args[] = {(void*)&A,   (void*)&m,   (void*)&ksv, (void*)&wsv,  (void*)&R,   (void*)&pvp,
                        (void*)&pip, (void*)&sgp, (void*)&rcp, (void*)&pivp, (void*)&stp, (void*)&bar};
        STOKES_CUDA(cudaLaunchCooperativeKernel((const void*)k_panel_lu32_smem, dim3(coop_grid), dim3(256), args,
                                                (size_t)R * kNb * 256 * sizeof(float), s));
      } else {
        void* args[] = {(void*)&A,   (void*)&m,   (void*)&ksv,  (void*)&wsv, (void*)&pvp,
                        (void*)&pip, (void*)&sgp, (void*)&pivp, (void*)&stp, (void*)&bar};
        STOKES_CUDA(
            cudaLaunchCooperativeKernel((const void*)k_panel_lu32, dim3(coop_grid), dim3(256), args, 0, s));
      }
      if (m > ws)
        k_laswp32<<<(unsigned)std::min<int64_t>((m - ws + 255) / 256, 152 * 8), 256, 0, s>>>(A, m, ks, ws, pivp,
                                                                                            bar.err);
    } else {
      for (int64_t c = ks; c < ks + ws; ++c) {
        const int parts = (int)std::min<int64_t>(256, (m - c + 255) / 256);
        k_piv_partial32<<<parts, 256, 0, s>>>(A, m, c, pv.get(), pi.get());
        k_piv_swap32<<<(unsigned)std::min<int64_t>(64, (m + 255) / 256), 256, 0, s>>>(
            A, m, c, parts, pv.get(), pi.get(), t.piv.get(), t.status.get(), ivp.get());
        const int64_t nr = m - c - 1;
        if (nr > 0)
          k_panel_update32<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, (nr + 127) / 128)), 128, 0,
                             s>>>(A, m, c, ks + ws, ivp.get());
      }
    }
  };
  for (int64_t k0 = 0; k0 < m; k0 += nb) {
    const int kb = (int)std::min<int64_t>(nb, m - k0);
    mark();
    const int pp = g.prof.begin(kProfLuPanel, (double)kb, s);
    // the panel as sub-panels of kNb columns; after each, the panel's
    // columns to its right get their rows of U (row-panel solve) and the
    // product of the sub-panel's L and those rows subtracted below
    for (int64_t ks = k0; ks < k0 + kb; ks += kNb) {
      const int ws = (int)std::min<int64_t>(kNb, k0 + kb - ks);
      factor_subpanel(ks, ws);
      const int64_t q0 = ks + ws, q1 = k0 + kb;
      if (q1 > q0) {
        k_trsm_row_panel32<<<(unsigned)((q1 - q0 + kTrsmCols - 1) / kTrsmCols), 128, 0, s>>>(A, m, ks, ws, q0, q1);
        sgemm32(s, m - q0, q1 - q0, ws, -1.f, A + ks * m + q0, m, A + q0 * m + ks, m, 1.f, A + q0 * m + q0, m);
      }
    }
    g.prof.end(pp, s);
    const int64_t rest = m - k0 - kb;
    mark();
    if (rest > 0) {
      // U12 = L11^-1 A12 (rows of the panel, columns from k0 + kb on), by
      // blocks of kNb rows: solve the first block, subtract its product from
      // the rest of the panel's rows, solve the second
      const int64_t base = k0 + kb;
      const unsigned gq = (unsigned)((rest + kTrsmCols - 1) / kTrsmCols);
      k_trsm_row_panel32<<<gq, 128, 0, s>>>(A, m, k0, std::min(kb, kNb), base, m);
      if (kb > kNb) {
        sgemm32(s, kb - kNb, rest, kNb, -1.f, A + k0 * m + k0 + kNb, m, A + base * m + k0, m, 1.f,
                A + base * m + k0 + kNb, m);
        k_trsm_row_panel32<<<gq, 128, 0, s>>>(A, m, k0 + kNb, kb - kNb, base, m);
      }
      // A22 -= L21 U12 (rows and columns from k0 + kb on)
      const int pg = g.prof.begin(kProfLuGemm, 2.0 * (double)rest * (double)rest * kb, s);
      if (tc && kb % 32 == 0 && rest >= 256)
        tc_trailing_update(s, A, m, k0, kb, rest, tc_work.get(), (int*)(t.barrier.get() + 2));
      else
        sgemm32(s, rest, rest, kb, -1.f, A + k0 * m + base, m, A + base * m + k0, m, 1.f, A + base * m + base, m);
      g.prof.end(pg, s);
    }
    STOKES_LAUNCHED();
  }
  mark();
  if (tm.on) {
    STOKES_CUDA(cudaStreamSynchronize(s));
    double panel = 0.0, trail = 0.0;
    for (size_t e = 0; e + 1 < ev.size(); ++e) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[e], ev[e + 1]);
      (e % 2 == 0 ? panel : trail) += ms;
    }
    for (auto e : ev) cudaEventDestroy(e);
    std::fprintf(stderr, "[stokes] two-grid LU: panels %.3f s, row panel solves + trailing updates %.3f s\n",
                 panel / 1e3, trail / 1e3);
  }
  tm.lap("LU");
  std::vector<int> hpiv(m);
  int hstatus = 0;
  unsigned hbar = 0;
  STOKES_CUDA(cudaMemcpyAsync(hpiv.data(), t.piv.get(), 4 * m, cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaMemcpyAsync(&hstatus, t.status.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaMemcpyAsync(&hbar, t.barrier.get() + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  STOKES_CUDA(cudaStreamSynchronize(s));
  require(hbar == 0, "two-grid: a bounded wait of the coarse LU (panel barrier or tensor-core pipeline) timed out",
          STOKES_ECUDA);
  require(hstatus == 0, "two-grid: singular coarse operator (zero pivot)", STOKES_EBREAKDOWN);
  std::vector<int> perm(m);
  for (int64_t r = 0; r < m; ++r) perm[r] = (int)r;
  for (int64_t c = 0; c < m; ++c) {
    require(hpiv[c] >= c && hpiv[c] < m, "two-grid: coarse LU pivot out of range", STOKES_ECUDA);
    std::swap(perm[c], perm[hpiv[c]]);
  }
  t.perm.alloc(m);
  STOKES_CUDA(cudaMemcpyAsync(t.perm.get(), perm.data(), 4 * m, cudaMemcpyHostToDevice, s));
  t.rc.alloc(m);
  t.rc32.alloc(m);
  t.zc.alloc(m);
  t.gemv_part.alloc((size_t)kGemvSplits * m);
  int64_t max_nf = 0;
  for (int k = 0; k < nc; ++k) max_nf = std::max<int64_t>(max_nf, g.off[k + 1] - g.off[k]);
  t.max_chunks = (max_nf + kRc - 1) / kRc;
  t.rpart.alloc((size_t)t.max_chunks * Nc);
  t.h.alloc(2 * g.N);
  // Coarse solve: an explicit float inverse (each apply one memory-bound
  // matrix-vector product) while forming it is cheap (2 m^3 flops); beyond
  // kMaxExplicitCoarse unknowns, or on request, the LU factors are applied
  // by the persistent triangular solves instead (the same bytes per apply,
  // no inversion).
  t.use_lu = coarse_mode == STOKES_TG_COARSE_LU || (coarse_mode == STOKES_TG_COARSE_AUTO && m > kMaxExplicitCoarse);
  if (t.use_lu) {
    t.inv.release();
    t.trsv_work.alloc(lu_solve_work_words(m, sizeof(float)));
    STOKES_CUDA(cudaMemsetAsync(t.trsv_work.get(), 0, lu_solve_work_words(m, sizeof(float)) * 8, s));
    t.trsv_gen = 0;
    t.tinv.alloc(lu_tile_inverse_elems(m));
    lu_tile_inverses<float>(s, t.lu.get(), m, t.tinv.get());
  } else {
    t.inv.alloc((size_t)m * m);
    invert_from_lu32(g, t.lu.get(), m, t.perm.get(), t.inv.get());
    t.lu.release();
    tm.lap("inverse");
  }
  g.prof.end(ps, s);
  // fine blocks of the pores (the wall block is replaced by -2 I)
  bd_setup_pores(g, /*skip_wall=*/true);
  STOKES_CUDA(cudaStreamSynchronize(s));
  tm.lap("pore blocks");
  t.ready = true;
}

static void twogrid_apply(Geom& g, const double* r, double* z, const int* done, bool f32) {
  TwoGrid& t = g.tg;
  cudaStream_t s = g.stream;
  const int nc = g.n_comp;
  k_restrict_part<<<dim3((unsigned)t.max_chunks, (unsigned)nc), 128, 0, s>>>(
      g.d_off.get(), t.d_off_c.get(), t.d_ioff.get(), t.interp.get(), r, t.Nc, t.rpart.get(), done);
  k_restrict_sum<<<(unsigned)std::min<int64_t>(152 * 4, (t.Nc + 255) / 256), 256, 0, s>>>(
      t.Nc, t.comp_c.get(), g.d_off.get(), t.d_off_c.get(), t.rpart.get(), t.rc.get(), t.rc32.get(), done);
  STOKES_LAUNCHED();
  const int64_t m = 2 * t.Nc;
  const int pc = g.prof.begin(kProfCoarseSolve, 4.0 * (double)m * (double)m, s);
  if (t.use_lu) {
    lu_solve_persistent<float>(g, t.lu.get(), m, t.perm.get(), t.tinv.get(), t.rc.get(), t.zc.get(),
                               t.trsv_work.get(), t.trsv_gen, done);
  } else {
    k_dense_gemv32_part<<<dim3((unsigned)((m + 1023) / 1024), kGemvSplits), 256, 0, s>>>(
        t.inv.get(), m, t.rc32.get(), t.gemv_part.get(), done);
    k_dense_gemv32_sum<<<(unsigned)std::min<int64_t>(152 * 4, (m + 255) / 256), 256, 0, s>>>(t.gemv_part.get(), m,
                                                                                           t.zc.get(), done);
  }
  g.prof.end(pc, s);
  STOKES_LAUNCHED();
  k_prolong<<<(unsigned)std::min<int64_t>(152 * 16, (g.N + 7) / 8), 256, 0, s>>>(
      g.N, g.outer, g.comp.get(), g.d_off.get(), t.d_off_c.get(), t.d_ioff.get(), t.interp.get(), r, t.rc.get(),
      t.zc.get(), z, t.h.get(), done);
  STOKES_LAUNCHED();
  bd_apply_pores_accumulate(g, t.h.get(), z, done, f32);
}

void precond_apply(Geom& g, const double* v, double* z, const int* done, bool f32) {
  if (g.tg.ready) {
    const TwoGrid& t = g.tg;
    const BlockDiag& b = g.bd;
    const double coarse = 4.0 * (double)(2 * t.Nc) * (double)(2 * t.Nc);
    const double transfers = 4.0 * (double)t.interp.n;
    const double pores = (f32 ? 4.0 : 8.0) * (double)(b.elem_off.empty() ? 0 : b.elem_off.back());
    const int pb = g.prof.begin(kProfBdApply, coarse + transfers + pores + 32.0 * (double)g.N, g.stream);
    twogrid_apply(g, v, z, done, f32);
    g.prof.end(pb, g.stream);
  } else if (g.cl.ready) {
    coarse_apply(g, v, z, done, f32);
  } else {
    bd_apply(g, v, z, done, f32);
  }
}

unsigned long long launches_twogrid() { return tu_launches(); }

}  // namespace stokes
