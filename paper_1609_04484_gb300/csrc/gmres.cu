// Restarted GMRES on the device (Sec. 4: GMRES of Saad and Schultz with a
// relative-residual tolerance; Sec. 4.1: preconditioning).
//
// Each Arnoldi step: z = P^-1 v_j (right) or t = A v_j (left), w = A z or
// P^-1 t, classical Gram-Schmidt applied twice (CGS2: dot products as
// warp-level reductions over chunks of the vector, deterministic two-level
// sums), normalisation, then one thread applies the Givens rotations,
// updates the least-squares residual and raises a device flag when it drops
// below tol. Every kernel of a cycle reads that flag and returns at once
// once it is set, so the host only synchronises at the end of each cycle to
// read the column count and the true residual.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kChunk = 2048;  // vector elements per CTA in the reductions
constexpr int kMaxRestart = 8192;
constexpr double kF32Refine = 1e4;   // residual reduction a double-float cycle may leave to the FP32 operator
constexpr double kDfResMargin = 0.3;  // target of a cycle started from a double-float residual, in units of tol

// partial[b * ldp + k] = sum_{i in chunk b} V[k][i] w[i], k < ncols
__global__ void __launch_bounds__(256)
k_dot_partial(const double* __restrict__ V, int64_t ldv, int ncols, const double* __restrict__ w, int64_t n,
              double* __restrict__ partial, int ldp, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double sw[kChunk];
  const int64_t i0 = blockIdx.x * (int64_t)kChunk;
  const int cn = (int)imin64(kChunk, n - i0);
  for (int e = threadIdx.x; e < cn; e += blockDim.x) sw[e] = w[i0 + e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = wid; k < ncols; k += nw) {
    const double* v = V + k * ldv + i0;
    double acc = 0.0;
    for (int e = lane; e < cn; e += 32) acc = fma(v[e], sw[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) partial[blockIdx.x * ldp + k] = acc;
  }
}

// h_k = sum_b partial[b][k] for k < ncols (fixed order), written to hvec and
// to the Hessenberg column (pass 0: =, pass 1: +=).
__global__ void k_reduce_partials(const double* __restrict__ partial, int ldp, int nblk, int ncols,
                                  double* __restrict__ hvec, double* __restrict__ hcol, int accumulate,
                                  const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncols) return;
  double h = 0.0;
  for (int b = 0; b < nblk; ++b) h += partial[(int64_t)b * ldp + k];
  hvec[k] = h;
  hcol[k] = accumulate ? hcol[k] + h : h;
}

// w -= sum_k h_k V[k]; normpart[b] = sum_{i in chunk b} w_i^2 (if given).
__global__ void __launch_bounds__(256)
k_orth_update(const double* __restrict__ V, int64_t ldv, int ncols, const double* __restrict__ hvec,
              double* __restrict__ w, int64_t n, double* __restrict__ normpart, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  __shared__ double sred[32];
  const int64_t i0 = blockIdx.x * (int64_t)kChunk;
  const int cn = (int)imin64(kChunk, n - i0);
  double sq = 0.0;
  for (int e = threadIdx.x; e < cn; e += blockDim.x) {
    const int64_t i = i0 + e;
    double acc = w[i];
    for (int k = 0; k < ncols; ++k) acc = fma(-hvec[k], V[k * ldv + i], acc);
    w[i] = acc;
    sq = fma(acc, acc, sq);
  }
  if (normpart) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if (lane == 0) sred[wid] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sred[q];
      normpart[blockIdx.x] = s;
    }
  }
}

// normpart[b] = sum_{i in chunk b} x_i^2 (and optionally r = f - t first)
__global__ void __launch_bounds__(256)
k_residual_norm(const double* __restrict__ f, const double* __restrict__ t, double* __restrict__ r, int64_t n,
                double* __restrict__ normpart) {
  count_launch();
  __shared__ double sred[32];
  const int64_t i0 = blockIdx.x * (int64_t)kChunk;
  const int cn = (int)imin64(kChunk, n - i0);
  double sq = 0.0;
  for (int e = threadIdx.x; e < cn; e += blockDim.x) {
    const int64_t i = i0 + e;
    const double v = t ? f[i] - t[i] : f[i];
    if (r) r[i] = v;
    sq = fma(v, v, sq);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if (lane == 0) sred[wid] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sred[q];
    normpart[blockIdx.x] = s;
  }
}

// scal[slot] = sqrt(sum normpart), scal[slot + 1] = 1 / that (0 if zero)
__global__ void k_norm_final(const double* __restrict__ normpart, int nblk, double* __restrict__ scal, int slot) {
  count_launch();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += normpart[b];
    const double nr = sqrt(s);
    scal[slot] = nr;
    scal[slot + 1] = nr > 0.0 ? 1.0 / nr : 0.0;
  }
}

// y = x * scal[slot]
__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ scal, int slot,
                        double* __restrict__ y, int64_t n, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  const double a = scal[slot];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * a;
}

// Start of a cycle: g = (beta, 0, ...), flags cleared.
__global__ void k_cycle_start(double* __restrict__ g, int m, const double* __restrict__ scal, int slot,
                              int* __restrict__ state) {
  count_launch();
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? scal[slot] : 0.0;
  if (threadIdx.x == 0) {
    state[0] = 0;
    state[1] = 0;
    state[2] = 0;
  }
}

// Column j of the Hessenberg matrix is complete except H[j+1][j]: finish it,
// apply the previous rotations, form the new one and test convergence.
// H is column-major with leading dimension m + 1.
__global__ void k_arnoldi_finish(int j, int m, const double* __restrict__ normpart, int nblk,
                                 double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                                 double* __restrict__ g, double* __restrict__ scal, int* __restrict__ state,
                                 double rhsnorm, double tol) {
  count_launch();
  if (state[0]) return;
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += normpart[b];
  const double hnext = sqrt(s);
  double* h = H + (int64_t)j * (m + 1);
  double colnorm = 0.0;
  for (int i = 0; i <= j; ++i) colnorm = fmax(colnorm, fabs(h[i]));
  h[j + 1] = hnext;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
    h[i] = t;
  }
  const double den = hypot(h[j], hnext);
  const double c = den > 0.0 ? h[j] / den : 1.0;
  const double sv = den > 0.0 ? hnext / den : 0.0;
  cs[j] = c;
  sn[j] = sv;
  h[j] = den;
  h[j + 1] = 0.0;
  g[j + 1] = -sv * g[j];
  g[j] = c * g[j];
  state[1] = j + 1;
  scal[0] = hnext > 0.0 ? 1.0 / hnext : 0.0;
  const double est = fabs(g[j + 1]) / rhsnorm;
  scal[4] = est;
  if (!isfinite(est) || !isfinite(hnext)) {
    state[2] = 1;
    state[0] = 1;
  } else if (est <= tol || hnext <= 1e-14 * colnorm) {  // converged or happy breakdown
    state[0] = 1;
  }
}

// y = R^-1 g over the completed columns: column-oriented back substitution
// by one CTA (after y_i is known, every thread updates its rows above).
__global__ void __launch_bounds__(256)
k_lsq_solve(const double* __restrict__ H, int m, const double* __restrict__ g, const int* __restrict__ state,
            double* __restrict__ y, double* __restrict__ work) {
  count_launch();
  const int jd = state[1];
  for (int i = threadIdx.x; i < jd; i += blockDim.x) work[i] = g[i];
  __syncthreads();
  for (int i = jd - 1; i >= 0; --i) {
    __shared__ double yi;
    if (threadIdx.x == 0) {
      const double d = H[(int64_t)i * (m + 1) + i];
      yi = d != 0.0 ? work[i] / d : 0.0;
      y[i] = yi;
    }
    __syncthreads();
    const double v = yi;
    for (int r = threadIdx.x; r < i; r += blockDim.x) work[r] -= H[(int64_t)i * (m + 1) + r] * v;
    __syncthreads();
  }
}

// t = sum_{k < jd} y_k V[k]
__global__ void k_combine(const double* __restrict__ V, int64_t ldv, const double* __restrict__ y,
                          const int* __restrict__ state, double* __restrict__ t, int64_t n) {
  count_launch();
  const int jd = state[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < jd; ++k) acc = fma(y[k], V[k * ldv + i], acc);
    t[i] = acc;
  }
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ z, int64_t n) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += z[i];
}

__global__ void k_copy(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  count_launch();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}

unsigned grid_for(int64_t n) { return (unsigned)imin64((n + 255) / 256, 152 * 16); }

}  // namespace

void apply_operator(Geom& g, const double* sigma, double* y, int precision, const int* done) {
  switch (precision) {
    case STOKES_FP64:
      dlp_apply_f64(g, (const double2*)sigma, (double2*)y, true, g.pos.get(), g.N, done);
      break;
    case STOKES_FP32:
      dlp_apply_f32(g, (const double2*)sigma, (double2*)y, true, g.pos.get(), g.N, done);
      break;
    case STOKES_DF64:
      dlp_apply_df64(g, (const double2*)sigma, (double2*)y, true, g.pos.get(), g.N, done);
      break;
    default:
      throw Error(STOKES_EINVAL, "precision not supported by this operator");
  }
}

// Workspace of the Krylov solver for restart length m (grows on demand).
static void krylov_alloc(Geom& g, int m) {
  Krylov& k = g.kr;
  const int64_t n = 2 * g.N;
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  const int ldp = std::max(m, k.m) + 1;
  if (k.m < m || k.n2 != n) {
    k.V.alloc((size_t)(m + 1) * n);
    k.Z.alloc(n);
    k.w.alloc(n);
    k.t.alloc(n);
    k.r.alloc(n);
    k.H.alloc((size_t)(m + 1) * m);
    k.cs.alloc(m);
    k.sn.alloc(m);
    k.g.alloc(m + 1);
    k.y.alloc(2 * (size_t)(m + 1));  // projection coefficients / y, then back-substitution work
    k.Zb.release();
    k.m = m;
    k.n2 = n;
  }
  k.partial.alloc((size_t)nblk * ldp + 8);
  k.scal.alloc(8);
  k.state.alloc(4);
  k.nblk = nblk;
  if (!k.ring_ready) {
    STOKES_CUDA(cudaMallocHost(&k.h_done, Krylov::kRing * sizeof(int)));
    for (auto& e : k.ev) STOKES_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    k.ring_ready = true;
  }
}

// ||v|| on the device, copied to the host (synchronises). Needs krylov_alloc.
static double device_norm(Geom& g, const double* v, int64_t n) {
  Krylov& k = g.kr;
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  k_residual_norm<<<nblk, 256, 0, g.stream>>>(v, nullptr, nullptr, n, k.partial.get());
  k_norm_final<<<1, 32, 0, g.stream>>>(k.partial.get(), nblk, k.scal.get(), 2);
  STOKES_LAUNCHED();
  double h = 0.0;
  STOKES_CUDA(cudaMemcpyAsync(&h, k.scal.get() + 2, sizeof(double), cudaMemcpyDeviceToHost, g.stream));
  STOKES_CUDA(cudaStreamSynchronize(g.stream));
  return h;
}

// inner = true (correction solves of the refinement): stop as soon as the
// Arnoldi estimate of the residual meets tol, without re-checking the true
// residual of the (single-precision) operator, whose rounding floor is near
// the inner tolerance.
static SolveResult gmres_core(Geom& g, const double* f, double* x, double tol, int restart, int max_iter,
                              int precision, int side, bool inner = false) {
  // single-precision block inverses for the FP32 and double-float operators
  // (a fixed linear preconditioner: the converged solution is unchanged);
  // STOKES_BD_F32=0 keeps the double-precision ones
  static const bool bd_f32_ok = !(std::getenv("STOKES_BD_F32") && std::getenv("STOKES_BD_F32")[0] == '0');
  const bool bd32 = (precision == STOKES_FP32 || precision == STOKES_DF64) && bd_f32_ok;
  const bool trace = std::getenv("STOKES_TRACE") != nullptr;
  require(restart >= 1 && restart <= kMaxRestart, "restart must be in [1, 8192]");
  require(max_iter >= 1, "max_iter must be >= 1");
  require(tol > 0 && std::isfinite(tol), "tol must be > 0");
  const bool use_pc = g.bd.ready || g.tg.ready;
  const bool left = side == STOKES_PC_LEFT && use_pc;
  require(!(left && g.tg.ready), "the two-grid preconditioner is applied from the right only");
  cudaStream_t s = g.stream;
  const int64_t n = 2 * g.N;
  const int m = restart;
  Krylov& k = g.kr;
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  const int ldp = m + 1;
  krylov_alloc(g, m);
  const bool use_pc_any = g.bd.ready || g.tg.ready;
  if (use_pc_any && side != STOKES_PC_LEFT) k.Zb.alloc((size_t)m * n);
  double* normpart = k.partial.get();  // reductions of norms share the partial buffer
  DevBuf<double> np2;                  // separate buffer for the norm partials inside a step
  np2.alloc(nblk);
  int* state = k.state.get();
  const unsigned gv = grid_for(n);

  SolveResult res;
  const double fnorm = device_norm(g, f, n);
  if (fnorm == 0.0) {
    STOKES_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    STOKES_CUDA(cudaStreamSynchronize(s));
    return res;
  }
  double rhsnorm = fnorm;
  if (left) {
    precond_apply(g, f, k.t.get(), nullptr, bd32);
    rhsnorm = device_norm(g, k.t.get(), n);
  }
  const double xnorm0 = device_norm(g, x, n);
  bool x_is_zero = xnorm0 == 0.0;
  int iters = 0;
  // r = f - A x with the operator of precision p (x = 0: r = f); |r|
  auto residual = [&](int p) {
    if (x_is_zero) {
      k_residual_norm<<<nblk, 256, 0, s>>>(f, nullptr, k.r.get(), n, normpart);
    } else {
      apply_operator(g, x, k.t.get(), p, nullptr);
      k_residual_norm<<<nblk, 256, 0, s>>>(f, k.t.get(), k.r.get(), n, normpart);
    }
    k_norm_final<<<1, 32, 0, s>>>(normpart, nblk, k.scal.get(), 2);
    STOKES_LAUNCHED();
    double rn = 0.0;
    STOKES_CUDA(cudaMemcpyAsync(&rn, k.scal.get() + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    STOKES_CUDA(cudaStreamSynchronize(s));
    return rn;
  };
  // Double-float solves (right preconditioner): the residual a restart
  // starts from is taken with the double-float operator, whose error (a
  // small multiple of 2^-44 times the sum of the terms' magnitudes,
  // amplified by large densities) is small against a residual well above
  // the tolerance;
  // convergence is decided by the native FP64 operator only, which
  // recomputes the residual whenever the double-float one is at the
  // tolerance or stopped falling (from then on every restart uses FP64).
  // A cycle that starts from a double-float residual aims kDfResMargin
  // below the tolerance, to cover that residual's error.
  // A refinement cycle (started from a double-float residual) that reports
  // convergence goes straight to the FP64 residual: its double-float one
  // would only confirm what the FP64 one decides.
  bool df_res = precision == STOKES_DF64 && !inner && !left;
  double df_prev = -1.0;
  bool from_df = false;
  bool refined_converged = false;  // the last cycle started from a double-float residual and converged
  while (true) {
    // true residual r = f - A x
    if (refined_converged) df_res = false;
    const int rprec = (precision == STOKES_DF64 && !inner) ? (df_res ? STOKES_DF64 : STOKES_FP64) : precision;
    double rn = residual(rprec);
    from_df = false;
    if (rprec == STOKES_DF64 && !x_is_zero) {
      const double rel = rn / fnorm;
      if (rel <= tol || (df_prev > 0.0 && rel > 0.5 * df_prev) || iters >= max_iter || !std::isfinite(rel)) {
        df_res = false;
        rn = residual(STOKES_FP64);
      } else {
        from_df = true;
        df_prev = rel;
      }
    }
    res.relres = rn / fnorm;
    double beta = rn;
    if (left) {
      precond_apply(g, k.r.get(), k.Z.get(), nullptr, bd32);
      k_copy<<<gv, 256, 0, s>>>(k.r.get(), k.Z.get(), n);
      beta = device_norm(g, k.r.get(), n);
    }
    res.pc_relres = beta / rhsnorm;
    res.iters = iters;
    if (!std::isfinite(res.relres) || !std::isfinite(res.pc_relres)) {
      res.status = STOKES_EBREAKDOWN;
      return res;
    }
    const bool conv = left ? res.pc_relres <= tol : res.relres <= tol;
    if (conv) return res;
    if (iters >= max_iter) {
      res.status = STOKES_ENOTCONV;
      return res;
    }
    // v_0 = r / beta: the last norm computed (of r, or of P^-1 r) left
    // beta and 1 / beta in scal[2], scal[3]
    k_scale<<<gv, 256, 0, s>>>(k.r.get(), k.scal.get(), 3, k.V.get(), n, nullptr);
    k_cycle_start<<<1, 256, 0, s>>>(k.g.get(), m, k.scal.get(), 2, state);
    STOKES_LAUNCHED();
    // A double-float cycle that starts within kF32Refine tol of the tolerance
    // only has to reduce the residual by at most kF32Refine: a refinement
    // step, which the FP32 operator does at a seventh of the cost; the
    // FP64 residual decides convergence.
    const int op_prec =
        (precision == STOKES_DF64 && !inner && !left && !x_is_zero && res.relres <= kF32Refine * tol) ? STOKES_FP32
                                                                                                      : precision;
    const double ctol = from_df ? kDfResMargin * tol : tol;
    const int mc = std::min(m, max_iter - iters);
    std::vector<size_t> iter_first(mc + 1, g.prof.entries.size());
    for (int j = 0; j < mc; ++j) {
      iter_first[j] = g.prof.entries.size();
      double* vj = k.V.get() + (int64_t)j * n;
      double* vnext = k.V.get() + (int64_t)(j + 1) * n;  // k.w normalised into it
      if (!use_pc) {
        apply_operator(g, vj, k.w.get(), op_prec, state);
      } else if (!left) {
        // flexible GMRES: keep z_j = P^-1 v_j, the iterate is x0 + Z y
        double* zj = k.Zb.get() + (int64_t)j * n;
        precond_apply(g, vj, zj, state, bd32);
        apply_operator(g, zj, k.w.get(), op_prec, state);
      } else {
        apply_operator(g, vj, k.t.get(), op_prec, state);
        precond_apply(g, k.t.get(), k.w.get(), state, bd32);
      }
      const int pa = g.prof.begin(kProfArnoldi, 8.0 * n * (4.0 * (j + 1) + 4.0), s);
      for (int pass = 0; pass < 2; ++pass) {
        k_dot_partial<<<nblk, 256, 0, s>>>(k.V.get(), n, j + 1, k.w.get(), n, k.partial.get(), ldp, state);
        k_reduce_partials<<<(j + 1 + 255) / 256, 256, 0, s>>>(k.partial.get(), ldp, nblk, j + 1, k.y.get(),
                                                              k.H.get() + (int64_t)j * (m + 1), pass, state);
        k_orth_update<<<nblk, 256, 0, s>>>(k.V.get(), n, j + 1, k.y.get(), k.w.get(), n,
                                           pass ? np2.get() : nullptr, state);
      }
      k_arnoldi_finish<<<1, 32, 0, s>>>(j, m, np2.get(), nblk, k.H.get(), k.cs.get(), k.sn.get(), k.g.get(),
                                        k.scal.get(), state, rhsnorm, ctol);
      k_scale<<<gv, 256, 0, s>>>(k.w.get(), k.scal.get(), 0, vnext, n, state);
      g.prof.end(pa, s);
      STOKES_LAUNCHED();
      // The host runs at most kAhead iterations ahead of the GPU and stops
      // enqueueing once the GPU reports convergence: the done flag after
      // each iteration goes to pinned memory behind an event, and the flag
      // of iteration j - kAhead is read once that event has completed (the
      // GPU still has kAhead iterations queued, so it does not idle).
      constexpr int kAhead = 16;
      static_assert(Krylov::kRing > kAhead, "ring must outlast the run-ahead");
      STOKES_CUDA(cudaMemcpyAsync(k.h_done + j % Krylov::kRing, state, sizeof(int), cudaMemcpyDeviceToHost, s));
      STOKES_CUDA(cudaEventRecord(k.ev[j % Krylov::kRing], s));
      if (j >= kAhead) {
        const int jj = j - kAhead;
        STOKES_CUDA(cudaEventSynchronize(k.ev[jj % Krylov::kRing]));
        if (k.h_done[jj % Krylov::kRing]) break;
      }
      if (trace && (j + 1) % 100 == 0) {
        double est = 0.0;
        int st = 0;
        STOKES_CUDA(cudaMemcpyAsync(&est, k.scal.get() + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
        STOKES_CUDA(cudaMemcpyAsync(&st, state, sizeof(int), cudaMemcpyDeviceToHost, s));
        STOKES_CUDA(cudaStreamSynchronize(s));
        std::fprintf(stderr, "[stokes]   iteration %d: residual estimate %.3e\n", iters + j + 1, est);
        if (st) break;
      }
    }
    iter_first[mc] = g.prof.entries.size();
    int hstate[3] = {0, 0, 0};
    STOKES_CUDA(cudaMemcpyAsync(hstate, state, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    k_lsq_solve<<<1, 256, 0, s>>>(k.H.get(), m, k.g.get(), state, k.y.get(), k.y.get() + (m + 1));
    k_combine<<<gv, 256, 0, s>>>((use_pc && !left) ? k.Zb.get() : k.V.get(), n, k.y.get(), state, k.t.get(), n);
    k_axpy<<<gv, 256, 0, s>>>(x, k.t.get(), n);
    STOKES_LAUNCHED();
    STOKES_CUDA(cudaStreamSynchronize(s));
    bd_check_barrier(g);
    // launches of iterations after convergence returned at once: not timed work
    for (size_t e = iter_first[hstate[1]]; e < iter_first[mc]; ++e) g.prof.entries[e].valid = false;
    iters += hstate[1];
    x_is_zero = false;
    if (std::getenv("STOKES_TRACE"))
      std::fprintf(stderr,
                   "[stokes]   cycle: %d columns, converged flag %d, breakdown %d, relres at start %.3e (%s), "
                   "operator %s\n",
                   hstate[1], hstate[0], hstate[2], res.relres, from_df ? "df64 residual" : "true residual",
                   op_prec == STOKES_FP32 ? "fp32" : (op_prec == STOKES_DF64 ? "df64" : "fp64"));
    refined_converged = from_df && hstate[0] && !hstate[2];
    if (inner && hstate[0] && !hstate[2]) {
      res.iters = iters;
      res.relres = res.pc_relres = -1.0;  // not evaluated
      return res;
    }
    if (hstate[2]) {
      res.iters = iters;
      res.status = STOKES_EBREAKDOWN;
      return res;
    }
    if (hstate[1] == 0) {  // no progress possible
      res.iters = iters;
      res.status = STOKES_ENOTCONV;
      return res;
    }
  }
}

}  // namespace stokes

namespace stokes {

// Mixed-precision iterative refinement: the outer residual r = f - A x uses
// the native FP64 operator; each correction solves A d = r
// with GMRES on the FP32 operator until its Arnoldi residual estimate drops
// below max(1e-4, tol / (2 |r| / |f|)) (Arnoldi, Givens and least squares
// stay FP64), then x += d. STOKES_TRACE=1 prints each refinement step.
static SolveResult ir_solve(Geom& g, const double* f, double* x, double tol, int restart, int max_iter, int side) {
  cudaStream_t s = g.stream;
  const int64_t n = 2 * g.N;
  DevBuf<double> r, d, t;
  r.alloc(n);
  d.alloc(n);
  t.alloc(n);
  require(restart >= 1 && restart <= kMaxRestart, "restart must be in [1, 8192]");
  krylov_alloc(g, restart);  // device_norm and the residual below use its buffers
  SolveResult res;
  const double fnorm = device_norm(g, f, n);
  if (fnorm == 0.0) {
    STOKES_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    STOKES_CUDA(cudaStreamSynchronize(s));
    return res;
  }
  const unsigned gv = grid_for(n);
  int iters = 0;
  for (int outer = 0;; ++outer) {
    apply_operator(g, x, t.get(), STOKES_FP64, nullptr);
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    k_residual_norm<<<nblk, 256, 0, s>>>(f, t.get(), r.get(), n, g.kr.partial.get());
    k_norm_final<<<1, 32, 0, s>>>(g.kr.partial.get(), nblk, g.kr.scal.get(), 2);
    STOKES_LAUNCHED();
    double rn = 0.0;
    STOKES_CUDA(cudaMemcpyAsync(&rn, g.kr.scal.get() + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    STOKES_CUDA(cudaStreamSynchronize(s));
    res.relres = rn / fnorm;
    res.pc_relres = res.relres;
    res.iters = iters;
    if (!std::isfinite(res.relres)) {
      res.status = STOKES_EBREAKDOWN;
      return res;
    }
    if (res.relres <= tol) return res;
    if (iters >= max_iter || outer >= 30) {
      res.status = STOKES_ENOTCONV;
      return res;
    }
    STOKES_CUDA(cudaMemsetAsync(d.get(), 0, n * sizeof(double), s));
    const double inner_tol = std::max(1e-4, 0.5 * tol / res.relres);
    SolveResult in = gmres_core(g, r.get(), d.get(), inner_tol, restart, max_iter - iters, STOKES_FP32, side,
                                /*inner=*/true);
    if (std::getenv("STOKES_TRACE"))
      std::fprintf(stderr, "[stokes] refinement step %d: relres %.3e, inner tol %.1e, inner iterations %d (status %d)\n",
                   outer, res.relres, inner_tol, in.iters, in.status);
    iters += in.iters;
    if (in.status == STOKES_EBREAKDOWN) {
      res.status = in.status;
      res.iters = iters;
      return res;
    }
    k_axpy<<<gv, 256, 0, s>>>(x, d.get(), n);
    STOKES_LAUNCHED();
  }
}

SolveResult gmres_solve(Geom& g, const double* f, double* x, double tol, int restart, int max_iter, int precision,
                        int side) {
  if (precision == STOKES_MIXED_IR) return ir_solve(g, f, x, tol, restart, max_iter, side);
  return gmres_core(g, f, x, tol, restart, max_iter, precision, side);
}

}  // namespace stokes

namespace stokes {
unsigned long long launches_gmres() { return tu_launches(); }
}  // namespace stokes
