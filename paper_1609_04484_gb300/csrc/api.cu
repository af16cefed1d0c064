// extern "C" entry points of libstokes (declared in include/stokes.h).
// Each call validates its arguments, stages host arrays through handle-owned
// device buffers, runs the device path and maps failures to status codes.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace stokes {
Geom* geometry_create(const double*, const double*, const double*, const double*, const int64_t*, int, int,
                      const double*, void*);
bool is_device_pointer(const void* p);
}  // namespace stokes

namespace {

thread_local std::string g_last_error;

template <class F>
int guarded(F&& fn) {
  try {
    fn();
    g_last_error.clear();
    return STOKES_OK;
  } catch (const stokes::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return STOKES_ECUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return STOKES_ECUDA;
  }
}

using stokes::DevBuf;
using stokes::Geom;

}  // namespace

int stokes::guarded_call(void (*fn)(void*), void* ctx) {
  return guarded([&] { fn(ctx); });
}

namespace {

// A device view of a caller array: the caller's pointer if it is device
// memory, else a handle-owned staging buffer filled from the host.
const double* input_view(Geom& g, const double* p, size_t count, DevBuf<double2>& stage) {
  if (stokes::is_device_pointer(p)) return p;
  stage.alloc((count + 1) / 2);
  STOKES_CUDA(cudaMemcpyAsync(stage.get(), p, count * sizeof(double), cudaMemcpyHostToDevice, g.stream));
  return (const double*)stage.get();
}

double* output_view(Geom& g, double* p, size_t count, DevBuf<double2>& stage, bool& staged) {
  staged = !stokes::is_device_pointer(p);
  if (!staged) return p;
  stage.alloc((count + 1) / 2);
  return (double*)stage.get();
}

void finish_output(Geom& g, double* user, const double* dev, size_t count, bool staged) {
  if (staged) {
    STOKES_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(double), cudaMemcpyDeviceToHost, g.stream));
    STOKES_CUDA(cudaStreamSynchronize(g.stream));
  }
}

Geom& handle(stokes_geom* h) {
  stokes::require(h && h->g, "null handle");
  return *h->g;
}

}  // namespace

extern "C" {

int stokes_geometry_create(const double* nodes, const double* normals, const double* weights,
                           const double* curvature, const int64_t* offsets, int n_comp, int outer_comp,
                           const double* centres, void* stream, stokes_geom** out) {
  return guarded([&] {
    stokes::require(out != nullptr, "out is null");
    Geom* g = stokes::geometry_create(nodes, normals, weights, curvature, offsets, n_comp, outer_comp, centres,
                                      stream);
    *out = new stokes_geom{g};
  });
}

int stokes_geometry_destroy(stokes_geom* h) {
  return guarded([&] {
    if (!h) return;
    if (h->g) {
      cudaStreamSynchronize(h->g->stream);
      delete h->g;
    }
    delete h;
  });
}

int64_t stokes_geometry_num_nodes(const stokes_geom* h) { return (h && h->g) ? h->g->N : -1; }

int stokes_matvec(stokes_geom* h, const double* sigma, double* y, int precision) {
  return guarded([&] {
    Geom& g = handle(h);
    stokes::require(sigma && y, "null array argument");
    stokes::require(sigma != y, "sigma and y may not alias");
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64,
                    "precision must be FP64, FP32 or DF64");
    const size_t n = 2 * g.N;
    const double* s = input_view(g, sigma, n, g.stage_in);
    bool staged;
    double* yo = output_view(g, y, n, g.stage_out, staged);
    stokes::apply_operator(g, s, yo, precision, nullptr);
    STOKES_LAUNCHED();
    finish_output(g, y, yo, n, staged);
  });
}

int stokes_precond_setup_twogrid(stokes_geom* h, int coarsen) {
  return stokes_precond_setup_twogrid_ex(h, coarsen, STOKES_TG_COARSE_AUTO);
}

int stokes_precond_setup_twogrid_ex(stokes_geom* h, int coarsen, int coarse_mode) {
  return guarded([&] {
    Geom& g = handle(h);
    stokes::require(coarse_mode == STOKES_TG_COARSE_AUTO || coarse_mode == STOKES_TG_COARSE_INVERSE ||
                        coarse_mode == STOKES_TG_COARSE_LU,
                    "unknown coarse_mode");
    g.tg.ready = false;
    g.bd.ready = false;
    g.cl.ready = false;
    stokes::twogrid_setup(g, coarsen, coarse_mode);
  });
}

int stokes_precond_apply(stokes_geom* h, const double* v, double* z) {
  return stokes_precond_apply_prec(h, v, z, STOKES_FP64);
}

int stokes_precond_apply_prec(stokes_geom* h, const double* v, double* z, int precision) {
  return guarded([&] {
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32, "precision must be FP64 or FP32");
    Geom& g = handle(h);
    stokes::require(v && z && v != z, "bad array arguments");
    stokes::require(g.bd.ready || g.tg.ready, "preconditioner not set up", STOKES_ESTATE);
    const size_t n = 2 * g.N;
    const double* vi = input_view(g, v, n, g.stage_in);
    bool staged;
    double* zo = output_view(g, z, n, g.stage_out, staged);
    stokes::precond_apply(g, vi, zo, nullptr, precision == STOKES_FP32);
    STOKES_LAUNCHED();
    finish_output(g, z, zo, n, staged);
    stokes::bd_check_barrier(g);
  });
}

int stokes_gmres_solve(stokes_geom* h, const double* f, double tol, int restart, int max_iter, int precision,
                       int pc_side, double* sigma, int* iters_out, double* true_relres_out,
                       double* pc_relres_out) {
  int solve_status = STOKES_OK;
  const int rc = guarded([&] {
    Geom& g = handle(h);
    stokes::require(f && sigma && f != sigma, "bad array arguments");
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64 ||
                        precision == STOKES_MIXED_IR,
                    "precision must be FP64, FP32, DF64 or MIXED_IR");
    stokes::require(pc_side == STOKES_PC_RIGHT || pc_side == STOKES_PC_LEFT, "bad pc_side");
    const size_t n = 2 * g.N;
    const double* fi = input_view(g, f, n, g.stage_in);
    // sigma is read (initial guess) and written: work in a device copy when on the host
    bool staged = !stokes::is_device_pointer(sigma);
    double* x = sigma;
    if (staged) {
      g.stage_out.alloc(g.N);
      x = (double*)g.stage_out.get();
      STOKES_CUDA(cudaMemcpyAsync(x, sigma, n * sizeof(double), cudaMemcpyHostToDevice, g.stream));
    }
    stokes::SolveResult r = stokes::gmres_solve(g, fi, x, tol, restart, max_iter, precision, pc_side);
    finish_output(g, sigma, x, n, staged);
    if (iters_out) *iters_out = r.iters;
    if (true_relres_out) *true_relres_out = r.relres;
    if (pc_relres_out) *pc_relres_out = r.pc_relres;
    solve_status = r.status;
  });
  if (rc != STOKES_OK) return rc;
  if (solve_status != STOKES_OK) {
    g_last_error = solve_status == STOKES_ENOTCONV ? "GMRES reached max_iter" : "GMRES: non-finite residual";
  }
  return solve_status;
}

int stokes_eval_velocity(stokes_geom* h, const double* sigma, const double* targets, int64_t n_targets, double* u,
                         int precision) {
  return guarded([&] {
    Geom& g = handle(h);
    stokes::require(sigma && targets && u, "null array argument");
    stokes::require(n_targets >= 0, "n_targets must be >= 0");
    stokes::require(precision == STOKES_FP64 || precision == STOKES_FP32 || precision == STOKES_DF64,
                    "precision must be FP64, FP32 or DF64");
    if (n_targets == 0) return;
    const double* s = input_view(g, sigma, 2 * g.N, g.stage_in);
    const double* t = input_view(g, targets, 2 * n_targets, g.stage_tgt);
    bool staged;
    double* uo = output_view(g, u, 2 * n_targets, g.stage_out, staged);
    const auto* sv = (const double2*)s;
    const auto* tv = (const double2*)t;
    if (precision == STOKES_FP64) stokes::dlp_apply_f64(g, sv, (double2*)uo, false, tv, n_targets, nullptr);
    else if (precision == STOKES_FP32) stokes::dlp_apply_f32(g, sv, (double2*)uo, false, tv, n_targets, nullptr);
    else stokes::dlp_apply_df64(g, sv, (double2*)uo, false, tv, n_targets, nullptr);
    finish_output(g, u, uo, 2 * n_targets, staged);
  });
}

int stokes_profile_enable(stokes_geom* h, int on) {
  return guarded([&] {
    Geom& g = handle(h);
    STOKES_CUDA(cudaStreamSynchronize(g.stream));
    g.prof.clear();
    g.prof.on = on != 0;
  });
}

int stokes_profile_read(stokes_geom* h, int kind, int64_t* launches, double* total_ms, double* total_units) {
  return guarded([&] {
    Geom& g = handle(h);
    stokes::require(kind >= 0 && kind < stokes::kProfKinds, "unknown profile kind");
    STOKES_CUDA(cudaStreamSynchronize(g.stream));
    int64_t cnt = 0;
    double ms = 0.0, units = 0.0;
    for (const auto& e : g.prof.entries) {
      if (e.kind != kind || !e.valid) continue;
      float t = 0.f;
      STOKES_CUDA(cudaEventElapsedTime(&t, e.a, e.b));
      ++cnt;
      ms += t;
      units += e.units;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    if (total_units) *total_units = units;
  });
}

int64_t stokes_kernel_launches(void) {
  try {
    return (int64_t)(stokes::launches_geometry() + stokes::launches_dlp_f64() + stokes::launches_dlp_f32() +
                     stokes::launches_dlp_df64() + stokes::launches_bd() + stokes::launches_bd_trsv() + stokes::launches_bd_inv32() + stokes::launches_twogrid() +
                     stokes::launches_gmres() + stokes::launches_batch() + stokes::launches_noalloc() +
                     stokes::launches_mlp() + stokes::launches_coarse() + stokes::launches_tc_gemm());
  } catch (...) {
    return -1;
  }
}

int stokes_batch_matvec(stokes_geom* const* geoms, int n_geoms, int n_rhs, const double* const* sigma,
                        double* const* y, int precision) {
  return guarded([&] {
    stokes::require(geoms && sigma && y, "null argument");
    stokes::require(n_geoms >= 1, "n_geoms must be >= 1");
    std::vector<Geom*> gs(n_geoms);
    for (int k = 0; k < n_geoms; ++k) gs[k] = &handle(geoms[k]);
    stokes::batch_matvec(gs.data(), n_geoms, n_rhs, sigma, y, precision);
  });
}

int stokes_batch_solve(stokes_geom* const* geoms, int n_geoms, int n_rhs, const double* const* f, double tol,
                       int restart, int max_iter, int precision, double* const* sigma, int* iters,
                       double* relres, int* status) {
  return guarded([&] {
    stokes::require(geoms && f && sigma, "null argument");
    stokes::require(n_geoms >= 1, "n_geoms must be >= 1");
    std::vector<Geom*> gs(n_geoms);
    for (int k = 0; k < n_geoms; ++k) gs[k] = &handle(geoms[k]);
    stokes::batch_solve(gs.data(), n_geoms, n_rhs, f, tol, restart, max_iter, precision, sigma, iters, relres,
                        status);
  });
}

int stokes_rcp_f64(const double* x, double* y, int64_t n, void* stream) {
  return guarded([&] {
    stokes::require(n >= 0, "n must be >= 0");
    if (n == 0) return;
    stokes::require(x && y && stokes::is_device_pointer(x) && stokes::is_device_pointer(y),
                    "x and y must be device arrays");
    stokes::rcp_newton_apply(x, y, n, (cudaStream_t)stream);
  });
}

const char* stokes_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
