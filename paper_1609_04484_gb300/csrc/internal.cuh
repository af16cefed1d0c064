// Internal declarations of libstokes: the geometry handle, device buffers,
// error handling and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "stokes.h"

namespace stokes {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define STOKES_CUDA(call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::stokes::Error(e_ == cudaErrorMemoryAllocation ? STOKES_ENOMEM : STOKES_ECUDA, \
                            std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

#define STOKES_LAUNCHED() STOKES_CUDA(cudaGetLastError())

inline void require(bool ok, const std::string& msg, int code = STOKES_EINVAL) {
  if (!ok) throw Error(code, msg);
}

// Owning device buffer (cudaMalloc / cudaFree), grows on demand.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    STOKES_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  T* get() const { return p; }
};

// Device-side launch counter, one per translation unit: thread 0 of block 0
// of every kernel adds one when the kernel starts.
static __device__ unsigned long long g_tu_launches;
__device__ __forceinline__ void count_launch() {
  if ((threadIdx.x | threadIdx.y | blockIdx.x | blockIdx.y | blockIdx.z) == 0) atomicAdd(&g_tu_launches, 1ull);
}
static inline unsigned long long tu_launches() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_tu_launches, sizeof(v));
  return v;
}

__host__ __device__ inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr double kPi = 3.14159265358979323846;
constexpr double kInvPi = 0.31830988618379067154;
constexpr double kInv4Pi = 0.07957747154594766788;

// Per-block data of the block-diagonal preconditioner.
struct BlockDiag {
  bool ready = false;
  std::vector<int64_t> rows;      // 2 n_k per component
  std::vector<int64_t> elem_off;  // offset of each block's m x m matrix (prefix sums of m^2)
  std::vector<int64_t> piv_off;   // offset of each block's pivots (prefix sums of m)
  std::vector<int> small_ids;     // factorised and inverted by one CTA each
  std::vector<int> inv_ids;       // applied through their explicit inverse
  std::vector<int> tri_ids;       // applied by blocked triangular solves
  int64_t max_inv_rows = 0;
  DevBuf<double> lu;              // column-major LU in place (unit-lower L below the diagonal)
  DevBuf<double> inv;             // explicit inverses (same offsets as lu)
  DevBuf<int> piv;                // interchanges: row c was swapped with piv[c]
  DevBuf<int> perm;               // row r of P A is row perm[r] of A
  DevBuf<int64_t> d_elem_off, d_piv_off, d_rows, d_node_off;
  DevBuf<int> d_small_ids, d_inv_ids;
  DevBuf<int> status;             // 0 ok, 1 zero pivot
  DevBuf<double> pv, ivp;         // pivot search scratch
  DevBuf<int64_t> pi;
  // single-precision copies for the inner solves of the refinement
  DevBuf<float> inv32;            // inverses (same offsets as lu)
  DevBuf<float> lu32;             // factors of the triangular-solve blocks, packed
  std::vector<int64_t> lu32_off;  // per component offset into lu32 (-1 if none)
  DevBuf<int> d_tri_ids;          // blocks applied by triangular solves in FP64
  int64_t max_tri_rows = 0;
  DevBuf<unsigned long long> trsv_work;  // tagged solutions of the persistent triangular solves
  DevBuf<double> tinv64;          // diagonal-tile inverses of the FP64 triangular-solve blocks
  std::vector<int64_t> tinv_off;  // per component offset into tinv64 (-1 if none)
  DevBuf<unsigned> barrier;       // count, generation, sticky error
  unsigned trsv_gen = 0;          // generation of the last solve tagged in trsv_work (0: buffer zeroed)
};

// Workspace of the Krylov solver.
struct Krylov {
  int m = 0;          // restart length the buffers are sized for
  int64_t n2 = 0;     // vector length 2N
  DevBuf<double> V, Z, Zb, w, t, x, f, r, partial, H, cs, sn, g, y, scal;
  DevBuf<int> state;  // [0] done, [1] columns completed, [2] breakdown
  int nblk = 0;
  // bounded run-ahead of the host: the done flag after each iteration is
  // copied to pinned memory behind an event (a ring of kRing slots)
  static constexpr int kRing = 32;
  int* h_done = nullptr;
  cudaEvent_t ev[kRing] = {};
  bool ring_ready = false;
  Krylov() = default;
  Krylov(const Krylov&) = delete;
  Krylov& operator=(const Krylov&) = delete;
  ~Krylov() {
    if (h_done) cudaFreeHost(h_done);
    if (ring_ready)
      for (auto e : ev) cudaEventDestroy(e);
  }
};

// Kernel timing: launches of each kernel class bracketed by CUDA events on
// the handle's stream while enabled; read back (synchronising) on demand.
enum ProfKind {
  kProfPairsF64 = 0, kProfPairsF32 = 1, kProfPairsDF64 = 2, kProfEpilogue = 3,
  kProfBdApply = 4, kProfArnoldi = 5, kProfBdSetup = 6, kProfLuGemm = 7, kProfLuPanel = 8,
  kProfCoarseSolve = 9, kProfKinds = 10
};
struct ProfEntry {
  cudaEvent_t a, b;
  int kind;
  double units;
  bool valid;
};
struct Prof {
  bool on = false;
  std::vector<ProfEntry> entries;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  cudaEvent_t take() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      STOKES_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
  int begin(int kind, double units, cudaStream_t s) {
    if (!on) return -1;
    ProfEntry e{take(), take(), kind, units, true};
    STOKES_CUDA(cudaEventRecord(e.a, s));
    entries.push_back(e);
    return (int)entries.size() - 1;
  }
  void end(int idx, cudaStream_t s) {
    if (idx >= 0) STOKES_CUDA(cudaEventRecord(entries[idx].b, s));
  }
  void clear() {
    entries.clear();
    pool_used = 0;
  }
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Two-grid preconditioner: an exact solve with the operator on every q-th
// node (dense float LU) plus the pores' diagonal blocks on the remainder.
struct TwoGrid {
  bool ready = false;
  int q = 0;
  int64_t Nc = 0;
  std::vector<int64_t> off_c;      // coarse component offsets
  DevBuf<int64_t> d_off_c;
  DevBuf<int64_t> d_ioff;          // per component: offset of its interpolation matrix
  DevBuf<float> interp;            // row-major n_f x n_c matrices
  DevBuf<double2> pos_c, nrm_c;
  DevBuf<double> w_c;
  DevBuf<double4_32a> selfc_c;
  DevBuf<int> comp_c;
  DevBuf<float> lu;                // 2Nc x 2Nc, column-major, LU in place (setup only)
  DevBuf<float> inv;               // its explicit inverse
  DevBuf<int> piv, perm, status;
  DevBuf<double> rc, zc, h;
  DevBuf<float> rc32;
  DevBuf<float> gemv_part;         // column-split partial sums of the coarse apply
  DevBuf<float2> rpart;            // row-chunk partial sums of the restriction
  bool use_lu = false;             // coarse solve by the LU factors (else the explicit inverse)
  DevBuf<unsigned> barrier;        // grid barrier of the cooperative panel factorisation
  int64_t max_chunks = 0;
  DevBuf<unsigned long long> trsv_work;  // tagged solutions of the coarse triangular solves
  unsigned trsv_gen = 0;                 // generation of the last solve tagged in trsv_work (0: buffer zeroed)
  DevBuf<float> tinv;              // diagonal-tile inverses of the coarse LU factors
  DevBuf<int> d_pore_ids;
};

// Launch shape of a pair kernel: a compiled variant (threads per CTA,
// targets per thread, sources per shared-memory tile) and the number of CTAs
// per SM that the source splitting aims for.
struct PairVariant {
  int threads, tpt, tile;
};
struct PairShape {
  int variant = -1;     // < 0: not chosen (defaults or the tuner's cache decide)
  int ctas_per_sm = 4;
};

// Coarse level of the two-level preconditioner (rigid-motion modes of each
// pore; see coarse.cu).
struct CoarseLevel {
  bool ready = false;
  bool learned = false;
  int M = 0;                   // pores
  std::vector<int> pores;      // component of each pore
  DevBuf<int> d_pores;         // component of pore p
  DevBuf<int> pore_of;         // pore number of each component (-1 for the wall)
  DevBuf<double> stats;        // per pore: L = sum w, r = L / 2 pi, sum w dx, sum w dy, sum w |d|^2
  DevBuf<double> Y;            // A Z, 2N x 3M column-major
  DevBuf<double> C;            // coarse inverse, 3M x 3M row-major
  DevBuf<double> rc, c, t;     // Z^T W r, C rc, r - Y c
};

struct Geom {
  int64_t N = 0;
  int n_comp = 0;
  int outer = -1;
  int M = 0;  // number of pores
  cudaStream_t stream = nullptr;
  std::vector<int64_t> off;      // host copy of offsets
  std::vector<double> centre_h;  // host copy of centres (2 per component)

  // FP64 node data
  DevBuf<double4_32a> src;    // x, y, w n_x / pi, w n_y / pi
  DevBuf<double2> pos;    // x, y
  DevBuf<double2> nrm;    // n
  DevBuf<double> w;       // weights
  DevBuf<double4_32a> selfc;  // t_x, t_y, -kappa w / (2 pi), w
  DevBuf<int> comp;       // component of each node
  DevBuf<int64_t> d_off;  // offsets
  DevBuf<double2> centre; // completion centre per component
  DevBuf<int> pore_ids;   // the M pore components

  // Float copies for the FP32 and double-float kernels: every double v is
  // split into hi = fl32(v) and lo = fl32(v - hi).
  DevBuf<float4> f32_src;   // x_hi, y_hi, (w n_x / pi)_hi, (w n_y / pi)_hi
  DevBuf<float2> f32_lo;    // x_lo, y_lo
  DevBuf<float2> df_grid;   // x, y rounded to multiples of 2^-8 (exact differences)
  DevBuf<float4> df_pos;    // remainder x - grid as a float pair: rx_hi, ry_hi, rx_lo, ry_lo
  DevBuf<float4> df_a;      // a_x hi, a_y hi, a_x lo, a_y lo  (a = w n / pi)

  // log |x_i - c_k|^2 for every node and pore (double-float completion)
  DevBuf<float2> logtab;
  bool logtab_ready = false;

  // workspaces
  DevBuf<double4_32a> mom;    // lambda_x, lambda_y, xi, s0 per component
  DevBuf<double2> part;   // split partial sums of the pair kernel
  DevBuf<double2> stage_in, stage_out, stage_tgt;  // host<->device staging
  DevBuf<double2> tmp2;

  // launch shapes of the pair kernels set on this handle (by the tuner or
  // explicitly), indexed by precision (FP64, FP32, DF64)
  PairShape shape[3];

  BlockDiag bd;
  TwoGrid tg;
  CoarseLevel cl;
  Krylov kr;
  Prof prof;
};

// per-translation-unit launch counters
unsigned long long launches_geometry();
unsigned long long launches_dlp_f64();
unsigned long long launches_dlp_f32();
unsigned long long launches_dlp_df64();
unsigned long long launches_bd();
unsigned long long launches_bd_trsv();
unsigned long long launches_bd_inv32();
unsigned long long launches_twogrid();
unsigned long long launches_gmres();
unsigned long long launches_batch();
unsigned long long launches_noalloc();
unsigned long long launches_mlp();
unsigned long long launches_tc_gemm();
unsigned long long launches_coarse();

// ---- geometry.cu ----
// component moments (lambda_x, lambda_y, xi, s0) of sigma into `out`
// (default: the handle's buffer)
void moments_f64(Geom& g, const double2* sigma, const int* done, double4_32a* out = nullptr);

// ---- dlp_f64.cu ----
// y = A sigma on the boundary (boundary=true, targets = nodes), or the
// interior velocity at T targets (boundary=false). All pointers device.
void dlp_apply_f64(Geom& g, const double2* sigma, double2* y, bool boundary,
                   const double2* targets, int64_t T, const int* done);

// y[i] = the FP64 pair kernel's reciprocal of x[i] (device arrays)
void rcp_newton_apply(const double* x, double* y, int64_t n, cudaStream_t s);

// pair kernels alone (into g.part; returns the number of source splits)
int pairs_f64(Geom& g, const double2* sigma, const double2* targets, int64_t T, bool boundary, PairShape sh,
              const int* done);
int pairs_f32(Geom& g, const double2* sigma, const double2* targets, int64_t T, PairShape sh, const int* done);
int pairs_df64(Geom& g, const double2* sigma, const double2* targets, int64_t T, PairShape sh, const int* done);
// compiled shape variants of each pair kernel (entry 0 = default); returns the count
int pair_variants_f64(PairVariant* out, int cap);
int pair_variants_f32(PairVariant* out, int cap);
int pair_variants_df64(PairVariant* out, int cap);

// ---- tune.cu ----
// The launch shape of the pair kernel of `precision` for T targets on this
// handle: the handle's own choice, else the process-wide tuning cache entry
// of its size class, else the default.
PairShape pair_shape(const Geom& g, int precision, int64_t T);

// ---- dlp_f32.cu / dlp_df64.cu ----
void dlp_apply_f32(Geom& g, const double2* sigma, double2* y, bool boundary,
                   const double2* targets, int64_t T, const int* done);
void dlp_apply_df64(Geom& g, const double2* sigma, double2* y, bool boundary,
                    const double2* targets, int64_t T, const int* done);

// ---- bd.cu ----
void bd_setup(Geom& g);
// f32: use the single-precision inverses and factors (inner solves)
void bd_apply(Geom& g, const double* v, double* z, const int* done, bool f32 = false);
void bd_check_barrier(Geom& g);
// ---- twogrid.cu ----
void twogrid_setup(Geom& g, int q, int coarse_mode = STOKES_TG_COARSE_AUTO);
// z = P^-1 v with the current preconditioner (two-grid if set up, else block diagonal)
void precond_apply(Geom& g, const double* v, double* z, const int* done, bool f32);
void invert_from_lu32(Geom& g, const float* LU, int64_t m, const int* perm, float* X);
// C = alpha A B + beta C, column-major float (M x K times K x N)
void sgemm32(cudaStream_t s, int64_t M, int64_t N, int K, float alpha, const float* A, int64_t lda, const float* B,
             int64_t ldb, float beta, float* C, int64_t ldc);

// ---- tc_gemm.cu ----
// false when STOKES_TG_GEMM=simt selects the CUDA-core trailing updates
bool tc_trailing_enabled();
// A[b.., b..] -= A[b.., k0..k0+kb) A[k0..k0+kb), b..), b = k0 + kb, kb in {32, 64,
// 96, 128} (column-major float m x m) on the tensor cores (three TF32
// products); work: tc_trailing_work_floats(m)
void tc_trailing_update(cudaStream_t s, float* A, int64_t m, int64_t k0, int kb, int64_t rest, float* work,
                        int* err);
int64_t tc_trailing_work_floats(int64_t m);

// ---- bd_trsv.cu ----
// elements of the diagonal-tile inverses of an m x m LU (L's, then U's)
int64_t lu_tile_inverse_elems(int64_t m);
template <class T>
void lu_tile_inverses(cudaStream_t s, const T* A, int64_t m, T* tinv);
// 64-bit words of the work buffer of lu_solve_persistent for m rows of elem_bytes values
int64_t lu_solve_work_words(int64_t m, int elem_bytes);
// z = U^-1 L^-1 P v by the persistent solve that publishes tile solutions as
// generation-tagged words; work: lu_solve_work_words(m, sizeof(T)) words and gen
// its generation counter (0 when the buffer was zeroed)
template <class T>
void lu_solve_persistent(Geom& g, const T* A, int64_t m, const int* perm, const T* tinv, const double* v, double* z,
                         unsigned long long* work, unsigned& gen, const int* done);

// ---- coarse.cu ----
// z = Z c + B^-1 (r - Y c), c = C Z^T W r (needs cl.ready and the block diagonal)
void coarse_apply(Geom& g, const double* r, double* z, const int* done, bool f32);

// ---- gmres.cu ----
struct SolveResult {
  int iters = 0;
  double relres = 0, pc_relres = 0;
  int status = STOKES_OK;
};
SolveResult gmres_solve(Geom& g, const double* f, double* x, double tol, int restart, int max_iter,
                        int precision, int side);

// operator dispatch used by the solver and the API
void apply_operator(Geom& g, const double* sigma, double* y, int precision, const int* done);

// ---- batch.cu ----
// y[k R + r] = A_k sigma[k R + r] for geometries k and right-hand sides r < R
// (device arrays), FP32 or DF64, one persistent pair launch.
void batch_matvec(Geom* const* geoms, int n_geoms, int R, const double* const* sigma, double* const* y,
                  int precision);
// lockstep flexible GMRES of all (geometry, right-hand side) systems
void batch_solve(Geom* const* geoms, int n_geoms, int R, const double* const* f, double tol, int restart,
                 int max_iter, int precision, double* const* sigma, int* iters, double* relres, int* status);

// ---- api.cu ----
// runs fn(ctx), mapping exceptions to a status code and the thread's last error
int guarded_call(void (*fn)(void*), void* ctx);

}  // namespace stokes

// the opaque handle of the C ABI
struct stokes_geom {
  stokes::Geom* g;
};
