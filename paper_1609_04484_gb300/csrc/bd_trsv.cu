// Triangular solves with the LU factors of the largest preconditioner
// blocks (too large to invert explicitly), one persistent kernel per solve.
//
// z = U^-1 L^-1 P v for a column-major m x m block (L unit lower below the
// diagonal, U on and above it). Rows are cut into tiles of kTs; tile u
// belongs to CTA u mod gridDim.x, which keeps the tile's running right-hand
// side in shared memory. The inverses of the diagonal tiles are formed once
// at setup (lu_tile_inverses), so solving a tile is one small product.
// Forward sweep over t = 0, 1, ...: the owner of tile t publishes x_t, each
// value in 64-bit words that carry this launch's generation number in their
// upper half (a float in one word, a double in two); every CTA waits until
// the words of tile t carry the generation, then subtracts L[u, t] x_t from
// each of its tiles u > t, the owner of t + 1 first, which solves and
// publishes t + 1 at once. A 64-bit store is seen whole or not at all, so the
// word that shows the generation holds the value: no fence, flag or second
// load sits on the chain of dependent tile solves, the only serial part; the
// other updates stream the factors at the memory's rate behind it. The
// owner of the next tile polls all of the tile's words, other CTAs one word
// with one thread before reading the rest (fewer polls of the same lines).
// The backward sweep mirrors it with U from the last tile.
//
// Every wait polls with an iteration limit: on timeout the CTA raises the
// sticky error word, every other CTA sees it at its next check and leaves,
// and the host reports the failure instead of hanging. All CTAs are
// resident (cooperative launch, one CTA per SM), so a value that will be
// published is always published by a running CTA.
#include <algorithm>

#include "grid_sync.cuh"

namespace stokes {

namespace {

constexpr int kTs = 64;
constexpr int kThreads = 512;
constexpr int kPh = kThreads / kTs;  // column phases of a tile
constexpr int kGroupF = 4;  // float factor blocks per group of the bulk updates (16 KB each)
constexpr int kGroupD = 1;  // double factor blocks per group (32 KB each)
template <class T>
__host__ __device__ constexpr int group_blocks() { return sizeof(T) == 4 ? kGroupF : kGroupD; }
// dynamic shared memory of the bulk updates' two group buffers
template <class T>
constexpr size_t update_buffer_bytes() { return 2 * (size_t)group_blocks<T>() * kTs * kTs * sizeof(T); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

typedef unsigned long long u64;

__device__ __forceinline__ u64 ld_volatile_u64(const u64* p) { return *(volatile const u64*)p; }

// Wait until word p carries generation gen and return it; false on timeout
// (raising *err) or when another CTA raised *err.
__device__ __forceinline__ bool wait_word(const u64* p, unsigned gen, int* err, long long limit, u64& w) {
  long long spins = 0;
  while (((w = ld_volatile_u64(p)) >> 32) != gen) {
    if (++spins > limit || ((spins & 63) == 0 && *(volatile int*)err)) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(20);
  }
  return true;
}

// Value val published as sizeof(T) / 4 tagged words at p.
template <class T>
__device__ __forceinline__ void put_tagged(u64* p, unsigned gen, T val) {
  constexpr int kW = sizeof(T) / 4;
  unsigned u[kW];
  memcpy(u, &val, sizeof(T));
#pragma unroll
  for (int i = 0; i < kW; ++i) *(volatile u64*)(p + i) = ((u64)gen << 32) | u[i];
}
template <class T>
__device__ __forceinline__ bool get_tagged(const u64* p, unsigned gen, int* err, long long limit, T& val) {
  constexpr int kW = sizeof(T) / 4;
  unsigned u[kW];
#pragma unroll
  for (int i = 0; i < kW; ++i) {
    u64 w;
    if (!wait_word(p + i, gen, err, limit, w)) return false;
    u[i] = (unsigned)w;
  }
  memcpy(&val, u, sizeof(T));
  return true;
}

// x (forward solutions) and y (backward solutions): m tagged values each.
// Thread (rr, ph) of the CTA handles row rr of a tile and its columns
// ph, ph + kPh, ...; the step that gates the next tile's solve has its
// factor block and tile inverse loaded into registers before the wait for
// the previous tile, so only arithmetic and two block syncs remain on the
// serial path; the other tiles are updated kGroup at a time (all of their
// loads issued before any use, for memory-level parallelism). The bulk
// updates read their factor blocks from shared memory: a group of four blocks
// is copied in (cp.async, 16 bytes per copy) while the previous group is used,
// and the first group of a step's updates is requested before the wait for
// that step's solution, since the factors do not depend on it. The CTA that
// will gate the next step (it owns tile t + 2) updates only that tile with
// x_t and defers the rest of x_t's updates until it has solved and published
// t + 2, so its share of the bulk updates never delays the chain; every tile
// still receives x_0, x_1, ... in that order.
template <class T>
__global__ void __launch_bounds__(kThreads, 1)
k_lu_solve_flags(const T* __restrict__ A, int64_t m, const int* __restrict__ perm, const T* __restrict__ tinv,
                 const double* __restrict__ v, u64* __restrict__ work, double* __restrict__ out, unsigned gen,
                 int* __restrict__ err, long long limit, const int* __restrict__ done) {
  count_launch();
  if (done && *done) return;
  constexpr int kW = sizeof(T) / 4;  // tagged words per value
  constexpr int kGa = group_blocks<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sbuf = reinterpret_cast<T*>(smem_raw);  // [2][kGa][kTs columns][kTs rows]: factor blocks
  T* acc = sbuf + 2 * kGa * kTs * kTs;       // [my tiles][kTs]
  __shared__ T szb[2][kTs];  // x_t (or y_t) in slot t & 1: the current column and a deferred one
  __shared__ T red[1][kPh][kTs];         // partial sums of the gate's products
  __shared__ T redb[2][kGa][kPh][kTs];   // partial sums of the bulk updates, by group parity
  __shared__ int s_fail;
  const int64_t nt = (m + kTs - 1) / kTs;
  const int G = gridDim.x, me = blockIdx.x;
  const int mine = (int)((nt - me + G - 1) / G);  // tiles me, me + G, ...
  if (mine <= 0) return;                          // nothing to solve or update here
  const int64_t last = me + (int64_t)(mine - 1) * G;
  const int rr = threadIdx.x & (kTs - 1), ph = threadIdx.x / kTs;
  const T* invL = tinv;
  const T* invU = tinv + nt * kTs * kTs;
  u64* x = work;           // forward solutions, tagged
  u64* y = work + m * kW;  // backward solutions, tagged
  constexpr int kPer = kTs / kPh;  // columns per thread

  // acc_u = (P v)_u
  for (int e = threadIdx.x; e < mine * kTs; e += kThreads) {
    const int64_t row = (int64_t)(me + (e / kTs) * G) * kTs + (e % kTs);
    acc[e] = row < m ? (T)v[perm[row]] : (T)0;
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();

  // this thread's values of the block A[u tile rows, t tile columns]
  auto load_block = [&](int64_t u, int64_t t, T (&r)[kPer]) {
    const int64_t r0 = u * kTs, c0 = t * kTs;
    const int nc = (int)imin64(kTs, m - c0);
    const bool rowok = r0 + rr < m;
    const T* col = A + c0 * m + r0 + rr;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int c = ph + kPh * j;
      r[j] = (rowok && c < nc) ? col[(int64_t)c * m] : (T)0;
    }
  };
  // this thread's values of the inverse of diagonal tile t (column-major)
  auto load_inv = [&](int64_t t, const T* inv, T (&r)[kPer]) {
    const T* X = inv + t * kTs * kTs;
#pragma unroll
    for (int j = 0; j < kPer; ++j) r[j] = X[(ph + kPh * j) * kTs + rr];
  };
  // a -= block z
  auto apply_block = [&](const T (&r)[kPer], T* a, const T* z) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) s += r[j] * z[ph + kPh * j];
    red[0][ph][rr] = s;
    __syncthreads();
    if (ph == 0) {
      T t = 0;
#pragma unroll
      for (int q = 0; q < kPh; ++q) t += red[0][q][rr];
      a[rr] -= t;
    }
    __syncthreads();
  };
  // a = inv a, also published (tagged) in dst for the other CTAs
  auto solve_block = [&](int64_t t, const T (&r)[kPer], T* a, u64* dst) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) s += r[j] * a[ph + kPh * j];
    red[0][ph][rr] = s;
    __syncthreads();
    if (ph == 0) {
      T val = 0;
#pragma unroll
      for (int q = 0; q < kPh; ++q) val += red[0][q][rr];
      a[rr] = val;
      if (t * kTs + rr < m) put_tagged(dst + (t * kTs + rr) * kW, gen, val);
    }
    __syncthreads();
  };
  // Copies of group gi of the blocks A[u0 + i step, t], i < count, into
  // buffer bsel, as one cp.async group per thread (possibly empty); rows and
  // columns past m are zero-filled. With m a multiple of 16 / sizeof(T) every
  // copy is 16-byte aligned; otherwise the group is loaded synchronously.
  constexpr int kEpc = 16 / (int)sizeof(T);  // elements per 16-byte copy
  constexpr int kCpc = kTs / kEpc;            // copies per column of a block
  const bool async_ok = m % kEpc == 0;
  auto issue_group = [&](int64_t u0, int64_t step, int64_t count, int64_t t, int gi, int bsel) {
    const int64_t i0 = (int64_t)gi * kGa;
    const int n = (int)imin64(kGa, count - i0);
    T* dstb = sbuf + (size_t)bsel * kGa * kTs * kTs;
    const int64_t c0 = t * kTs;
    for (int e = threadIdx.x; e < n * kTs * kCpc; e += kThreads) {
      const int q = e / (kTs * kCpc), w = e - q * (kTs * kCpc);
      const int c = w / kCpc, r0 = (w - c * kCpc) * kEpc;
      const int64_t row = (u0 + (i0 + q) * step) * kTs + r0, col = c0 + c;
      T* dst = dstb + ((size_t)q * kTs + c) * kTs + r0;
      const int valid = (col < m && row < m) ? (int)imin64(kEpc, m - row) : 0;
      if (async_ok) {
        cp_async16(dst, valid > 0 ? (const void*)(A + col * m + row) : (const void*)A, valid * (int)sizeof(T));
      } else {
#pragma unroll
        for (int k = 0; k < kEpc; ++k) dst[k] = k < valid ? A[col * m + row + k] : (T)0;
      }
    }
    cp_async_commit();
  };
  bool pending = false;  // group 0 of (pend_u0, pend_t) is in flight into buffer 0
  int64_t pend_u0 = -1, pend_t = -1;
  auto prefetch = [&](int64_t u0, int64_t step, int64_t count, int64_t t) {
    if (count <= 0) return;
    issue_group(u0, step, count, t, 0, 0);
    pending = true;
    pend_u0 = u0;
    pend_t = t;
  };
  // a_u -= A[u, t] z for `count` of this CTA's tiles u0, u0 + step, ...
  auto update_many = [&](int64_t u0, int64_t step, int64_t count, int64_t t, const T* z) {
    if (count <= 0) return;
    if (pending && (pend_u0 != u0 || pend_t != t)) {  // not the prefetched updates: let it land first
      cp_async_wait<0>();
      __syncthreads();
      pending = false;
    }
    if (!pending) issue_group(u0, step, count, t, 0, 0);
    pending = false;
    const int ngroups = (int)((count + kGa - 1) / kGa);
    for (int gi = 0; gi < ngroups; ++gi) {
      if (gi + 1 < ngroups) {
        issue_group(u0, step, count, t, gi + 1, (gi + 1) & 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int n = (int)imin64(kGa, count - (int64_t)gi * kGa);
      const T* bufp = sbuf + (size_t)(gi & 1) * kGa * kTs * kTs;
      T(*rd)[kPh][kTs] = redb[gi & 1];
#pragma unroll
      for (int q = 0; q < kGa; ++q)
        if (q < n) {
          T s = 0;
#pragma unroll
          for (int j = 0; j < kPer; ++j) s += bufp[((size_t)q * kTs + ph + kPh * j) * kTs + rr] * z[ph + kPh * j];
          rd[q][ph][rr] = s;
        }
      // after this barrier every thread is done with the buffer of group gi
      // (the next group's copies may overwrite it) and the partial sums are
      // complete; the sums of group gi + 1 go to the other half of redb, so
      // no barrier is needed after the accumulation below
      __syncthreads();
      if (ph < n) {
        T sum = 0;
#pragma unroll
        for (int q = 0; q < kPh; ++q) sum += rd[ph][q][rr];
        acc[((u0 + ((int64_t)gi * kGa + ph) * step) / G) * kTs + rr] -= sum;
      }
    }
    __syncthreads();  // the accumulators are complete before anything reads them
  };
  // sz = the solution of tile t: this CTA's own copy, or the published one
  // (waiting for its words to carry this launch's generation; `all`: every
  // thread polls its word at once, else thread 0 polls the tile's first
  // word before the others read theirs); false if a wait gave up
  auto fetch = [&](int64_t t, const u64* src, bool all, T* sz) -> bool {
    if (t % G == me) {
      if (threadIdx.x < kTs) sz[threadIdx.x] = acc[(t / G) * kTs + threadIdx.x];
    } else {
      if (!all) {
        if (threadIdx.x == 0) {
          u64 w;
          if (!wait_word(src + t * kTs * kW, gen, err, limit, w)) s_fail = 1;
        }
        __syncthreads();
      }
      if (threadIdx.x < kTs && !s_fail) {
        T val = (T)0;
        if (t * kTs + threadIdx.x < m && !get_tagged(src + (t * kTs + threadIdx.x) * kW, gen, err, limit, val))
          s_fail = 1;
        sz[threadIdx.x] = val;
      }
    }
    __syncthreads();
    return !s_fail;
  };

  T pa[kPer], pinv[kPer];
  // forward sweep: L (unit lower)
  if (me == 0) {
    load_inv(0, invL, pinv);
    solve_block(0, pinv, acc, x);
  }
  int deferred = -1;  // a column whose updates of this CTA's later tiles wait (tile counts fit an int)
  for (int64_t t = 0; t < last; ++t) {  // beyond `last` this CTA has no tile to update
    const int64_t nxt = t + 1;
    T* zt = szb[t & 1];
    int64_t u = nxt + ((me - nxt) % G + G) % G;  // this CTA's first tile after t
    const bool gate = u == nxt;                  // it gates the next step
    if (gate) {
      load_block(nxt, t, pa);
      load_inv(nxt, invL, pinv);
    }
    {  // the first group of this step's first bulk update, before the wait
      const int64_t ua = gate ? u + G : u;
      if (ua < nt) {
        if (deferred >= 0) prefetch(ua, G, (nt - 1 - ua) / G + 1, deferred);
        else if (!gate && u == t + 2) prefetch(u, G, 1, t);
        else prefetch(ua, G, (nt - 1 - ua) / G + 1, t);
      }
    }
    if (!fetch(t, x, gate, zt)) {
      cp_async_wait<0>();  // own copies in flight land before the CTA leaves
      return;
    }
    if (gate) {
      T* a = acc + (nxt / G) * kTs;
      apply_block(pa, a, zt);
      solve_block(nxt, pinv, a, x);
      u += G;
    }
    if (deferred >= 0) {  // (tile t + 1 received it before)
      if (u < nt) update_many(u, G, (nt - 1 - u) / G + 1, deferred, szb[deferred & 1]);
      deferred = -1;
    }
    if (u < nt) {
      if (!gate && u == t + 2) {  // this CTA gates the next step: that tile first, the rest after it
        update_many(u, G, 1, t, zt);
        deferred = (int)t;
      } else {
        update_many(u, G, (nt - 1 - u) / G + 1, t, zt);
      }
    }
  }

  // backward sweep: U (upper, with its diagonal) from the forward solution in acc
  if (last == nt - 1) {
    load_inv(nt - 1, invU, pinv);
    solve_block(nt - 1, pinv, acc + ((nt - 1) / G) * kTs, y);
  }
  deferred = -1;
  for (int64_t t = nt - 1; t > me; --t) {  // at or below `me` this CTA has no tile to update
    const int64_t prv = t - 1;
    T* zt = szb[t & 1];
    int64_t u = prv - ((prv - me) % G + G) % G;  // this CTA's last tile before t
    const bool gate = u == prv;
    if (gate) {
      load_block(prv, t, pa);
      load_inv(prv, invU, pinv);
    }
    {
      const int64_t ua = gate ? u - G : u;
      if (ua >= 0) {
        if (deferred >= 0) prefetch(ua, -(int64_t)G, (ua - me) / G + 1, deferred);
        else if (!gate && u == t - 2) prefetch(u, -(int64_t)G, 1, t);
        else prefetch(ua, -(int64_t)G, (ua - me) / G + 1, t);
      }
    }
    if (!fetch(t, y, gate, zt)) {
      cp_async_wait<0>();  // own copies in flight land before the CTA leaves
      return;
    }
    if (gate) {
      T* a = acc + (prv / G) * kTs;
      apply_block(pa, a, zt);
      solve_block(prv, pinv, a, y);
      u -= G;
    }
    if (deferred >= 0) {
      if (u >= 0) update_many(u, -(int64_t)G, (u - me) / G + 1, deferred, szb[deferred & 1]);
      deferred = -1;
    }
    if (u >= 0) {
      if (!gate && u == t - 2) {
        update_many(u, -(int64_t)G, 1, t, zt);
        deferred = (int)t;
      } else {
        update_many(u, -(int64_t)G, (u - me) / G + 1, t, zt);
      }
    }
  }
  for (int e = threadIdx.x; e < mine * kTs; e += kThreads) {
    const int64_t row = (int64_t)(me + (e / kTs) * G) * kTs + (e % kTs);
    if (row < m) out[row] = (double)acc[e];
  }
}

// Inverse of each diagonal tile of L (unit lower; lower = 1) or U (upper),
// kTs x kTs, column-major into out[t * kTs * kTs]; a partial last tile is
// completed with the identity. One CTA per tile; thread q solves for column q.
template <class T>
__global__ void __launch_bounds__(kTs)
k_tile_inverse_t(const T* __restrict__ A, int64_t m, int lower, T* __restrict__ out) {
  count_launch();
  const int64_t t = blockIdx.x;
  const int64_t r0 = t * kTs;
  const int n = (int)imin64(kTs, m - r0);
  __shared__ T sT[kTs][kTs + 1];  // [col][row]
  __shared__ T sX[kTs][kTs + 1];
  for (int e = threadIdx.x; e < kTs * kTs; e += blockDim.x) {
    const int c = e / kTs, r = e % kTs;
    sT[c][r] = (c < n && r < n) ? A[(r0 + c) * m + r0 + r] : (c == r ? (T)1 : (T)0);
    sX[c][r] = c == r ? (T)1 : (T)0;
  }
  __syncthreads();
  const int q = threadIdx.x;
  if (lower) {
    for (int c = 0; c < kTs; ++c) {
      const T xc = sX[q][c];
      for (int r = c + 1; r < kTs; ++r) sX[q][r] -= sT[c][r] * xc;
    }
  } else {
    for (int c = kTs - 1; c >= 0; --c) {
      const T xc = sX[q][c] / sT[c][c];
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

}  // namespace

int64_t lu_tile_inverse_elems(int64_t m) { return 2 * ((m + kTs - 1) / kTs) * kTs * kTs; }

// tinv: lu_tile_inverse_elems(m) elements, the L tile inverses then the U ones.
template <class T>
void lu_tile_inverses(cudaStream_t s, const T* A, int64_t m, T* tinv) {
  const int64_t nt = (m + kTs - 1) / kTs;
  k_tile_inverse_t<T><<<(unsigned)nt, kTs, 0, s>>>(A, m, 1, tinv);
  k_tile_inverse_t<T><<<(unsigned)nt, kTs, 0, s>>>(A, m, 0, tinv + nt * kTs * kTs);
  STOKES_LAUNCHED();
}

int64_t lu_solve_work_words(int64_t m, int elem_bytes) { return 2 * m * (elem_bytes / 4); }

// z (block rows) = factors^-1 v for one block. T = double uses the FP64
// factors, T = float a float copy of them; work: lu_solve_work_words(m,
// sizeof(T)) words with their own generation counter gen, which the caller
// sets to 0 when it zeroes the buffer (a word is current only when its
// generation matches the launch's, and generations start at 1).
template <class T>
void lu_solve_persistent(Geom& g, const T* A, int64_t m, const int* perm, const T* tinv, const double* v, double* z,
                         unsigned long long* work, unsigned& gen_counter, const int* done) {
  static int grid = 0;
  const int64_t nt = (m + kTs - 1) / kTs;
  BlockDiag& b = g.bd;
  if (grid == 0) {
    int dev = 0, nsm = 0;
    STOKES_CUDA(cudaGetDevice(&dev));
    STOKES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    grid = nsm;  // one CTA per SM: all resident
  }
  const size_t tiles_bytes = (size_t)((nt + grid - 1) / grid) * kTs * sizeof(T);
  require(tiles_bytes <= 64 * 1024, "triangular solve: block too large for the per-CTA tile store");
  const size_t smem = update_buffer_bytes<T>() + tiles_bytes;
  STOKES_CUDA(cudaFuncSetAttribute(k_lu_solve_flags<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  STOKES_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_solve_flags<T>, kThreads, smem));
  require(per_sm >= 1, "persistent triangular solve does not fit on an SM", STOKES_ECUDA);
  if (!b.barrier.get()) {
    b.barrier.alloc(4);
    STOKES_CUDA(cudaMemsetAsync(b.barrier.get(), 0, 4 * sizeof(unsigned), g.stream));
  }
  unsigned gen = ++gen_counter;
  if (gen == 0) {  // wrapped: clear the buffer so that no stale generation matches
    STOKES_CUDA(cudaMemsetAsync(work, 0, lu_solve_work_words(m, sizeof(T)) * sizeof(unsigned long long), g.stream));
    gen = gen_counter = 1;
  }
  int* err = (int*)(b.barrier.get() + 2);
  long long limit = gsync::spin_limit();
  void* args[] = {(void*)&A,   (void*)&m,   (void*)&perm, (void*)&tinv,  (void*)&v,    (void*)&work,
                  (void*)&z,   (void*)&gen, (void*)&err,  (void*)&limit, (void*)&done};
  STOKES_CUDA(cudaLaunchCooperativeKernel((const void*)k_lu_solve_flags<T>, dim3(grid), dim3(kThreads), args, smem,
                                          g.stream));
}

// Throws if a persistent solve ever timed out waiting (synchronises).
void bd_check_barrier(Geom& g) {
  if (!g.bd.barrier.get()) return;
  unsigned err = 0;
  STOKES_CUDA(cudaMemcpyAsync(&err, g.bd.barrier.get() + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, g.stream));
  STOKES_CUDA(cudaStreamSynchronize(g.stream));
  require(err == 0, "block-diagonal triangular solve: a wait for another CTA's tile timed out", STOKES_ECUDA);
}

template void lu_tile_inverses<double>(cudaStream_t, const double*, int64_t, double*);
template void lu_tile_inverses<float>(cudaStream_t, const float*, int64_t, float*);
template void lu_solve_persistent<double>(Geom&, const double*, int64_t, const int*, const double*, const double*,
                                          double*, unsigned long long*, unsigned&, const int*);
template void lu_solve_persistent<float>(Geom&, const float*, int64_t, const int*, const float*, const double*,
                                         double*, unsigned long long*, unsigned&, const int*);

unsigned long long launches_bd_trsv() { return tu_launches(); }

}  // namespace stokes
