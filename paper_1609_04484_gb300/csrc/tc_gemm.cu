// Trailing update of the two-grid preconditioner's coarse LU on the
// fifth-generation tensor cores (tcgen05 MMA with TMEM accumulators, TMA
// tile loads, mbarrier pipeline):
//   C[base.., base..] -= L21 U12,  L21 = rest x kb, U12 = kb x rest
// (one rank-kb update of the right-looking blocked LU; kb a multiple of 32,
// at most 128). The LU is factorised
// in single precision; TF32 alone keeps ~11 bits, so each product is split
// into three TF32 products (a = a_hi + a_lo, a_hi = a rounded to TF32):
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi     (relative error ~2^-21)
// with float accumulation in TMEM.
//
// Per panel a small kernel writes the hi and lo parts of both operands as
// K-major [rows][kb] float arrays (L21 is stored column-major, so it is
// transposed on the way). The GEMM is persistent and warp-specialised:
//   warp 0     TMA producer: for each 128 x 128 output tile and each slice of
//              K (32 floats = one 128-byte swizzle row) it loads the four
//              operand slabs (A_hi, A_lo, B_hi, B_lo: 16 KB each) into a ring
//              of kStages shared-memory stages (128-byte swizzle);
//   warp 1     MMA issuer (one thread): 3 x 4 MMAs (M = 128, N = 128, K = 8)
//              per stage into one of two TMEM accumulators, commits that free
//              the stage and, after the tile, signal the epilogue;
//   warps 2-9  epilogue: each warp reads its 32 TMEM lanes (rows) for 64 of
//              the 128 columns (tcgen05.ld 32x32b), 32 columns at a time,
//              writes the negated 32 x 32 product to its shared-memory
//              buffer and adds it to C with one TMA reduction
//              (cp.reduce.async.bulk.tensor ... add: L2 does the
//              read-modify-write, so the warp waits on no load of C), then
//              frees the accumulator. Where C's column stride is not a
//              multiple of 16 bytes (TMA's rule) the warp instead loads and
//              stores C itself (for each column, 32 consecutive rows: 128
//              contiguous bytes).
// The epilogue of one tile overlaps the loads and MMAs of the next.
// Every wait is bounded: on timeout the CTA raises the caller's error word,
// drains its own copies and MMAs (again bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace stokes {

namespace {

constexpr int kBM = 128, kBN = 128, kKH = 32;  // tile rows, tile columns, K slice (floats)
constexpr int kMaxPanel = 128;                 // largest K of one trailing update
constexpr int kPrepRows = 64;                  // rows per CTA of the operand preparation
constexpr int kStages = 3;
constexpr int kSlab = kBM * kKH * 4;           // bytes of one operand slab (16 KB)
constexpr int kStageBytes = 4 * kSlab;         // A_hi, A_lo, B_hi, B_lo
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 2 * kBN;             // two accumulators of 128 columns
constexpr long long kWaitLimit = 1ll << 22;    // polls of try_wait (each up to ~1 us): seconds at most
constexpr int kEpiBuf = 32 * 32;               // floats of one epilogue warp's staging tile (4 KB)
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + (size_t)kEpiWarps * kEpiBuf * 4 + 1024 + 256;

static_assert(kBM == kBN, "the operand slabs of A and B have the same shape");

// Instruction descriptor of tcgen05.mma kind::tf32: D float (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
// Wait until the phase of parity `parity` has completed; false on timeout
// (raising *err) or when another thread of the grid raised *err.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  const uint32_t a = saddr(b);
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255) == 255 && *(volatile int*)err) return false;
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, void* dst, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major slab with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading byte offset (unused by
// swizzled K-major layouts; 16 B) >> 4 at bits 16-29, stride byte offset
// (8 rows x 128 B = 1024 B between row groups) >> 4 at bits 32-45,
// descriptor version 1 at bits 46-47, layout SWIZZLE_128B (2) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
// C[x.., y..] += the 32 x 32 tile at src (column-major: element (r, c) at
// src[32 c + r]), x = row, y = column of C; completes through a bulk group.
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, const float* src, int x, int y) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   map),
               "r"(saddr(src)), "r"(x), "r"(y)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Two adjacent 32-column slices (columns [0, 32) and [32, 64) from taddr) with
// one wait for both loads.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr, float (&v0)[32], float (&v1)[32]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr + 32u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    v0[i] = __uint_as_float(r[i]);
    v1[i] = __uint_as_float(r[32 + i]);
  }
}

__device__ __forceinline__ float to_tf32(float a) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return __uint_as_float(r);
}

// hi / lo TF32 parts of both operands of one trailing update, K-major with
// row length kb (each CTA kPrepRows rows):
//   a_hi[r][k], a_lo[r][k] from L21[r][k] = A[(k0 + k) m + base + r]   (blockIdx.y = 0)
//   b_hi[n][k], b_lo[n][k] from U12[k][n] = A[(base + n) m + k0 + k]   (blockIdx.y = 1)
__global__ void __launch_bounds__(256)
k_tc_prep(const float* __restrict__ A, int64_t m, int64_t k0, int kb, int64_t base, int64_t rest,
          float* __restrict__ ahi, float* __restrict__ alo, float* __restrict__ bhi, float* __restrict__ blo) {
  count_launch();
  const int64_t r0 = blockIdx.x * (int64_t)kPrepRows;
  const int n = kb * kPrepRows;
  if (blockIdx.y == 0) {
    __shared__ float t[kMaxPanel][kPrepRows + 1];  // [k][r]: L21 is column-major, read along r
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int k = e / kPrepRows, r = e % kPrepRows;
      t[k][r] = r0 + r < rest ? A[(k0 + k) * m + base + r0 + r] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r = e / kb, k = e % kb;
      if (r0 + r >= rest) continue;
      const float a = t[k][r], h = to_tf32(a);
      ahi[(r0 + r) * kb + k] = h;
      alo[(r0 + r) * kb + k] = a - h;
    }
  } else {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int c = e / kb, k = e % kb;
      if (r0 + c >= rest) continue;
      const float a = A[(base + r0 + c) * m + k0 + k], h = to_tf32(a);
      bhi[(r0 + c) * kb + k] = h;
      blo[(r0 + c) * kb + k] = a - h;
    }
  }
}

// Output tile t of the mt x mt tiles: groups of G row tiles (G = the grid
// size) taken one after the other, and inside a group the row index fastest.
// At each moment the CTAs then work on G vertically adjacent tiles of one or
// two column strips: C is read and written in runs of G x 512 contiguous
// bytes per column (the 512-byte segments of a single tile are 272 KB apart
// at 68k rows, which costs DRAM page locality), every CTA keeps its row
// tile for the whole group (its operand slabs stay in L2: G x 128 KB), and
// one column tile's slabs serve all CTAs at once.
__device__ __forceinline__ void tile_of(int64_t t, int64_t mt, int64_t G, int64_t& tr, int64_t& tcol) {
  const int64_t span = G * mt;
  const int64_t grp = t / span, within = t - grp * span;
  const int64_t width = imin64(G, mt - grp * G);  // row tiles in this group
  tcol = within / width;
  tr = grp * G + (within - tcol * width);
}

struct TcMaps {
  CUtensorMap ahi, alo, bhi, blo;
  CUtensorMap c;  // the whole matrix, 32 x 32 boxes (used when reduce_c)
};

__global__ void __launch_bounds__(kThreads, 1)
k_tc_trailing(const __grid_constant__ TcMaps maps, float* __restrict__ C, int64_t ldc, int64_t base, int64_t rest,
              int nslices, int reduce_c, int* __restrict__ err) {
  count_launch();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* epi = reinterpret_cast<float*>(smem + (size_t)kStages * kStageBytes);  // [kEpiWarps][kEpiBuf]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * kStageBytes + (size_t)kEpiWarps * kEpiBuf * 4);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drained = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t mt = (rest + kBM - 1) / kBM;
  const int64_t ntiles = mt * mt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(drained, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int64_t it = 0;
      int armed_round[kStages];
      for (int s = 0; s < kStages; ++s) armed_round[s] = -1;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int64_t tr, tcol;
        tile_of(t, mt, gridDim.x, tr, tcol);
        const int rm = (int)(tr * kBM), rn = (int)(tcol * kBN);
        for (int h = 0; h < nslices && ok; ++h, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t round = (uint32_t)(it / kStages);
          if (!mbar_wait(&empty[s], (round & 1) ^ 1, err)) { ok = false; break; }
          unsigned char* st = smem + (size_t)s * kStageBytes;
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(&maps.ahi, st, &full[s], kKH * h, rm);
          tma_load_2d(&maps.alo, st + kSlab, &full[s], kKH * h, rm);
          tma_load_2d(&maps.bhi, st + 2 * kSlab, &full[s], kKH * h, rn);
          tma_load_2d(&maps.blo, st + 3 * kSlab, &full[s], kKH * h, rn);
          armed_round[s] = (int)round;
        }
      }
      // the stages' last copies have landed before the CTA may leave
      for (int s = 0; s < kStages; ++s)
        if (armed_round[s] >= 0) mbar_wait(&full[s], (uint32_t)armed_round[s] & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int64_t it = 0, ti = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++ti) {
        const int b = (int)(ti & 1);
        const uint32_t use = (uint32_t)(ti >> 1);
        if (!mbar_wait(&tempty[b], (use & 1) ^ 1, err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kBN);
        for (int h = 0; h < nslices; ++h, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t round = (uint32_t)(it / kStages);
          if (!mbar_wait(&full[s], round & 1, err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = saddr(smem + (size_t)s * kStageBytes);
#pragma unroll
          for (int kk = 0; kk < kKH / 8; ++kk) {  // K = 8 floats = 32 bytes per MMA
            const uint64_t ah = sdesc(st + 32 * kk), al = sdesc(st + kSlab + 32 * kk);
            const uint64_t bh = sdesc(st + 2 * kSlab + 32 * kk), bl = sdesc(st + 3 * kSlab + 32 * kk);
            umma_tf32(d, ah, bh, (h | kk) ? 1u : 0u);
            umma_tf32(d, ah, bl, 1u);
            umma_tf32(d, al, bh, 1u);
          }
          umma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (ok) umma_commit(&tfull[b]);
      }
      umma_commit(drained);  // every MMA issued above has completed once this arrives
      mbar_wait(drained, 0, err);
    }
  } else {  // epilogue warps
    const int g = warp & 3;                 // TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;       // columns [64 half, 64 half + 64)
    float* buf = epi + (warp - 2) * kEpiBuf;
    bool issued = false;                    // a reduction of this warp may still read buf
    int64_t ti = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
      const int b = (int)(ti & 1);
      const uint32_t use = (uint32_t)(ti >> 1);
      if (!mbar_wait(&tfull[b], use & 1, err)) break;
      tc_fence_after();
      int64_t tr, tcol;
      tile_of(t, mt, gridDim.x, tr, tcol);
      const int64_t row = tr * kBM + 32 * g + lane;
      const int64_t col0 = tcol * kBN + 64 * half;
      // both 32-column slices into registers, then the accumulator is free:
      // the MMAs of tile ti + 2 need not wait for C's update below
      float v0[32], v1[32];
      tmem_ld32x2(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(b * kBN + 64 * half), v0, v1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
      auto emit = [&](const float (&v)[32], int j) {
        if (reduce_c) {
          // a box that starts inside the trailing block may reach past it:
          // those rows and columns fall outside the map (base + rest = m)
          // and the TMA unit drops them; a box that starts past it is not
          // issued
          if (row - lane < rest && col0 + 32 * j < rest) {
            if (issued) {
              if (lane == 0) bulk_wait_read();
              __syncwarp();
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) buf[32 * c + lane] = -v[c];
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
              tma_reduce_add_2d(&maps.c, buf, (int)(base + row - lane), (int)(base + col0 + 32 * j));
            issued = true;
          }
        } else if (row < rest) {
          float* cp = C + (base + col0 + 32 * j) * ldc + base + row;
          const int ncol = (int)imin64(32, rest - (col0 + 32 * j));
#pragma unroll
          for (int h = 0; h < 32; h += 16) {  // 16 columns of loads in flight, then their stores
            float old[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) old[c] = h + c < ncol ? cp[(int64_t)(h + c) * ldc] : 0.f;
#pragma unroll
            for (int c = 0; c < 16; ++c)
              if (h + c < ncol) cp[(int64_t)(h + c) * ldc] = old[c] - v[h + c];
          }
        }
      };
      emit(v0, 0);
      emit(v1, 1);
    }
    if (issued && lane == 0) bulk_wait_all();  // C is complete before the CTA leaves
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    STOKES_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    require(q == cudaDriverEntryPointSuccess && p, "cuTensorMapEncodeTiled is not available", STOKES_ECUDA);
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D map of a K-major [rows][kb] float array: boxes of 32 floats x 128 rows,
// 128-byte swizzle, zero fill out of range.
void make_map(CUtensorMap* map, const float* base, int64_t rows, int kb) {
  const cuuint64_t dims[2] = {(cuuint64_t)kb, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kb * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKH, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  require(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")", STOKES_ECUDA);
}

// 2D map of the whole column-major m x m float matrix A (row index
// innermost): 32 x 32 boxes, no swizzle, for the epilogue's reductions.
// Needs m * 4 bytes between columns to be a multiple of 16 (m % 4 == 0).
void make_map_c(CUtensorMap* map, const float* A, int64_t m) {
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)m};
  const cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  require(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed for C (" + std::to_string((int)r) + ")", STOKES_ECUDA);
}

}  // namespace

bool tc_trailing_enabled() {
  const char* e = std::getenv("STOKES_TG_GEMM");
  return !(e && std::string(e) == "simt");
}

// A[base.., base..] -= A[base.., k0..k0+kb) A[k0..k0+kb), base..) for the
// column-major m x m float matrix A (base = k0 + kb; kb a multiple of 32, at
// most 128), on the tensor cores. work: 4 kb rest floats; err: device error
// word (sticky).
void tc_trailing_update(cudaStream_t s, float* A, int64_t m, int64_t k0, int kb, int64_t rest, float* work,
                        int* err) {
  if (rest <= 0) return;
  require(kb > 0 && kb % kKH == 0 && kb <= kMaxPanel, "tensor-core trailing update: panel width must be 32, 64, 96 or 128",
          STOKES_EINVAL);
  static bool attr = false;
  if (!attr) {
    STOKES_CUDA(cudaFuncSetAttribute(k_tc_trailing, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    attr = true;
  }
  const int64_t base = k0 + kb;
  float* ahi = work;
  float* alo = ahi + rest * kb;
  float* bhi = alo + rest * kb;
  float* blo = bhi + rest * kb;
  k_tc_prep<<<dim3((unsigned)((rest + kPrepRows - 1) / kPrepRows), 2), 256, 0, s>>>(A, m, k0, kb, base, rest, ahi, alo,
                                                                                    bhi, blo);
  STOKES_LAUNCHED();
  TcMaps maps;
  make_map(&maps.ahi, ahi, rest, kb);
  make_map(&maps.alo, alo, rest, kb);
  make_map(&maps.bhi, bhi, rest, kb);
  make_map(&maps.blo, blo, rest, kb);
  const int reduce_c = (m % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
  if (reduce_c) make_map_c(&maps.c, A, m);
  else std::memset(&maps.c, 0, sizeof(maps.c));
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    STOKES_CUDA(cudaGetDevice(&dev));
    STOKES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t mt = (rest + kBM - 1) / kBM;
  const unsigned grid = (unsigned)std::min<int64_t>(nsm, mt * mt);
  k_tc_trailing<<<grid, kThreads, kSmemBytes, s>>>(maps, A, m, base, rest, kb / kKH, reduce_c, err);
  STOKES_LAUNCHED();
}

int64_t tc_trailing_work_floats(int64_t m) { return 4 * (int64_t)kMaxPanel * m; }

unsigned long long launches_tc_gemm() { return tu_launches(); }

}  // namespace stokes
