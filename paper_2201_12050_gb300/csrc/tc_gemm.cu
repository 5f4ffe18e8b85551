// Offset-indexed complex block products on the 5th-generation tensor cores.
//
// The near field of the FMPBEM (Sec. 3.2: y_c = sum_delta S_delta p_{c-delta})
// and the P2M / L2P steps shared by all cells (Sec. 3.5: M_c = V_0 p_c,
// y_c += U_0 L_c) are the same operation: for every cell c and right-hand
// side r, a sum over cell offsets delta of a complex block times the vector
// of the source cell c - delta.  Seen from all cells at once, each offset is
// one dense GEMM whose columns are the (cell, rhs) pairs, so with many
// right-hand sides this is where the method becomes tensor-core work.
//
// Arithmetic: BF16 inputs, FP32 accumulation (tcgen05.mma kind::f16).  A
// complex product is carried as the real product of the interleaved 2 x 2
// representation [[re, -im], [im, re]], so one real GEMM of twice the size
// gives real and imaginary parts in adjacent accumulator rows.
//
// The per-frequency block products of the circulant engine (Sec. 2.4:
// Y_f = Lambda_f X_f for every padded-grid frequency f) are the other dense
// complex GEMMs of the method once many right-hand sides share the spectrum.
//
// Two kernels, both fed by the tensor memory accelerator (TMA) into rings of
// 128-byte-swizzled shared-memory stages, with one producer lane, one
// MMA-issuing lane (tcgen05.mma into FP32 accumulators in tensor memory) and
// the epilogue read back by tcgen05.ld:
//   - k_tc_gemm_tma: the offset GEMM, one CTA per output tile of 128 or 256
//     rows and a brick of (cell, right-hand side) columns (see there);
//   - k_tc_freq_tma: the per-frequency products on a persistent grid with a
//     double-buffered accumulator (see there).
// Every wait is bounded (one second of wall time); a wait that gives up sets
// an error word for the host, and the CTA still drains its copies and frees
// its tensor memory before it returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "tc_gemm.cuh"

namespace fmpb {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr int TC_THREADS = 256;
constexpr uint64_t TC_WAIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Waits for the completion of the phase with the given parity; false after TC_WAIT_NS.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > TC_WAIT_NS) return false;
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// D (tensor memory) = A B (+ D if accumulate), one 128 x N x 16 step.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier receives one arrival when all MMAs issued so far by this thread have completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
// 16 consecutive FP32 columns of this thread's accumulator lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Offset GEMM fed by the tensor memory accelerator.
//
// The columns of one output tile are a brick of source cells x right-hand
// sides (bx x by x bz cells, br right-hand sides, x fastest), so the B tile of
// offset delta is one 5-D TMA box of X viewed as (Kp, Mx, My, Mz, R nblk)
// starting at the brick's origin minus delta: source cells outside the grid
// (negative or too large coordinates) arrive as zeros from the copy engine.
// A is a 2-D box (64 x 128 rows) of the realified tables viewed as
// (Kp, n_off Mp).  Both use the 128-byte swizzle, which is the canonical
// K-major layout the MMA descriptors name.  An optional tail of kt2 more
// K-steps adds A2 X2 (offset zero, depth Kp2) into the same accumulator: the
// L2P term U_0 L_c of the FMM product joins the near field in one pass.
//
// Warp roles (256 threads):
//   - warp 0, one lane: producer.  For K-step kt it waits until stage
//     kt % NS is free (the MMAs of step kt - NS have completed), announces
//     the stage's bytes on its `full` mbarrier and issues the TMA copies;
//   - warp 1, one lane: MMA issuer.  It waits for `full`, issues the step's
//     four 128 x N x 16 MMAs per accumulator and commits them to `empty`;
//     after the last step it commits to `done`;
//   - warp 2 allocates and frees the tensor memory;
//   - all eight warps wait for `done` and run the epilogue (tcgen05.ld of
//     their 32-lane quarter, coalesced complex-double stores).
// Every wait is bounded (one second).  A wait that gives up raises a shared
// abort flag that ends the other role's loop, the CTA then waits (bounded)
// for every copy it issued and for its MMAs, sets the error word, frees its
// tensor memory and returns.
struct TcMaps {
  CUtensorMap a[TC_MAX_BATCH];    // per operator: A as (Kp, n_off Mp) BF16
  CUtensorMap a2[TC_MAX_BATCH];   // per operator: the tail's A2 as (Kp2, Mp) BF16
  CUtensorMap x;                  // X as (Kp, Mx, My, Mz, R nblk) BF16
  CUtensorMap x2;                 // the tail's X2 as (Kp2, Mx, My, Mz, R nblk) BF16
};
// The tail product of the offset GEMM: per operator A2 (Mp x tc_depth(k)
// rows, offset zero) times X2 (rows of depth tc_depth(k), the columns of X).
struct TcTail {
  const __nv_bfloat16* A[TC_MAX_BATCH];
  int64_t k;
  const __nv_bfloat16* X;
};
struct TcBrick {
  int bx, by, bz, br;       // cells along x, y, z and right-hand sides per tile
  int ntx, nty, ntz, ntr;   // tiles along each of them (per operator)
  int rows;                 // bx by bz br: B rows of one stage
  int n;                    // MMA N: rows rounded up to 16
};

template <int MT, int BNC>
struct TmaTile {
  static constexpr int A_HALF = TC_BM * TC_BK * 2;   // one 128-row A box
  static constexpr int A_BYTES = MT * A_HALF;
  static constexpr int B_BYTES = BNC * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // a multiple of 1024
  static constexpr int CTRL = 128;                         // mbarriers, TMEM address, flags
  static constexpr int FIT = (227 * 1024 - 1024 - CTRL) / STAGE_BYTES;
  static constexpr int STAGES = FIT < 6 ? FIT : 6;
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + CTRL;   // 1024: alignment slack
  static constexpr int TMEM_COLS = MT * BNC;
  static_assert(STAGES >= 3, "tile too large for the shared-memory ring");
  static_assert(2 * STAGES * 8 + 8 + 16 <= CTRL, "control block too small");
};

// Shared-memory descriptor of a K-major operand in the 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset),
// layout type 2 (bits 61-63); the leading byte offset is unused for this
// layout (field 1).  Advancing the start address by 32 bytes selects the
// next 16-element K slice within the swizzle atom.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], "
      "[%2];\n" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
// As mbar_wait_bounded, but also gives up when another role raised the abort
// flag; a timeout raises it.
__device__ bool mbar_wait_abortable(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > TC_WAIT_NS) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
// The long wait of the idle warps for the end of the main loop: polls with a
// short sleep so that they take few issue slots from the two working lanes.
__device__ bool mbar_wait_sleepy(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > TC_WAIT_NS) return false;
    __nanosleep(256);
  }
  return true;
}

template <int MT, int BNC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm_tma(const __grid_constant__ TcMaps maps, const TcBatch batch, const TcBrick bk, int Kp, int Mp,
                  void* __restrict__ y_, int m, int64_t ncols, int Mx, int My, int Mz, int R,
                  const TcOffsets offs, int kt2, int accumulate, int out_f32, unsigned* err) {
  using Tile = TmaTile<MT, BNC>;
  constexpr int NS = Tile::STAGES;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;   // the 128-byte swizzle wants 1024-byte aligned stages
  unsigned char* ctrl = smem_raw + (sbase - raw) + NS * Tile::STAGE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* n_loaded = abort_flag + 1;   // K-steps whose copies the producer issued
  volatile int* n_mma = abort_flag + 2;      // K-steps whose MMAs were issued

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM * MT;
  const bool two = MT == 2 && m0 + TC_BM < Mp;   // second row half present
  const int64_t tiles = (int64_t)bk.ntx * bk.nty * bk.ntz * bk.ntr;
  const int bop = (int)(blockIdx.y / tiles);
  int64_t rem = (int64_t)blockIdx.y - (int64_t)bop * tiles;
  const int tx = (int)(rem % bk.ntx);
  rem /= bk.ntx;
  const int ty = (int)(rem % bk.nty);
  rem /= bk.nty;
  const int tz = (int)(rem % bk.ntz);
  const int tr = (int)(rem / bk.ntz);
  const int x0 = tx * bk.bx, y0 = ty * bk.by, z0 = tz * bk.bz, r0 = tr * bk.br;
  const int blk = batch.blk[bop];

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    *n_loaded = 0;
    *n_mma = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    tmem_alloc(smem_u32(tmem_slot), Tile::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int kt_per_off = Kp / TC_BK;
  const int KT1 = offs.n * kt_per_off;
  const int KT = KT1 + kt2;

  if (warp == 0 && lane == 0) {
    // producer
    const void* amap = &maps.a[bop];
    const void* xmap = &maps.x;
    const void* amap2 = &maps.a2[bop];
    const void* xmap2 = &maps.x2;
    const uint32_t tx_bytes = (uint32_t)((two ? 2 : 1) * Tile::A_HALF + bk.rows * TC_BK * 2);
    int kt = 0;
    for (; kt < KT; ++kt) {
      const int s = kt % NS;
      if (kt >= NS && !mbar_wait_abortable(smem_u32(&empty[s]), ((kt / NS) - 1) & 1, abort_flag)) break;
      const uint32_t sa = sbase + s * Tile::STAGE_BYTES, sb = sa + Tile::A_BYTES;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, tx_bytes);
      if (kt < KT1) {
        const int o = kt / kt_per_off;
        const int k0 = (kt - o * kt_per_off) * TC_BK;
        tma_load_2d(sa, amap, fb, k0, o * Mp + m0);
        if (two) tma_load_2d(sa + Tile::A_HALF, amap, fb, k0, o * Mp + m0 + TC_BM);
        tma_load_5d(sb, xmap, fb, k0, x0 - offs.d[o][0], y0 - offs.d[o][1], z0 - offs.d[o][2], blk * R + r0);
      } else {
        const int k0 = (kt - KT1) * TC_BK;
        tma_load_2d(sa, amap2, fb, k0, m0);
        if (two) tma_load_2d(sa + Tile::A_HALF, amap2, fb, k0, m0 + TC_BM);
        tma_load_5d(sb, xmap2, fb, k0, x0, y0, z0, blk * R + r0);
      }
    }
    *n_loaded = kt;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bk.n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    int kt = 0;
    for (; kt < KT; ++kt) {
      const int s = kt % NS;
      if (!mbar_wait_abortable(smem_u32(&full[s]), (kt / NS) & 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t a0 = sbase + s * Tile::STAGE_BYTES, b0 = a0 + Tile::A_BYTES;
#pragma unroll
      for (int q = 0; q < TC_BK / 16; ++q) {
        tc_mma(tmem, smem_desc_sw128(a0 + 32 * q), smem_desc_sw128(b0 + 32 * q), idesc, (kt | q) != 0);
        if (two)
          tc_mma(tmem + BNC, smem_desc_sw128(a0 + Tile::A_HALF + 32 * q), smem_desc_sw128(b0 + 32 * q), idesc,
                 (kt | q) != 0);
      }
      tc_commit(smem_u32(&empty[s]));
    }
    *n_mma = kt;
    tc_commit(smem_u32(done));   // arrives once every MMA issued above has completed
  }
  __syncwarp();
  const bool mma_done = mbar_wait_sleepy(smem_u32(done), 0);
  const bool bad = __syncthreads_or(!mma_done || *abort_flag != 0);
  if (bad) {
    // copies issued for steps whose MMAs never ran are still landing
    if (tid == 0) {
      for (int kt = *n_mma; kt < *n_loaded; ++kt) mbar_wait_bounded(smem_u32(&full[kt % NS]), (kt / NS) & 1);
      atomicOr(err, 1u);
    }
  } else {
    // output column of every tile column (-1: outside the grid), decoded
    // once per CTA into the first stage's shared memory (the main loop has
    // finished with it) instead of per thread and column in the stores
    const int Nc = Mx * My * Mz;
    int64_t* colj = reinterpret_cast<int64_t*>(smem_raw + (sbase - raw));
    for (int col = tid; col < bk.rows; col += TC_THREADS) {
      int q = col;
      const int cx = x0 + q % bk.bx;
      q /= bk.bx;
      const int cy = y0 + q % bk.by;
      q /= bk.by;
      const int cz = z0 + q % bk.bz;
      const int r = r0 + q / bk.bz;
      colj[col] = (cx < Mx && cy < My && cz < Mz && r < R)
                      ? (int64_t)r * Nc + ((int64_t)cz * My + cy) * Mx + cx
                      : (int64_t)-1;
    }
    __syncthreads();
    tc_fence_after();
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t gm = (int64_t)m0 + (MT == 2 ? half * TC_BM : 0) + quarter * 32 + lane;
    const bool row_ok = gm < 2 * (int64_t)m;
    const int64_t i = gm >> 1;
    const int part = (int)(gm & 1);
    // MT = 1: warps 0-3 and 4-7 read the two column halves of the accumulator;
    // MT = 2: warps 0-3 read accumulator 0 (rows 0..127), warps 4-7 accumulator 1
    const int cbeg = MT == 2 ? 0 : half * (BNC / 2);
    const int cend = MT == 2 ? ((half == 0 || two) ? bk.n : 0) : min(bk.n, cbeg + BNC / 2);
    const uint32_t tcol = MT == 2 ? (uint32_t)(half * BNC) : 0u;
    const int64_t yoff = (int64_t)blk * ncols * m;
#pragma unroll 1
    for (int c0 = cbeg; c0 < cend; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + tcol + (uint32_t)c0, v);
      if (row_ok) {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int col = c0 + t;
          if (col >= bk.rows) break;
          const int64_t jc = colj[col];
          if (jc >= 0) {
            const int64_t e = yoff + jc * m + i;
            if (out_f32) {
              float* d = reinterpret_cast<float*>(reinterpret_cast<float2*>(y_) + e) + part;
              *d = accumulate ? *d + v[t] : v[t];
            } else {
              double* d = reinterpret_cast<double*>(reinterpret_cast<cd*>(y_) + e) + part;
              *d = accumulate ? *d + (double)v[t] : (double)v[t];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, Tile::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Per-frequency products Y_f = Lambda_f X_f (the circulant engine's block
// products with many right-hand sides) on a persistent grid.
//
// Work item = (frequency f, operator, column tile, 128-row tile); one CTA per
// SM takes items blockIdx.x, blockIdx.x + gridDim.x, ...  Each item is
// Kp / 64 K-steps of a 128 x N x 64 MMA group, A from the realified spectrum
// (a 2-D box of (Kp, F Mp)) and B from the rows f ctot + column of X (a 2-D
// box of (Kp, F ctot)), both TMA copies into a ring of up to eight stages.
// The spectrum is read once per product and only from HBM, so the kernel is a
// stream: the producer runs ahead across items, and the accumulator is
// double-buffered in tensor memory so that the epilogue of item c overlaps
// the MMAs of item c + 1.
//   - warp 0, one lane: producer (TMA);
//   - warp 1, one lane: MMA issuer; before reusing accumulator c & 1 it waits
//     for the epilogue's `tempty`, after an item's last step it commits `tfull`;
//   - warp 2: tensor-memory allocation;
//   - warps 4-7: epilogue, one 32-lane quarter each (tcgen05.ld), then one
//     arrival per warp on `tempty`.
// Waits are bounded as in the offset kernel (shared abort flag, drain of the
// copies in flight, error word).
template <int BNC>
struct FreqTile {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BNC * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // a multiple of 1024 for BNC >= 8
  static constexpr int CTRL = 256;
  static constexpr int FIT = (227 * 1024 - 1024 - CTRL) / STAGE_BYTES;
  static constexpr int STAGES = FIT < 8 ? FIT : 8;
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + CTRL;
  static constexpr int TMEM_COLS = 2 * BNC < 32 ? 32 : 2 * BNC;   // two accumulators
  static_assert(STAGES >= 3, "tile too large for the shared-memory ring");
  static_assert((2 * STAGES + 5) * 8 + 16 <= CTRL, "control block too small");
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// As mbar_wait_sleepy, but also gives up when the abort flag is raised, and
// raises it on a timeout.
__device__ bool mbar_wait_sleepy_abortable(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > TC_WAIT_NS) {
      *abort_flag = 1;
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

template <int BNC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_freq_tma(const __grid_constant__ TcMaps maps, const TcBatch batch, int Kp, int Mp, int64_t F, int B, int R,
                  int64_t ctot, int bn_rows, int n, void* __restrict__ y_, int f32_out, unsigned* err) {
  using Tile = FreqTile<BNC>;
  constexpr int NS = Tile::STAGES;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  unsigned char* ctrl = smem_raw + (sbase - raw) + NS * Tile::STAGE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;   // [2]
  uint64_t* tempty = tfull + 2;   // [2]
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* n_loaded = abort_flag + 1;   // K-steps whose copies were issued
  volatile int* n_mma = abort_flag + 2;      // K-steps whose MMAs were issued

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RT = Mp / TC_BM;
  const int CT = (R + BNC - 1) / BNC;
  const int64_t items = F * batch.n * CT * RT;
  const int64_t my_items = (int64_t)blockIdx.x < items ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int KS = Kp / TC_BK;
  // item -> (f, operator, column tile, row tile), row tiles fastest
  auto decode = [&](int64_t it, int64_t& f, int& op, int& ct, int& rt) {
    rt = (int)(it % RT);
    it /= RT;
    ct = (int)(it % CT);
    it /= CT;
    op = (int)(it % batch.n);
    f = it / batch.n;
  };

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 4);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    *n_loaded = 0;
    *n_mma = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    tmem_alloc(smem_u32(tmem_slot), Tile::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint32_t tx_bytes = (uint32_t)(Tile::A_BYTES + bn_rows * TC_BK * 2);
    int64_t kt = 0;
    bool stop = false;
    for (int64_t c = 0; c < my_items && !stop; ++c) {
      int64_t f;
      int op, ct, rt;
      decode(blockIdx.x + c * gridDim.x, f, op, ct, rt);
      const int arow = (int)(f * Mp + rt * TC_BM);
      const int xrow = (int)(f * ctot + (int64_t)batch.blk[op] * R + ct * BNC);
      for (int ks = 0; ks < KS; ++ks, ++kt) {
        const int s = (int)(kt % NS);
        if (kt >= NS && !mbar_wait_abortable(smem_u32(&empty[s]), (uint32_t)(((kt / NS) - 1) & 1), abort_flag)) {
          stop = true;
          break;
        }
        const uint32_t sa = sbase + s * Tile::STAGE_BYTES, sb = sa + Tile::A_BYTES;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, tx_bytes);
        tma_load_2d(sa, &maps.a[op], fb, ks * TC_BK, arow);
        tma_load_2d(sb, &maps.x, fb, ks * TC_BK, xrow);
      }
    }
    *n_loaded = (int)kt;
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    int64_t kt = 0;
    bool stop = false;
    for (int64_t c = 0; c < my_items && !stop; ++c) {
      const int buf = (int)(c & 1);
      if (c >= 2 && !mbar_wait_abortable(smem_u32(&tempty[buf]), (uint32_t)(((c >> 1) - 1) & 1), abort_flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(buf * BNC);
      for (int ks = 0; ks < KS; ++ks, ++kt) {
        const int s = (int)(kt % NS);
        if (!mbar_wait_abortable(smem_u32(&full[s]), (uint32_t)((kt / NS) & 1), abort_flag)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = sbase + s * Tile::STAGE_BYTES, b0 = a0 + Tile::A_BYTES;
#pragma unroll
        for (int q = 0; q < TC_BK / 16; ++q)
          tc_mma(d, smem_desc_sw128(a0 + 32 * q), smem_desc_sw128(b0 + 32 * q), idesc, (ks | q) != 0);
        tc_commit(smem_u32(&empty[s]));
      }
      if (!stop) tc_commit(smem_u32(&tfull[buf]));
    }
    *n_mma = (int)kt;
    tc_commit(smem_u32(done));
  } else if (warp >= 4) {
    const int quarter = warp & 3;
    for (int64_t c = 0; c < my_items; ++c) {
      const int buf = (int)(c & 1);
      if (!mbar_wait_sleepy_abortable(smem_u32(&tfull[buf]), (uint32_t)((c >> 1) & 1), abort_flag)) break;
      tc_fence_after();
      int64_t f;
      int op, ct, rt;
      decode(blockIdx.x + c * gridDim.x, f, op, ct, rt);
      const int gm = rt * TC_BM + quarter * 32 + lane;
      const bool row_ok = gm < 2 * B;
      const int b = gm >> 1, part = gm & 1;
      const int64_t ybase = f * ctot + (int64_t)batch.blk[op] * R;
#pragma unroll 1
      for (int c0 = 0; c0 < n; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BNC + c0), v);
        if (row_ok) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int j = ct * BNC + c0 + t;
            if (j < R && c0 + t < bn_rows) {
              const int64_t e = (ybase + j) * B + b;
              if (f32_out)
                reinterpret_cast<float*>(reinterpret_cast<float2*>(y_) + e)[part] = v[t];
              else
                reinterpret_cast<float2*>(reinterpret_cast<float4*>(y_) + e)[part] = make_float2(v[t], 0.f);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
    }
  }
  __syncwarp();
  const bool mma_done = mbar_wait_sleepy(smem_u32(done), 0);
  const bool bad = __syncthreads_or(!mma_done || *abort_flag != 0);
  if (bad && tid == 0) {
    for (int kt = *n_mma; kt < *n_loaded; ++kt) mbar_wait_bounded(smem_u32(&full[kt % NS]), (kt / NS) & 1);
    atomicOr(err, 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, Tile::TMEM_COLS);
}

__device__ __forceinline__ __nv_bfloat16 to_bf16(double v) { return __float2bfloat16_rn(__double2float_rn(v)); }

__global__ void k_tc_realify(const cd* __restrict__ T, int64_t m, int64_t k, int64_t Mh, int64_t Kh, int64_t total,
                             __nv_bfloat162* __restrict__ A) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t per = Mh * Kh;
  const int64_t o = idx / per, rem = idx - o * per;
  const int64_t i = rem / Kh, j = rem - i * Kh;
  cd v = mkc(0.0, 0.0);
  if (i < m && j < k) v = T[(o * m + i) * k + j];
  const __nv_bfloat16 re = to_bf16(v.x), im = to_bf16(v.y), nim = to_bf16(-v.y);
  // rows 2i and 2i+1 of the realified block, each Kp = 2 Kh values (Kh pairs)
  __nv_bfloat162* base = A + o * (2 * Mh) * Kh;
  __nv_bfloat162 top, bot;
  top.x = re;
  top.y = nim;
  bot.x = im;
  bot.y = re;
  base[(2 * i) * Kh + j] = top;
  base[(2 * i + 1) * Kh + j] = bot;
}

// Float-float (float4: re_hi, re_lo, im_hi, im_lo) sources: the value is
// hi + lo, whose FP32 rounding is hi for normalised pairs.
__device__ __forceinline__ __nv_bfloat16 ff_to_bf16(float hi, float lo) {
  return __float2bfloat16_rn(__double2float_rn((double)hi + (double)lo));
}

__global__ void k_tc_realify_ff(const float4* __restrict__ T, int64_t m, int64_t k, int64_t Mh, int64_t Kh,
                                int64_t total, __nv_bfloat162* __restrict__ A) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t per = Mh * Kh;
  const int64_t o = idx / per, rem = idx - o * per;
  const int64_t i = rem / Kh, j = rem - i * Kh;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < m && j < k) v = T[(o * m + i) * k + j];
  const __nv_bfloat16 re = ff_to_bf16(v.x, v.y), im = ff_to_bf16(v.z, v.w), nim = ff_to_bf16(-v.z, -v.w);
  __nv_bfloat162* base = A + o * (2 * Mh) * Kh;
  __nv_bfloat162 top, bot;
  top.x = re;
  top.y = nim;
  bot.x = im;
  bot.y = re;
  base[(2 * i) * Kh + j] = top;
  base[(2 * i + 1) * Kh + j] = bot;
}

__device__ __forceinline__ __nv_bfloat162 bf16_pair(cd v) {
  __nv_bfloat162 p;
  p.x = to_bf16(v.x);
  p.y = to_bf16(v.y);
  return p;
}
__device__ __forceinline__ __nv_bfloat162 bf16_pair(float4 v) {
  __nv_bfloat162 p;
  p.x = ff_to_bf16(v.x, v.y);
  p.y = ff_to_bf16(v.z, v.w);
  return p;
}
__device__ __forceinline__ __nv_bfloat162 bf16_pair(float2 v) {
  __nv_bfloat162 p;
  p.x = __float2bfloat16_rn(v.x);
  p.y = __float2bfloat16_rn(v.y);
  return p;
}
// Rows of X: one warp per row, the lanes over its Kh (re, im) pairs (reads of
// consecutive complex values, 4-byte stores, zeros past k).
template <typename Src>
__global__ void k_tc_rows(const Src* __restrict__ x, int k, int Kh, int64_t rows, __nv_bfloat162* __restrict__ X) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const int lane = threadIdx.x & 31;
  const Src* __restrict__ xr = x + row * k;
  __nv_bfloat162* __restrict__ Xr = X + row * Kh;
  for (int j = lane; j < Kh; j += 32) {
    __nv_bfloat162 p;
    p.x = p.y = __float2bfloat16_rn(0.f);
    if (j < k) p = bf16_pair(xr[j]);
    Xr[j] = p;
  }
}

// cuTensorMapEncodeTiled, fetched from the driver once (the library does not
// link the driver library itself).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// A BF16 tensor of `rank` dimensions (dims innermost first, byte strides of
// dims 1..rank-1) read in boxes `box` with the 128-byte swizzle; elements
// outside the tensor read as zero.
fmpb_status encode_map(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                       const cuuint64_t* strides, const cuuint32_t* box) {
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) {
    set_error("tensor-core product: the driver offers no cuTensorMapEncodeTiled");
    return FMPB_ECUDA;
  }
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor-core product: tensor map encoding failed (driver status %d)", (int)r);
    return FMPB_ECUDA;
  }
  return FMPB_OK;
}

// The brick of cells x right-hand sides per output tile, at most `cap`
// columns: the one with the least work counted as tiles x (N + 128), N the
// MMA width of a tile (its columns rounded up to 16) and 128 the rows of A a
// tile copies per K-step in units of B rows (ties: more columns per tile).
TcBrick pick_brick(int Mx, int My, int Mz, int R, int cap) {
  TcBrick best{};
  double best_cost = INFINITY;
  for (int bx = 1; bx <= std::min(Mx, cap); ++bx)
    for (int by = 1; by <= std::min(My, cap / bx); ++by)
      for (int bz = 1; bz <= std::min(Mz, cap / (bx * by)); ++bz) {
        const int br = std::min(R, cap / (bx * by * bz));
        TcBrick b{bx, by, bz, br, (Mx + bx - 1) / bx, (My + by - 1) / by, (Mz + bz - 1) / bz, (R + br - 1) / br,
                  bx * by * bz * br, 0};
        b.n = (b.rows + 15) / 16 * 16;
        const double cost = (double)b.ntx * b.nty * b.ntz * b.ntr * (b.n + 128);
        if (cost < best_cost || (cost == best_cost && b.rows > best.rows)) {
          best_cost = cost;
          best = b;
        }
      }
  return best;
}

template <int MT, int BNC>
fmpb_status launch_tma(const TcBatch& A, int64_t Mp, int64_t Kp, const __nv_bfloat16* X, void* y, int64_t m,
                       int64_t ncols, const int M[3], int R, const TcOffsets& offs, const TcTail* tail,
                       bool accumulate, bool y_f32, unsigned* err, cudaStream_t st) {
  using Tile = TmaTile<MT, BNC>;
  const TcBrick bk = pick_brick(M[0], M[1], M[2], R, BNC);
  const int64_t tiles = (int64_t)bk.ntx * bk.nty * bk.ntz * bk.ntr;
  if (tiles * A.n > 65535 || Mp * offs.n > INT32_MAX || (int64_t)R * A.nblk > INT32_MAX) {
    set_error("tensor-core product: %lld column tiles exceed the launch limit", (long long)(tiles * A.n));
    return FMPB_EINVAL;
  }
  TcMaps maps;
  memset(&maps, 0, sizeof(maps));
  {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)(Mp * offs.n)};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    for (int o = 0; o < A.n; ++o) FMPB_TRY(encode_map(&maps.a[o], A.A[o], 2, dims, strides, box));
  }
  {
    // the rows' real extent: their padding up to Kp reads as zero from the
    // copy engine, so whoever writes them may leave it untouched
    const cuuint64_t dims[5] = {(cuuint64_t)(A.kx > 0 ? A.kx : Kp), (cuuint64_t)M[0], (cuuint64_t)M[1], (cuuint64_t)M[2],
                                (cuuint64_t)R * A.nblk};
    const cuuint64_t strides[4] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * M[0], (cuuint64_t)Kp * 2 * M[0] * M[1],
                                   (cuuint64_t)Kp * 2 * M[0] * M[1] * M[2]};
    const cuuint32_t box[5] = {(cuuint32_t)TC_BK, (cuuint32_t)bk.bx, (cuuint32_t)bk.by, (cuuint32_t)bk.bz,
                               (cuuint32_t)bk.br};
    FMPB_TRY(encode_map(&maps.x, X, 5, dims, strides, box));
  }
  int kt2 = 0;
  if (tail) {
    const int64_t Kp2 = tc_depth(tail->k);
    kt2 = (int)(Kp2 / TC_BK);
    const cuuint64_t adims[2] = {(cuuint64_t)Kp2, (cuuint64_t)Mp};
    const cuuint64_t astrides[1] = {(cuuint64_t)Kp2 * 2};
    const cuuint32_t abox[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    for (int o = 0; o < A.n; ++o) FMPB_TRY(encode_map(&maps.a2[o], tail->A[o], 2, adims, astrides, abox));
    const cuuint64_t dims[5] = {(cuuint64_t)(2 * tail->k), (cuuint64_t)M[0], (cuuint64_t)M[1], (cuuint64_t)M[2],
                                (cuuint64_t)R * A.nblk};
    const cuuint64_t strides[4] = {(cuuint64_t)Kp2 * 2, (cuuint64_t)Kp2 * 2 * M[0],
                                   (cuuint64_t)Kp2 * 2 * M[0] * M[1], (cuuint64_t)Kp2 * 2 * M[0] * M[1] * M[2]};
    const cuuint32_t box[5] = {(cuuint32_t)TC_BK, (cuuint32_t)bk.bx, (cuuint32_t)bk.by, (cuuint32_t)bk.bz,
                               (cuuint32_t)bk.br};
    FMPB_TRY(encode_map(&maps.x2, tail->X, 5, dims, strides, box));
  }
  const int64_t rows = (int64_t)TC_BM * MT;
  const dim3 grid((unsigned)((Mp + rows - 1) / rows), (unsigned)(tiles * A.n));
  FMPB_CUDA((smem_limit_once<k_tc_gemm_tma<MT, BNC>>(Tile::SMEM)));
  FMPB_LAUNCH("tc_gemm", st,
              (k_tc_gemm_tma<MT, BNC><<<grid, TC_THREADS, Tile::SMEM, st>>>(
                  maps, A, bk, (int)Kp, (int)Mp, y, (int)m, ncols, M[0], M[1], M[2], R, offs, kt2,
                  accumulate ? 1 : 0, y_f32 ? 1 : 0, err)));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// Tile variants of the offset GEMM: (row tiles per CTA, output columns per CTA).
struct TcVariant {
  int mt, bn;
};
constexpr TcVariant TC_VARIANTS[] = {{1, 256}, {2, 256}, {2, 128}, {1, 128}};
constexpr int TC_NVARIANTS = sizeof(TC_VARIANTS) / sizeof(TC_VARIANTS[0]);

fmpb_status launch_offset_variant(int v, const TcBatch& A, int64_t Mp, int64_t Kp, const __nv_bfloat16* X,
                                  void* y, int64_t m, int64_t ncols, const int M[3], int R, const TcOffsets& offs,
                                  const TcTail* tail, bool accumulate, bool y_f32, unsigned* err, cudaStream_t st) {
  switch (v) {
    case 0: return launch_tma<1, 256>(A, Mp, Kp, X, y, m, ncols, M, R, offs, tail, accumulate, y_f32, err, st);
    case 1: return launch_tma<2, 256>(A, Mp, Kp, X, y, m, ncols, M, R, offs, tail, accumulate, y_f32, err, st);
    case 2: return launch_tma<2, 128>(A, Mp, Kp, X, y, m, ncols, M, R, offs, tail, accumulate, y_f32, err, st);
    default: return launch_tma<1, 128>(A, Mp, Kp, X, y, m, ncols, M, R, offs, tail, accumulate, y_f32, err, st);
  }
}

// Autotuner of the offset GEMM: the first call of a shape (device, m, k,
// columns, offsets) times every variant on the caller's stream with CUDA
// events (after one untimed launch each) and keeps the fastest; later calls
// of the shape launch it directly.  The variants compute the same sums in the
// same order (they only assign output tiles to CTAs differently).  Tuning runs
// of an accumulating call write into a scratch output, so the caller's y
// receives the product exactly once.
struct TuneKey {
  int dev;
  int64_t m, k, ncols;
  int noff, nbatch;
  int64_t k2;   // depth of a tail product (0: none)
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, m, k, ncols, noff, nbatch, k2) < std::tie(o.dev, o.m, o.k, o.ncols, o.noff, o.nbatch, o.k2);
  }
};
struct TuneEntry {
  int variant;
  float ms[TC_NVARIANTS];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;
int g_forced_variant = -1;   // >= 0: fmpb_set_tile_variant override

fmpb_status tune_offset_gemm(const TuneKey& key, const TcBatch& A, int64_t Mp, int64_t Kp,
                             const __nv_bfloat16* X, void* y, int64_t m, int64_t ncols, const int M[3], int R,
                             const TcOffsets& offs, const TcTail* tail, bool accumulate, bool y_f32, unsigned* err,
                             cudaStream_t st, int* chosen) {
  void* out = y;
  cd* scratch = nullptr;
  if (accumulate) {
    FMPB_CUDA(cudaMalloc(&scratch, sizeof(cd) * (size_t)ncols * A.nblk * m));
    out = scratch;
  }
  TuneEntry e{};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  fmpb_status s = FMPB_OK;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "tune events");
  float best = 1e30f;
  int bestv = 0;
  for (int v = 0; v < TC_NVARIANTS && s == FMPB_OK; ++v) {
    s = launch_offset_variant(v, A, Mp, Kp, X, out, m, ncols, M, R, offs, tail, false, y_f32, err, st);
    if (s == FMPB_OK && cudaEventRecord(t0, st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tune");
    if (s == FMPB_OK) s = launch_offset_variant(v, A, Mp, Kp, X, out, m, ncols, M, R, offs, tail, false, y_f32, err, st);
    if (s == FMPB_OK && (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess))
      s = cuda_status(cudaGetLastError(), "tune");
    float ms = 0.f;
    if (s == FMPB_OK && cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tune");
    e.ms[v] = ms;
    if (s == FMPB_OK && ms < best) {
      best = ms;
      bestv = v;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (scratch) {
    cudaStreamSynchronize(st);
    cudaFree(scratch);
  }
  if (s != FMPB_OK) return s;
  e.variant = bestv;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = e;
  }
  *chosen = bestv;
  return FMPB_OK;
}

}  // namespace

fmpb_status tc_realify(const cd* T, int n_off, int64_t m, int64_t k, __nv_bfloat16* A, cudaStream_t st) {
  const int64_t Mh = tc_rows(m) / 2, Kh = tc_depth(k) / 2;
  const int64_t total = (int64_t)n_off * Mh * Kh;
  FMPB_LAUNCH("tc_realify", st,
              k_tc_realify<<<grid_for((size_t)total, 256), 256, 0, st>>>(T, m, k, Mh, Kh, total,
                                                                          reinterpret_cast<__nv_bfloat162*>(A)));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

template <typename Src>
fmpb_status rows_to_bf16(const Src* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st) {
  const int64_t Kh = tc_depth(k) / 2;
  if (rows == 0) return FMPB_OK;
  if (Kh > INT32_MAX) {
    set_error("tensor-core rows: depth %lld too large", (long long)k);
    return FMPB_EINVAL;
  }
  FMPB_LAUNCH("tc_to_bf16", st,
              k_tc_rows<Src><<<grid_for((size_t)rows * 32, 256), 256, 0, st>>>(
                  x, (int)k, (int)Kh, rows, reinterpret_cast<__nv_bfloat162*>(X)));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status tc_rows_to_bf16(const cd* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st) {
  return rows_to_bf16(x, rows, k, X, st);
}

fmpb_status tc_realify_ff(const float4* T, int n_off, int64_t m, int64_t k, __nv_bfloat16* A, cudaStream_t st) {
  const int64_t Mh = tc_rows(m) / 2, Kh = tc_depth(k) / 2;
  const int64_t total = (int64_t)n_off * Mh * Kh;
  FMPB_LAUNCH("tc_realify", st,
              k_tc_realify_ff<<<grid_for((size_t)total, 256), 256, 0, st>>>(T, m, k, Mh, Kh, total,
                                                                             reinterpret_cast<__nv_bfloat162*>(A)));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status tc_rows_from_ff(const float4* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st) {
  return rows_to_bf16(x, rows, k, X, st);
}

fmpb_status tc_rows_from_f32(const float2* x, int64_t rows, int64_t k, __nv_bfloat16* X, cudaStream_t st) {
  return rows_to_bf16(x, rows, k, X, st);
}

fmpb_status tc_offset_gemm(const __nv_bfloat16* A, const TcOffsets& offs, int64_t m, int64_t k, const int M[3], int R,
                           const __nv_bfloat16* X, cd* y, bool accumulate, unsigned* err, cudaStream_t st) {
  return tc_offset_gemm_batch(&A, 1, offs, m, k, M, R, X, y, accumulate, err, st);
}

fmpb_status tc_offset_gemm_batch(const __nv_bfloat16* const* Aops, int n_ops, const TcOffsets& offs, int64_t m,
                                 int64_t k, const int M[3], int R, const __nv_bfloat16* X, void* y, bool accumulate,
                                 unsigned* err, cudaStream_t st, const int* blk, const __nv_bfloat16* const* A2,
                                 int64_t k2, const __nv_bfloat16* X2, bool y_f32) {
  if (n_ops < 1 || n_ops > TC_MAX_BATCH) {
    set_error("tc_offset_gemm: %d operators in a batch (1..%d)", n_ops, TC_MAX_BATCH);
    return FMPB_EINVAL;
  }
  TcBatch A{};
  A.n = n_ops;
  A.nblk = 0;
  for (int o = 0; o < n_ops; ++o) {
    A.A[o] = Aops[o];
    A.blk[o] = blk ? blk[o] : o;
    A.nblk = std::max(A.nblk, A.blk[o] + 1);
  }
  A.kx = 2 * k;
  const int64_t Mp = tc_rows(m), Kp = tc_depth(k);
  const int64_t Nc = (int64_t)M[0] * M[1] * M[2];
  const int64_t ncols = Nc * R;
  if (offs.n < 1 || offs.n > TC_MAX_OFF || m < 1 || k < 1 || R < 1 || Nc < 1) {
    set_error("tc_offset_gemm: bad shape (offsets %d, m %lld, k %lld, R %d)", offs.n, (long long)m, (long long)k, R);
    return FMPB_EINVAL;
  }
  if ((ncols + 127) / 128 > 65535 || Mp / TC_BM > 65535 || Kp > (1 << 24) || Nc > (1 << 30)) {
    set_error("tc_offset_gemm: %lld columns exceed the launch limit", (long long)ncols);
    return FMPB_EINVAL;
  }
  TcTail tail{};
  const bool has_tail = A2 != nullptr;
  if (has_tail) {
    if (!X2 || k2 < 1 || tc_depth(k2) > (1 << 24)) {
      set_error("tc_offset_gemm: bad tail product (depth %lld)", (long long)k2);
      return FMPB_EINVAL;
    }
    for (int o = 0; o < n_ops; ++o) tail.A[o] = A2[o];
    tail.k = k2;
    tail.X = X2;
  }
  int dev = 0;
  FMPB_CUDA(cudaGetDevice(&dev));
  // single products and batches tune apart; a batch's choice holds for any
  // operator count (the tile grid only grows by whole copies of one
  // operator's), so operators dropping out of a batched solve cost no retuning
  const TuneKey key{dev, m, k, ncols, offs.n, n_ops == 1 ? 1 : 2, has_tail ? k2 : 0};
  int v = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (g_forced_variant >= 0)
      v = g_forced_variant;
    else if (it != g_tune.end())
      v = it->second.variant;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FMPB_CUDA(cudaStreamIsCapturing(st, &cap));
  if (v < 0 && cap == cudaStreamCaptureStatusNone)
    FMPB_TRY(tune_offset_gemm(key, A, Mp, Kp, X, y, m, ncols, M, R, offs, has_tail ? &tail : nullptr, accumulate,
                              y_f32, err, st, &v));
  if (v < 0) v = 0;   // no tuning inside a stream capture
  return launch_offset_variant(v, A, Mp, Kp, X, y, m, ncols, M, R, offs, has_tail ? &tail : nullptr, accumulate,
                               y_f32, err, st);
}

fmpb_status tc_force_variant(int v) {
  if (v < -1 || v >= TC_NVARIANTS) {
    set_error("set_tile_variant: variant %d outside -1..%d", v, TC_NVARIANTS - 1);
    return FMPB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_forced_variant = v;
  return FMPB_OK;
}

fmpb_status tc_tuning_summary(std::string& out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  out = "[";
  bool first = true;
  char buf[512];
  for (const auto& kv : g_tune) {
    const TcVariant t = TC_VARIANTS[kv.second.variant];
    int n = snprintf(buf, sizeof(buf),
                     "%s{\"kernel\": \"tc_gemm\", \"device\": %d, \"m\": %lld, \"k\": %lld, \"columns\": %lld, "
                     "\"offsets\": %d, \"batched\": %s, \"rows_per_cta\": %d, \"columns_per_cta\": %d, \"ms\": [",
                     first ? "" : ", ", kv.first.dev, (long long)kv.first.m, (long long)kv.first.k,
                     (long long)kv.first.ncols, kv.first.noff, kv.first.nbatch > 1 ? "true" : "false",
                     TC_BM * t.mt, t.bn);
    out.append(buf, n);
    for (int v = 0; v < TC_NVARIANTS; ++v) {
      n = snprintf(buf, sizeof(buf), "%s%.4f", v ? ", " : "", kv.second.ms[v]);
      out.append(buf, n);
    }
    out += "]}";
    first = false;
  }
  out += "]";
  return FMPB_OK;
}

// SMs of the current device (the persistent grids' size), read once per device.
int sm_count() {
  static std::mutex mu;
  static std::map<int, int> counts;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = counts.find(dev);
  if (it != counts.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  counts[dev] = n;
  return n;
}

template <int BNC>
fmpb_status launch_freq(const TcBatch& A, int64_t F, int64_t B, int R, const __nv_bfloat16* X, void* Y, bool y_f32,
                        unsigned* err, cudaStream_t st) {
  using Tile = FreqTile<BNC>;
  const int64_t Mp = tc_rows(B), Kp = tc_depth(B);
  const int64_t ctot = (int64_t)R * A.nblk;
  const int bn_rows = std::min(R, BNC);
  const int n = (bn_rows + 15) / 16 * 16;
  TcMaps maps;
  memset(&maps, 0, sizeof(maps));
  {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)(F * Mp)};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    for (int o = 0; o < A.n; ++o) FMPB_TRY(encode_map(&maps.a[o], A.A[o], 2, dims, strides, box));
  }
  {
    // the rows' real extent is 2 B values: the padding up to Kp reads as zero
    // from the copy engine, so whoever writes the rows may leave it untouched
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * B), (cuuint64_t)(F * ctot)};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)bn_rows};
    FMPB_TRY(encode_map(&maps.x, X, 2, dims, strides, box));
  }
  const int64_t items = F * A.n * ((R + BNC - 1) / BNC) * (Mp / TC_BM);
  const unsigned grid = (unsigned)std::min<int64_t>(items, sm_count());
  FMPB_CUDA((smem_limit_once<k_tc_freq_tma<BNC>>(Tile::SMEM)));
  FMPB_LAUNCH("tc_block_product", st,
              (k_tc_freq_tma<BNC><<<grid, TC_THREADS, Tile::SMEM, st>>>(maps, A, (int)Kp, (int)Mp, F, (int)B, R, ctot,
                                                                       bn_rows, n, Y, y_f32 ? 1 : 0, err)));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status tc_freq_gemm(const __nv_bfloat16* A, int64_t F, int64_t B, int R, const __nv_bfloat16* X, void* Y,
                         unsigned* err, cudaStream_t st, bool y_f32) {
  return tc_freq_gemm_batch(&A, 1, F, B, R, X, Y, err, st, y_f32);
}

fmpb_status tc_freq_gemm_batch(const __nv_bfloat16* const* Aops, int n_ops, int64_t F, int64_t B, int R,
                               const __nv_bfloat16* X, void* Y, unsigned* err, cudaStream_t st, bool y_f32,
                               const int* blk, int n_blocks) {
  if (n_ops < 1 || n_ops > TC_MAX_BATCH) {
    set_error("tc_freq_gemm: %d operators in a batch (1..%d)", n_ops, TC_MAX_BATCH);
    return FMPB_EINVAL;
  }
  TcBatch A{};
  A.n = n_ops;
  A.nblk = n_blocks > 0 ? n_blocks : n_ops;
  for (int o = 0; o < n_ops; ++o) {
    A.A[o] = Aops[o];
    A.blk[o] = blk ? blk[o] : o;
    if (A.blk[o] < 0 || A.blk[o] >= A.nblk) {
      set_error("tc_freq_gemm: operator block %d outside 0..%d", A.blk[o], A.nblk - 1);
      return FMPB_EINVAL;
    }
  }
  const int64_t Mp = tc_rows(B), Kp = tc_depth(B);
  if (F < 1 || B < 1 || R < 1 || Mp / TC_BM > 65535 || Kp > (1 << 24)) {
    set_error("tc_freq_gemm: bad shape (F %lld, B %lld, R %d)", (long long)F, (long long)B, R);
    return FMPB_EINVAL;
  }
  if ((int64_t)F * Mp > INT32_MAX || (int64_t)F * R * A.nblk > INT32_MAX) {
    set_error("tc_freq_gemm: %lld frequencies exceed the copy coordinates", (long long)F);
    return FMPB_EINVAL;
  }
  const int BN = R <= 32 ? 32 : (R <= 64 ? 64 : (R <= 128 ? 128 : 256));
  switch (BN) {
    case 32: return launch_freq<32>(A, F, B, R, X, Y, y_f32, err, st);
    case 64: return launch_freq<64>(A, F, B, R, X, Y, y_f32, err, st);
    case 128: return launch_freq<128>(A, F, B, R, X, Y, y_f32, err, st);
    default: return launch_freq<256>(A, F, B, R, X, Y, y_f32, err, st);
  }
}

}  // namespace fmpb
