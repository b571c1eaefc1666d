// Row probes of a mixed-precision plan: X = G A (the product behind the row
// estimate of Sec. 3.3) at FP64 grade from the complex64 A, in one pass over
// A.  The arithmetic is the exact-slice emulation of rid_sketch_tc.cu: G' and
// A' in the real view, balanced base-256 digits relative to a row exponent
// (G') and a 256-real chunk exponent (A'), BF16 x BF16 products summed in FP32
// per chunk and flushed into double-FP32 running sums.  What differs:
//
// No digit tiles of A in memory.  Tensor copies bring each K stage of raw
// complex64 A (16 rows x 128 columns) into a shared-memory ring; slicer warps
// cut it into the stage's seven digit tiles of A' in shared memory and hand
// them to the MMA warp.  (The plan's FP64-emulated sketch writes A's digits to
// HBM first, 3.5 times A's bytes for complex64, and reads them back.)  The
// chunk exponents are taken by the mixed sketch's BF16x3 slicer, which reads
// every entry of A first anyway (rid_sketch_mixed.cu); they are stored as
// [chunk][column].  The digits are formed by FP32 rounding steps
// (digit_words_fp).
//
// Seven MMAs per K16 step instead of 28.  G' has only 2 r <= 32 rows (W rows
// per digit, W = 16 or 32), so a product of one A digit tile t with one G
// digit block s is a narrow MMA.  Each stage's G digit blocks sit one after
// the other in shared memory, so B_t = [G_0, ..., G_(6-t)] is one operand of
// W (7 - t) rows; one MMA A_t x B_t, whose accumulator starts at column W t,
// adds the product of digit pair (s, t) to columns W (s + t) .. + W - 1.  So
// column block d holds diagonal d = s + t, and the pairs with s + t > 6 are
// not formed, as in the wide product.  Every diagonal has its own columns
// (the wide product shares one group for d >= 3), which keeps every chunk
// sum of a diagonal exact.
//
// Each CTA keeps its own running exponent per column (the largest chunk
// exponent it has seen; the double-FP32 sums are rescaled by a power of two
// when it grows), and the reduction scales each K-split's partial sum by
// its own exponent.  Results depend only on the column and the plan's
// K-split, so column panels give the one-call X bit for bit.
#include <cudaTypedefs.h>

#include "rid_internal.cuh"
#include "rid_tc.cuh"
#include "rid_tc_digits.cuh"

using namespace rid_tc;

namespace {

constexpr int PB_SLICE_WARPS = 16;           // warps that cut A's digits
constexpr int PB_NS = 2;                     // digit stages in flight
constexpr int PB_MAX_RAW = 6;                // raw A stages in flight, at most
constexpr int PB_RAW_ROWS = 16;              // complex rows of A per K stage
constexpr uint32_t PB_RAW_BYTES = 128 * PB_RAW_ROWS * 8;   // one raw stage: 128 columns x 128 bytes

// Shared memory of one digit stage: seven A digit tiles (128 rows x 64
// bytes), then seven G digit blocks of W rows x 64 bytes.
__host__ __device__ constexpr uint32_t pb_block_bytes(int W) { return (uint32_t)W * TC_KS * 2; }
__host__ __device__ constexpr uint32_t pb_om_off(int) { return (uint32_t)(TC_S * TC_TILE_BYTES); }
__host__ __device__ constexpr uint32_t pb_om_bytes(int W) { return TC_S * pb_block_bytes(W); }
__host__ __device__ constexpr uint32_t pb_slot_bytes(int W) { return (pb_om_off(W) + pb_om_bytes(W) + 1023) / 1024 * 1024; }
// raw stages: what shared memory holds after the digit stages (2 KB for the
// static part, 1 KB for alignment)
__host__ __device__ constexpr int pb_raw_stages(int W) {
  return (int)((TC_SMEM_LIMIT - 2048 - 1024 - PB_NS * pb_slot_bytes(W)) / PB_RAW_BYTES) < PB_MAX_RAW
             ? (int)((TC_SMEM_LIMIT - 2048 - 1024 - PB_NS * pb_slot_bytes(W)) / PB_RAW_BYTES)
             : PB_MAX_RAW;
}
__host__ __device__ constexpr uint32_t pb_raw_off(int W) { return PB_NS * pb_slot_bytes(W); }
__host__ __device__ constexpr int pb_dyn_smem(int W) {
  return (int)(pb_raw_off(W) + pb_raw_stages(W) * PB_RAW_BYTES + 1024);
}

// Warp roles, by W (rows of G' per digit block):
//   warps 0 .. FW-1      flush (FW = W / 4): TMEM lane quarter w % 4, digit-block
//                        columns 16 (w / 4) .. + 15, one column of A per thread;
//   FW .. FW+15          slicers: per stage, thread t cuts the 16-byte piece
//                        t % 4 (4 complex rows) of column t / 4;
//   FW+16                lane 0 issues the tensor copies of raw A and the bulk
//                        copies of G's digit blocks;
//   FW+17                MMA issuer (whole warp, one elected lane issues), TMEM owner.
__host__ __device__ constexpr int pb_flush_warps(int W) { return W / 4; }
__host__ __device__ constexpr int pb_threads(int W) { return 32 * (pb_flush_warps(W) + PB_SLICE_WARPS + 2); }

struct ProbeState {
  int nrows;            // probe rows r
  int W;                // rows of G' per digit block: 2 r rounded up to 16 or 32
  int NC;               // chunks of 128 complex rows (256 reals of K = 2m)
  int64_t KP;           // NC x 256
  int ksplit, chunks_per_split;
  uint16_t* om_tiles;   // [K stage][digit][W rows x TC_KS] bf16, swizzled
  int* om_exp;          // [2 r]
  int* cexp;            // [NC][n]: chunk exponents of A (written by the mixed slicer)
  float2* partial;      // [ksplit][n][W]: (hi, lo) of each running sum
  int* part_exp;        // [ksplit][n]: the exponent the split's sums are relative to
  int* err;             // device error word
};

struct PbArgs {
  const float2* A;      // the plan's first column
  int64_t lda, m, n;    // n: the plan's columns (the strides of cexp and the partials)
  int64_t col0;         // first column of the launch (a multiple of 128)
  int64_t j_end;        // columns below this are in the launch
  int NC, chunks_per_split;
  const uint16_t* om_tiles;
  const int* cexp;
  float2* partial;
  int* part_exp;
  int* err;
};

// N complex rows r0 .. r0 + N - 1 of a column from global memory (zeros past
// m or for a column outside the launch); the path for A whose columns are
// not 16-byte aligned (no tensor copies).
template <int N>
__device__ __forceinline__ void load_rows(const float2* __restrict__ col, int64_t r0, bool ok, int64_t m,
                                          float2 (&v)[N]) {
#pragma unroll
  for (int u = 0; u < N; ++u) v[u] = (ok && r0 + u < m) ? __ldg(col + r0 + u) : make_float2(0.f, 0.f);
}

// Digits of a float x in a chunk with exponent e (|x| < 2^e), by FP32
// arithmetic.  With t = x 2^(8-e) (|t| < 256; exact, or below 2^-126 where
// every digit is zero), for s = 0 .. 6 the digit v_s is t rounded to a
// multiple of 2^(-8s) (adding and subtracting M = 1.5 2^(23-8s) rounds to
// that grid, ties to even) and t -= v_s (exact).  So v_0 in [-256, 256],
// |v_s| <= 2^(-8s) 128, every v_s is exact in BF16, and sum v_s is
// x 2^(8-e) rounded to 2^-48: the value the integer cutter of
// rid_sketch_tc.cu forms, except at ties of the last digit (to even here,
// half up in magnitude there), under the same digit bounds.  Where 2^(8-e)
// is not a normal float (chunks of subnormals), x is first scaled by part
// of it.
struct ChunkScale {
  float pre;     // applied to x first when `split`
  float s;       // x (pre) s = x 2^(8-e)
  bool split;
};
__device__ __forceinline__ ChunkScale chunk_scale(int e) {
  if (e == TC_EXP_ZERO) return {1.f, 0.f, false};     // an all-zero chunk
  int p = 8 - e;
  if (p < -126) p = -126;                             // only for infinities and NaNs
  if (p <= 127) return {1.f, __int_as_float((127 + p) << 23), false};
  const int p1 = p >> 1;
  return {__int_as_float((127 + p1) << 23), __int_as_float((127 + p - p1) << 23), true};
}

// The real and imaginary parts go through the steps together as FP32 pairs
// (one packed instruction per step): t = x sc, then per digit d = (t + M) - M
// and t = t - d (as d (-1) + t, exact).  Result: the TC_S packed words
// (re digit | im digit << 16) of one complex64 entry.
__device__ __forceinline__ void digit_words_fp(float2 x, float sc, uint32_t (&w)[TC_S]) {
  float2 t = __fmul2_rn(x, make_float2(sc, sc));
#pragma unroll
  for (int s = 0; s < TC_S; ++s) {
    const float M = __int_as_float(((150 - 8 * s) << 23) | 0x400000);   // 1.5 2^(23 - 8s)
    const float2 d = __fadd2_rn(__fadd2_rn(t, make_float2(M, M)), make_float2(-M, -M));
    w[s] = __byte_perm(__float_as_uint(d.x), __float_as_uint(d.y), 0x7632);
    if (s < TC_S - 1) t = __ffma2_rn(d, make_float2(-1.f, -1.f), t);
  }
}

// 2^k as a float for -126 <= k <= 127, else 0 (k < -126; only used there).
__device__ __forceinline__ float pow2f_or_zero(int k) { return k >= -126 ? __int_as_float((127 + k) << 23) : 0.f; }

// A 2-D tensor copy of rows x .. x + 15 of columns y .. y + 127 of A (8-byte
// elements) into a raw stage: 128 rows of 128 bytes, column after column, in
// the 128-byte swizzle (so the slicers' reads are free of bank conflicts);
// out-of-range rows and columns arrive as zeros.
__device__ __forceinline__ void tma_load_raw(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Grid (column blocks of the launch, K-splits).  TMA: raw A arrives by tensor
// copies (every column 16-byte aligned); otherwise the slicers load it.
template <int W, bool TMA>
__global__ void __launch_bounds__(pb_threads(W), 1)
probe_tc_kernel(const __grid_constant__ CUtensorMap map_a, PbArgs a) {
  constexpr int NB = W == 16 ? 4 : 2;          // accumulator buffers in TMEM
  constexpr int BUF = 512 / NB;                // their column stride
  constexpr int N = TC_S * W;                  // MMA N: seven diagonal blocks
  constexpr int NS = PB_NS, R = pb_raw_stages(W);
  constexpr int FW = pb_flush_warps(W);
  constexpr int SLICER0 = FW, PRODUCER = FW + PB_SLICE_WARPS, MMA = PRODUCER + 1;
  constexpr uint32_t SLOT = pb_slot_bytes(W), OOFF = pb_om_off(W), OBYTES = pb_om_bytes(W);
  constexpr uint32_t ROFF = pb_raw_off(W);
  static_assert(N <= 256 && N % 16 == 0, "MMA N");
  static_assert(R >= 2, "two raw stages at least");
  static_assert(PB_SLICE_WARPS == 16, "a slicer thread per 16-byte piece of a stage row");

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[NS], empty_bar[NS], raw_full[R], raw_empty[R], acc_full[NB], acc_empty[NB];
  __shared__ uint64_t mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ks = blockIdx.y;
  const int64_t jbase = a.col0 + (int64_t)blockIdx.x * 128;
  const int c_begin = ks * a.chunks_per_split;
  const int c_end = min(a.NC, c_begin + a.chunks_per_split);
  const int nchunks = max(0, c_end - c_begin);
  const int iters = nchunks * TC_SPC;

  if (warp == MMA) tmem_alloc(&tmem_slot, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full_bar[i], PB_SLICE_WARPS + 1);   // the slicer warps and the G copy
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < R; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], PB_SLICE_WARPS);
    }
    for (int g = 0; g < NB; ++g) {
      mbar_init(&acc_full[g], 1);
      mbar_init(&acc_empty[g], FW);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  auto fail = [&](int code) {
    s_abort = 1;
    atomicCAS(a.err, 0, code);
  };

  if (warp == PRODUCER) {
    if (lane == 0) {
      // ---------------- raw A (up to R stages ahead) and G's digit blocks ----------------
      if (TMA) prefetch_tensormap(&map_a);
      const uint16_t* src = a.om_tiles + (int64_t)c_begin * TC_SPC * (OBYTES / 2);
      int it = 0, rit = 0;
      for (; it < iters && !s_abort; ++it) {
        for (; TMA && rit < iters && rit < it + R; ++rit) {
          const int rs = rit % R;
          if (rit >= R && !mbar_wait(&raw_empty[rs], ((rit / R) - 1) & 1, TC_WAIT_BUDGET)) {
            fail(13);
            break;
          }
          mbar_arrive_expect_tx(&raw_full[rs], PB_RAW_BYTES);
          tma_load_raw(smem + ROFF + rs * PB_RAW_BYTES, &map_a, (c_begin * TC_SPC + rit) * PB_RAW_ROWS, (int)jbase,
                       &raw_full[rs]);
        }
        if (s_abort) break;
        const int ds = it % NS;
        if (it >= NS && !mbar_wait(&empty_bar[ds], ((it / NS) - 1) & 1, TC_WAIT_BUDGET)) {
          fail(11);
          break;
        }
        mbar_arrive_expect_tx(&full_bar[ds], OBYTES);
        bulk_load(smem + ds * SLOT + OOFF, src, OBYTES, &full_bar[ds]);
        src += OBYTES / 2;
      }
      // before the CTA may exit: every stage consumed, or after an error every
      // copy issued into this CTA landed
      for (int k = max(0, it - NS); k < it; ++k) {
        const bool ok = s_abort ? mbar_wait(&full_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET)
                                : mbar_wait(&empty_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET);
        if (!ok) fail(12);
      }
      for (int k = max(0, rit - R); k < rit; ++k) {
        const bool ok = s_abort ? mbar_wait(&raw_full[k % R], (k / R) & 1, TC_WAIT_BUDGET)
                                : mbar_wait(&raw_empty[k % R], (k / R) & 1, TC_WAIT_BUDGET);
        if (!ok) fail(14);
      }
    }
  } else if (warp == MMA) {
    // ---------------- MMA issuer ----------------
    for (int it = 0; it < iters && !s_abort; ++it) {
      const int cl = it / TC_SPC, b = it - cl * TC_SPC, g = cl % NB, ds = it % NS;
      if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[ds], (it / NS) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(21);
        break;
      }
      if (b == 0 && cl >= NB &&
          !__all_sync(0xffffffffu, mbar_wait(&acc_empty[g], ((cl / NB) - 1) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(22);
        break;
      }
      tc_fence_after();
      unsigned char* base = smem + ds * SLOT;
      const uint64_t db = tile_desc(base + OOFF);                   // B_t = G_0 .. G_(6-t)
#pragma unroll
      for (int t = 0; t < TC_S; ++t) {
        const uint64_t da = tile_desc(base + t * TC_TILE_BYTES);
        const uint32_t idesc = idesc_bf16_f32(128, W * (TC_S - t));
#pragma unroll
        for (int kk = 0; kk < TC_KS / 16; ++kk)
          mma_bf16_w(tmem + (uint32_t)(g * BUF + W * t), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                     (b == 0 && t == 0 && kk == 0) ? 0u : 1u);
      }
      mma_commit_w(&empty_bar[ds]);
      if (b == TC_SPC - 1) mma_commit_w(&acc_full[g]);
    }
    mma_commit_w(&mma_done);
  } else if (warp >= SLICER0 && warp < SLICER0 + PB_SLICE_WARPS) {
    // ---------------- slicers ----------------
    const int ti = threadIdx.x - 32 * SLICER0;
    const int jl = ti >> 2, q4 = ti & 3;         // column of the block; rows 4 q4 .. 4 q4 + 3 of each stage
    const int64_t j = jbase + jl;
    const bool j_ok = j < a.j_end;
    const float2* col = a.A + (j_ok ? j : 0) * a.lda;
    // the chunk exponent of this thread's column, a chunk ahead
    auto chunk_exp = [&](int cl) { return (j_ok && cl < nchunks) ? __ldg(a.cexp + (c_begin + cl) * a.n + j) : TC_EXP_ZERO; };
    const int pc = (q4 ^ ((jl >> 1) & 3)) << 4;  // the piece's swizzled place in its row
    int e_cur = chunk_exp(0), e_next = chunk_exp(1);
    float2 xg[4];                                // the direct-load path: the next stage's rows
    if (!TMA && iters > 0) load_rows<4>(col, (int64_t)c_begin * 128 + 4 * q4, j_ok, a.m, xg);
    for (int it = 0; it < iters && !s_abort; ++it) {
      const int cl = it / TC_SPC, b = it - cl * TC_SPC, ds = it % NS;
      if (b == 0 && cl > 0) {
        e_cur = e_next;
        e_next = chunk_exp(cl + 1);
      }
      float2 x[4];
      if (TMA) {
        const int rs = it % R;
        if (!__all_sync(0xffffffffu, mbar_wait(&raw_full[rs], (it / R) & 1, TC_WAIT_BUDGET))) {
          if (lane == 0) fail(43);
          break;
        }
        // the copy's 128-byte swizzle: 16-byte piece c of column jl sits at c ^ (jl % 8)
        const unsigned char* row = smem + ROFF + rs * PB_RAW_BYTES + jl * (PB_RAW_ROWS * 8);
        const float4 f0 = *(const float4*)(row + (((2 * q4) ^ (jl & 7)) << 4));
        const float4 f1 = *(const float4*)(row + (((2 * q4 + 1) ^ (jl & 7)) << 4));
        x[0] = make_float2(f0.x, f0.y);
        x[1] = make_float2(f0.z, f0.w);
        x[2] = make_float2(f1.x, f1.y);
        x[3] = make_float2(f1.z, f1.w);
        __syncwarp();
        if (lane == 0) mbar_arrive(&raw_empty[rs]);   // the raw stage is read
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = xg[u];
        if (it + 1 < iters) {
          const int c1 = c_begin + (it + 1) / TC_SPC, b1 = (it + 1) % TC_SPC;
          load_rows<4>(col, (int64_t)c1 * 128 + b1 * 16 + 4 * q4, j_ok, a.m, xg);
        }
      }
      const ChunkScale cs = chunk_scale(e_cur);
      if (cs.split) {
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = make_float2(x[u].x * cs.pre, x[u].y * cs.pre);
      }
      uint32_t w[4][TC_S];
#pragma unroll
      for (int u = 0; u < 4; ++u) digit_words_fp(x[u], cs.s, w[u]);
      if (it >= NS && !__all_sync(0xffffffffu, mbar_wait(&empty_bar[ds], ((it / NS) - 1) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(41);
        break;
      }
      unsigned char* piece = smem + ds * SLOT + jl * (TC_KS * 2) + pc;
#pragma unroll
      for (int s = 0; s < TC_S; ++s)
        *(uint4*)(piece + s * TC_TILE_BYTES) = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> the MMAs' reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[ds]);
    }
  } else if (warp < FW) {
    // ---------------- flush ----------------
    const int quarter = warp & 3, cbase = 16 * (warp >> 2);
    const int jl = 32 * quarter + lane;
    const int64_t j = jbase + jl;
    const bool j_ok = j < a.j_end;
    float hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      hi[i] = 0.f;
      lo[i] = 0.f;
    }
    int E = TC_EXP_ZERO;
    auto chunk_exp = [&](int cl) { return (j_ok && cl < nchunks) ? __ldg(a.cexp + (c_begin + cl) * a.n + j) : TC_EXP_ZERO; };
    int e_next = chunk_exp(0);
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cbase;
    for (int cl = 0; cl < nchunks && !s_abort; ++cl) {
      const int g = cl % NB;
      const int e = e_next;
      e_next = chunk_exp(cl + 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[g], (cl / NB) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(31);
        break;
      }
      tc_fence_after();
      if (e > E) {                       // a larger exponent: rescale the running sums (exact)
        const float f = pow2f_or_zero(E - e);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          hi[i] *= f;
          lo[i] *= f;
        }
        E = e;
      }
      const float scale = e == TC_EXP_ZERO ? 0.f : pow2f_or_zero(e - E);
#pragma unroll
      for (int d = 0; d < TC_S; ++d) {
        uint32_t r[16];
        tmem_ld16(lane_base + (uint32_t)(g * BUF + d * W), r);
        tmem_ld_wait();
        if (d == TC_S - 1) {             // the buffer is read: the MMAs may overwrite it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[g]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float v = __fmul_rn(__uint_as_float(r[i]), scale);
          const float s = __fadd_rn(hi[i], v);
          const float bp = __fsub_rn(s, hi[i]);
          const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(s, bp)), __fsub_rn(v, bp));
          hi[i] = s;
          lo[i] = __fadd_rn(lo[i], err);
        }
      }
    }
    if (!s_abort && j_ok) {
      float4* dst = (float4*)(a.partial + ((int64_t)ks * a.n + j) * W + cbase);
#pragma unroll
      for (int i = 0; i < 16; i += 2) dst[i / 2] = make_float4(hi[i], lo[i], hi[i + 1], lo[i + 1]);
      if (cbase == 0) a.part_exp[(int64_t)ks * a.n + j] = E;
    }
  }

  // ---------------- teardown ----------------
  tc_fence_before();
  __syncthreads();
  if (warp == MMA) {
    if (!mbar_wait(&mma_done, 0, TC_WAIT_BUDGET)) fail(91);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// X(i, j) = sum over the K-splits of 2^(E_split(j) + e_G(2i) - 16) (hi + lo) of
// rows 2i (real part) and 2i + 1 (imaginary part), the splits in order.
__global__ void probe_reduce_kernel(const float2* __restrict__ partial, const int* __restrict__ part_exp, int ksplit,
                                    int64_t n, int nrows, int W, const int* __restrict__ om_exp,
                                    double2* __restrict__ X, int64_t ldx, int64_t j0, int64_t ncols) {
  const int64_t total = ncols * nrows;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + e / nrows;
    const int i = (int)(e - (j - j0) * nrows);
    const int er = om_exp[2 * i] - 16, ei = om_exp[2 * i + 1] - 16;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ksplit; ++s) {
      const int E = part_exp[(int64_t)s * n + j];
      if (E == TC_EXP_ZERO) continue;
      const float4 q = *(const float4*)(partial + ((int64_t)s * n + j) * W + 2 * i);
      re += ldexp((double)q.x + (double)q.y, E + er);
      im += ldexp((double)q.z + (double)q.w, E + ei);
    }
    X[i + j * ldx] = make_double2(re, im);
  }
}

void probe_free_state(rid_plan_s* p, ProbeState* st) {
  if (!st) return;
  rid_dev_free(st->om_tiles, p->stream);   // start of the single allocation
  free(st);
}

const void* probe_kernel_fn(int W, bool tma) {
  if (W == 16) return tma ? (const void*)probe_tc_kernel<16, true> : (const void*)probe_tc_kernel<16, false>;
  return tma ? (const void*)probe_tc_kernel<32, true> : (const void*)probe_tc_kernel<32, false>;
}

// The tensor map of A for the raw stages: A as m x n 8-byte elements (columns
// lda apart), boxes of 16 rows x 128 columns, 128-byte swizzle (the raw
// stages start on 1024-byte boundaries).  False if A's base or column
// stride is not 16-byte aligned (the slicers then load A themselves).
bool make_map_a(CUtensorMap* map, const void* A, int64_t lda, int64_t m, int64_t n) {
  if (((uintptr_t)A & 15u) != 0 || lda % 2 != 0) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t gstride[1] = {(cuuint64_t)lda * 8};
  cuuint32_t box[2] = {PB_RAW_ROWS, 128};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, (void*)A, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// A mixed-precision plan's probe state: G's digit tiles (rows l .. l + r - 1 of
// Omega), A's chunk exponents, the partial sums and the error word.
rid_status rid_tc_probe_init(rid_plan_s* p) {
  if (p->nrow < 1 || p->nrow > 16 || p->dtype != RID_C64) return RID_EUNSUPPORTED;
  ProbeState* st = (ProbeState*)calloc(1, sizeof(ProbeState));
  if (!st) return RID_ENOMEM;
  st->nrows = p->nrow;
  st->W = 2 * p->nrow <= 16 ? 16 : 32;
  st->NC = (int)((2 * p->m + TC_KC - 1) / TC_KC);
  st->KP = (int64_t)st->NC * TC_KC;
  const int nblocks = (int)((p->n + 127) / 128);
  st->ksplit = rid_tc_choose_ksplit(nblocks, st->NC, p->num_sms > 0 ? p->num_sms : 1);
  st->chunks_per_split = (st->NC + st->ksplit - 1) / st->ksplit;
  st->ksplit = (st->NC + st->chunks_per_split - 1) / st->chunks_per_split;

  const size_t om_bytes = (size_t)TC_S * st->W * st->KP * 2;
  const size_t cexp_bytes = (size_t)st->NC * p->n * 4;
  const size_t part_bytes = (size_t)st->ksplit * p->n * st->W * 8;
  const size_t pexp_bytes = (size_t)st->ksplit * p->n * 4;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t total = al(om_bytes) + al((size_t)2 * st->nrows * 4) + al(cexp_bytes) + al(part_bytes) +
                       al(pexp_bytes) + al(4);
  char* base = nullptr;
  if (rid_dev_alloc((void**)&base, total, p->stream, p->device) != cudaSuccess) {
    free(st);
    return RID_ENOMEM;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { char* ptr = base + off; off += al(bytes); return ptr; };
  st->om_tiles = (uint16_t*)take(om_bytes);
  st->om_exp = (int*)take((size_t)2 * st->nrows * 4);
  st->cexp = (int*)take(cexp_bytes);
  st->partial = (float2*)take(part_bytes);
  st->part_exp = (int*)take(pexp_bytes);
  st->err = (int*)take(4);

  cudaError_t e = cudaMemsetAsync(st->err, 0, 4, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->om_tiles, 0, om_bytes, p->stream);   // rows 2 r .. W - 1
  if (e == cudaSuccess)
    e = rid_tc_cut_omega(p->omega + (int64_t)p->l * p->ldo, p->ldo, p->m, st->nrows, st->KP, st->W, false,
                         st->om_exp, st->om_tiles, p->num_sms, p->stream);
  for (int v = 0; v < 2 && e == cudaSuccess; ++v)
    e = cudaFuncSetAttribute(probe_kernel_fn(st->W, v == 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pb_dyn_smem(st->W));
  if (e != cudaSuccess) {
    probe_free_state(p, st);
    return RID_ECUDA;
  }
  p->tc_probe_state = st;
  p->tc_probe_bytes = total;
  return RID_OK;
}

void rid_tc_probe_free(rid_plan_s* p) {
  probe_free_state(p, (ProbeState*)p->tc_probe_state);
  p->tc_probe_state = nullptr;
  p->tc_probe_bytes = 0;
}

int* rid_tc_probe_chunk_exp(const rid_plan_s* p, int* nc) {
  const ProbeState* st = (const ProbeState*)p->tc_probe_state;
  if (!st) return nullptr;
  *nc = st->NC;
  return st->cexp;
}

// X(:, col0 .. col0 + ncols - 1) = G A(:, those columns); col0 a multiple of 128.
// The chunk exponents of these columns are in place (the mixed slicer ran).
cudaError_t rid_tc_probe_sketch_cols(const rid_plan_s* p, const void* A_, int64_t lda, int64_t col0, int64_t ncols) {
  const ProbeState* st = (const ProbeState*)p->tc_probe_state;
  if (!st) return cudaErrorNotSupported;
  if (ncols <= 0) return cudaSuccess;
  const int nblocks = (int)((ncols + 127) / 128);
  PbArgs args{(const float2*)A_, lda, p->m, p->n, col0, col0 + ncols, st->NC, st->chunks_per_split,
              st->om_tiles, st->cexp, st->partial, st->part_exp, st->err};
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const bool tma = make_map_a(&map, A_, lda, p->m, p->n);
  const dim3 grid((unsigned)nblocks, (unsigned)st->ksplit);
  void* params[] = {&map, &args};
  cudaError_t e = cudaLaunchKernel(probe_kernel_fn(st->W, tma), grid, dim3((unsigned)pb_threads(st->W)), params,
                                   (size_t)pb_dyn_smem(st->W), p->stream);
  if (e != cudaSuccess) return e;
  const int64_t total = ncols * (int64_t)st->nrows;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
  probe_reduce_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(st->partial, st->part_exp, st->ksplit, p->n,
                                                               st->nrows, st->W, st->om_exp, p->xrow, p->nrow, col0,
                                                               ncols);
  return cudaGetLastError();
}

cudaError_t rid_tc_probe_sketch(const rid_plan_s* p, const void* A_, int64_t lda) {
  return rid_tc_probe_sketch_cols(p, A_, lda, 0, p->n);
}

int rid_tc_probe_error_word(const rid_plan_s* p) {
  const ProbeState* st = (const ProbeState*)p->tc_probe_state;
  if (!st) return 0;
  int h = 0;
  cudaMemcpyAsync(&h, st->err, 4, cudaMemcpyDeviceToHost, p->stream);
  cudaStreamSynchronize(p->stream);
  return h;
}
