// Row probes of a mixed-precision plan: X = G A (the product behind the row
// estimate of Sec. 3.3) at FP64 grade from the complex64 A, in one pass over
// A.  The arithmetic is the exact-slice emulation of rid_sketch_tc.cu: G' and
// A' in the real view, balanced base-256 digits relative to a row exponent
// (G') and a 256-real chunk exponent (A'), BF16 x BF16 products summed in FP32
// per chunk and flushed into double-FP32 running sums.  Two things differ.
//
// No digit tiles of A in memory.  The complex64 A is read once; the kernel's
// slicer warps cut each K stage's seven digit tiles of A' into shared memory
// and hand them to the MMA warp (the plan's FP64-emulated sketch writes A's
// digits to HBM first, 3.5 times A's bytes for complex64, and reads them
// back).  A chunk's exponent is known before its digits are cut: the slicers
// take the maxima of chunk c + 1 while they cut chunk c.
//
// Seven MMAs per K16 step instead of 28.  G' has only 2 r <= 32 rows (W rows
// per digit, W = 16 or 32), so a product of one A digit tile t with one G
// digit block s is a narrow MMA.  Each stage's G digit blocks sit in shared
// memory behind six zero blocks: B_t = [0 (t blocks), G_0, ..., G_(6-t)]
// (7 W rows) starts (6 - t) blocks before G_0.  One MMA A_t x B_t (N = 7 W)
// adds the product of digit pair (s, t) to columns W (s + t) .. of the
// accumulator, so column block d holds diagonal d = s + t; the pairs with
// s + t > 6 are not formed, as in the wide product.  Every diagonal has its
// own columns (the wide product shares one group for d >= 3), which keeps
// every chunk sum of a diagonal exact.
//
// Each CTA keeps its own running exponent per column (the largest chunk
// exponent it has seen; the double-FP32 sums are rescaled by a power of two
// when it grows), and the reduction scales each K-split's partial sum by
// its own exponent.  Results depend only on the column and the plan's
// K-split, so column panels give the one-call X bit for bit.
#include "rid_internal.cuh"
#include "rid_tc.cuh"
#include "rid_tc_digits.cuh"

using namespace rid_tc;

namespace {

constexpr int PB_SLICE_WARPS = 8;            // warps 4..11 cut A's digits
constexpr int PB_FIRST_SLICER = 4;
constexpr int PB_EXP_RING = 8;               // chunks of exponents kept in shared memory
constexpr int PB_MAX_STAGES = 4;

// Shared memory of one pipeline stage: seven A digit tiles (128 rows x 64
// bytes), six zero blocks and seven G digit blocks of W rows x 64 bytes.
__host__ __device__ constexpr uint32_t pb_block_bytes(int W) { return (uint32_t)W * TC_KS * 2; }
__host__ __device__ constexpr uint32_t pb_zero_off() { return (uint32_t)(TC_S * TC_TILE_BYTES); }
__host__ __device__ constexpr uint32_t pb_om_off(int W) { return pb_zero_off() + (TC_S - 1) * pb_block_bytes(W); }
__host__ __device__ constexpr uint32_t pb_om_bytes(int W) { return TC_S * pb_block_bytes(W); }
__host__ __device__ constexpr uint32_t pb_slot_bytes(int W) { return (pb_om_off(W) + pb_om_bytes(W) + 1023) / 1024 * 1024; }
__host__ __device__ constexpr int pb_stages(int W) {
  return (int)((TC_SMEM_LIMIT - 8192 - 1024) / pb_slot_bytes(W)) < PB_MAX_STAGES
             ? (int)((TC_SMEM_LIMIT - 8192 - 1024) / pb_slot_bytes(W))
             : PB_MAX_STAGES;
}

struct ProbeState {
  int nrows;            // probe rows r
  int W;                // rows of G' per digit block: 2 r rounded up to 16 or 32
  int NC;               // chunks of 256 reals of K = 2m
  int64_t KP;           // NC x 256
  int ksplit, chunks_per_split;
  uint16_t* om_tiles;   // [K stage][digit][W rows x TC_KS] bf16, swizzled
  int* om_exp;          // [2 r]
  float2* partial;      // [ksplit][n][W]: (hi, lo) of each running sum
  int* part_exp;        // [ksplit][n]: the exponent the split's sums are relative to
  int* err;             // device error word
};

struct PbArgs {
  const float2* A;      // the plan's first column
  int64_t lda, m, n;    // n: the plan's columns (the partials' stride)
  int64_t col0;         // first column of the launch (a multiple of 128)
  int64_t j_end;        // columns below this are in the launch
  int NC, chunks_per_split;
  const uint16_t* om_tiles;
  float2* partial;
  int* part_exp;
  int* err;
};

// N complex rows r0 .. r0 + N - 1 of a column (zeros past m or for a column
// outside the launch); 16-byte loads when the column is 16-byte aligned.
template <int N, bool VEC>
__device__ __forceinline__ void load_rows(const float2* __restrict__ col, int64_t r0, bool ok, int64_t m,
                                          float2 (&v)[N]) {
  if (VEC && ok && r0 + N <= m) {
    const float4* p = (const float4*)(col + r0);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const float4 f = __ldg(p + q);
      v[2 * q] = make_float2(f.x, f.y);
      v[2 * q + 1] = make_float2(f.z, f.w);
    }
  } else {
#pragma unroll
    for (int u = 0; u < N; ++u) v[u] = (ok && r0 + u < m) ? __ldg(col + r0 + u) : make_float2(0.f, 0.f);
  }
}

// Digits of a float x in a chunk with exponent e (|x| < 2^e), by FP32
// arithmetic: t = x 2^(8-e) (|t| < 256; exact, or below 2^-126 where every
// digit is zero), then for s = 0 .. 6 the digit v_s = t rounded to a multiple
// of 2^(-8s) (adding and subtracting 1.5 2^(23-8s) rounds to that grid, ties
// to even) and t -= v_s (exact).  So v_0 in [-256, 256], |v_s| <= 2^(-8s) 128,
// every v_s is exact in BF16, and sum v_s is x 2^(8-e) rounded to 2^-48: the
// digits the integer cutter of rid_sketch_tc.cu forms, up to a different
// choice between equal sums and ties of the last digit rounded to even.
__device__ __forceinline__ float chunk_scaled(float x, int e) {
  if (e == TC_EXP_ZERO) return 0.f;
  int p = 8 - e;
  if (p < -126) p = -126;                        // only for infinities and NaNs
  if (p <= 127) return __fmul_rn(x, __int_as_float((127 + p) << 23));
  const int p1 = p >> 1;                         // chunks of subnormal floats: two exact steps
  return __fmul_rn(__fmul_rn(x, __int_as_float((127 + p1) << 23)), __int_as_float((127 + p - p1) << 23));
}

__device__ __forceinline__ void fp_digits(float t, float (&v)[TC_S]) {
#pragma unroll
  for (int s = 0; s < TC_S; ++s) {
    const float M = __int_as_float(((150 - 8 * s) << 23) | 0x400000);   // 1.5 2^(23 - 8s)
    const float d = __fsub_rn(__fadd_rn(t, M), M);
    v[s] = d;
    if (s < TC_S - 1) t = __fsub_rn(t, d);
  }
}

// The TC_S packed words (re digit | im digit << 16) of one complex64 entry.
__device__ __forceinline__ void digit_words_fp(float2 x, int e, uint32_t (&w)[TC_S]) {
  float vr[TC_S], vi[TC_S];
  fp_digits(chunk_scaled(x.x, e), vr);
  fp_digits(chunk_scaled(x.y, e), vi);
#pragma unroll
  for (int s = 0; s < TC_S; ++s) w[s] = __byte_perm(__float_as_uint(vr[s]), __float_as_uint(vi[s]), 0x7632);
}

// 2^k as a float for -126 <= k <= 127, else 0 (k < -126; only used there).
__device__ __forceinline__ float pow2f_or_zero(int k) { return k >= -126 ? __int_as_float((127 + k) << 23) : 0.f; }

// Grid (column blocks of the launch, K-splits), 512 threads:
//   warps 0-3   flush: TMEM lane quarter w, one column of A per thread;
//   warps 4-11  slicers: per stage, thread t cuts 8 complex rows of column t / 2;
//   warp 12     lane 0 loads each stage's G digit blocks (bulk copy);
//   warp 13     MMA issuer (whole warp, one elected lane issues) and TMEM owner.
template <int W, bool VEC>
__global__ void __launch_bounds__(TC_THREADS, 1) probe_tc_kernel(PbArgs a) {
  constexpr int NB = W == 16 ? 4 : 2;          // accumulator buffers in TMEM
  constexpr int BUF = 512 / NB;                // their column stride
  constexpr int N = TC_S * W;                  // MMA N: seven diagonal blocks
  constexpr int NS = pb_stages(W);
  constexpr uint32_t SLOT = pb_slot_bytes(W), ZOFF = pb_zero_off(), OOFF = pb_om_off(W), OBYTES = pb_om_bytes(W);
  constexpr uint32_t BLK = pb_block_bytes(W);
  static_assert(N <= 256 && N % 16 == 0, "MMA N");
  static_assert(NS >= 2, "two stages at least");

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[NS], empty_bar[NS], acc_full[NB], acc_empty[NB], exp_bar, mma_done;
  __shared__ int s_exp[PB_EXP_RING][128];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ks = blockIdx.y;
  const int64_t jbase = a.col0 + (int64_t)blockIdx.x * 128;
  const int c_begin = ks * a.chunks_per_split;
  const int c_end = min(a.NC, c_begin + a.chunks_per_split);
  const int nchunks = max(0, c_end - c_begin);
  const int iters = nchunks * TC_SPC;

  if (warp == 13) tmem_alloc(&tmem_slot, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full_bar[i], PB_SLICE_WARPS + 1);   // the slicer warps and the G copy
      mbar_init(&empty_bar[i], 1);
    }
    for (int g = 0; g < NB; ++g) {
      mbar_init(&acc_full[g], 1);
      mbar_init(&acc_empty[g], 4);
    }
    mbar_init(&exp_bar, PB_SLICE_WARPS);
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

  if (warp == 12) {
    if (lane == 0) {
      // ---------------- G digit blocks, one bulk copy per stage ----------------
      const uint16_t* src = a.om_tiles + (int64_t)c_begin * TC_SPC * (OBYTES / 2);
      int it = 0, slot = 0, round = 0;
      for (; it < iters && !s_abort; ++it) {
        if (round > 0 && !mbar_wait(&empty_bar[slot], (round - 1) & 1, TC_WAIT_BUDGET)) {
          fail(11);
          break;
        }
        mbar_arrive_expect_tx(&full_bar[slot], OBYTES);
        bulk_load(smem + slot * SLOT + OOFF, src, OBYTES, &full_bar[slot]);
        src += OBYTES / 2;
        if (++slot == NS) {
          slot = 0;
          ++round;
        }
      }
      // before the CTA may exit: every stage consumed, or after an error every
      // copy issued into this CTA landed
      for (int k = max(0, it - NS); k < it; ++k) {
        const bool ok = s_abort ? mbar_wait(&full_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET)
                                : mbar_wait(&empty_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET);
        if (!ok) fail(12);
      }
    }
  } else if (warp == 13) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = idesc_bf16_f32(128, N);
    int slot = 0, round = 0;
    for (int it = 0; it < iters && !s_abort; ++it) {
      const int cl = it / TC_SPC, b = it - cl * TC_SPC, g = cl % NB;
      if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[slot], round & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(21);
        break;
      }
      if (b == 0 && cl >= NB &&
          !__all_sync(0xffffffffu, mbar_wait(&acc_empty[g], ((cl / NB) - 1) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(22);
        break;
      }
      tc_fence_after();
      unsigned char* base = smem + slot * SLOT;
#pragma unroll
      for (int t = 0; t < TC_S; ++t) {
        const uint64_t da = tile_desc(base + t * TC_TILE_BYTES);
        const uint64_t db = tile_desc(base + ZOFF + (TC_S - 1 - t) * BLK);   // B_t: t zero blocks, then G_0 ..
#pragma unroll
        for (int kk = 0; kk < TC_KS / 16; ++kk)
          mma_bf16_w(tmem + (uint32_t)(g * BUF), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc,
                     (b == 0 && t == 0 && kk == 0) ? 0u : 1u);
      }
      mma_commit_w(&empty_bar[slot]);
      if (b == TC_SPC - 1) mma_commit_w(&acc_full[g]);
      if (++slot == NS) {
        slot = 0;
        ++round;
      }
    }
    mma_commit_w(&mma_done);
  } else if (warp >= PB_FIRST_SLICER && warp < PB_FIRST_SLICER + PB_SLICE_WARPS) {
    // ---------------- slicers ----------------
    const int sw = warp - PB_FIRST_SLICER;
    const int ti = threadIdx.x - 32 * PB_FIRST_SLICER;
    const int jl = ti >> 1, h = ti & 1;          // column of the block; rows 8h .. 8h + 7 of each stage
    const int64_t j = jbase + jl;
    const bool j_ok = j < a.j_end;
    const float2* col = a.A + (j_ok ? j : 0) * a.lda;
    // the zero blocks of every stage (generic stores, read by the MMAs: the
    // proxy fence before each stage's arrival covers them)
    for (int s = 0; s < NS; ++s)
      for (uint32_t o = (uint32_t)ti * 16; o < (TC_S - 1) * BLK; o += 256 * 16)
        *(uint4*)(smem + s * SLOT + ZOFF + o) = make_uint4(0u, 0u, 0u, 0u);

    // 8 complex rows of this thread's column for stage `it` of the split
    auto load_stage = [&](int it, float2 (&v)[8]) {
      const int c = c_begin + it / TC_SPC, b = it % TC_SPC;
      load_rows<8, VEC>(col, (int64_t)c * 128 + b * 16 + 8 * h, j_ok, a.m, v);
    };
    // chunk exponents: column jc of the block, the lane's 4 complex rows of chunk c
    auto exp_load = [&](int c, int jc, float2 (&v)[4]) {
      const int64_t jj = jbase + jc;
      const bool ok = jj < a.j_end;
      load_rows<4, VEC>(a.A + (ok ? jj : 0) * a.lda, (int64_t)c * 128 + 4 * lane, ok, a.m, v);
    };
    auto exp_reduce = [&](const float2 (&v)[4]) {
      int e = TC_EXP_ZERO;
#pragma unroll
      for (int u = 0; u < 4; ++u) e = max(e, max(exp_of_f(v[u].x), exp_of_f(v[u].y)));
      return __reduce_max_sync(0xffffffffu, e);
    };
    auto exp_store = [&](int c, int pair, int e0, int e1) {
      if (lane == 0) {
        s_exp[c & (PB_EXP_RING - 1)][16 * sw + 2 * pair] = e0;
        s_exp[c & (PB_EXP_RING - 1)][16 * sw + 2 * pair + 1] = e1;
      }
    };
    // every slicer warp has stored its exponents of a chunk
    auto exp_sync = [&](int phase) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&exp_bar);
      return __all_sync(0xffffffffu, mbar_wait(&exp_bar, phase & 1, TC_WAIT_BUDGET));
    };

    // The exponents run two chunks ahead of the cutting: those of chunks 0
    // and 1 first; then during chunk cl, stage b loads column pair b of chunk
    // cl + 2 and reduces the pair the previous stage loaded, so each load has
    // a stage of cutting to land.
    int ephase = 0;
    bool ok = true;
    for (int c = 0; c < min(2, nchunks); ++c)
      for (int pr = 0; pr < 8; ++pr) {
        float2 v0[4], v1[4];
        exp_load(c_begin + c, 16 * sw + 2 * pr, v0);
        exp_load(c_begin + c, 16 * sw + 2 * pr + 1, v1);
        exp_store(c, pr, exp_reduce(v0), exp_reduce(v1));
      }
    if (nchunks > 0) {
      ok = exp_sync(ephase++);
      if (!ok && lane == 0) fail(42);
    }
    float2 x[8];
    if (iters > 0) load_stage(0, x);
    float2 pa[4], pb[4];                         // the pending exponent pair
    int p_chunk = -1, p_pair = 0;
    const int swz = (jl >> 1) & 3;
    int slot = 0, round = 0;
    for (int it = 0; it < iters && ok && !s_abort; ++it) {
      const int cl = it / TC_SPC, b = it - cl * TC_SPC;
      float2 y[8];
      if (it + 1 < iters) load_stage(it + 1, y);
      float2 na[4], nb[4];
      const bool n_exp = cl + 2 < nchunks;
      if (n_exp) {
        exp_load(c_begin + cl + 2, 16 * sw + 2 * b, na);
        exp_load(c_begin + cl + 2, 16 * sw + 2 * b + 1, nb);
      }
      const int e = s_exp[cl & (PB_EXP_RING - 1)][jl];
      if (round > 0 && !__all_sync(0xffffffffu, mbar_wait(&empty_bar[slot], (round - 1) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(41);
        break;
      }
      unsigned char* row = smem + slot * SLOT + jl * (TC_KS * 2);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t w[4][TC_S];
#pragma unroll
        for (int u = 0; u < 4; ++u) digit_words_fp(x[4 * half + u], e, w[u]);
        const int pc = ((2 * h + half) ^ swz) << 4;
#pragma unroll
        for (int s = 0; s < TC_S; ++s)
          *(uint4*)(row + s * TC_TILE_BYTES + pc) = make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> the MMAs' reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[slot]);
      if (p_chunk >= 0) {
        exp_store(p_chunk, p_pair, exp_reduce(pa), exp_reduce(pb));
        if (p_pair == 7) {               // chunk p_chunk's exponents complete
          ok = exp_sync(ephase++);
          if (!ok && lane == 0) fail(42);
        }
      }
      p_chunk = n_exp ? cl + 2 : -1;
      p_pair = b;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        pa[u] = na[u];
        pb[u] = nb[u];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = y[u];
      if (++slot == NS) {
        slot = 0;
        ++round;
      }
    }
  } else if (warp < 4) {
    // ---------------- flush ----------------
    const int jl = 32 * warp + lane;
    const int64_t j = jbase + jl;
    const bool j_ok = j < a.j_end;
    float hi[W], lo[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      hi[i] = 0.f;
      lo[i] = 0.f;
    }
    int E = TC_EXP_ZERO;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int cl = 0; cl < nchunks && !s_abort; ++cl) {
      const int g = cl % NB;
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[g], (cl / NB) & 1, TC_WAIT_BUDGET))) {
        if (lane == 0) fail(31);
        break;
      }
      tc_fence_after();
      const int e = s_exp[cl & (PB_EXP_RING - 1)][jl];
      if (e > E) {                       // a larger exponent: rescale the running sums (exact)
        const float f = pow2f_or_zero(E - e);
#pragma unroll
        for (int i = 0; i < W; ++i) {
          hi[i] *= f;
          lo[i] *= f;
        }
        E = e;
      }
      const float scale = e == TC_EXP_ZERO ? 0.f : pow2f_or_zero(e - E);
#pragma unroll
      for (int d = 0; d < TC_S; ++d) {
        uint32_t r[W];
#pragma unroll
        for (int q = 0; q < W / 16; ++q)
          tmem_ld16(lane_base + (uint32_t)(g * BUF + d * W + 16 * q), *(uint32_t(*)[16])(r + 16 * q));
        tmem_ld_wait();
        if (d == TC_S - 1) {             // the buffer is read: the MMAs may overwrite it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[g]);
        }
#pragma unroll
        for (int i = 0; i < W; ++i) {
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
      float4* dst = (float4*)(a.partial + ((int64_t)ks * a.n + j) * W);
#pragma unroll
      for (int i = 0; i < W; i += 2) dst[i / 2] = make_float4(hi[i], lo[i], hi[i + 1], lo[i + 1]);
      a.part_exp[(int64_t)ks * a.n + j] = E;
    }
  }

  // ---------------- teardown ----------------
  tc_fence_before();
  __syncthreads();
  if (warp == 13) {
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

const void* probe_kernel_fn(int W, bool vec) {
  if (W == 16) return vec ? (const void*)probe_tc_kernel<16, true> : (const void*)probe_tc_kernel<16, false>;
  return vec ? (const void*)probe_tc_kernel<32, true> : (const void*)probe_tc_kernel<32, false>;
}

int probe_dyn_smem(int W) {
  return (int)(pb_stages(W) * pb_slot_bytes(W) + 1024);
}

}  // namespace

// A mixed-precision plan's probe state: G's digit tiles (rows l .. l + r - 1 of
// Omega), the partial sums and the error word.
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
  const size_t part_bytes = (size_t)st->ksplit * p->n * st->W * 8;
  const size_t pexp_bytes = (size_t)st->ksplit * p->n * 4;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t total = al(om_bytes) + al((size_t)2 * st->nrows * 4) + al(part_bytes) + al(pexp_bytes) + al(4);
  char* base = nullptr;
  if (rid_dev_alloc((void**)&base, total, p->stream, p->device) != cudaSuccess) {
    free(st);
    return RID_ENOMEM;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { char* ptr = base + off; off += al(bytes); return ptr; };
  st->om_tiles = (uint16_t*)take(om_bytes);
  st->om_exp = (int*)take((size_t)2 * st->nrows * 4);
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
                             probe_dyn_smem(st->W));
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

// X(:, col0 .. col0 + ncols - 1) = G A(:, those columns); col0 a multiple of 128.
cudaError_t rid_tc_probe_sketch_cols(const rid_plan_s* p, const void* A_, int64_t lda, int64_t col0, int64_t ncols) {
  const ProbeState* st = (const ProbeState*)p->tc_probe_state;
  if (!st) return cudaErrorNotSupported;
  if (ncols <= 0) return cudaSuccess;
  const int nblocks = (int)((ncols + 127) / 128);
  PbArgs args{(const float2*)A_, lda, p->m, p->n, col0, col0 + ncols, st->NC, st->chunks_per_split,
              st->om_tiles, st->partial, st->part_exp, st->err};
  const dim3 grid((unsigned)nblocks, (unsigned)st->ksplit);
  const bool vec = ((uintptr_t)A_ & 15u) == 0 && lda % 2 == 0;   // every column 16-byte aligned
  const void* fn = probe_kernel_fn(st->W, vec);
  void* params[] = {&args};
  cudaError_t e = cudaLaunchKernel(fn, grid, dim3(TC_THREADS), params, (size_t)probe_dyn_smem(st->W), p->stream);
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
