// Shared pieces of the exact-slice tensor-core products (the plan's sketch and
// the batched sketch): stage and tile constants, the swizzled tile layout, the
// balanced base-256 digits of a value, and one K stage of slice-pair MMAs.
// The digit scheme and the exactness argument are described at the top of
// rid_sketch_tc.cu.
#pragma once

#include <stdint.h>

#include "rid_tc.cuh"

#ifdef __CUDACC__

namespace rid_tc {

constexpr int TC_S = 7;                 // digits per value: 56 bits
constexpr int TC_G = 4;                 // accumulator groups
constexpr int TC_KC = 256;              // chunk of the reduction with exact FP32 sums
constexpr int TC_KS = 32;               // K per pipeline stage: 64-byte tile rows, 2 MMAs per slice pair
constexpr int TC_SPC = TC_KC / TC_KS;   // stages per chunk
constexpr int TC_MAX_STAGES = 6;        // stages in flight: as many as fit in shared memory, at most this
constexpr int TC_TILE_BYTES = 128 * TC_KS * 2;     // an A tile: 128 rows x (2 TC_KS) bytes
constexpr int TC_TILE_ELEMS = 128 * TC_KS;         // the same in bf16 elements
constexpr int TC_SMEM_LIMIT = 232448;   // dynamic + static shared memory of one CTA
// The dynamic shared memory attribute is process-wide and plans of other
// shapes launch the kernel from other host threads: it is always set to this
// bound, which every plan's stages fit under.
constexpr int TC_DYN_SMEM_MAX = TC_SMEM_LIMIT - 2048;
constexpr int TC_THREADS = 512;         // warps 0-11 flush, 12 TMA, 13 MMA + TMEM, 14-15 idle
constexpr int TC_FLUSH_WARPS = 12;
constexpr int TC_LAUNCH_REGS = 128;    // 65536 / 512: the pool the setmaxnreg split assumes
constexpr int TC_EXP_ZERO = -30000;     // exponent of an all-zero chunk / row
constexpr long long TC_WAIT_BUDGET = 4000000000ll;   // clock cycles (~2 s)

// Byte offset of element k (0 <= k < TC_KS) of row r within a tile of 64-byte
// rows in the 64-byte swizzle: the row's 16-byte chunk c sits at position
// c ^ ((r >> 1) & 3), the image a tensor copy with that swizzle leaves in
// shared memory (tiles start at multiples of 1024 bytes there).
__host__ __device__ __forceinline__ int tile_offset(int r, int k) {
  return r * (TC_KS * 2) + ((((k * 2) >> 4) ^ ((r >> 1) & 3)) << 4) + ((k * 2) & 15);
}

// Columns of one N-tile's MMA: its rows rounded up to 16; pairs take at least
// 32 (each CTA supplies half).  The Omega slicer splits a pair's tile at half
// of this.
__host__ __device__ __forceinline__ int tile_mma_n(int tile_w, int l2, int nt, bool pair) {
  const int rest = l2 - nt * tile_w;
  const int nm = ((rest < tile_w ? rest : tile_w) + 15) & ~15;
  return !pair ? nm : nm < 32 ? (tile_w < 32 ? tile_w : 32) : nm;
}

// ---- digits --------------------------------------------------------------------
// Exponent e of x (|x| < 2^e, x = f 2^e with 1/2 <= |f| < 1); subnormals and
// zero count as zero.
__device__ __forceinline__ int exp_of(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  return ex == 0 ? TC_EXP_ZERO : ex - 1022;
}

// Balanced base-256 digits of x relative to exponent e (|x| < 2^e):
// round(|x| 2^(8S-e)) = sum_s d_s 256^(S-1-s), d_0 in [0, 256], others in
// [-128, 127]; stored as BF16 bits of +-d_s 2^(-8s).
__device__ __forceinline__ void digits_of(double x, int e, uint16_t (&out)[TC_S]) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long q = 0;
  if (ex != 0 && e != TC_EXP_ZERO) {
    const unsigned long long mant = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (ex - 1075) + 8 * TC_S - e;
    if (sh >= 0) {
      q = mant << sh;
    } else if (sh > -62) {
      q = (mant + (1ull << (-sh - 1))) >> (-sh);
    }
  }
  const bool neg = b < 0;
  int d[TC_S];
#pragma unroll
  for (int s = TC_S - 1; s >= 1; --s) {
    int v = (int)(q & 0xFF);
    q >>= 8;
    if (v >= 128) {
      v -= 256;
      q += 1;
    }
    d[s] = v;
  }
  d[0] = (int)q;
#pragma unroll
  for (int s = 0; s < TC_S; ++s) {
    float f = (float)(neg ? -d[s] : d[s]);
    f = __fmul_rn(f, __int_as_float((127 - 8 * s) << 23));   // * 2^(-8s)
    out[s] = (uint16_t)(__float_as_uint(f) >> 16);
  }
}

// The same digits as digits_of, computed for the hot path with few integer
// operations.  q' = q + B with B = sum_{s=1..6} 128 * 256^(6-s) holds the
// balanced digits as plain bytes (byte 6-s of q' is d_s + 128 for s >= 1, and
// q' >> 48 = d_0), so no carries are propagated.  A digit u becomes its BF16
// value with one FFMA: the float with exponent field 150 - 8s and low bits u is
// 2^(-8s) (2^23 + u), so sgn * that - sgn * 2^(-8s) (2^23 + bias) = sgn d 2^(-8s)
// exactly (and +0 for a zero digit, as the integer conversion gives).
__device__ __forceinline__ unsigned long long digit_bytes(double x, int e, float& sgn) {
  const long long b = __double_as_longlong(x);
  sgn = b < 0 ? -1.0f : 1.0f;
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long q = 0;
  if (ex != 0 && e != TC_EXP_ZERO) {
    const unsigned long long mant = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (ex - 1075) + 8 * TC_S - e;
    if (sh >= 0) {
      q = mant << sh;
    } else if (sh > -62) {
      q = (mant + (1ull << (-sh - 1))) >> (-sh);
    }
  }
  return q + 0x0000808080808080ull;
}

template <int S>
__device__ __forceinline__ float digit_value(uint32_t u, float sgn) {
  constexpr uint32_t kExp = (uint32_t)(150 - 8 * S) << 23;
  // 2^(-8S) (2^23 + 128) for S >= 1 (the bias), 2^23 for the leading digit
  const float c = S == 0 ? 8388608.0f : __uint_as_float(kExp | 128u);
  return __fmaf_rn(sgn, __uint_as_float(kExp | u), __fmul_rn(-sgn, c));
}

// The TC_S packed words (re digit | im digit << 16) of one complex entry.
__device__ __forceinline__ void digit_words(double2 x, int e, uint32_t (&w)[TC_S]) {
  static_assert(TC_S == 7, "digit byte layout assumes 7 digits");
  float sr, si;
  const unsigned long long qr = digit_bytes(x.x, e, sr), qi = digit_bytes(x.y, e, si);
  const uint32_t rl = (uint32_t)qr, rh = (uint32_t)(qr >> 32), il = (uint32_t)qi, ih = (uint32_t)(qi >> 32);
#define RID_DIGIT_PAIR(S, RB, IB) \
  w[S] = __byte_perm(__float_as_uint(digit_value<S>(RB, sr)), __float_as_uint(digit_value<S>(IB, si)), 0x7632);
  RID_DIGIT_PAIR(0, rh >> 16, ih >> 16)
  RID_DIGIT_PAIR(1, (rh >> 8) & 0xFF, (ih >> 8) & 0xFF)
  RID_DIGIT_PAIR(2, rh & 0xFF, ih & 0xFF)
  RID_DIGIT_PAIR(3, rl >> 24, il >> 24)
  RID_DIGIT_PAIR(4, (rl >> 16) & 0xFF, (il >> 16) & 0xFF)
  RID_DIGIT_PAIR(5, (rl >> 8) & 0xFF, (il >> 8) & 0xFF)
  RID_DIGIT_PAIR(6, rl & 0xFF, il & 0xFF)
#undef RID_DIGIT_PAIR
}

// exp_of of a float converted to double (exact), from the float bits: a
// float is its 24-bit significand times 2^(ex - 150), or the raw field times
// 2^-149 when subnormal; infinities and NaNs take their double's exponent.
__device__ __forceinline__ int exp_of_f(float x) {
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFF);
  const uint32_t mant = b & 0x7FFFFFu;
  if (ex == 0) return mant ? (32 - __clz((int)mant)) - 149 : TC_EXP_ZERO;
  return ex == 255 ? 1025 : ex - 126;
}

__device__ __forceinline__ int group_of(int d) { return d >= 3 ? 3 : d; }

// Descriptor of a tile of TC_KS bf16 per row (the swizzle of tile_offset).
__device__ __forceinline__ uint64_t tile_desc(const void* p) { return desc_sw64(p); }

// One stage's products: the slice pairs (s, t) with s < SO (the Omega digits
// that can be non-zero), t < S and s + t <= S - 1, diagonal by diagonal from
// the smallest (group 3 holds d >= 3), each group waiting for its flush before
// its first product of a chunk.  Descriptor start addresses are in 16-byte
// units (low 14 bits): a tile offset within shared memory adds without carry.
// Called by the whole MMA warp (converged); one elected lane issues.
template <int SO, bool PAIR>
__device__ __forceinline__ bool mma_stage(uint32_t tmem, uint64_t da0, uint64_t db0, uint64_t o_step, uint32_t idesc,
                                          int b, int cl, int stages_per_chunk, uint64_t* acc_empty,
                                          uint64_t* acc_full) {
  constexpr uint64_t a_step = TC_TILE_BYTES >> 4;
#pragma unroll
  for (int d = TC_S - 1; d >= 0; --d) {
    const int g = group_of(d);
    const bool group_start = (d == TC_S - 1) || (d < 3);   // first diagonal of its group
    if (b == 0 && group_start && cl > 0) {
      // a pair's barrier also counts the other CTA's flush warps
      const bool ok = PAIR ? mbar_wait_cluster(&acc_empty[g], (cl - 1) & 1, TC_WAIT_BUDGET)
                           : mbar_wait(&acc_empty[g], (cl - 1) & 1, TC_WAIT_BUDGET);
      if (!__all_sync(0xffffffffu, ok)) return false;
      tc_fence_after();
    }
#pragma unroll
    for (int s = 0; s <= d; ++s) {
      const int t = d - s;
      if (s >= SO || t >= TC_S) continue;
      const uint64_t da = da0 + a_step * t, db = db0 + o_step * s;
#pragma unroll
      for (int kk = 0; kk < TC_KS / 16; ++kk) {   // K16 steps are 32 bytes apart in a row
        const uint32_t acc = (b == 0 && group_start && s == 0 && kk == 0) ? 0u : 1u;
        if (PAIR) mma_bf16_pair_w(tmem + (uint32_t)(g * 128), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, acc);
        else mma_bf16_w(tmem + (uint32_t)(g * 128), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, acc);
      }
    }
    const bool group_end = (d <= 3);     // last diagonal of its group in this stage
    if (b == stages_per_chunk - 1 && group_end) {
      if (PAIR) mma_commit_pair_multicast_w(&acc_full[g], 3);   // both CTAs flush their rows
      else mma_commit_w(&acc_full[g]);
    }
  }
  return true;
}

}  // namespace rid_tc

#endif  // __CUDACC__
