// Randomization Y = Omega A (Sec. 2) on the tcgen05 tensor cores with an
// FP64-grade result: an exact-slice (Ozaki-type) emulation of the complex128
// product from BF16 digits with FP32 accumulation.
//
// Real view.  With A and Omega stored as interleaved complex numbers, the
// complex product is the real product Y' = Omega' A' of a (2l x 2m) matrix
// Omega' (row 2i = (Re w, -Im w, ...), row 2i+1 = (Im w, Re w, ...)) with the
// (2m x n) matrix A' whose column j is A's column j read as 2m doubles.  Y'
// column j is Y's column j read as 2l doubles, so no data is reordered.
//
// Digits.  Each real value x in a 256-long chunk c of a column (of A') or in a
// row (of Omega') is written x = 2^(e-8) sum_s v_s with e the chunk's (row's)
// binary exponent (|x| < 2^e), v_s = d_s 2^(-8s), d_0 in [0, 256] and
// d_s in [-128, 127] for s >= 1 (balanced base-256 digits of x rounded to
// 8S bits).  Every v_s is exact in BF16.  The products of a slice pair (s, t)
// carry the scale 2^(-8(s+t)); pairs with s + t <= S-1 are kept.
//
// Exact accumulation.  Within one chunk (256 products per pair) the tensor
// core's FP32 sums are exact for the diagonals s+t = 0, 1 and 2 kept apart
// (|sum| < 2^24 units of each diagonal's last bit); the diagonals s+t >= 3 go
// to a fourth accumulator whose rounding error is below 2^-48 of the chunk's
// leading term.  So a CTA holds four TMEM accumulators of 128 x 128 FP32
// (all 512 columns).  After each chunk the flush warps read the four groups,
// scale them by 2^(e_A(j,c) - E_A(j)) (E_A = the column's largest chunk
// exponent) and add them to a double-FP32 (hi + lo) running sum.  The
// groups are released to the MMA warp one by one, in the order the next
// chunk needs them, so flushing overlaps the next chunk's products.
//
// Tiles.  M = 128 columns of A (TMEM lanes), N <= 128 rows of Omega' (TMEM
// columns; the 2l rows are split evenly into N-tiles, a multiple of 16 each),
// K in 32-element stages of 64-byte rows with the 64-byte swizzle: one stage
// holds S A-slice tiles and S Omega-slice tiles.  The N-tiles of one column
// block form a cluster: each A tile is loaded once and multicast to them, and
// a stage is released by a multicast commit.  A K-split over CTAs balances
// the waves; partial sums are reduced in a fixed order, so results are
// deterministic.  Row probes (rows l.. of Omega) are sliced and multiplied
// like the test matrix's rows and reduced into X instead of Y.
#include <climits>
#include <cudaTypedefs.h>

#include "rid_internal.cuh"
#include "rid_tc.cuh"

using namespace rid_tc;

namespace {

constexpr int TC_S = 7;                 // digits per value: 56 bits
constexpr int TC_G = 4;                 // accumulator groups
constexpr int TC_KC = 256;              // chunk of the reduction with exact FP32 sums
#ifndef RID_TC_KS
#define RID_TC_KS 32
#endif
constexpr int TC_KS = RID_TC_KS;        // K per pipeline stage (32: 64-byte tile rows, 2 MMAs per slice pair)
constexpr int TC_MAX_STAGES = 6;        // stages in flight: as many as fit in shared memory, at most this
constexpr int TC_TILE_BYTES = 128 * TC_KS * 2;     // an A tile: 128 rows x (2 TC_KS) bytes
constexpr int TC_SMEM_LIMIT = 232448;   // dynamic + static shared memory of one CTA
// The dynamic shared memory attribute is process-wide and plans of other
// shapes launch the kernel from other host threads: it is always set to this
// bound, which every plan's stages fit under.
constexpr int TC_DYN_SMEM_MAX = TC_SMEM_LIMIT - 2048;
#ifndef RID_TC_PREFETCH
#define RID_TC_PREFETCH 0
#endif
constexpr int TC_PREFETCH = RID_TC_PREFETCH;   // stages ahead whose A tiles are prefetched into L2
#ifndef RID_TC_OPAD
#define RID_TC_OPAD 1024
#endif
constexpr int TC_OPAD = RID_TC_OPAD;           // Omega tiles start at multiples of this in a stage
constexpr int TC_THREADS = 512;         // warps 0-11 flush, 12 TMA, 13 MMA + TMEM, 14-15 idle
constexpr int TC_FLUSH_WARPS = 12;
constexpr int TC_LAUNCH_REGS = 128;    // 65536 / 512: the pool the setmaxnreg split assumes
constexpr int TC_EXP_ZERO = -30000;     // exponent of an all-zero chunk / row
constexpr long long TC_WAIT_BUDGET = 4000000000ll;   // clock cycles (~2 s)

struct TcState {
  int S;
  int row0, nrows;        // the rows of Omega this state multiplies
  bool a_c64;             // A is complex64 (converted exactly to FP64 before slicing)
  int nstages;            // pipeline stages that fit in shared memory
  uint32_t stage_smem, o_off, o_tile_smem;
  int dyn_smem;           // dynamic shared memory of the product kernel
  int so;                 // Omega digits used: S, or bits / 8 for a rounded Omega
  int64_t KP;             // padded reduction length (multiple of TC_KC)
  int NC;                 // chunks
  int l2;                 // 2l rows of Omega'
  int ntiles;             // N-tiles of tile_w <= 128 rows (balanced: the cluster runs at the widest)
  int tile_w;             // rows of Omega' per N-tile, a multiple of 16
  int nblocks;            // column blocks of 128
  int ksplit;             // K-splits
  int chunks_per_split;
  int cx, cy;             // cluster shape (N-tiles x column blocks)
  int nblocks_p;          // column blocks padded to a multiple of cy
  uint16_t* om_slices;    // [S][l2][KP] bf16
  int* om_exp;            // [l2]
  uint16_t* a_slices;     // [S][n][KP] bf16
  int* a_exp;             // [n][NC]
  int* a_exp_max;         // [n]
  float2* partial;        // [ksplit][n][l2p]: (hi, lo) of each running sum
  int l2p;
  int* err;               // device error word
  CUtensorMap map_a, map_om;
};

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

// ---- Omega' slices (plan time) ---------------------------------------------------
// Row exponent of Omega' rows 2i and 2i+1 (same values): max over the row.
__global__ void omega_exp_kernel(const double2* __restrict__ om, int64_t ldo, int64_t m, int* __restrict__ om_exp) {
  __shared__ int red[8];
  const int i = blockIdx.x;
  int e = TC_EXP_ZERO;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
    const double2 w = om[i * ldo + r];
    e = max(e, max(exp_of(w.x), exp_of(w.y)));
  }
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = max(v, red[w]);
    om_exp[2 * i] = v;
    om_exp[2 * i + 1] = v;
  }
}

// Digits of Omega' rows: row 2i = (Re w_r, -Im w_r), row 2i+1 = (Im w_r, Re w_r).
__global__ void omega_slice_kernel(const double2* __restrict__ om, int64_t ldo, int64_t m, int l, int64_t KP,
                                   const int* __restrict__ om_exp, uint16_t* __restrict__ slices) {
  const int64_t per_row = KP / 2;      // complex positions per row, incl. padding
  const int64_t total = (int64_t)l * per_row;
  const int64_t slice_stride = (int64_t)2 * l * KP;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / per_row);
    const int64_t r = e - (int64_t)i * per_row;
    const double2 w = r < m ? om[i * ldo + r] : make_double2(0.0, 0.0);
    const int ex = om_exp[2 * i];
    uint16_t re[TC_S], nim[TC_S], im[TC_S];
    digits_of(w.x, ex, re);
    digits_of(-w.y, ex, nim);
    digits_of(w.y, ex, im);
    for (int s = 0; s < TC_S; ++s) {
      uint16_t* row0 = slices + s * slice_stride + (int64_t)(2 * i) * KP + 2 * r;
      uint16_t* row1 = row0 + KP;
      *(uint32_t*)row0 = (uint32_t)re[s] | ((uint32_t)nim[s] << 16);
      *(uint32_t*)row1 = (uint32_t)im[s] | ((uint32_t)re[s] << 16);
    }
  }
}

// ---- A' slices (every call) -------------------------------------------------------
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

// One warp per (column j, chunk c): 128 complex rows = 256 real values; a
// lane takes 4 consecutive complex rows, so every slice row is written with
// one 16-byte store per lane.
template <typename TA>
__global__ void __launch_bounds__(256) a_slice_kernel(const TA* __restrict__ A, int64_t lda, int64_t m,
                                                      int64_t n, int NC, int64_t KP, int64_t slice_stride,
                                                      uint16_t* __restrict__ slices, int* __restrict__ a_exp,
                                                      int* __restrict__ a_exp_max) {
  // A, slices, a_exp and a_exp_max start at the first column of the range
  // (n columns); slice_stride separates the digit planes of the whole matrix
  const int lane = threadIdx.x & 31;
  const int64_t tasks = n * NC;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tasks;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t j = t / NC;
    const int c = (int)(t - j * NC);
    const int64_t r0 = (int64_t)c * 128 + 4 * lane;
    const TA* col = A + j * lda;
    double2 x[4];
    int e = TC_EXP_ZERO;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (r0 + u < m) {
        const TA v = __ldcs(col + r0 + u);
        x[u] = make_double2((double)v.x, (double)v.y);     // exact for complex64 input
      } else {
        x[u] = make_double2(0.0, 0.0);
      }
      e = max(e, max(exp_of(x[u].x), exp_of(x[u].y)));
    }
    e = __reduce_max_sync(0xffffffffu, e);
    uint32_t w[4][TC_S];
#pragma unroll
    for (int u = 0; u < 4; ++u) digit_words(x[u], e, w[u]);
#pragma unroll
    for (int s = 0; s < TC_S; ++s)
      __stcs((uint4*)(slices + s * slice_stride + j * KP + 2 * r0), make_uint4(w[0][s], w[1][s], w[2][s], w[3][s]));
    if (lane == 0) {
      a_exp[j * NC + c] = e;
      atomicMax(a_exp_max + j, e);
    }
  }
}

// ---- the tensor-core product ----------------------------------------------------------
struct TcArgs {
  int n, l2, l2p, NC, chunks_per_split, ntiles, tile_w;
  uint32_t stage_bytes;   // bytes landing in one stage: S A tiles of 128 rows + so Omega tiles of tile_w rows
  int so;                 // Omega digits that can be non-zero (S, or fewer for a rounded Omega)
  int nstages;            // pipeline stages
  uint32_t stage_smem;    // shared memory of one stage (1024-byte multiple)
  uint32_t o_off;         // offset of the Omega tiles in a stage
  uint32_t o_tile_smem;   // shared memory of one Omega tile (1024-byte multiple)
  int cx, cy;             // cluster: cx N-tiles (share A tiles) x cy column blocks (share Omega tiles)
  int jb0;                // first column block of the launch (a column range of the sketch)
  const int* a_exp;
  const int* a_exp_max;
  float2* partial;
  int* err;
};

__device__ __forceinline__ int group_of(int d) { return d >= 3 ? 3 : d; }

// Descriptor of a 128-row tile of TC_KS bf16 per row (swizzle matching the tensor map).
__device__ __forceinline__ uint64_t tile_desc(const void* p) { return TC_KS == 16 ? desc_sw32(p) : desc_sw64(p); }

// One stage's products: the slice pairs (s, t) with s < SO (the Omega digits
// that can be non-zero), t < S and s + t <= S - 1, diagonal by diagonal from
// the smallest (group 3 holds d >= 3), each group waiting for its flush before
// its first product of a chunk.  Descriptor start addresses are in 16-byte
// units (low 14 bits): a tile offset within shared memory adds without carry.
template <int SO>
__device__ __forceinline__ bool mma_stage(uint32_t tmem, uint64_t da0, uint64_t db0, uint64_t o_step, uint32_t idesc,
                                          int b, int cl, int stages_per_chunk, uint64_t* acc_empty,
                                          uint64_t* acc_full) {
  constexpr uint64_t a_step = TC_TILE_BYTES >> 4;
#pragma unroll
  for (int d = TC_S - 1; d >= 0; --d) {
    const int g = group_of(d);
    const bool group_start = (d == TC_S - 1) || (d < 3);   // first diagonal of its group
    if (b == 0 && group_start && cl > 0) {
      if (!mbar_wait(&acc_empty[g], (cl - 1) & 1, TC_WAIT_BUDGET)) return false;
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
        mma_bf16(tmem + (uint32_t)(g * 128), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, acc);
      }
    }
    const bool group_end = (d <= 3);     // last diagonal of its group in this stage
    if (b == stages_per_chunk - 1 && group_end) mma_commit(&acc_full[g]);
  }
  return true;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_om, TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[TC_MAX_STAGES], empty_bar[TC_MAX_STAGES];
  __shared__ uint64_t acc_full[TC_G], acc_empty[TC_G], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Grid (N-tiles, column blocks, K-splits); a cluster of cx x cy CTAs covers
  // all N-tiles of cy column blocks.  Each A tile is loaded once per cluster
  // row and multicast to the cx CTAs that use it; each Omega tile once per
  // cluster column and multicast to the cy CTAs that use it.
  const int nb = blockIdx.x, jb = blockIdx.y + a.jb0, ks = blockIdx.z;
  const int rx = nb % a.cx, ry = jb % a.cy;
  const uint32_t my_rank = (uint32_t)(rx + ry * a.cx);
  const uint16_t row_mask = (uint16_t)(((1u << a.cx) - 1u) << (ry * a.cx));
  uint16_t col_mask = 0;
  for (int y = 0; y < a.cy; ++y) col_mask |= (uint16_t)(1u << (rx + y * a.cx));
  const uint16_t all_mask = (uint16_t)((1u << (a.cx * a.cy)) - 1u);
  const int c_begin = ks * a.chunks_per_split;
  const int c_end = min(a.NC, c_begin + a.chunks_per_split);
  const int nchunks = max(0, c_end - c_begin);
  const int row0 = nb * a.tile_w;
  const int n_tile = min(a.tile_w, a.l2 - row0);
  const int n_mma = (n_tile + 15) & ~15;

  if (warp == 13) tmem_alloc(&tmem_slot, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nstages; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], a.cx * a.cy);   // every CTA of the cluster releases the slot
    }
    for (int g = 0; g < TC_G; ++g) {
      mbar_init(&acc_full[g], 1);
      mbar_init(&acc_empty[g], TC_FLUSH_WARPS);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
    s_abort = cluster_rank() != my_rank ? 1 : 0;      // grid and cluster layout disagree
    if (s_abort) atomicCAS(a.err, 0, 1);
  }
  tc_fence_before();
  cluster_sync();          // barriers of every CTA initialised before any multicast
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  auto a_tile = [&](int slot, int s) { return smem + slot * a.stage_smem + s * TC_TILE_BYTES; };
  auto o_tile = [&](int slot, int s) { return smem + slot * a.stage_smem + a.o_off + s * a.o_tile_smem; };
  const int NS = a.nstages;
  auto fail = [&](int code) {
    s_abort = 1;
    atomicCAS(a.err, 0, code);
  };

  if (warp >= 12) {
    // Warpgroup 3 (producer, MMA, two idle warps) gives registers to the flush
    // warpgroups: 128 x 56 + 384 x 152 = 512 x 128, the launch allocation.
    asm volatile("setmaxnreg.dec.sync.aligned.u32 56;\n" ::: "memory");
    if (warp == 12 && lane == 0) {
      // ---------------- TMA producer ----------------
      prefetch_tensormap(&map_a);
      prefetch_tensormap(&map_om);
      const int iters = nchunks * (TC_KC / TC_KS);
      int it = 0, slot = 0, round = 0;
      for (; it < iters && !s_abort; ++it) {
        if (round > 0 && !mbar_wait(&empty_bar[slot], (round - 1) & 1, TC_WAIT_BUDGET)) {
          fail(11);
          break;
        }
        const int c = c_begin + it / (TC_KC / TC_KS);
        const int x = c * TC_KC + (it % (TC_KC / TC_KS)) * TC_KS;
        if (TC_PREFETCH > 0 && it + TC_PREFETCH < iters) {
          const int ip = it + TC_PREFETCH;
          const int xp = (c_begin + ip / (TC_KC / TC_KS)) * TC_KC + (ip % (TC_KC / TC_KS)) * TC_KS;
          for (int s = rx; s < TC_S; s += a.cx) tma_prefetch_3d(&map_a, xp, jb * 128, s);
        }
        // the stage's 2S tiles arrive here whoever issued them
        mbar_arrive_expect_tx(&full_bar[slot], a.stage_bytes);
        for (int s = rx; s < TC_S; s += a.cx)
          tma_load_3d_multicast(&map_a, &full_bar[slot], a_tile(slot, s), x, jb * 128, s, row_mask);
        for (int s = ry; s < a.so; s += a.cy)
          tma_load_3d_multicast(&map_om, &full_bar[slot], o_tile(slot, s), x, row0, s, col_mask);
        if (++slot == NS) {
          slot = 0;
          ++round;
        }
      }
      // tail: before the CTA may exit, every slot must have been released by
      // every CTA of the cluster (their commits arrive here), or, after an
      // error, every load issued into this CTA must have landed
      for (int k = max(0, it - NS); k < it; ++k) {
        const bool ok = s_abort ? mbar_wait(&full_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET)
                                : mbar_wait(&empty_bar[k % NS], (k / NS) & 1, TC_WAIT_BUDGET);
        if (!ok) fail(12);
      }
    } else if (warp == 13 && lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = idesc_bf16_f32(128, n_mma);
      const int stages_per_chunk = TC_KC / TC_KS;
      // descriptor start addresses are in 16-byte units (low 14 bits): a tile
      // offset within the CTA's shared memory adds without carry
      const uint64_t o_step = a.o_tile_smem >> 4;
      int slot = 0, round = 0;
      for (int cl = 0; cl < nchunks && !s_abort; ++cl) {
        for (int b = 0; b < stages_per_chunk && !s_abort; ++b) {
          if (!mbar_wait(&full_bar[slot], round & 1, TC_WAIT_BUDGET)) {
            fail(21);
            break;
          }
          tc_fence_after();
          const uint64_t da0 = tile_desc(a_tile(slot, 0)), db0 = tile_desc(o_tile(slot, 0));
          bool ok = true;
          switch (a.so) {      // the Omega digit count picks a fully unrolled issue sequence
#define RID_MMA_STAGE(SO) \
            case SO: ok = mma_stage<SO>(tmem, da0, db0, o_step, idesc, b, cl, stages_per_chunk, acc_empty, acc_full); break;
            RID_MMA_STAGE(1) RID_MMA_STAGE(2) RID_MMA_STAGE(3) RID_MMA_STAGE(4) RID_MMA_STAGE(5) RID_MMA_STAGE(6)
            RID_MMA_STAGE(7)
#undef RID_MMA_STAGE
            default: ok = false;
          }
          if (!ok) {
            fail(22);
            break;
          }
          mma_commit_multicast(&empty_bar[slot], all_mask);
          if (++slot == NS) {
            slot = 0;
            ++round;
          }
        }
      }
      mma_commit(&mma_done);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 152;\n" ::: "memory");
    // ---------------- flush warps (0..11) ----------------
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 (the hardware's lane quarter
    // of the warp) and tile columns 48 (w / 4) .. : 48, 48 and 32 columns.
    const int quarter = warp & 3, third = warp >> 2;
    const int col0 = third * 48;
    const int nblk = third < 2 ? 3 : 2;              // 16-column blocks of this warp
    const int64_t j = (int64_t)jb * 128 + quarter * 32 + lane;
    const bool j_ok = j < a.n;
    const int emax = j_ok ? a.a_exp_max[j] : TC_EXP_ZERO;
    float hi[48], lo[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) {
      hi[i] = 0.f;
      lo[i] = 0.f;
    }
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    for (int cl = 0; cl < nchunks && !s_abort; ++cl) {
      const int c = c_begin + cl;
      const int e = j_ok ? a.a_exp[j * a.NC + c] : TC_EXP_ZERO;
      const int delta = e - emax;
      const float scale = delta >= -126 ? __int_as_float((127 + delta) << 23) : 0.f;
      for (int gi = 0; gi < TC_G; ++gi) {
        const int g = TC_G - 1 - gi;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[g], cl & 1, TC_WAIT_BUDGET));
        if (!ok) {                       // the whole warp leaves together
          if (lane == 0) fail(31);
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int h2 = 0; h2 < 3; ++h2) {
          if (h2 < nblk) {
            uint32_t r[16];
            tmem_ld16(lane_base + (uint32_t)(g * 128 + h2 * 16), r);
            tmem_ld_wait();
            if (h2 == nblk - 1) {        // all columns read: the group may be overwritten
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&acc_empty[g]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int i = h2 * 16 + q;
              const float v = __fmul_rn(__uint_as_float(r[q]), scale);
              const float s = __fadd_rn(hi[i], v);
              const float bp = __fsub_rn(s, hi[i]);
              const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(s, bp)), __fsub_rn(v, bp));
              hi[i] = s;
              lo[i] = __fadd_rn(lo[i], err);
            }
          }
        }
      }
    }
    if (!s_abort && j_ok) {
      float2* dst = a.partial + ((int64_t)ks * a.n + j) * a.l2p + row0 + col0;
#pragma unroll
      for (int i = 0; i < 48; ++i)
        if (i < nblk * 16 && col0 + i < n_tile) dst[i] = make_float2(hi[i], lo[i]);
    }
  }

  // ---------------- teardown ----------------
  tc_fence_before();
  cluster_sync();          // no CTA of the cluster sends anything after this

  if (warp == 13) {
    if (!mbar_wait(&mma_done, 0, TC_WAIT_BUDGET)) fail(91);
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Y(i, j) = 2^(E_om + E_A - 16) sum_split partial, rows 2i / 2i+1 -> Re / Im;
// rows i >= ly (the row probes) go to X.
__global__ void tc_reduce_kernel(const float2* __restrict__ partial, int ksplit, int64_t n, int l, int l2p,
                                 const int* __restrict__ om_exp, const int* __restrict__ a_exp_max,
                                 double2* __restrict__ Y, int64_t ldy, int ly, double2* __restrict__ X,
                                 int64_t ldx, int64_t j0, int64_t ncols) {
  // columns j0 .. j0 + ncols - 1 of the n-column partial sums
  const int64_t total = ncols * l;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + e / l;
    const int i = (int)(e - (j - j0) * l);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ksplit; ++s) {
      const float2* p = partial + ((int64_t)s * n + j) * l2p + 2 * i;
      re += (double)p[0].x + (double)p[0].y;
      im += (double)p[1].x + (double)p[1].y;
    }
    const int ea = a_exp_max[j];
    const double2 v = make_double2(ea == TC_EXP_ZERO ? 0.0 : ldexp(re, om_exp[2 * i] + ea - 16),
                                   ea == TC_EXP_ZERO ? 0.0 : ldexp(im, om_exp[2 * i + 1] + ea - 16));
    if (i < ly) Y[i + j * ldy] = v;
    else X[(i - ly) + j * ldx] = v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  return enc;
}

// 3D bf16 tensor [slices][rows][KP] with a box of TC_KS x box_rows x 1 and the matching swizzle.
int make_slice_map(CUtensorMap* map, const void* base, int64_t KP, int64_t rows, int slices, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return -1;
  cuuint64_t gdim[3] = {(cuuint64_t)KP, (cuuint64_t)rows, (cuuint64_t)slices};
  cuuint64_t gstride[2] = {(cuuint64_t)KP * 2, (cuuint64_t)(KP * 2 * rows)};
  cuuint32_t box[3] = {TC_KS, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, gdim, gstride, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, TC_KS == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

// K-splits so that the clusters fill whole waves; `slots` = clusters resident at once.
int choose_ksplit(int units, int NC, int sms) {
  int best = 1;
  double best_eff = 0.0;
  const int max_split = max(1, NC / 8);
  for (int ks = 1; ks <= min(max_split, 64); ++ks) {
    const double waves = (double)units * ks / sms;
    const double eff = waves / ceil(waves);
    // prefer fuller waves; among equals, fewer splits
    if (eff > best_eff + 1e-9 && (waves >= 1.0 || ks == max_split)) {
      best_eff = eff;
      best = ks;
    }
    if (best_eff > 0.999) break;
  }
  if (best_eff == 0.0) best = min(max_split, (sms + units - 1) / units);
  return best;
}

}  // namespace

void rid_tc_plan_free_fp64(rid_plan_s* p);

// dry_run: compute p->tc_bytes (the device bytes the state needs) and return
// without allocating or launching anything.
namespace {

void tc_free_state(rid_plan_s* p, TcState* st) {
  if (!st) return;
  rid_dev_free(st->om_slices, p->stream);   // start of the single allocation, released in stream order
  free(st);
}

// A tensor-core state for rows row0 .. row0 + nrows - 1 of Omega: their digit
// planes, the A digit buffers, partial sums and tensor maps.  dry_run: only
// the device bytes.
rid_status tc_setup(rid_plan_s* p, int dry_run, int row0, int nrows, bool a_c64, TcState** out,
                    size_t* bytes_out) {
  *out = nullptr;
  TcState* st = (TcState*)calloc(1, sizeof(TcState));
  if (!st) return RID_ENOMEM;
  st->S = TC_S;
  st->row0 = row0;
  st->nrows = nrows;
  st->a_c64 = a_c64;
  // a rounded Omega holds omega_bits / 8 digits relative to its row exponent,
  // the same exponent omega_exp_kernel takes, so the others are exactly zero
  st->so = p->omega_bits > 0 ? (p->omega_bits + 7) / 8 : TC_S;
  st->NC = (int)((2 * p->m + TC_KC - 1) / TC_KC);
  st->KP = (int64_t)st->NC * TC_KC;
  st->l2 = 2 * nrows;
  st->ntiles = (st->l2 + 127) / 128;
  st->tile_w = ((st->l2 + st->ntiles - 1) / st->ntiles + 15) / 16 * 16;
  st->l2p = st->ntiles * st->tile_w;
  st->nblocks = (int)((p->n + 127) / 128);
  if (st->ntiles > 8) {
    free(st);
    return RID_EUNSUPPORTED;
  }
  // Stage layout: S A tiles, then so Omega tiles of tile_w rows, each a
  // multiple of 1024 bytes; as many stages as shared memory holds.
  st->o_tile_smem = (uint32_t)((st->tile_w * TC_KS * 2 + TC_OPAD - 1) / TC_OPAD * TC_OPAD);
  st->o_off = (uint32_t)(TC_S * TC_TILE_BYTES);
  st->stage_smem = st->o_off + (uint32_t)st->so * st->o_tile_smem;
  st->nstages = (int)((TC_SMEM_LIMIT - 2048 - 1024) / st->stage_smem);
  if (st->nstages > TC_MAX_STAGES) st->nstages = TC_MAX_STAGES;
  if (st->nstages < 2) {
    free(st);
    return RID_EUNSUPPORTED;
  }
  st->dyn_smem = (int)(st->nstages * st->stage_smem + 1024);
  // Clusters span the N-tiles of one column block (they share its A tiles).
  // Sharing Omega tiles across column blocks too (cy > 1) measured slower:
  // larger clusters pack GPCs less densely and run in lockstep.
  st->cx = st->ntiles;
  st->cy = 1;
  st->nblocks_p = (st->nblocks + st->cy - 1) / st->cy * st->cy;
  {
    // how many clusters of this shape are resident at once
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(st->cx, st->nblocks_p, 1);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = st->dyn_smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = st->cx;
    attr[0].val.clusterDim.y = st->cy;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM_MAX);
    if (cudaOccupancyMaxActiveClusters(&clusters, sketch_tc_kernel, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      clusters = p->num_sms / (st->cx * st->cy);
    }
    st->ksplit = choose_ksplit(st->nblocks_p / st->cy, st->NC, clusters > 0 ? clusters : 1);
  }
  st->chunks_per_split = (st->NC + st->ksplit - 1) / st->ksplit;
  st->ksplit = (st->NC + st->chunks_per_split - 1) / st->chunks_per_split;

  const size_t om_bytes = (size_t)TC_S * st->l2 * st->KP * 2;
  const size_t a_bytes = (size_t)TC_S * p->n * st->KP * 2;
  const size_t aexp_bytes = (size_t)p->n * st->NC * 4;
  const size_t part_bytes = (size_t)st->ksplit * p->n * st->l2p * 8;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t total = al(om_bytes) + al(a_bytes) + al(aexp_bytes) + al((size_t)p->n * 4) +
                       al((size_t)st->l2 * 4) + al(part_bytes) + al(4);
  *bytes_out = total;
  if (dry_run) {
    free(st);
    return RID_OK;
  }
  char* base = nullptr;
  if (rid_dev_alloc((void**)&base, total, p->stream, p->device) != cudaSuccess) {
    free(st);
    return RID_ENOMEM;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { char* ptr = base + off; off += al(bytes); return ptr; };
  st->om_slices = (uint16_t*)take(om_bytes);
  st->a_slices = (uint16_t*)take(a_bytes);
  st->a_exp = (int*)take(aexp_bytes);
  st->a_exp_max = (int*)take((size_t)p->n * 4);
  st->om_exp = (int*)take((size_t)st->l2 * 4);
  st->partial = (float2*)take(part_bytes);
  st->err = (int*)take(4);

  if (make_slice_map(&st->map_a, st->a_slices, st->KP, p->n, TC_S, 128) ||
      make_slice_map(&st->map_om, st->om_slices, st->KP, st->l2, TC_S, st->tile_w)) {
    tc_free_state(p, st);
    return RID_ECUDA;
  }
  cudaError_t e = cudaMemsetAsync(st->err, 0, 4, p->stream);
  if (e == cudaSuccess) {
    omega_exp_kernel<<<nrows, 256, 0, p->stream>>>(p->omega + (int64_t)row0 * p->ldo, p->ldo, p->m, st->om_exp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    int64_t blocks = ((int64_t)nrows * (st->KP / 2) + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    omega_slice_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(p->omega + (int64_t)row0 * p->ldo, p->ldo, p->m,
                                                                 nrows, st->KP, st->om_exp, st->om_slices);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sketch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM_MAX);
  if (e == cudaSuccess) {
    // setmaxnreg moves registers between warpgroups inside the launch
    // allocation; it is only safe if the kernel launches with exactly the
    // 128 registers per thread the split adds up to.
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, sketch_tc_kernel);
    if (e == cudaSuccess && fa.numRegs != TC_LAUNCH_REGS) {
      tc_free_state(p, st);
      return RID_EUNSUPPORTED;
    }
  }
  if (e != cudaSuccess) {
    tc_free_state(p, st);
    return RID_ECUDA;
  }
  *out = st;
  return RID_OK;
}

}  // namespace

rid_status rid_tc_plan_setup_fp64(rid_plan_s* p, int dry_run) {
  if (p->mode != RID_FP64_EMULATED || p->dtype != RID_C128) return RID_EUNSUPPORTED;
  TcState* st = nullptr;
  size_t bytes = 0;
  const rid_status s = tc_setup(p, dry_run, 0, p->ls, false, &st, &bytes);   // the test matrix and the row probes
  if (s != RID_OK) return s;
  p->tc_bytes = bytes;
  if (!dry_run) {
    p->tc_state = st;
    p->tc_sketch_launches = 3;
  }
  return RID_OK;
}

void rid_tc_plan_free_fp64(rid_plan_s* p) {
  tc_free_state(p, (TcState*)p->tc_state);
  p->tc_state = nullptr;
  p->tc_bytes = 0;
}

// Mixed-precision plans with row probes: an FP64-emulated state for the probe
// rows alone, multiplied into X from the complex64 A (exact in FP64), so the
// error estimate keeps FP64 grade while Y takes the BF16x3 product.
rid_status rid_tc_probe_init(rid_plan_s* p) {
  TcState* st = nullptr;
  size_t bytes = 0;
  const rid_status s = tc_setup(p, 0, p->l, p->nrow, p->dtype == RID_C64, &st, &bytes);
  if (s != RID_OK) return s;
  p->tc_probe_state = st;
  p->tc_probe_bytes = bytes;
  return RID_OK;
}

void rid_tc_probe_free(rid_plan_s* p) {
  tc_free_state(p, (TcState*)p->tc_probe_state);
  p->tc_probe_state = nullptr;
  p->tc_probe_bytes = 0;
}

namespace {

// Columns col0 .. col0 + ncols - 1 (col0 a multiple of 128) of the product of
// the state's rows of Omega with A: rows below ly go to Y, the others to X.
// The K-split is the state's, so any set of column ranges gives the same
// result as one call over all columns.
cudaError_t tc_sketch(const rid_plan_s* p, const TcState* st, const void* A_, int64_t lda, double2* Y, int64_t ldy,
                      int ly, double2* X, int64_t ldx, int64_t col0, int64_t ncols, bool timing) {
  if (!st) return cudaErrorNotSupported;
  if (ncols <= 0) return cudaSuccess;
  timing = timing && p->timing;
  if (timing) cudaEventRecord(p->ev[0], p->stream);
  // 0x80808080 is below every exponent: the running maximum starts there
  cudaError_t e = cudaMemsetAsync(st->a_exp_max + col0, 0x80, (size_t)ncols * 4, p->stream);
  if (e != cudaSuccess) return e;
  {
    const int64_t tasks = ncols * (int64_t)st->NC;
    int64_t blocks = (tasks * 32 + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 16) blocks = (int64_t)p->num_sms * 16;
    if (st->a_c64)
      a_slice_kernel<float2><<<(unsigned)blocks, 256, 0, p->stream>>>(
          (const float2*)A_ + col0 * lda, lda, p->m, ncols, st->NC, st->KP, p->n * st->KP,
          st->a_slices + col0 * st->KP, st->a_exp + col0 * st->NC, st->a_exp_max + col0);
    else
      a_slice_kernel<double2><<<(unsigned)blocks, 256, 0, p->stream>>>(
          (const double2*)A_ + col0 * lda, lda, p->m, ncols, st->NC, st->KP, p->n * st->KP,
          st->a_slices + col0 * st->KP, st->a_exp + col0 * st->NC, st->a_exp_max + col0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (timing) cudaEventRecord(p->ev[1], p->stream);
  const int jb0 = (int)(col0 / 128);
  const int nblocks = (int)((ncols + 127) / 128);
  TcArgs args{(int)p->n, st->l2, st->l2p, st->NC, st->chunks_per_split, st->ntiles, st->tile_w,
              (uint32_t)(TC_S * TC_TILE_BYTES + st->so * st->tile_w * TC_KS * 2), st->so, st->nstages,
              st->stage_smem, st->o_off, st->o_tile_smem, st->cx, st->cy, jb0,
              st->a_exp, st->a_exp_max, st->partial, st->err};
  {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)st->ntiles, (unsigned)((nblocks + st->cy - 1) / st->cy * st->cy), (unsigned)st->ksplit);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = st->dyn_smem;
    cfg.stream = p->stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = st->cx;
    attr[0].val.clusterDim.y = st->cy;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, sketch_tc_kernel, st->map_a, st->map_om, args);
    if (e != cudaSuccess) return e;
  }
  if (timing) cudaEventRecord(p->ev[2], p->stream);
  {
    const int64_t total = ncols * (int64_t)st->nrows;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)p->num_sms * 32) blocks = (int64_t)p->num_sms * 32;
    tc_reduce_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(st->partial, st->ksplit, p->n, st->nrows, st->l2p,
                                                               st->om_exp, st->a_exp_max, Y, ldy, ly, X, ldx, col0,
                                                               ncols);
    e = cudaGetLastError();
  }
  if (timing) cudaEventRecord(p->ev[3], p->stream);
  return e;
}

}  // namespace

cudaError_t rid_tc_sketch_cols_fp64(const rid_plan_s* p, const void* A_, int64_t lda, double2* Y, int64_t ldy,
                                    int64_t col0, int64_t ncols) {
  return tc_sketch(p, (const TcState*)p->tc_state, A_, lda, Y, ldy, p->l, p->xrow, p->nrow > 0 ? p->nrow : 1, col0,
                   ncols, true);
}

cudaError_t rid_tc_sketch_fp64(const rid_plan_s* p, const void* A_, int64_t lda, double2* Y, int64_t ldy) {
  return rid_tc_sketch_cols_fp64(p, A_, lda, Y, ldy, 0, p->n);
}

// X = G A for a mixed-precision plan's row probes (every row goes to X).
cudaError_t rid_tc_probe_sketch(const rid_plan_s* p, const void* A_, int64_t lda) {
  return tc_sketch(p, (const TcState*)p->tc_probe_state, A_, lda, nullptr, 0, 0, p->xrow, p->nrow, 0, p->n, false);
}

namespace {
int state_error_word(const rid_plan_s* p, const TcState* st) {
  if (!st) return 0;
  int h = 0;
  cudaMemcpyAsync(&h, st->err, 4, cudaMemcpyDeviceToHost, p->stream);
  cudaStreamSynchronize(p->stream);
  return h;
}
}  // namespace

int rid_tc_error_word_fp64(const rid_plan_s* p) { return state_error_word(p, (const TcState*)p->tc_state); }

int rid_tc_probe_error_word(const rid_plan_s* p) { return state_error_word(p, (const TcState*)p->tc_probe_state); }

rid_status rid_tc_plan_init_fp64(rid_plan_s* p) { return rid_tc_plan_setup_fp64(p, 0); }
